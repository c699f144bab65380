"""Time-to-target arithmetic of the paper (Sec. II.B, eq. (1)-(2); Sec. III.A).

* eq. (1): r = max(1, log(1 - 0.99) / log(1 - P_s)) repetitions are needed to
  reach the target with at least 99 % probability when one trial succeeds
  with probability P_s;
* eq. (2): TTT = t_trial * r;
* Sec. III.A: sweeps-to-target = sweeps per run * r;
* Appendix I, footnote 4: a projected time per run from an average time per
  success, successes and runs.

Plain host arithmetic for reporting; no device work.
"""
from __future__ import annotations

import math

CONFIDENCE = 0.99


def repetitions(p_success: float, confidence: float = CONFIDENCE) -> float:
    """eq. (1): repetitions r needed for the given confidence (r >= 1)."""
    if not 0.0 <= p_success <= 1.0:
        raise ValueError("success probability must lie in [0, 1]")
    if p_success == 0.0:
        return math.inf
    if p_success == 1.0:
        return 1.0
    return max(1.0, math.log(1.0 - confidence) / math.log(1.0 - p_success))


def time_to_target(t_trial: float, p_success: float, confidence: float = CONFIDENCE) -> float:
    """eq. (2): TTT = t_trial * r."""
    return t_trial * repetitions(p_success, confidence)


def sweeps_to_target(sweeps_per_run: float, p_success: float,
                     confidence: float = CONFIDENCE) -> float:
    """Sec. III.A: sweeps per run multiplied by the repetitions of eq. (1)."""
    return sweeps_per_run * repetitions(p_success, confidence)


def projected_time_per_run(avg_time_per_success: float, successes: int, runs: int) -> float:
    """Appendix I, footnote 4: total time = average time per success x successes,
    spread over all runs."""
    return avg_time_per_success * successes / runs


def percentile(values, q: float) -> float:
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    xs = sorted(values)
    if not xs:
        return math.nan
    pos = (len(xs) - 1) * q / 100.0
    lo = math.floor(pos)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (pos - lo)


def cut_value(total_weight: int, energy: int) -> int:
    """MaxCut value of a configuration of energy E = sum w_ij s_i s_j: (W - E) / 2."""
    return (total_weight - energy) // 2


def bitstring_hex(spins) -> str:
    """Hex string of a configuration, variables 1..n left to right, most
    significant bit first, bit 1 for spin +1 (the encoding of Appendix II/III);
    the last digit is padded with zero bits."""
    bits = ["1" if int(x) > 0 else "0" for x in spins]
    bits += ["0"] * (-len(bits) % 4)
    return "".join("%X" % int("".join(bits[k:k + 4]), 2) for k in range(0, len(bits), 4))


def spins_from_hex(text: str, n: int | None = None):
    """Inverse of ``bitstring_hex``: spins (+1/-1) of the first n variables."""
    digits = "".join(ch for ch in text if not ch.isspace())
    bits = []
    for ch in digits:
        v = int(ch, 16)
        bits.extend((v >> (3 - b)) & 1 for b in range(4))
    if n is not None:
        bits = bits[:n]
    return [1 if b else -1 for b in bits]
