"""Writes served_oracle_64.txt: the oracle's results for a seeded sample of 64
requests of the served workload (Poisson stream of +-1 tori 40..100 x 40..200
and unweighted random graphs of 2,000..20,000 vertices with mean degree 2..4;
32 replicas; a budget of 10,000 geometric sweeps from 0.1 to 5.0).

For each sampled request j: the target is the oracle's lowest best energy over
the whole budget (the plain form's best), then the oracle runs the request to
that target.  One line per request:

  j target hit_sweep sweeps_done best_energy best_replica sha256(final spins)
  sha256(best spins) e_final[0..31] e_best[0..31]

the spin arrays being int8 [replica][vertex] in the request's vertex order.
Only the oracle and the seeded input generators are called.  Run from the
repository root: python tests/golden/make_served_oracle.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2311_09275_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "served_oracle_64.txt")


def sample():
    """The seeded sample of 64 request indices of the 2,000-request stream."""
    rng = np.random.default_rng(55)
    return sorted(int(x) for x in rng.choice(2000, size=64, replace=False))


def main():
    reqs = I.served_stream(count=2000, sweeps=10000)
    cores = os.cpu_count() or 1
    lines = []
    for j in sample():
        sv = reqs[j].solve
        c = oracle.csr_of(sv.problem)
        full = oracle.anneal(c, sv.replicas, sv.betas, sv.seed, nthreads=cores)
        target = int(full.e_best.min())
        o = oracle.anneal(c, sv.replicas, sv.betas, sv.seed, target=target, nthreads=cores)
        be, br = o.best
        hf = hashlib.sha256(np.ascontiguousarray(o.s_final, np.int8).tobytes()).hexdigest()
        hb = hashlib.sha256(np.ascontiguousarray(o.s_best, np.int8).tobytes()).hexdigest()
        row = [j, target, o.hit_sweep, o.sweeps_done, be, br, hf, hb]
        row += [int(x) for x in o.e_final] + [int(x) for x in o.e_best]
        lines.append(" ".join(str(x) for x in row))
        print(j, target, o.hit_sweep, flush=True)
    with open(OUT, "w") as f:
        f.write("# oracle results for 64 sampled served requests; written by "
                "make_served_oracle.py (see its docstring for the columns)\n")
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
