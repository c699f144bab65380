"""Python binding of libisg (the C ABI of ``include/isg.h``).

Argument marshalling only: every step of the annealing path runs in the CUDA
library.  Functions carry the C names; arrays are numpy; handles are opaque
integers wrapped in small owner classes.  PyTorch is used for one thing: when
no stream is given, work is enqueued on ``torch.cuda.current_stream()``.

The library is built in-tree by ``paper_2311_09275_gb300.build``.  Importing
this module without the built library raises ImportError: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libisg.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libisg is not built ({_LIB_PATH}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
_lib = ctypes.CDLL(_LIB_PATH)

ISG_OK, ISG_EINVAL, ISG_ENOMEM, ISG_ECUDA, ISG_ETIMEOUT, ISG_EBUSY, ISG_ECANCELLED = range(7)
ISG_NO_TARGET = -(2 ** 63)
KERNEL_AUTO, KERNEL_TORUS_MSC, KERNEL_CSR, KERNEL_PLAIN = range(4)

_P = ctypes.c_void_p
_i32, _i64, _u64, _dbl, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, \
    ctypes.c_size_t


class isg_options(ctypes.Structure):
    _fields_ = [("kernel", _i32), ("cluster_ctas", _i32), ("threads", _i32),
                ("time_kernels", _i32), ("quads_per_cta", _i32), ("first_replica", _i32),
                ("mask_chunk", _i32)]


class isg_stats(ctypes.Structure):
    _fields_ = [("sweep_kernel_ms", ctypes.c_float), ("launches", _i32),
                ("sweep_launches", _i32), ("kernel", _i32), ("ctas", _i32),
                ("cluster_ctas", _i32), ("threads", _i32), ("h2d_bytes", _i64),
                ("staged", _i32), ("first_replica", _i32), ("mask_chunks", _i32)]


class isg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("queued", _i32), ("active", _i32),
                ("peak_active", _i32), ("passes", _i64), ("replays", _i64), ("cancelled", _i64)]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("isg_problem_create_edges", [_i32, _i64, _P, _P, _P, ctypes.POINTER(_P)])
_sig("isg_problem_create_csr", [_i32, _P, _P, _P, ctypes.POINTER(_P)])
_sig("isg_problem_create_fields", [_i32, _i64, _P, _P, _P, _P, ctypes.POINTER(_P)])
_sig("isg_problem_create_torus", [_i32, _i32, _P, _P, ctypes.POINTER(_P)])
_sig("isg_problem_info", [_P, _P, _P, _P, _P, _P])
_sig("isg_problem_set_colouring", [_P, _i32])
_sig("isg_problem_destroy", [_P], None)
_sig("isg_anneal", [_P, _i32, _P, _i32, _u64, _i64, _P, ctypes.POINTER(_P)])
_sig("isg_anneal_ex", [_P, _i32, _P, _i32, _u64, _i64, ctypes.POINTER(isg_options), _P,
                       ctypes.POINTER(_P)])
_sig("isg_anneal_batch", [_P, _i32, _i32, _P, _i32, _P, _P, _P, _P])
_sig("isg_anneal_continue", [_P, _P, _P, _i32, _P])
_sig("isg_autotune_batch", [_P, _i32, _i32, _P, _i32, _i32, _P, _P, _P])
_sig("isg_debug_fail_allocations", [_i32])
_sig("isg_anneal_resume", [_P, _i32, _P, _i32, _u64, _i32, _P, _P, ctypes.POINTER(isg_options),
                           _P, ctypes.POINTER(_P)])
_sig("isg_autotune", [_P, _i32, _i32, _P, ctypes.POINTER(isg_options)])
_sig("isg_energy", [_P, _P, _i32, _P])
_sig("isg_energy_noalloc", [_i32, _P, _P, _P, _P, _i32, _P, _P])
_sig("isg_result_final", [_P, _P, _P, _P])
_sig("isg_best", [_P, _P, _P, _P, _P, _P])
_sig("isg_result_shape", [_P, _P, _P, _P])
_sig("isg_result_best_all", [_P, _P])
_sig("isg_result_stats", [_P, ctypes.POINTER(isg_stats)])
_sig("isg_result_destroy", [_P], None)
_sig("isg_server_create", [_sz, _i32, _i32, ctypes.POINTER(_P)])
_sig("isg_server_submit", [_P, _P, _i32, _P, _i32, _u64, _i64, ctypes.POINTER(_u64)])
_sig("isg_server_poll", [_P, ctypes.POINTER(_u64), ctypes.POINTER(_P), _dbl])
_sig("isg_server_destroy", [_P])
_sig("isg_server_get_stats", [_P, ctypes.POINTER(isg_server_stats)])
_sig("isg_server_cancel", [_P, _u64])
_sig("isg_integer_peaks", [_P, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)])
_sig("isg_acceptance_table", [_P, _i32, _i32, _P])
_sig("isg_philox_rates", [_P, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)])
_sig("isg_parallel_tempering", [_P, _i32, _P, _i32, _i32, _i32, _u64,
                                ctypes.POINTER(isg_options), _P, ctypes.POINTER(_P)])
_sig("isg_result_cluster_flips", [_P, _P, _i32])
_sig("isg_result_exchanges", [_P, _P, _P, _i32])
_sig("isg_last_error", [], ctypes.c_char_p)
_sig("isg_version", [], ctypes.c_char_p)


class IsgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"isg status {status}: {message}")
        self.status = status


def _check(st: int):
    if st != ISG_OK:
        raise IsgError(st, (_lib.isg_last_error() or b"").decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def _stream(stream):
    """Raw cudaStream_t: an int, a torch stream, or None = torch's current stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def library_path() -> str:
    return _LIB_PATH


def isg_version() -> str:
    return _lib.isg_version().decode()


# ------------------------------------------------------------------ problems
class Problem:
    """Owner of an isg_problem handle."""

    def __init__(self, handle: int):
        self.handle = handle
        info = isg_problem_info(self)
        self.n, self.m, self.total_weight, self.n_colors = (info["n"], info["m"],
                                                            info["total_weight"],
                                                            info["n_colors"])

    def close(self):
        if self.handle:
            _lib.isg_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(x):
    return x.handle if hasattr(x, "handle") else x


def isg_problem_create_edges(n: int, u, v, w) -> Problem:
    u, v, w = _arr(u, np.int32), _arr(v, np.int32), _arr(w, np.int32)
    out = _P()
    _check(_lib.isg_problem_create_edges(n, int(u.shape[0]), _ptr(u), _ptr(v), _ptr(w),
                                         ctypes.byref(out)))
    return Problem(out.value)


def isg_problem_create_fields(n: int, u, v, w, h) -> Problem:
    u, v, w = _arr(u, np.int32), _arr(v, np.int32), _arr(w, np.int32)
    hh = None if h is None else _arr(h, np.int32)
    if hh is not None and hh.shape != (n,):
        raise ValueError("fields need one entry per vertex")
    out = _P()
    _check(_lib.isg_problem_create_fields(n, int(u.shape[0]), _ptr(u), _ptr(v), _ptr(w),
                                          _ptr(hh) if hh is not None else None,
                                          ctypes.byref(out)))
    return Problem(out.value)


def isg_problem_create_csr(n: int, rowptr, col, w) -> Problem:
    rowptr, col, w = _arr(rowptr, np.int64), _arr(col, np.int32), _arr(w, np.int32)
    out = _P()
    _check(_lib.isg_problem_create_csr(n, _ptr(rowptr), _ptr(col), _ptr(w), ctypes.byref(out)))
    return Problem(out.value)


def isg_problem_create_torus(L: int, W: int, j_right, j_down) -> Problem:
    jr, jd = _arr(j_right, np.int8), _arr(j_down, np.int8)
    out = _P()
    _check(_lib.isg_problem_create_torus(L, W, _ptr(jr), _ptr(jd), ctypes.byref(out)))
    return Problem(out.value)


def isg_problem_info(p, colors: bool = False) -> dict:
    n, m, tw, nc = _i32(), _i64(), _i64(), _i32()
    _check(_lib.isg_problem_info(_h(p), ctypes.byref(n), ctypes.byref(m), ctypes.byref(tw),
                                 ctypes.byref(nc), None))
    d = {"n": n.value, "m": m.value, "total_weight": tw.value, "n_colors": nc.value}
    if colors:
        c = np.zeros(n.value, dtype=np.int32)
        _check(_lib.isg_problem_info(_h(p), None, None, None, None, _ptr(c)))
        d["colors"] = c
    return d


COLOURING_GREEDY, COLOURING_SMALLEST_LAST = 0, 1


def isg_problem_set_colouring(p, method: int):
    """Colour classes of a graph instance: 0 greedy by id (default), 1 smallest-last."""
    _check(_lib.isg_problem_set_colouring(_h(p), int(method)))


def isg_problem_destroy(p):
    if isinstance(p, Problem):
        p.close()
    else:
        _lib.isg_problem_destroy(p)


def problem_of(instance, colouring: int = COLOURING_GREEDY) -> Problem:
    """libisg instance of a generator object from ``paper_2311_09275_gb300.inputs``
    (graphs coloured by ``colouring``, an isg_colouring)."""
    if hasattr(instance, "L"):
        return isg_problem_create_torus(instance.L, instance.W, instance.j_right,
                                        instance.j_down)
    if getattr(instance, "h", None) is not None:
        p = isg_problem_create_fields(instance.n, instance.u, instance.v, instance.w,
                                      instance.h)
    else:
        p = isg_problem_create_edges(instance.n, instance.u, instance.v, instance.w)
    if colouring != COLOURING_GREEDY:
        isg_problem_set_colouring(p, colouring)
    return p


# ------------------------------------------------------------------ results
class Result:
    """Owner of an isg_result handle."""

    def __init__(self, handle: int):
        self.handle = handle
        n, R, S = _i32(), _i32(), _i32()
        _check(_lib.isg_result_shape(handle, ctypes.byref(n), ctypes.byref(R), ctypes.byref(S)))
        self.n, self.replicas, self.sweeps = n.value, R.value, S.value

    def final(self, spins: bool = True):
        return isg_result_final(self, spins)

    def best(self, spins: bool = True):
        return isg_best(self, spins)

    def best_all(self):
        return isg_result_best_all(self)

    def stats(self) -> dict:
        return isg_result_stats(self)

    def close(self):
        if self.handle:
            _lib.isg_result_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def isg_anneal(p, replicas: int, betas, seed: int, target=None, stream=None, kernel: int = 0,
               cluster_ctas: int = 0, threads: int = 0, time_kernels: bool = False,
               quads_per_cta: int = 0, first_replica: int = 0, mask_chunk: int = 0) -> Result:
    """Anneal `replicas` replicas (global indices first_replica + 0..replicas-1,
    first_replica a multiple of 32) through isg_anneal_ex; mask_chunk as in
    isg_options (-1: the graph kernel builds its acceptance masks itself)."""
    b = _arr(betas, np.float64)
    opts = isg_options(kernel, cluster_ctas, threads, 1 if time_kernels else 0, quads_per_cta,
                       first_replica, mask_chunk)
    out = _P()
    _check(_lib.isg_anneal_ex(_h(p), int(replicas), _ptr(b), int(b.shape[0]),
                              int(seed) & 0xFFFFFFFFFFFFFFFF,
                              ISG_NO_TARGET if target is None else int(target),
                              ctypes.byref(opts), _stream(stream), ctypes.byref(out)))
    return Result(out.value)


def isg_anneal_continue(p, res, betas, stream=None) -> None:
    """Run len(betas) more sweeps of the solve `res` (of problem p, no target):
    afterwards `res` equals one solve of the concatenated schedule."""
    b = _arr(betas, np.float64)
    _check(_lib.isg_anneal_continue(_h(p), _h(res), _ptr(b), int(b.shape[0]), _stream(stream)))
    if isinstance(res, Result):
        res.sweeps += int(b.shape[0])


def isg_anneal_resume(p, replicas: int, betas, seed: int, sweeps_done: int, spins, best_spins,
                      stream=None, kernel: int = 0, cluster_ctas: int = 0, threads: int = 0,
                      quads_per_cta: int = 0, first_replica: int = 0,
                      mask_chunk: int = 0) -> Result:
    """A solve restarted from a checkpoint (final and best int8 states after
    `sweeps_done` sweeps); equal to one solve of the whole schedule."""
    b = _arr(betas, np.float64)
    s = _arr(spins, np.int8)
    bs = _arr(best_spins, np.int8)
    if s.size != int(replicas) * _lib_n(p) or bs.size != s.size:
        raise ValueError("spins and best_spins must hold replicas x n values")
    opts = isg_options(kernel, cluster_ctas, threads, 0, quads_per_cta, first_replica, mask_chunk)
    out = _P()
    _check(_lib.isg_anneal_resume(_h(p), int(replicas), _ptr(b), int(b.shape[0]),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(sweeps_done), _ptr(s),
                                  _ptr(bs), ctypes.byref(opts), _stream(stream),
                                  ctypes.byref(out)))
    return Result(out.value)


def _lib_n(p) -> int:
    return isg_problem_info(p)["n"]


def isg_debug_fail_allocations(count: int) -> None:
    """Make the next `count` solve-state allocations fail with ISG_ENOMEM (tests)."""
    _check(_lib.isg_debug_fail_allocations(int(count)))


def isg_autotune(p, replicas: int, probe_sweeps: int = 64, stream=None) -> dict:
    """Measure launch shapes for (instance, replicas); later solves use the best."""
    best = isg_options()
    _check(_lib.isg_autotune(_h(p), int(replicas), int(probe_sweeps), _stream(stream),
                             ctypes.byref(best)))
    return {"kernel": best.kernel, "cluster_ctas": best.cluster_ctas, "threads": best.threads,
            "quads_per_cta": best.quads_per_cta}


def isg_autotune_batch(problems, replicas: int, betas, probe_sweeps: int = 128,
                       stream=None) -> dict:
    """Measured launch shape of the batched form for this batch's size histogram
    (remembered for later isg_anneal_batch calls of the same histogram), probed
    on sweeps sampled evenly from the schedule `betas`."""
    count = len(problems)
    hs = (_P * count)(*[_h(p) for p in problems])
    b = _arr(betas, np.float64)
    t, c = _i32(), _i32()
    _check(_lib.isg_autotune_batch(ctypes.cast(hs, _P), count, int(replicas), _ptr(b),
                                   int(b.shape[0]), int(probe_sweeps), _stream(stream),
                                   ctypes.byref(t), ctypes.byref(c)))
    return {"threads": t.value, "ctas_per_sm": c.value}


def isg_anneal_batch(problems, replicas: int, betas, seeds, targets=None, stream=None):
    count = len(problems)
    hs = (_P * count)(*[_h(p) for p in problems])
    b = _arr(betas, np.float64)
    sd = _arr([int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds], np.uint64)
    tg = None
    if targets is not None:
        tg = _arr([ISG_NO_TARGET if t is None else int(t) for t in targets], np.int64)
    outs = (_P * count)()
    _check(_lib.isg_anneal_batch(ctypes.cast(hs, _P), count, int(replicas), _ptr(b),
                                 int(b.shape[0]), _ptr(sd), _ptr(tg) if tg is not None else None,
                                 _stream(stream), ctypes.cast(outs, _P)))
    return [Result(outs[k]) for k in range(count)]


def isg_energy(p, spins) -> np.ndarray:
    s = _arr(spins, np.int8)
    if s.ndim == 1:
        s = s[None, :]
    e = np.zeros(s.shape[0], dtype=np.int64)
    _check(_lib.isg_energy(_h(p), _ptr(s), int(s.shape[0]), _ptr(e)))
    return e


def isg_energy_noalloc(n: int, rowptr_dev: int, col_dev: int, w_dev: int, spins_dev: int,
                       replicas: int, energies_dev: int, stream=None):
    """Energies of device-resident configurations with no device allocation.

    For callers that cannot allocate device memory at call time (device memory
    fully reserved by another allocator, or a loop that must stay out of the
    driver's allocator).  Every argument is a raw device address the caller
    owns (e.g. ``tensor.data_ptr()``); see ``isg_energy_noalloc`` in isg.h for
    layouts, the replica limit and the rule on overlapping calls.
    """
    _check(_lib.isg_energy_noalloc(int(n), rowptr_dev, col_dev, w_dev, spins_dev, int(replicas),
                                   energies_dev, _stream(stream)))


def isg_parallel_tempering(p, betas, rounds: int, sweeps_per_round: int, seed: int,
                           stream=None, cluster_ctas: int = 0, threads: int = 0,
                           time_kernels: bool = False, icm_slots: int = 0,
                           quads_per_cta: int = 0) -> "Result":
    """Parallel tempering over len(betas) slots x 32 chains (replica r = 32 k + c),
    with Houdayer cluster moves on the last icm_slots slots."""
    b = _arr(betas, np.float64)
    opts = isg_options(0, cluster_ctas, threads, 1 if time_kernels else 0, quads_per_cta, 0)
    out = _P()
    _check(_lib.isg_parallel_tempering(_h(p), int(b.shape[0]), _ptr(b), int(rounds),
                                       int(sweeps_per_round), int(icm_slots),
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(opts),
                                       _stream(stream), ctypes.byref(out)))
    res = Result(out.value)
    res.pairs = int(b.shape[0]) - 1
    return res


def isg_result_exchanges(r, pairs: int):
    """(accepted[pairs], attempted[pairs]) exchange counts of a tempering result."""
    acc = np.zeros(max(pairs, 1), dtype=np.int64)
    att = np.zeros(max(pairs, 1), dtype=np.int64)
    _check(_lib.isg_result_exchanges(_h(r), _ptr(acc), _ptr(att), int(pairs)))
    return acc[:pairs], att[:pairs]


def isg_result_cluster_flips(r, temperatures: int) -> np.ndarray:
    """Sites flipped by cluster moves per slot (summed over pairs and rounds)."""
    f = np.zeros(temperatures, dtype=np.int64)
    _check(_lib.isg_result_cluster_flips(_h(r), _ptr(f), int(temperatures)))
    return f


def isg_acceptance_table(betas, kmax: int) -> np.ndarray:
    """[S][kmax + 1] uint32 thresholds the solve paths use (host computation)."""
    b = _arr(betas, np.float64)
    out = np.empty((b.shape[0], kmax + 1), dtype=np.uint32)
    _check(_lib.isg_acceptance_table(_ptr(b), int(b.shape[0]), int(kmax), _ptr(out)))
    return out


def isg_philox_rates(stream=None) -> dict:
    """Measured uniforms/s of the sweeps' Philox stream alone and with the threshold masks."""
    a, b = _dbl(), _dbl()
    _check(_lib.isg_philox_rates(_stream(stream), ctypes.byref(a), ctypes.byref(b)))
    return {"uniforms_per_s": a.value, "masked_per_s": b.value}


def isg_integer_peaks(stream=None) -> dict:
    """Measured device-wide rates (thread-instructions/s) of lop3 and mul.wide.u32."""
    a, b = _dbl(), _dbl()
    _check(_lib.isg_integer_peaks(_stream(stream), ctypes.byref(a), ctypes.byref(b)))
    return {"lop3_per_s": a.value, "mul_wide_per_s": b.value}


def isg_result_final(r: Result, spins: bool = True):
    """(spins [R][n] int8 or None, energies [R] int32, sweeps_done)."""
    sp = np.empty((r.replicas, r.n), dtype=np.int8) if spins else None
    e = np.empty(r.replicas, dtype=np.int32)
    done = _i32()
    _check(_lib.isg_result_final(_h(r), _ptr(sp) if sp is not None else None, _ptr(e),
                                 ctypes.byref(done)))
    return sp, e, done.value


def isg_best(r: Result, spins: bool = True):
    """(best energy, best replica, its spins [n] or None, per-replica best [R], hit sweep)."""
    be, br, hit = _i32(), _i32(), _i32()
    sp = np.empty(r.n, dtype=np.int8) if spins else None
    per = np.empty(r.replicas, dtype=np.int32)
    _check(_lib.isg_best(_h(r), ctypes.byref(be), ctypes.byref(br),
                         _ptr(sp) if sp is not None else None, _ptr(per), ctypes.byref(hit)))
    return be.value, br.value, sp, per, hit.value


def isg_result_best_all(r: Result) -> np.ndarray:
    sp = np.empty((r.replicas, r.n), dtype=np.int8)
    _check(_lib.isg_result_best_all(_h(r), _ptr(sp)))
    return sp


def isg_result_stats(r: Result) -> dict:
    st = isg_stats()
    _check(_lib.isg_result_stats(_h(r), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in isg_stats._fields_}


def isg_result_destroy(r):
    if isinstance(r, Result):
        r.close()
    else:
        _lib.isg_result_destroy(r)


# ------------------------------------------------------------------ serving
class Server:
    """Owner of an isg_server handle (continuous batching on the current device)."""

    def __init__(self, device_mem_budget: int, max_slots: int, sweeps_per_chunk: int):
        out = _P()
        _check(_lib.isg_server_create(int(device_mem_budget), int(max_slots),
                                      int(sweeps_per_chunk), ctypes.byref(out)))
        self.handle = out.value

    def submit(self, p, replicas: int, betas, seed: int, target=None) -> int:
        return isg_server_submit(self, p, replicas, betas, seed, target)

    def poll(self, timeout_s: float = 1.0):
        return isg_server_poll(self, timeout_s)

    def stats(self) -> dict:
        return isg_server_get_stats(self)

    def cancel(self, request_id: int) -> None:
        isg_server_cancel(self, request_id)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(_lib.isg_server_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def isg_server_create(device_mem_budget: int, max_slots: int, sweeps_per_chunk: int) -> Server:
    return Server(device_mem_budget, max_slots, sweeps_per_chunk)


def isg_server_cancel(s, request_id: int) -> None:
    _check(_lib.isg_server_cancel(_h(s), int(request_id)))


def isg_server_get_stats(s) -> dict:
    st = isg_server_stats()
    _check(_lib.isg_server_get_stats(_h(s), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in isg_server_stats._fields_}


def isg_server_submit(s, p, replicas: int, betas, seed: int, target=None) -> int:
    b = _arr(betas, np.float64)
    rid = _u64()
    _check(_lib.isg_server_submit(_h(s), _h(p), int(replicas), _ptr(b), int(b.shape[0]),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF,
                                  ISG_NO_TARGET if target is None else int(target),
                                  ctypes.byref(rid)))
    return rid.value


def isg_server_poll(s, timeout_s: float = 1.0):
    """(request id, Result) of a finished request, or None after the timeout."""
    rid, out = _u64(), _P()
    st = _lib.isg_server_poll(_h(s), ctypes.byref(rid), ctypes.byref(out), float(timeout_s))
    if st == ISG_ETIMEOUT:
        return None
    _check(st)
    return rid.value, Result(out.value)


def isg_server_destroy(s):
    if isinstance(s, Server):
        s.close()
    else:
        _check(_lib.isg_server_destroy(s))
