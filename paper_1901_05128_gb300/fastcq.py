"""ctypes binding of the fastcq C ABI (``include/fastcq.h``).

Argument marshalling only: every function forwards to the entry point of the
same name in ``_build/libfastcq.so`` and raises :class:`CQError` on a non-zero
status. Device buffers are passed as torch CUDA tensors (float64, contiguous)
or raw integer addresses; the CUDA stream defaults to torch's current stream.
There is no CPU implementation behind these names: when the library is not
built, loading fails with an ImportError.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfastcq.so")

CQ_OK, CQ_EINVAL, CQ_ENOMEM, CQ_ECUDA, CQ_ESINGULAR, CQ_ENONFINITE, CQ_ETIMEOUT, CQ_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
CQ_BE, CQ_BDF2 = 1, 2
CQ_DIRECT, CQ_FAST = 0, 1
CQ_F64, CQ_F32, CQ_BF16X3, CQ_TF32X3, CQ_DF64 = 0, 1, 2, 3, 4
FP2S_ASYNC = 1


class CQError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, strerror(status), status))


class FastCfg(C.Structure):
    _fields_ = [("np1", C.c_int32), ("np2", C.c_int32), ("ns", C.c_int32)]


class Problem(C.Structure):
    """fp2s_problem_t."""
    _fields_ = [("alpha1", C.c_double), ("alpha2", C.c_double), ("m", C.c_double), ("T", C.c_double),
                ("N", C.c_int64), ("dim", C.c_int32), ("M", C.c_int32), ("scheme", C.c_int32),
                ("form", C.c_int32), ("fast", FastCfg), ("prec", C.c_int32), ("flags", C.c_int32)]


class BatchPlan(C.Structure):
    """fp2s_batch_t."""
    _fields_ = [("n_inst", C.c_int32), ("n_units", C.c_int32), ("warps_per_block", C.c_int32),
                ("max_np", C.c_int32), ("max_L", C.c_int32), ("max_N", C.c_int32), ("max_M", C.c_int32),
                ("flags", C.c_int32), ("ctas_per_sm", C.c_int32), ("tuned_candidates", C.c_int32),
                ("node_unroll", C.c_int32),
                ("max_modes", C.c_int64), ("field_elems", C.c_int64),
                ("ws_bytes", C.c_int64), ("off", C.c_int64 * 16)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("fastcq CUDA library not built (%s missing); run paper_1901_05128_gb300.build.build()"
                          % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.POINTER(C.c_size_t)
    sig = {
        "cq_strerror": (C.c_char_p, [C.c_int]),
        "cq_launch_count": (I64, []),
        "cq_timing_enable": (C.c_int, [C.c_int]),
        "cq_timing_last": (C.c_int, [C.POINTER(C.c_double)]),
        "cq_timing_part": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
        "cq_test_expire_waits": (C.c_int, [C.c_int]),
        "cq_weights": (C.c_int, [I32, D, D, I64, P, P]),
        "cq_gauss_jacobi": (C.c_int, [I32, D, D, P, P, P]),
        "cq_fast_coeffs": (C.c_int, [I32, D, D, C.POINTER(FastCfg), P, P, SZ, P]),
        "cq_history_direct": (C.c_int, [I32, D, D, I64, I64, I64, P, I64, P, I64, I32, P, SZ, P]),
        "cq_split": (C.c_int, [I32, P, I64, P, P, P]),
        "cq_history_fast": (C.c_int, [I32, D, D, C.POINTER(FastCfg), I64, I64, P, P, I32, P, SZ, P]),
        "cq_history_fast_noalloc": (C.c_int, [I32, D, D, C.POINTER(FastCfg), I64, I64, P, P, I32, P]),
        "fp2s_solve": (C.c_int, [C.POINTER(Problem), P, P, P, SZ, P]),
        "fp2s_solve_modes": (C.c_int, [C.POINTER(Problem), I64, I64, P, P, P, SZ, P]),
        "fp2s_init": (C.c_int, [C.POINTER(Problem), P, P, SZ, P]),
        "fp2s_step": (C.c_int, [C.POINTER(Problem), I64, P, C.c_size_t, P, P]),
        "fp2s_modal": (C.c_int, [C.POINTER(Problem), P, C.c_size_t, P, P]),
        "fp2s_status": (C.c_int, [C.POINTER(Problem), P, C.c_size_t, P]),
        "fp2s_gradient": (C.c_int, [C.POINTER(Problem), P, P, C.POINTER(C.c_double), P, C.POINTER(C.c_double), P,
                                    SZ, P]),
        "fp2s_vjp": (C.c_int, [C.POINTER(Problem), P, P, P, C.POINTER(C.c_double), P, SZ, P]),
        "fp2s_batch_plan": (C.c_int, [C.POINTER(Problem), I32, I32, C.POINTER(BatchPlan), P, SZ, P]),
        "fp2s_solve_batched": (C.c_int, [C.POINTER(BatchPlan), P, P, P, P]),
        "fp2s_batch_status": (C.c_int, [C.POINTER(BatchPlan), P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTS = ("cq_strerror", "cq_launch_count", "cq_timing_enable", "cq_timing_last", "cq_timing_part",
           "cq_test_expire_waits", "cq_weights",
           "cq_gauss_jacobi", "cq_fast_coeffs", "cq_history_direct", "cq_split", "cq_history_fast",
           "cq_history_fast_noalloc", "fp2s_solve", "fp2s_solve_modes",
           "fp2s_init", "fp2s_step", "fp2s_modal", "fp2s_status", "fp2s_gradient", "fp2s_vjp", "fp2s_batch_plan",
           "fp2s_solve_batched", "fp2s_batch_status")


def strerror(status: int) -> str:
    return _lib.cq_strerror(int(status)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream, query=False):
    if query:
        return None                      # size queries enqueue nothing
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st, where):
    if st != CQ_OK:
        raise CQError(st, where)
    return st


def problem(alpha1, alpha2, m, T, N, dim, M, scheme=CQ_BE, form=CQ_DIRECT, np1=32, np2=32, ns=17,
            prec=CQ_F64, flags=0) -> Problem:
    return Problem(float(alpha1), float(alpha2), float(m), float(T), int(N), int(dim), int(M), int(scheme),
                   int(form), FastCfg(int(np1), int(np2), int(ns)), int(prec), int(flags))


def cq_launch_count() -> int:
    return int(_lib.cq_launch_count())


def cq_timing_enable(on: bool):
    _check(_lib.cq_timing_enable(1 if on else 0), "cq_timing_enable")


def cq_timing_last() -> float:
    ms = C.c_double()
    _check(_lib.cq_timing_last(C.byref(ms)), "cq_timing_last")
    return ms.value


def cq_timing_part(part: int) -> float:
    ms = C.c_double()
    _check(_lib.cq_timing_part(int(part), C.byref(ms)), "cq_timing_part")
    return ms.value


def cq_test_expire_waits(on: bool):
    """Failure-path test switch of the tensor-core kernels (see the C header)."""
    _lib.cq_test_expire_waits(1 if on else 0)


def cq_weights(scheme, beta, tau, n, w_dev, stream=None):
    _check(_lib.cq_weights(scheme, beta, tau, n, _ptr(w_dev), _stream(stream)), "cq_weights")


def cq_gauss_jacobi(n, a, b, nodes_dev, weights_dev, stream=None):
    _check(_lib.cq_gauss_jacobi(n, a, b, _ptr(nodes_dev), _ptr(weights_dev), _stream(stream)), "cq_gauss_jacobi")


def cq_fast_coeffs(scheme, beta, tau, np1, np2, ns, coef_dev, ws_dev=None, stream=None) -> int:
    """Returns the workspace size when ws_dev is None (size query)."""
    cfg = FastCfg(np1, np2, ns)
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    _check(_lib.cq_fast_coeffs(scheme, beta, tau, C.byref(cfg), _ptr(coef_dev), _ptr(ws_dev), C.byref(sz),
                               _stream(stream, ws_dev is None)), "cq_fast_coeffs")
    return sz.value


def cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, G_dev, ldg, H_dev, ldh, ws_dev=None, prec=CQ_F64,
                      stream=None) -> int:
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    _check(_lib.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, _ptr(G_dev), ldg, _ptr(H_dev), ldh, prec,
                                  _ptr(ws_dev), C.byref(sz), _stream(stream, ws_dev is None)), "cq_history_direct")
    return sz.value


def cq_split(prec, x_dev, hi_dev, lo_dev, stream=None):
    """Operand split of the tensor-core forms: hi / lo bit patterns (uint16 BF16 or uint32
    TF32-in-FP32) of every FP64 value of x_dev."""
    _check(_lib.cq_split(prec, _ptr(x_dev), x_dev.numel(), _ptr(hi_dev), _ptr(lo_dev), _stream(stream)), "cq_split")


def cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, n, G_prev_dev, H_dev, ws_dev=None, prec=CQ_F64,
                    stream=None) -> int:
    cfg = FastCfg(np1, np2, ns)
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    _check(_lib.cq_history_fast(scheme, beta, tau, C.byref(cfg), ndof, n, _ptr(G_prev_dev), _ptr(H_dev), prec,
                                _ptr(ws_dev), C.byref(sz), _stream(stream, ws_dev is None)), "cq_history_fast")
    return sz.value


def cq_history_fast_noalloc(scheme, beta, tau, np1, np2, ns, ndof, n, G_prev_dev, H_dev, prec=CQ_F64,
                            stream=None):
    """cq_history_fast without a workspace: the state lives in the library's own
    fixed-size device array (for callers that cannot allocate device memory)."""
    cfg = FastCfg(np1, np2, ns)
    _check(_lib.cq_history_fast_noalloc(scheme, beta, tau, C.byref(cfg), ndof, n, _ptr(G_prev_dev), _ptr(H_dev),
                                        prec, _stream(stream)), "cq_history_fast_noalloc")


def fp2s_solve(p: Problem, G0_dev, GN_dev, ws_dev=None, stream=None, check=True) -> int:
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    st = _lib.fp2s_solve(C.byref(p), _ptr(G0_dev), _ptr(GN_dev), _ptr(ws_dev), C.byref(sz),
                         _stream(stream, ws_dev is None))
    if check:
        _check(st, "fp2s_solve")
    elif st not in (CQ_OK, CQ_ENONFINITE):
        _check(st, "fp2s_solve")
    return sz.value if ws_dev is None else st


def fp2s_solve_modes(p: Problem, mode_lo, mode_hi, g0_dev, gN_dev, ws_dev=None, stream=None, check=True) -> int:
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    st = _lib.fp2s_solve_modes(C.byref(p), int(mode_lo), int(mode_hi), _ptr(g0_dev), _ptr(gN_dev), _ptr(ws_dev),
                               C.byref(sz), _stream(stream, ws_dev is None))
    if check:
        _check(st, "fp2s_solve_modes")
    elif st not in (CQ_OK, CQ_ENONFINITE):
        _check(st, "fp2s_solve_modes")
    return sz.value if ws_dev is None else st


def fp2s_init(p: Problem, G0_dev, ws_dev=None, stream=None) -> int:
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    _check(_lib.fp2s_init(C.byref(p), _ptr(G0_dev), _ptr(ws_dev), C.byref(sz), _stream(stream, ws_dev is None)),
           "fp2s_init")
    return sz.value


def fp2s_step(p: Problem, n, ws_dev, G_out_dev=None, stream=None):
    _check(_lib.fp2s_step(C.byref(p), n, _ptr(ws_dev), _nbytes(ws_dev), _ptr(G_out_dev), _stream(stream)),
           "fp2s_step")


def fp2s_modal(p: Problem, ws_dev, g_dev, stream=None):
    _check(_lib.fp2s_modal(C.byref(p), _ptr(ws_dev), _nbytes(ws_dev), _ptr(g_dev), _stream(stream)), "fp2s_modal")


def fp2s_gradient(p: Problem, G0_dev, Gt_dev, dJdG0_dev, ws_dev=None, stream=None):
    """Returns the workspace size when ws_dev is None, else (J, (dJ/dalpha1, dJ/dalpha2));
    dJ/dG0 is written to dJdG0_dev."""
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    J = C.c_double(0.0)
    da = (C.c_double * 2)()
    _check(_lib.fp2s_gradient(C.byref(p), _ptr(G0_dev), _ptr(Gt_dev), C.byref(J), _ptr(dJdG0_dev), da, _ptr(ws_dev),
                              C.byref(sz), _stream(stream, ws_dev is None)), "fp2s_gradient")
    if ws_dev is None:
        return sz.value
    return J.value, (da[0], da[1])


def fp2s_vjp(p: Problem, G0_dev, dGN_dev, dG0_dev, ws_dev=None, stream=None):
    """Returns the workspace size when ws_dev is None, else (dL/dalpha1, dL/dalpha2);
    dL/dG0 for the upstream gradient dGN_dev is written to dG0_dev."""
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    da = (C.c_double * 2)()
    _check(_lib.fp2s_vjp(C.byref(p), _ptr(G0_dev), _ptr(dGN_dev), _ptr(dG0_dev), da, _ptr(ws_dev), C.byref(sz),
                         _stream(stream, ws_dev is None)), "fp2s_vjp")
    if ws_dev is None:
        return sz.value
    return da[0], da[1]


def fp2s_batch_plan(problems, ws_dev=None, tune=False, stream=None):
    """Size query (ws_dev None) -> bytes; else -> BatchPlan."""
    arr = (Problem * len(problems))(*problems)
    plan = BatchPlan()
    sz = C.c_size_t(0 if ws_dev is None else _nbytes(ws_dev))
    _check(_lib.fp2s_batch_plan(arr, len(problems), 1 if tune else 0, C.byref(plan), _ptr(ws_dev), C.byref(sz),
                                _stream(stream, ws_dev is None)), "fp2s_batch_plan")
    return sz.value if ws_dev is None else plan


def fp2s_solve_batched(plan: BatchPlan, G0_dev, GN_dev, ws_dev, stream=None):
    _check(_lib.fp2s_solve_batched(C.byref(plan), _ptr(G0_dev), _ptr(GN_dev), _ptr(ws_dev), _stream(stream)),
           "fp2s_solve_batched")


def fp2s_batch_status(plan: BatchPlan, ws_dev, stream=None) -> int:
    return int(_lib.fp2s_batch_status(C.byref(plan), _ptr(ws_dev), _stream(stream)))


def fp2s_status(p: Problem, ws_dev, stream=None) -> int:
    return int(_lib.fp2s_status(C.byref(p), _ptr(ws_dev), _nbytes(ws_dev), _stream(stream)))


def _nbytes(t) -> int:
    if isinstance(t, int):
        raise TypeError("pass workspaces as tensors so that their size is known")
    return t.numel() * t.element_size()


def workspace(nbytes: int, device="cuda"):
    """A caller-owned workspace of at least ``nbytes`` bytes (256-byte aligned by the allocator)."""
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
