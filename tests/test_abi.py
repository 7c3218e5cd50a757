"""Host-side checks of the C ABI: the library builds, loads, exports every
function declared in include/fastcq.h, and rejects invalid arguments before
touching the GPU (size queries and argument errors need no device)."""
import ctypes as C
import os
import re

import pytest

import paper_1901_05128_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fc():
    pkg.build()
    return pkg.load()


def _declared(only=None):
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h") and (only is None or fn == only):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b((?:cq|fp2s)_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(fc):
    decl = _declared("fastcq.h")
    assert {"cq_weights", "cq_history_direct", "cq_history_fast", "fp2s_step", "fp2s_solve"} <= decl
    lib = C.CDLL(fc.LIB_PATH)
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fc.EXPORTS) == decl


def test_strerror(fc):
    assert fc.strerror(0) == "ok"
    assert "workspace" in fc.strerror(-2)


def test_invalid_arguments_rejected_on_host(fc):
    lib = fc._lib
    assert lib.cq_weights(1, 1.5, 0.1, 10, None, None) == fc.CQ_EINVAL
    assert lib.cq_weights(3, 0.5, 0.1, 10, None, None) == fc.CQ_EINVAL
    assert lib.cq_weights(1, 0.5, -0.1, 10, None, None) == fc.CQ_EINVAL
    assert lib.cq_gauss_jacobi(0, 0.5, 0.5, None, None, None) == fc.CQ_EINVAL
    assert lib.cq_gauss_jacobi(300, 0.5, 0.5, 8, 8, None) == fc.CQ_EINVAL
    sz = C.c_size_t(0)
    assert lib.cq_history_direct(1, 0.5, 0.1, 10, 0, 5, None, 10, None, 10, 0, None, C.byref(sz), None) == fc.CQ_EINVAL
    assert lib.cq_history_direct(1, 0.5, 0.1, 10, 1, 5, None, 10, None, 10, 7, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED
    cfg = fc.FastCfg(8, 8, 2)
    assert lib.cq_history_fast(2, 0.5, 0.1, C.byref(cfg), 10, 1, None, None, 0, None, C.byref(sz), None) == fc.CQ_EINVAL
    assert lib.cq_split(fc.CQ_F64, None, 0, None, None, None) == fc.CQ_EUNSUPPORTED
    assert lib.cq_split(fc.CQ_BF16X3, None, -1, None, None, None) == fc.CQ_EINVAL
    assert lib.cq_split(fc.CQ_TF32X3, None, 0, None, None, None) == fc.CQ_OK          # nothing to split
    assert lib.cq_split(fc.CQ_BF16X3, None, 5, None, None, None) == fc.CQ_EINVAL


def test_test_switch_toggles(fc):
    assert fc._lib.cq_test_expire_waits(1) == fc.CQ_OK
    assert fc._lib.cq_test_expire_waits(0) == fc.CQ_OK


def test_batch_size_limit(fc):
    probs = (fc.Problem * 65536)()
    plan = fc.BatchPlan()
    sz = C.c_size_t(0)
    assert fc._lib.fp2s_batch_plan(probs, 65536, 0, C.byref(plan), None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED
    assert fc._lib.fp2s_batch_plan(probs, 3, 0, C.byref(plan), None, C.byref(sz), None) == fc.CQ_EINVAL  # zeroed


@pytest.mark.parametrize("m", [0.5, 1.0, -0.1])
def test_problem_validation(fc, m):
    p = fc.problem(0.3, 0.7, m, 1.0, 64, 1, 15)
    sz = C.c_size_t(0)
    assert fc._lib.fp2s_solve(C.byref(p), None, None, None, C.byref(sz), None) == fc.CQ_EINVAL


def test_size_queries_need_no_device(fc):
    p = fc.problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, fc.CQ_BDF2, fc.CQ_FAST, 16, 64, 17)
    n_fast = fc.fp2s_solve(p, None, None, None)
    assert 0 < n_fast < 64 << 20            # tables and modal vectors only: the state lives on chip
    pd = fc.problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, fc.CQ_BDF2, fc.CQ_DIRECT)
    n_dir = fc.fp2s_solve(pd, None, None, None)
    assert n_dir >= 4097 * 2 * 255 * 255 * 8  # the full modal history
    assert fc.fp2s_init(p, None, None) > n_fast
    n_h = fc.cq_history_direct(1, 0.3, 1e-3, 1000, 1, 512, None, 1000, None, 1000)
    assert n_h >= 512 * 8
    n_f = fc.cq_history_fast(2, 0.3, 1e-3, 16, 64, 17, 1000, 1, None, None)
    assert n_f >= (80 + 17) * 1000 * 8


def test_mixed_direct_size_query(fc):
    """The mixed-precision direct solve sizes its BF16 hi/lo level matrix (K-major, levels
    of all blocks but the last), the FP32 contraction rows of one block and of one pair of
    blocks, and the Toeplitz banks; it needs no FP64 history. The fast form and the step API reject the BF16x3 precision."""
    M, N = 511, 8192
    nm = M * M
    nmp = (nm + 3) // 4 * 4
    pm = fc.problem(0.2, 0.8, 0.45, 1.0, N, 2, M, fc.CQ_BE, fc.CQ_DIRECT, prec=fc.CQ_BF16X3)
    n_mx = fc.fp2s_solve(pm, None, None, None)
    levels = 2 * (2 * nmp) * (N - 128) * 2
    accs = (128 + 256) * 2 * nmp * 4          # one block's and one pair's contraction rows (FP32)
    assert levels + accs <= n_mx <= levels + accs + (64 << 20)
    pd = fc.problem(0.2, 0.8, 0.45, 1.0, N, 2, M, fc.CQ_BE, fc.CQ_DIRECT)
    assert fc.fp2s_solve(pd, None, None, None) > 1.9 * n_mx    # FP64 keeps (N + 1) x 2 x nm doubles
    one = fc.problem(0.2, 0.8, 0.45, 1.0, 128, 1, 15, fc.CQ_BE, fc.CQ_DIRECT, prec=fc.CQ_BF16X3)
    assert 0 < fc.fp2s_solve(one, None, None, None) < 1 << 20  # a single block: no levels, no accumulator
    pf = fc.problem(0.2, 0.8, 0.45, 1.0, N, 2, M, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2, prec=fc.CQ_BF16X3)
    sz = C.c_size_t(0)
    assert fc._lib.fp2s_solve(C.byref(pf), None, None, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED
    assert fc._lib.fp2s_init(C.byref(pm), None, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED


def test_df64_form_host_checks(fc):
    """The double-float solves (CQ_DF64): the fast form needs no more workspace than the FP64
    fast solve's tables and modal vectors and takes up to 128 points per state; the direct form
    keeps every level as a pair of FP32 numbers; larger node counts and the step API are
    rejected before touching the device."""
    sz = C.c_size_t(0)
    p = fc.problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, fc.CQ_BDF2, fc.CQ_FAST, 16, 64, 17, prec=fc.CQ_DF64)
    n_df = fc.fp2s_solve(p, None, None, None)
    assert 0 < n_df < 64 << 20
    ok = fc.problem(0.2, 0.8, 0.45, 1.0, 8192, 2, 511, fc.CQ_BE, fc.CQ_FAST, 128, 0, 2, prec=fc.CQ_DF64)
    assert 0 < fc.fp2s_solve(ok, None, None, None) < 64 << 20
    big = fc.problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, fc.CQ_BDF2, fc.CQ_FAST, 16, 113, 17, prec=fc.CQ_DF64)
    assert fc._lib.fp2s_solve(C.byref(big), None, None, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED
    dr = fc.problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, fc.CQ_BDF2, fc.CQ_DIRECT, prec=fc.CQ_DF64)
    assert fc.fp2s_solve(dr, None, None, None) >= 4097 * 2 * 255 * 255 * 8   # levels as hi + lo pairs
    assert fc._lib.fp2s_init(C.byref(p), None, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED


def test_dimension_limits(fc):
    sz = C.c_size_t(0)
    p3 = fc.problem(0.3, 0.7, 0.4, 1.0, 64, 3, 31)
    assert fc.fp2s_solve(p3, None, None, None) >= 65 * 2 * 31 ** 3 * 8     # direct history of 31^3 modes
    for dim, M in [(4, 5), (0, 5), (3, 1025), (2, 4097)]:
        p = fc.problem(0.3, 0.7, 0.4, 1.0, 64, dim, M)
        assert fc._lib.fp2s_solve(C.byref(p), None, None, None, C.byref(sz), None) == fc.CQ_EINVAL


def test_vjp_host_checks(fc):
    p = fc.problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, fc.CQ_BE, fc.CQ_DIRECT)
    n_g = fc.fp2s_gradient(p, None, None, None, None)
    assert fc.fp2s_vjp(p, None, None, None, None) == n_g
    sz = C.c_size_t(0)
    da = (C.c_double * 2)()
    pf = fc.problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2)
    assert fc.fp2s_vjp(pf, None, None, None, None) > 0                     # fast form: FP64
    pd = fc.problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2, prec=fc.CQ_DF64)
    assert fc.fp2s_vjp(pd, None, None, None, None) > 0                     # and its double-float sweep
    for prec in (fc.CQ_F32,):
        pq = fc.problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2, prec=prec)
        sz = C.c_size_t(0)
        assert fc._lib.fp2s_vjp(C.byref(pq), None, None, None, da, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED
    assert fc._lib.fp2s_vjp(C.byref(p), None, None, None, da, None, None, None) == fc.CQ_EINVAL
    sz = C.c_size_t(n_g)
    assert fc._lib.fp2s_vjp(C.byref(p), None, None, None, da, 1 << 20, C.byref(sz), None) == fc.CQ_EINVAL


def test_gradient_workspace_cap(fc):
    """FP64 gradient: a nonzero *ws_bytes in the size query is a cap; the library sizes the
    workspace for the largest slice of modes (a multiple of 32) that fits, or returns
    CQ_ENOMEM below one slice."""
    p = fc.problem(0.3, 0.7, 0.4, 1.0, 200, 2, 31, fc.CQ_BDF2, fc.CQ_DIRECT)
    full = fc.fp2s_gradient(p, None, None, None, None)
    J = C.c_double(0.0)
    da = (C.c_double * 2)()
    sz = C.c_size_t(full // 4)
    assert fc._lib.fp2s_gradient(C.byref(p), None, None, C.byref(J), None, da, None, C.byref(sz), None) == fc.CQ_OK
    assert 0 < sz.value <= full // 4
    hist_slice = 2 * 201 * 2 * 32 * 8                 # forward history + adjoint variables of 32 modes
    assert sz.value >= hist_slice
    sz = C.c_size_t(full + 12345)                      # room for everything: the unsliced size
    assert fc._lib.fp2s_gradient(C.byref(p), None, None, C.byref(J), None, da, None, C.byref(sz), None) == fc.CQ_OK
    assert sz.value == full
    sz = C.c_size_t(4096)
    assert fc._lib.fp2s_gradient(C.byref(p), None, None, C.byref(J), None, da, None, C.byref(sz), None) == \
        fc.CQ_ENOMEM


def test_mixed_gradient_size_query(fc):
    """The mixed-precision gradient keeps every level and the weight-derivative history
    (N x 2 x nmp FP32) beyond what the mixed solve needs; vjp shares the layout."""
    N, M = 300, 15
    p = fc.problem(0.3, 0.7, 0.4, 1.0, N, 1, M, fc.CQ_BDF2, fc.CQ_DIRECT, prec=fc.CQ_BF16X3)
    n_g = fc.fp2s_gradient(p, None, None, None, None)
    assert n_g >= fc.fp2s_solve(p, None, None, None) + N * 2 * 16 * 4
    assert fc.fp2s_vjp(p, None, None, None, None) == n_g
    pt = fc.problem(0.3, 0.7, 0.4, 1.0, N, 1, M, fc.CQ_BDF2, fc.CQ_DIRECT, prec=fc.CQ_TF32X3)
    assert fc.fp2s_gradient(pt, None, None, None, None) > n_g          # 4-byte TF32 operands
    sz = C.c_size_t(0)
    da = (C.c_double * 2)()
    p32 = fc.problem(0.3, 0.7, 0.4, 1.0, N, 1, M, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2, prec=fc.CQ_F32)
    assert fc._lib.fp2s_vjp(C.byref(p32), None, None, None, da, None, C.byref(sz), None) == fc.CQ_EUNSUPPORTED


def test_timing_part_needs_a_timed_call(fc):
    ms = C.c_double(0.0)
    assert fc._lib.cq_timing_part(3, C.byref(ms)) == fc.CQ_EINVAL
    assert fc._lib.cq_timing_part(1, None) == fc.CQ_EINVAL


def test_workspace_too_small(fc):
    import torch
    p = fc.problem(0.4, 0.6, 0.3, 1.0, 64, 1, 15)
    small = torch.empty(256, dtype=torch.uint8)
    sz = C.c_size_t(256)
    st = fc._lib.fp2s_solve(C.byref(p), 1 << 20, 1 << 20, small.data_ptr(), C.byref(sz), None)
    assert st == fc.CQ_ENOMEM


def test_mode_range_validation(fc):
    """fp2s_solve_modes: 0 <= mode_lo < mode_hi <= M^dim; the workspace follows the range length."""
    p = fc.problem(0.3, 0.7, 0.3, 1.0, 64, 2, 15, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2)
    sz = C.c_size_t(0)
    lib = fc._lib
    for lo, hi in ((-1, 10), (0, 226), (5, 5), (7, 3)):
        assert lib.fp2s_solve_modes(C.byref(p), lo, hi, None, None, None, C.byref(sz), None) == fc.CQ_EINVAL
    assert lib.fp2s_solve_modes(C.byref(p), 0, 225, None, None, None, C.byref(sz), None) == fc.CQ_OK
    whole = sz.value
    assert lib.fp2s_solve_modes(C.byref(p), 100, 110, None, None, None, C.byref(sz), None) == fc.CQ_OK
    assert 0 < sz.value < whole


def test_probe_library_exports_its_header(fc):
    """libcqprobe.so (the FMA-rate probe of the benchmark) exports what include/cqprobe.h declares."""
    import importlib
    B = importlib.import_module("paper_1901_05128_gb300.build")
    decl = _declared("cqprobe.h")
    assert decl == {"cq_probe_fma_rate"}
    lib = C.CDLL(B.PROBE_LIB)
    assert all(hasattr(lib, n) for n in decl)
    f = lib.cq_probe_fma_rate
    f.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    r = C.c_double(0)
    assert f(2, 1, 32, 1, None, C.byref(r), None) == -1          # invalid arguments, checked on the host
    assert f(0, 1, 48, 1, None, C.byref(r), None) == -1
