"""Batched persistent solve (fp2s_batch_plan / fp2s_solve_batched) against single
solves of the same problems and against the oracle (``-m gpu``). Also: autotuned block
width, repeated solves, capture of the batched solve in a CUDA graph, and batches in the
double-float form (CQ_DF64) at the FP64 bar."""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import scheme as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    return pkg.load()


MIXED = [ci.Problem(0.3, 0.7, 0.4, 1.0, 300, 1, 63, ci.BE, ci.FAST, 64, 0, 2),
         ci.Problem(0.4, 0.6, 0.3, 1.0, 257, 2, 19, ci.BDF2, ci.FAST, 9, 23, 7),
         ci.Problem(0.5, 0.5, 0.6, 1.0, 3, 1, 1, ci.BDF2, ci.FAST, 2, 2, 3),
         ci.Problem(0.25, 0.55, 0.7, 0.5, 333, 2, 21, ci.BE, ci.FAST, 40, 0, 2),
         ci.Problem(0.8, 0.2, 0.45, 1.0, 700, 1, 45, ci.BDF2, ci.FAST, 16, 48, 17),
         ci.Problem(0.6, 0.35, 0.0, 2.0, 111, 2, 40, ci.BDF2, ci.FAST, 12, 36, 15),
         ci.Problem(0.2, 0.9, 0.52, 1.0, 64, 1, 300, ci.BE, ci.FAST, 33, 0, 2),
         ci.Problem(0.45, 0.65, 0.35, 1.0, 1, 2, 3, ci.BE, ci.FAST, 4, 0, 2)]


def _cp(fc, p, prec=0):
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      prec=prec)


def _single(fc, p, G0):
    cp = _cp(fc, p)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    fc.fp2s_solve(cp, g0, gN, ws)
    return gN.cpu().numpy()


def _pack(fields):
    return torch.tensor(np.concatenate([f.reshape(-1) for f in fields]), dtype=torch.float64, device="cuda")


def _unpack(t, probs):
    out, o, a = [], 0, t.cpu().numpy()
    for p in probs:
        n = 2 * p.M ** p.dim
        out.append(a[o:o + n].reshape(2, -1))
        o += n
    return out


@pytest.mark.parametrize("tune", [False, True])
def test_batch_matches_single_solves_and_oracle(fc, tune):
    fields = [ci.g0_uniform(p.M, p.dim, 100 + i) for i, p in enumerate(MIXED)]
    cps = [_cp(fc, p) for p in MIXED]
    ws = fc.workspace(fc.fp2s_batch_plan(cps), "cuda")
    plan = fc.fp2s_batch_plan(cps, ws, tune=tune)
    assert plan.n_inst == len(MIXED) and plan.n_units >= len(MIXED)
    if tune:
        # block widths x (all, half of the CTAs per SM that fit) x node-loop widths, each timed
        # three times
        assert plan.flags & 1 and plan.tuned_candidates >= 6
        assert 2 <= plan.warps_per_block <= 16 and plan.ctas_per_sm >= 0 and plan.node_unroll in (2, 4, 8)
    else:
        assert plan.tuned_candidates == 0 and plan.ctas_per_sm == 0 and plan.node_unroll == 4
    assert plan.field_elems == sum(2 * p.M ** p.dim for p in MIXED)
    g0 = _pack(fields)
    gN = torch.empty_like(g0)
    fc.fp2s_solve_batched(plan, g0, gN, ws)
    assert fc.fp2s_batch_status(plan, ws) == fc.CQ_OK
    res = _unpack(gN, MIXED)
    for i, (p, f) in enumerate(zip(MIXED, fields)):
        single = _single(fc, p, f)
        # same per-mode arithmetic; only the sine transforms sum in another order
        assert np.max(np.abs(res[i] - single)) <= 1e-12 * np.max(np.abs(single)) + 1e-300, i
        if i in (0, 1, 4, 7):
            ref = OS.solve(p, f)
            assert np.linalg.norm(res[i] - ref) <= 1e-12 * np.linalg.norm(ref), i
    # a second solve on the same plan gives the same numbers (the work counter is reset)
    gN2 = torch.empty_like(g0)
    fc.fp2s_solve_batched(plan, g0, gN2, ws)
    torch.cuda.synchronize()
    assert torch.equal(gN, gN2)


def test_batch_in_cuda_graph(fc):
    probs = MIXED[:5]
    cps = [_cp(fc, p) for p in probs]
    ws = fc.workspace(fc.fp2s_batch_plan(cps), "cuda")
    plan = fc.fp2s_batch_plan(cps, ws)
    f1 = [ci.g0_uniform(p.M, p.dim, 7 + i) for i, p in enumerate(probs)]
    f2 = [ci.g0_uniform(p.M, p.dim, 70 + i) for i, p in enumerate(probs)]
    g0 = _pack(f1)
    gN = torch.empty_like(g0)
    fc.fp2s_solve_batched(plan, g0, gN, ws)          # eager reference for f1
    torch.cuda.synchronize()
    ref1 = gN.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            fc.fp2s_solve_batched(plan, g0, gN, ws)
    torch.cuda.synchronize()
    gN.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(gN, ref1)
    g0.copy_(_pack(f2))                              # new data, same graph
    graph.replay()
    torch.cuda.synchronize()
    res = _unpack(gN, probs)
    for i, (p, f) in enumerate(zip(probs, f2)):
        single = _single(fc, p, f)
        assert np.max(np.abs(res[i] - single)) <= 1e-12 * np.max(np.abs(single)) + 1e-300, i


def test_batch_rejects_invalid(fc):
    bad = [_cp(fc, MIXED[0]), fc.problem(0.3, 0.7, 0.4, 1.0, 64, 1, 15, fc.CQ_BE, fc.CQ_DIRECT)]
    with pytest.raises(fc.CQError) as e:
        fc.fp2s_batch_plan(bad)
    assert e.value.status == fc.CQ_EUNSUPPORTED


# node classes 16 .. 128 (above 80 the fastest slots in shared memory), both schemes, windows
# up to 17, and instances smaller than one 64-mode unit
DF_BATCH = MIXED + [ci.Problem(0.2, 0.8, 0.45, 1.0, 400, 2, 31, ci.BE, ci.FAST, 128, 0, 2),
                    ci.Problem(0.35, 0.55, 0.6, 1.0, 300, 1, 127, ci.BDF2, ci.FAST, 16, 96, 17),
                    ci.Problem(0.6, 0.25, 0.35, 1.0, 350, 2, 23, ci.BDF2, ci.FAST, 30, 60, 12)]


def test_df64_batch_matches_fp64_batch_and_oracle(fc):
    fields = [ci.g0_uniform(p.M, p.dim, 300 + i) for i, p in enumerate(DF_BATCH)]
    g0 = _pack(fields)
    res = {}
    for prec in (fc.CQ_F64, fc.CQ_DF64):
        cps = [_cp(fc, p, prec) for p in DF_BATCH]
        ws = fc.workspace(fc.fp2s_batch_plan(cps), "cuda")
        plan = fc.fp2s_batch_plan(cps, ws, tune=False)
        if prec == fc.CQ_DF64:
            assert plan.flags & 2 and plan.warps_per_block == 4 and plan.node_unroll == 0
        gN = torch.empty_like(g0)
        fc.fp2s_solve_batched(plan, g0, gN, ws)
        assert fc.fp2s_batch_status(plan, ws) == fc.CQ_OK
        res[prec] = _unpack(gN, DF_BATCH)
    for i, (p, f) in enumerate(zip(DF_BATCH, fields)):
        a, b = res[fc.CQ_DF64][i], res[fc.CQ_F64][i]
        for s_ in range(2):
            assert np.linalg.norm(a[s_] - b[s_]) <= 1e-12 * np.linalg.norm(b[s_]) + 1e-300, (i, s_)
        if i in (0, 4, 8, 9, 10):
            ref = OS.solve(p, f)
            for s_ in range(2):
                assert np.linalg.norm(a[s_] - ref[s_]) <= 1e-12 * np.linalg.norm(ref[s_]), (i, s_)


def test_batch_one_precision_per_plan(fc):
    mixed = [_cp(fc, MIXED[0]), _cp(fc, MIXED[1], fc.CQ_DF64)]
    with pytest.raises(fc.CQError) as e:
        fc.fp2s_batch_plan(mixed)
    assert e.value.status == fc.CQ_EUNSUPPORTED
