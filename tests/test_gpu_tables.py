"""The convergence studies of Sec. 5 on the GPU solver (``-m gpu``), against the values
printed in Tables 1-5 (``golden/tables_1_5.txt``).

What is checked, and why these bars:
- Rates of the plain and fast BE schemes (Tables 1-2): within 0.002 of every printed
  rate. With the reference step 1/6400 (the text says 1/3200, see the module
  ``paper_1901_05128_gb300.tables``) they agree to 1e-3 or better.
- Errors of the nonsmooth data (b), Table 2: within 1.5 % (the computed errors sit
  ~0.9 % below the printed ones at every step, a constant factor of the unstated
  spatial treatment). Data (a) (G2 = sin x, nonzero at x = 1) differs in magnitude
  and only its rates are compared.
- Plain SBD (Tables 3-4): the first two rates of every row within 0.015; all four
  rates of the rows the FP64 oracle pins (``golden/table3_4_sbd_rates.txt``: the
  (0.3,0.4) rows of Table 3 and the E1 rows of Table 4); Table 4 errors at the three coarsest steps within 1.5 % (rows other
  than the (0.2,0.4) E2 row, which the oracle puts 1.4x higher). The finer steps
  depend on the reference solution's own error. The printed fast-SBD rows carry the
  paper's own (unstated) quadrature split and are compared through the plain rows.
- Fast against plain (the claim of Tables 1-4): |E_fast / E_plain - 1| <= 2e-3.
- Table 5 (T = 10, 2 x 10^4 steps): the printed errors are not reproduced. The plain
  SBD scheme against its own half-step solution gives ~2e-12, about 100x below the
  printed 1e-10..1e-8 (below 1e-8 of |G_ref| here); the fast SBD form needs 240
  family-2 points at this length (see the module docstring) and then stays within
  1e-4 of |G_ref| (4e-5 measured).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tables_1_5.txt")


def _golden():
    err, rate = {}, {}
    with open(GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            key = (w[1], float(w[3]), float(w[4]), w[5], int(w[6][1]) - 1)
            (err if w[0] == "err" else rate)[key] = np.array([float(v) for v in w[7:]])
    return err, rate


@pytest.fixture(scope="module")
def results():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    fc = pkg.load()
    from paper_1901_05128_gb300 import tables as T
    out = {}
    for name in ("table1", "table2", "table3", "table4"):
        out[name] = T.run(name, fc, torch)
    ex5 = dict(T.EXPERIMENTS["table5"])
    ex5["alphas"] = [(0.3, 0.8)]
    T.EXPERIMENTS["table5_one"] = ex5
    try:
        out["table5"] = T.run("table5_one", fc, torch)
    finally:
        del T.EXPERIMENTS["table5_one"]
    return out


def _methods(table):
    return ("BE", "FBE") if table in ("table1", "table2") else ("SBD", "FSBD")


def _rows(results, table):
    for row in results[table]["rows"]:
        for form, meth in zip(("direct", "fast"), _methods(table)):
            yield row["alpha"], form, meth, row[form]


@pytest.mark.parametrize("table", ["table1", "table2"])
def test_be_rates(results, table):
    _, rate = _golden()
    for (a1, a2), _, meth, r in _rows(results, table):
        for c in range(2):
            printed = rate[(table, a1, a2, meth, c)]
            assert np.all(np.abs(r["rates"][:, c] - printed) <= 2e-3), (table, a1, a2, meth, c, r["rates"][:, c])


def test_be_nonsmooth_errors(results):
    err, _ = _golden()
    for (a1, a2), _, meth, r in _rows(results, "table2"):
        for c in range(2):
            ratio = r["E"][:, c] / err[("table2", a1, a2, meth, c)]
            assert np.all(np.abs(ratio - 1.0) <= 0.015), (a1, a2, meth, c, ratio)


ORACLE_ROWS = {("table3", 0.3, 0.4, 0), ("table3", 0.3, 0.4, 1), ("table4", 0.2, 0.4, 0),
               ("table4", 0.6, 0.8, 0)}


@pytest.mark.parametrize("table", ["table3", "table4"])
def test_sbd_rates(results, table):
    """Plain SBD rows only: the printed fast-SBD rates carry the paper's own quadrature
    error (its fast rows differ from its plain rows by up to 0.09); ours agree with the
    plain scheme (test_fast_matches_plain)."""
    _, rate = _golden()
    for (a1, a2), form, meth, r in _rows(results, table):
        if form != "direct":
            continue
        for c in range(2):
            printed = rate[(table, a1, a2, meth, c)]
            got = r["rates"][:, c]
            assert np.all(np.abs(got[:2] - printed[:2]) <= 0.015), (table, a1, a2, meth, c, got)
            if (table, a1, a2, c) in ORACLE_ROWS:
                assert np.all(np.abs(got - printed) <= 0.015), (table, a1, a2, meth, c, got)


def test_sbd_nonsmooth_errors(results):
    err, _ = _golden()
    for (a1, a2), form, meth, r in _rows(results, "table4"):
        for c in range(2):
            if (a1, a2, c) == (0.2, 0.4, 1) or form != "direct":
                continue
            ratio = r["E"][:3, c] / err[("table4", a1, a2, meth, c)][:3]
            assert np.all(np.abs(ratio - 1.0) <= 0.015), (a1, a2, meth, c, ratio)


@pytest.mark.parametrize("table", ["table1", "table2", "table3", "table4"])
def test_fast_matches_plain(results, table):
    for row in results[table]["rows"]:
        ratio = row["fast"]["E"] / row["direct"]["E"]
        assert np.all(np.abs(ratio - 1.0) <= 2e-3), (table, row["alpha"], ratio)


def test_table5_long_run(results):
    row = results["table5"]["rows"][0]
    Ed, Ef = row["direct"]["E"][0], row["fast"]["E"][0]
    ref = row["ref_norm"]
    assert np.all(Ed <= 1e-8 * ref)
    assert np.all(Ef <= 1e-4 * ref)
    print("table 5 (0.3,0.8): SBD E %s, FSBD E %s, |G_ref| %s" % (Ed, Ef, ref))
