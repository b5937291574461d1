"""Pins of the oracle's finite-difference weights and of the paper's
performance model against what the paper prints (Table tab:stab,
Table tab:cost, Table 1 / Eq. eqn_oi) and against closed forms."""
import math

import numpy as np
import pytest

from conftest import read_golden
from paper_1608_03984_gb300 import opmodel

ORDERS = [2, 4, 6, 8, 10, 12, 14, 16, 18, 24]


def closed_form(order):
    """Textbook central weights (offsets 0..r) of the first and second
    derivative at unit spacing."""
    r = order // 2
    w2 = np.zeros(r + 1)
    c1 = np.zeros(r + 1)
    for j in range(1, r + 1):
        ratio = math.factorial(r) ** 2 / (math.factorial(r - j) * math.factorial(r + j))
        w2[j] = 2.0 * (-1) ** (j + 1) * ratio / j ** 2
        c1[j] = (-1) ** (j + 1) * ratio / j
    w2[0] = -2.0 * w2[1:].sum()
    return w2, c1


@pytest.mark.parametrize("order", ORDERS)
def test_fornberg_matches_closed_form(O, order):
    w2, c1 = O.fd_weights(order)
    e2, e1 = closed_form(order)
    np.testing.assert_allclose(w2, e2, rtol=0, atol=1e-13 * max(1.0, abs(e2[0])))
    np.testing.assert_allclose(c1, e1, rtol=0, atol=1e-13)


@pytest.mark.parametrize("order", ORDERS)
def test_weights_exact_on_polynomials(O, order):
    """A stencil of order 2r differentiates x^p exactly for p <= 2r(+1):
    sum_j w_j j^p = p! [p == 2] and sum_j c_j j^p = [p == 1] (all offsets)."""
    r = order // 2
    w2, c1 = O.fd_weights(order)
    j = np.arange(-r, r + 1, dtype=np.float64)
    W2 = np.concatenate([w2[:0:-1], w2])
    C1 = np.concatenate([-c1[:0:-1], c1])
    for p in range(0, order + 1):
        m2 = float(np.sum(W2 * j ** p))
        m1 = float(np.sum(C1 * j ** p))
        assert abs(m2 - (2.0 if p == 2 else 0.0)) < 1e-9 * max(1, r ** p), (p, m2)
        assert abs(m1 - (1.0 if p == 1 else 0.0)) < 1e-9 * max(1, r ** p), (p, m1)


def test_fornberg_general_nodes(O):
    """Arbitrary node sets: weights reproduce derivatives of polynomials at z."""
    x = np.array([-0.7, 0.1, 0.4, 1.3, 2.0])
    z = 0.25
    W = O.fornberg(x, z, 3)
    for p in range(5):
        vals = x ** p
        for m in range(4):
            exact = 0.0 if m > p else math.factorial(p) / math.factorial(p - m) * z ** (p - m)
            assert abs(W[:, m] @ vals - exact) < 1e-10


def test_table_stab(O):
    """Table tab:stab: a2, dt = h sqrt(4/a2), N = (500/h)^3, nt ~ T/dt."""
    for row in read_golden("table_stab.txt"):
        order, a2, p, h, dt, N, nt = (float(v) for v in row)
        order = int(order)
        assert abs(O.laplacian_abs_weight_sum(order) - a2) < 0.005 + 1e-9, order
        got = opmodel.cost_setup(order, p)
        assert abs(got["a2"] - O.laplacian_abs_weight_sum(order)) < 1e-9
        assert abs(got["h"] - h) < 1e-12
        # printed to 4 decimals; the order-6 entry (0.5637) is 1e-4 above
        # h sqrt(4/a2) = 0.56360, the others agree to rounding
        assert abs(got["dt"] - dt) < 1.5e-4, (order, got["dt"], dt)
        assert abs(O.max_stable_dt(order, h, 1.0) - got["dt"]) < 1e-12
        assert abs(got["N"] / N - 1.0) < 5e-3
        # the paper rounds T/dt up except at order 6 (1024.4 -> 1024)
        assert abs(got["nt_exact"] - nt) < 1.0, (order, got["nt_exact"], nt)


def test_table_cost_and_oi():
    """Table tab:cost: I_alg(k) = 3k/8 + 1/4 and GFLOPs = F_kernel N nt."""
    stab = {int(float(r[0])): r for r in read_golden("table_stab.txt")}
    for row in read_golden("table_cost.txt"):
        order, I, gflops, fx, fp, tx, tp = (float(v) for v in row)
        order = int(order)
        k = order + 1
        assert opmodel.oi("acoustic", k) == pytest.approx(I, abs=1e-12)
        assert 3 * k / 8 + 1 / 4 == pytest.approx(I, abs=1e-12)
        N, nt = float(stab[order][5]), float(stab[order][6])
        work = opmodel.flops_per_point("acoustic", k) * N * nt / 1e9
        assert work == pytest.approx(gflops, rel=3e-3), (order, work, gflops)
        # predicted GFLOPS are I_alg x 100 GB/s (Xeon) and x 200 GB/s (Phi)
        assert opmodel.roofline(I, 100.0, 1e9) == pytest.approx(fx)
        assert opmodel.roofline(I, 200.0, 1e9) == pytest.approx(fp)
        assert math.ceil(gflops / fx) == pytest.approx(tx, abs=1)


def test_table1_and_oi_closed_forms():
    rows = {r[0]: (int(r[1]), int(r[2])) for r in read_golden("operational_intensity.txt")}
    for eq, (fields, bpp) in rows.items():
        assert opmodel.FIELDS[eq] == fields
        assert opmodel.bytes_per_point(eq) == bpp
    for k in range(3, 34, 2):
        assert opmodel.flops_per_point("acoustic", k) == 6 * k + 4
        assert opmodel.flops_per_point("vti", k) == 2 * (6 * k + 8)
        assert opmodel.flops_per_point("tti", k) == 12 * k * k - 12 * k + 100
        assert opmodel.oi("acoustic", k) == pytest.approx(3 * k / 8 + 1 / 4)
        assert opmodel.oi("vti", k) == pytest.approx(k / 3 + 4 / 9)
        assert opmodel.oi("tti", k) == pytest.approx(k * k / 5 - k / 5 + 5 / 3)
    # Section "Stencil operators": minimum compute-bound orders on the Xeon
    assert opmodel.min_compute_bound_order("acoustic", 9.3) == 24
    assert opmodel.min_compute_bound_order("vti", 9.3) == 26
    assert opmodel.min_compute_bound_order("tti", 9.3) == 6


def test_cfl_limits():
    """sqrt(4/a2) for orders 2/4/8/12/16: all above 0.4 (CFL 0.4 is stable)."""
    lim = {o: opmodel.cfl_limit(o) for o in (2, 4, 8, 12, 16)}
    assert lim[2] == pytest.approx(1 / math.sqrt(3))
    assert lim[4] == pytest.approx(0.5)
    assert all(v > 0.4 for v in lim.values())
    assert all(lim[a] > lim[b] for a, b in [(2, 4), (4, 8), (8, 12), (12, 16)])


def test_gb300_restatement_structure():
    """The restated model reproduces the paper's Xeon numbers when given the
    Xeon's achievable peaks (I_min 9.3 -> orders 24 / 26 / 6)."""
    r = opmodel.restate(100.0, 930.0)
    assert r["I_min"] == pytest.approx(9.3)
    assert r["min_compute_bound_order"] == {"acoustic": 24, "vti": 26, "tti": 6}
    assert r["table_cost"]["2"]["GFLOPS"] == pytest.approx(137.5)
    assert r["table_cost"]["2"]["runtime_s"] == pytest.approx(20.0, rel=1e-9)
    g = opmodel.restate(6784.2, opmodel.fp32_peak_gflops())
    assert g["min_compute_bound_order"]["tti"] == 8
