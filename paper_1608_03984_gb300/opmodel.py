"""The paper's first-principles performance model (host logic, no kernels).

* FLOPs per grid-point update, Table 1 (Section "Stencil operators"):
  derivative costs 2k (first), 2k (second), 2k^2 - 4k - 1 (cross), plus the
  per-equation multiplications/additions minus duplicates of Table 1.
* Bytes per point, B_global / N = 4 (l + s) with l loaded and s stored
  fields (Section "Performance Model", streaming stores): acoustic 4 fields,
  VTI 9, TTI 15 (6 of them precomputed trig tables).
* Operational intensity, Eq. eqn_oi: I_alg(k) = F_kernel(k) / (4 (l + s)).
* Roofline, Eq. perf-limits: F_ac = min(I B_peak, F_peak).
* Stability and dispersion set-up of Eq. stability and Table tab:stab.
k is the stencil width, k = order + 1.
"""
from __future__ import annotations

import math

FIELDS = {"acoustic": 4, "vti": 9, "tti": 15}  # l + s of Section "Operational intensity"


def flops_first(k):
    return 2 * k


def flops_second(k):
    return 2 * k


def flops_cross(k):
    return 2 * k * k - 4 * k - 1


def flops_per_point(equation: str, k: int) -> int:
    """F_kernel(k), Table 1."""
    if equation == "acoustic":
        return 3 * flops_second(k) + 3 + 5 - 4
    if equation == "vti":
        return 2 * (3 * flops_second(k) + 5 + 5 - 2)
    if equation == "tti":
        return 2 * (3 * flops_second(k) + 3 * flops_cross(k) + 44 + 17 - 8)
    raise ValueError(equation)


def bytes_per_point(equation: str, word: int = 4, write_allocate: bool = False) -> int:
    """B_global / N: word (l + s), or word (l + 2s) with write-allocate."""
    n = FIELDS[equation]
    stores = 1 if equation == "acoustic" else 2
    return word * (n + (stores if write_allocate else 0))


def oi(equation: str, k: int, word: int = 4) -> float:
    """I_alg(k) of Eq. eqn_oi."""
    return flops_per_point(equation, k) / bytes_per_point(equation, word)


def roofline(i_alg: float, b_peak: float, f_peak: float) -> float:
    """F_ac = min(I B_peak, F_peak), Eq. perf-limits (units of the inputs)."""
    return min(i_alg * b_peak, f_peak)


def min_compute_bound_order(equation: str, i_min: float, kmax: int = 101) -> int | None:
    """Smallest even order whose I_alg reaches i_min (None if none <= kmax-1)."""
    for order in range(2, kmax, 2):
        if oi(equation, order + 1) >= i_min:
            return order
    return None


# -- Eq. stability / Table tab:stab ---------------------------------------

def second_derivative_weights(order: int):
    """Central weights (offsets 0..r) of the second derivative, closed form."""
    r = order // 2
    w = [0.0] * (r + 1)
    for j in range(1, r + 1):
        w[j] = 2.0 * (-1) ** (j + 1) * math.factorial(r) ** 2 / (
            j * j * math.factorial(r - j) * math.factorial(r + j))
    w[0] = -2.0 * sum(w[1:])
    return w


def a2(order: int, dim: int = 3) -> float:
    """Sum of |weights| of the dim-D Laplacian stencil (a2 of Eq. stability)."""
    w = second_derivative_weights(order)
    return dim * (abs(w[0]) + 2.0 * sum(abs(x) for x in w[1:]))


def cfl_limit(order: int, a1: float = 4.0) -> float:
    """sqrt(a1/a2): the bound on vmax dt / h."""
    return math.sqrt(a1 / a2(order))


def fp32_peak_gflops(sms: int = 152, fma_lanes_per_sm: int = 128, clock_ghz: float = 2.07) -> float:
    """FP32 peak from unit counts: every SM issues fma_lanes_per_sm FMAs
    (2 FLOPs each) per clock."""
    return sms * fma_lanes_per_sm * 2 * clock_ghz


def restate(b_gbs: float, f_gflops: float, orders=(2, 4, 6, 8, 12, 16, 18, 24)):
    """The paper's model on a machine of bandwidth b_gbs and peak f_gflops:
    the ridge I_min = F/B, the minimum compute-bound order per equation
    (Section "Stencil operators"), and the Table tab:cost estimate for the
    Table tab:stab set-ups: GFLOPS = min(I B, F) and the runtime."""
    i_min = f_gflops / b_gbs
    out = {"B_GBs": b_gbs, "F_GFLOPs": f_gflops, "I_min": i_min,
           "min_compute_bound_order": {eq: min_compute_bound_order(eq, i_min)
                                       for eq in ("acoustic", "vti", "tti")},
           "table_cost": {}}
    ps = {2: 6, 6: 5, 12: 4, 18: 3, 24: 2}  # Table tab:stab
    for order, p in ps.items():
        k = order + 1
        st = cost_setup(order, p)
        nt = math.ceil(st["nt_exact"])
        gflop = flops_per_point("acoustic", k) * st["N"] * nt / 1e9
        gflops = roofline(oi("acoustic", k), b_gbs, f_gflops)
        out["table_cost"][str(order)] = {"I_alg": oi("acoustic", k), "GFLOPs": gflop,
                                         "GFLOPS": gflops, "runtime_s": gflop / gflops,
                                         "N": st["N"], "nt": nt}
    return out


def cost_setup(order: int, p: float, n2: int = 500, nt2: int = 1000):
    """Table tab:stab row for a physical box of n2 points at 2nd order
    (h = 6/p in units of the 2nd-order spacing, unit velocity)."""
    h = 6.0 / p
    dt = h * cfl_limit(order)
    N = (n2 / h) ** 3
    T = nt2 * cfl_limit(2)
    return {"a2": a2(order), "h": h, "dt": dt, "N": N, "nt_exact": T / dt}
