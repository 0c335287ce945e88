"""Inner-tolerance controller of the inexact LR-ADI (Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Notation follows the paper: c = 2 + sqrt(2) bounds the constants
check-c_k (Sec. 3.3.1, via Crouzeix-Palencia); xi in (0,1] is the
safeguard; eps is the absolute residual-gap target; kmax the maximum
number of outer steps; u, v the back-looking estimates of eq. (upd_resgap);
N_w = ||w_{k-1}||, N_t = ||t_{k-1}|| (spectral norms).
"""
from __future__ import annotations

import math

C_BOUND = 2.0 + math.sqrt(2.0)          # Sec. 3.3.1: check-c_k <= c = 2 + sqrt(2)

STRATEGIES = ("fixed", "nobl_mid", "bl_mid", "nobl_A", "bl_A", "nobl_B", "bl_B")


def eps_hat_nobl(eps: float, kmax: int, xi: float = 1.0) -> float:
    """eq. (ADI_relax1_prak): hat-eps^(1) = xi * eps / (2 c^2 kmax)."""
    return xi * eps / (2.0 * C_BOUND ** 2 * kmax)


def eps_hat_bl(eps: float, k: int, kmax: int, u_prev: float, v_prev: float,
               xi: float = 1.0) -> float:
    """eq. (ADI_relax2_prak): hat-eps^(2)_k = |xi k eps / (2 c kmax) - u - v| / c.

    The absolute value is taken literally, as printed.
    """
    return abs(xi * k * eps / (2.0 * C_BOUND * kmax) - u_prev - v_prev) / C_BOUND


def tol_B_from_A(eps_hat: float, dA: float, N_w: float, N_t: float) -> float:
    """eq. (tolBfromtolA) with check-c divided into hat-eps: the ||r^B|| on
    the curve dA*N_t + dB*N_w + 2 dA dB = eps_hat."""
    return (eps_hat - dA * N_t) / (2.0 * dA + N_w)


def tol_A_from_B(eps_hat: float, dB: float, N_w: float, N_t: float) -> float:
    """Mirror of eq. (tolBfromtolA): ||r^A|| on the same curve given dB."""
    return (eps_hat - dB * N_w) / (2.0 * dB + N_t)


def select_mid(eps_hat, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B):
    """eq. (simple_tols): delta^A from the middle of the admissible range,
    delta^B from eq. (tolBfromtolA), both clamped as in eq. (bound_tols).

    The midpoint is taken literally as printed: 1/2 (min(dmax, eps/N_t) - dmin).
    """
    dA = max(0.5 * (min(dmax_A, eps_hat / N_t) - dmin_A), dmin_A)
    dB = max(min(tol_B_from_A(eps_hat, dA, N_w, N_t), dmax_B), dmin_B)
    return dA, dB


def select_prefer_A(eps_hat, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B):
    """eq. (one_side): the A-systems are solved to delta^A_min, delta^B from
    eq. (simple_tols)'s second line."""
    dA = dmin_A
    dB = max(min(tol_B_from_A(eps_hat, dA, N_w, N_t), dmax_B), dmin_B)
    return dA, dB


def select_prefer_B(eps_hat, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B):
    """Mirror of eq. (one_side): delta^B = delta^B_min, largest admissible
    delta^A (used by the paper's 'B' settings in Table 2)."""
    dB = dmin_B
    dA = max(min(tol_A_from_B(eps_hat, dB, N_w, N_t), dmax_A), dmin_A)
    return dA, dB


def select_direct(direct, eps_hat, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B):
    """Sec. 3.3 "Combination of direct and iterative linear solves": the
    systems of one side are solved directly (||r|| ~ 0 there), and the
    criteria reduce to ||r^B_k|| <= hat-eps_k / ||w_{k-1}|| (A direct) or
    ||r^A_k|| <= hat-eps_k / ||t_{k-1}|| (B direct), the points of the
    admissible curve of eq. (tolBfromtolA) at delta = 0 on the direct side,
    clamped as in eq. (bound_tols).  The direct side's tolerance is 0."""
    if direct == "A":
        return 0.0, max(min(tol_B_from_A(eps_hat, 0.0, N_w, N_t), dmax_B), dmin_B)
    if direct == "B":
        return max(min(tol_A_from_B(eps_hat, 0.0, N_w, N_t), dmax_A), dmin_A), 0.0
    raise ValueError(f"direct side must be 'A' or 'B', not {direct!r}")


def inner_tolerances(strategy: str, *, k: int, kmax: int, eps: float, xi: float,
                     u_prev: float, v_prev: float, N_w: float, N_t: float,
                     dmin_A: float, dmax_A: float, dmin_B: float, dmax_B: float,
                     fixed_tol: float, direct: str | None = None):
    """(delta^A_k, delta^B_k, hat-eps_k) for outer step k (1-based).  With
    direct = "A" or "B" the systems of that side are solved directly and
    select_direct replaces the strategy's selection rule (its hat-eps rule
    is kept)."""
    if strategy not in STRATEGIES:
        raise ValueError(f"unknown strategy {strategy!r}")
    if strategy == "fixed":
        return (0.0 if direct == "A" else fixed_tol), (0.0 if direct == "B" else fixed_tol), float("nan")
    if strategy.startswith("bl_"):
        eh = eps_hat_bl(eps, k, kmax, u_prev, v_prev, xi)
    else:
        eh = eps_hat_nobl(eps, kmax, xi)
    if direct is not None:
        dA, dB = select_direct(direct, eh, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B)
        return dA, dB, eh
    side = strategy.split("_")[1]
    sel = {"mid": select_mid, "A": select_prefer_A, "B": select_prefer_B}[side]
    dA, dB = sel(eh, N_w, N_t, dmin_A, dmax_A, dmin_B, dmax_B)
    return dA, dB, eh
