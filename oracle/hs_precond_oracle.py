"""FP64 CPU oracle for the preconditioner mode.

TEST INFRASTRUCTURE ONLY (same rule as hs_oracle: only the test-suite, the
smoke check and the benchmark's CPU legs may import it; the solver library
never calls it and shares no code with it).

The paper's introduction (Section 1) names the second use of the direct
solver: a preconditioner for Helmholtz problems whose coefficient depends on
all three coordinates.  This module writes that out:

  * the compact operator for a coefficient K = k^2 that varies in x, y and z,
    on the interior of the box, zero Dirichlet data, scaled by h_z^2 like the
    per-row coefficients of Section 3.3 (so that for K = K(z) it is exactly the
    27-point matrix of eq. (stencil27) with those coefficients):
      4th order:  h_z^2 [ Lap_h U + sum_{a<b} (h_a^2 + h_b^2)/12 d_a^2 d_b^2 U
                          + K U + sum_a (h_a^2/12) d_a^2 (K U) ]
      2nd order:  h_z^2 [ Lap_h U + K U ]
    with d_a^2 the central second difference along a (U = 0 outside);
  * BiCGStab (van der Vorst's algorithm, right preconditioning) for A x = F,
    with the preconditioner M^{-1} = the Section 3.6 direct solve of the
    separable operator for a reference coefficient K_ref(z).
"""
from __future__ import annotations

import numpy as np

from . import hs_oracle as O


def _pad(U):
    P = np.zeros(tuple(n + 2 for n in U.shape))
    P[1:-1, 1:-1, 1:-1] = U
    return P


def _d2(P, axis, h):
    """Central second difference along an axis of a padded array, on the interior.

    Paper: delta_a^2 of Section 2."""
    sl = [slice(1, -1)] * 3
    lo, hi = list(sl), list(sl)
    lo[axis] = slice(0, -2)
    hi[axis] = slice(2, None)
    return (P[tuple(lo)] - 2.0 * P[tuple(sl)] + P[tuple(hi)]) / h ** 2


def _d2_full(P, axis, h):
    """Second difference along `axis` keeping the padded shape in the other axes
    (the padded axis shrinks by 2); used to form mixed differences.

    Paper: delta_a^2 of Section 2."""
    n = P.shape[axis]
    lo = [slice(None)] * 3
    mid = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis] = slice(0, n - 2)
    mid[axis] = slice(1, n - 1)
    hi[axis] = slice(2, n)
    return (P[tuple(lo)] - 2.0 * P[tuple(mid)] + P[tuple(hi)]) / h ** 2


def apply_general(order, K, U, h):
    """(A U) on the interior for a coefficient K = k^2 given on the interior
    nodes [z][y][x]; h = (hx, hy, hz).  Zero Dirichlet data.

    Paper: Section 2's 4th-order scheme (eq. scheme4) for a coefficient K(x, y, z); Section
    1 names the preconditioner use."""
    hx, hy, hz = h
    K = np.asarray(K, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    P = _pad(U)
    ax = {0: (2, hx), 1: (1, hy), 2: (0, hz)}   # our axis -> (array axis, step)
    lap = sum(_d2(P, ax[a][0], ax[a][1]) for a in range(3))
    if order == 2:
        return hz ** 2 * (lap + K * U)
    if order != 4:
        raise ValueError("general-coefficient operator: orders 2 and 4")
    out = lap + K * U
    # mixed fourth differences d_a^2 d_b^2 U with weights (h_a^2 + h_b^2)/12
    for a, b in ((0, 1), (0, 2), (1, 2)):
        (ia, ha), (ib, hb) = ax[a], ax[b]
        t = _d2_full(P, ia, ha)              # padded in the other two axes
        t = _d2_full(t, ib, hb)              # now interior in a and b
        rest = 3 - ia - ib                   # the third array axis
        sl = [slice(None)] * 3
        sl[rest] = slice(1, -1)
        out = out + (ha ** 2 + hb ** 2) / 12.0 * t[tuple(sl)]
    # (h_a^2 / 12) d_a^2 (K U)
    PK = _pad(K * U)
    for a in range(3):
        ia, ha = ax[a]
        out = out + ha ** 2 / 12.0 * _d2(PK, ia, ha)
    return hz ** 2 * out


def bicgstab(apply_A, apply_Minv, F, tol=1e-12, maxit=100, x0=None):
    """Right-preconditioned BiCGStab (van der Vorst 1992) for A x = F.

    Returns (x, history): history lists ||F - A x|| / ||F|| after each iteration
    (recomputed from the recurrence residual r)."""
    F = np.asarray(F, dtype=np.float64)
    x = np.zeros_like(F) if x0 is None else np.array(x0, dtype=np.float64)
    r = F - apply_A(x)
    rhat = r.copy()
    nF = np.linalg.norm(F)
    rho = alpha = omega = 1.0
    v = np.zeros_like(F)
    p = np.zeros_like(F)
    hist = []
    for _ in range(maxit):
        rho_new = float(np.vdot(rhat, r))
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = apply_Minv(p)
        v = apply_A(phat)
        alpha = rho_new / float(np.vdot(rhat, v))
        s = r - alpha * v
        shat = apply_Minv(s)
        t = apply_A(shat)
        omega = float(np.vdot(t, s)) / float(np.vdot(t, t))
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho = rho_new
        hist.append(float(np.linalg.norm(r) / nF))
        if hist[-1] <= tol:
            break
    return x, hist


def precond_solve(order, K, F, h, Kref, tol=1e-12, maxit=100):
    """Solve A(K) x = F (F assembled, interior) by BiCGStab preconditioned with
    the separable direct solve for Kref(z) (length Nz + 2, nodes l = 0..Nz+1).

    Paper: Section 1 (the separable solve as preconditioner); BiCGStab of van der Vorst
    (1992)."""
    C = O.stencil_coefficients(order, O.HELMHOLTZ, h, np.asarray(Kref, dtype=np.float64))
    return bicgstab(lambda u: apply_general(order, K, u, h),
                    lambda r: O.solve_assembled(C, r)[0], F, tol, maxit)


def reference_from_field(K):
    """K_ref(z_l) = mean of K over each interior plane, extended to the two
    boundary planes by the nearest interior plane (length Nz + 2).

    Paper: no paper counterpart (a choice of K_ref)."""
    m = np.asarray(K, dtype=np.float64).mean(axis=(1, 2))
    return np.concatenate([[m[0]], m, [m[-1]]])
