"""FP64 CPU oracle for the separation-of-variables compact-stencil solver.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plainly written reference
that the CUDA path is checked against.  Only the test-suite, the package's
smoke check and the benchmark's CPU-baseline leg may import it; the solver
library never calls it and shares no code with it.

What it computes (arXiv 1912.03565, Gonzales, Gryazin, Lee):

  * Section 2 grid: h_a = (L_a^r - L_a^l) / (N_a + 1), interior nodes 1..N_a.
  * Section 3.1, eq. (stencil27): every interior row l of the 27-point system is
        sum_{nu=l-1}^{l+1} a_nu [4 corners] + b_nu [2 x-neighbours]
                         + c_nu [2 y-neighbours] + d_nu [centre]  = F_ijl
    (the printed second x-neighbour "U_{i+1,j-1,nu}" is read as U_{i+1,j,nu}:
    Fig. 1 places b on both sides of the centre).  The coefficients depend on
    the row l as well as on nu, so they are stored as C[l, nu, {a,b,c,d}].
  * Sections 3.2-3.5: coefficients of the 2nd, 4th and 6th-order Helmholtz
    schemes and of the 4th-order convection-diffusion (CD) scheme.
  * Right-hand-side operators: F = h_z^2 f (2nd), h_z^2 f^(IV) (eq. scheme4),
    h_z^2 f^(VI) (eq. scheme6, see R6 below) and eq. (cd_rhs), with every
    derivative of f replaced by central differences on the node grid.
  * Dirichlet data on the six faces enter as F -= (stencil applied to the
    boundary values) (problem statement eq. (bc); the paper gives no formula).
  * Section 3.6: W_l = V^T U_l with the orthonormal 2-D sine basis V; the
    matrices C_m, C, C_p are diagonal in that basis with eigenvalues
        lambda_nu(p,q) = 4 a_nu cos(th_p) cos(th_q) + 2 b_nu cos(th_p)
                         + 2 c_nu cos(th_q) + d_nu,   th_p = p pi / (N_x + 1),
    (the paper's "(i+1) pi / (N_x+1), 0 <= i < N_x" is the mode p = i + 1),
    leaving N_x N_y independent tridiagonal systems in z, solved by LU
    (Thomas, no pivoting), followed by the inverse transform U_l = V W_l.

Readings where the paper is garbled (each one decided by the truncation order
it gives: with the reading taken, the scheme's local truncation error on a
smooth solution falls at the scheme's order when h is halved, which the test
suite checks; with the printed form it does not):
  * R6 (6th-order right-hand side, eq. scheme6).  The term k_l^2 U_ijl inside
    Delta_h(k^2 U) is k^2 f, and the nabla^4 f term is the sum of the pure fourth
    derivatives.  The f-derivatives are approximated explicitly (the paper's
    implicit compact approximation is not specified):
        F6 / h^2 = f + (1/12)(Dx + Dy + Dz) f - (1/240)(Dx^2 + Dy^2 + Dz^2) f
                   + (1/90)(Dx Dy + Dx Dz + Dy Dz) f - (h^2/20) K_l f
                   + (h^3/120) K_{z,l} (f_{l+1} - f_{l-1})
    with D_a the undivided second difference.  The +-2 neighbours outside the
    node grid are ghosts f_{-1} = 2 f_0 - f_1 + h^2 (f_nn)_face with face data
    f_nn defaulting to zero (the paper imposes zero derivative data).
  * CD with variable gamma(z): the printed coefficients freeze gamma at row l
    (variant CD_PAPER, second order for variable gamma); CD_CORRECTED adds
        d_{l+-1} += +-h_z^3 (gamma'' + gamma gamma')/24 + h_z^2 gamma'/6,
        d_l      += -h_z^2 gamma'/3,
    which restores fourth order.  Both reduce to the paper's for constant gamma.
"""
from __future__ import annotations

import numpy as np

HELMHOLTZ = 0
CONVDIFF = 1
CD_PAPER = 0
CD_CORRECTED = 1

# coefficient slots and plane offsets of C[l, nu, m]
A_, B_, C_, D_ = 0, 1, 2, 3
LOW, MID, UPP = 0, 1, 2


def grid_steps(N, L):
    """h_a = L_a / (N_a + 1) for a = x, y, z (Section 2)."""
    return tuple(float(L[a]) / (int(N[a]) + 1) for a in range(3))


# --------------------------------------------------------------------------
# stencil coefficients (Sections 3.2 - 3.5)


def stencil_coefficients(order, equation, h, c0, c1=None, c2=None, cd_variant=CD_CORRECTED):
    """Per-row coefficients C[l-1, nu, m] for interior rows l = 1..Nz.

    nu = 0, 1, 2 is the plane l-1, l, l+1; m = 0..3 is a (corners), b (x-neighbours),
    c (y-neighbours), d (centre).  c0, c1, c2 have length Nz + 2 (nodes l = 0..Nz+1):
    Helmholtz: K = k^2, K_z, K_zz; CD: gamma, gamma', gamma''.
    Paper: Sections 3.2 (2nd order), 3.3 (4th), 3.4 (6th) and 3.5 (convection-diffusion):
    the a, b, c, d of the stencil form, eq. stencil27.
    """
    hx, hy, hz = h
    c0 = np.asarray(c0, dtype=np.float64)
    Nz = c0.shape[0] - 2
    Rzx = hz * hz / (hx * hx)
    Rzy = hz * hz / (hy * hy)
    C = np.zeros((Nz, 3, 4))
    if equation == HELMHOLTZ:
        K, Km, Kp = c0[1:-1], c0[:-2], c0[2:]
        if order == 2:                                   # Section 3.2
            C[:, MID, B_] = Rzx
            C[:, MID, C_] = Rzy
            C[:, LOW, D_] = 1.0
            C[:, UPP, D_] = 1.0
            C[:, MID, D_] = -2.0 * (Rzx + Rzy + 1.0) + hz * hz * K
        elif order == 4:                                 # Section 3.3
            C[:, LOW, B_] = C[:, UPP, B_] = (1.0 + Rzx) / 12.0
            C[:, LOW, C_] = C[:, UPP, C_] = (1.0 + Rzy) / 12.0
            C[:, LOW, D_] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz * hz * Km / 12.0
            C[:, UPP, D_] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz * hz * Kp / 12.0
            C[:, MID, A_] = (Rzx + Rzy) / 12.0
            C[:, MID, B_] = (4.0 * Rzx - Rzy - 1.0 + hz * hz * K / 2.0) / 6.0
            C[:, MID, C_] = (4.0 * Rzy - Rzx - 1.0 + hz * hz * K / 2.0) / 6.0
            C[:, MID, D_] = -4.0 * (1.0 + Rzx + Rzy) / 3.0 + hz * hz * K / 2.0
        elif order == 6:                                 # Section 3.4 (h uniform)
            if c1 is None or c2 is None:
                raise ValueError("6th order needs K_z and K_zz")
            hh = hz
            Kz = np.asarray(c1, dtype=np.float64)[1:-1]
            Kzz = np.asarray(c2, dtype=np.float64)[1:-1]
            h2, h3, h4 = hh ** 2, hh ** 3, hh ** 4
            C[:, LOW, A_] = C[:, UPP, A_] = 1.0 / 30.0
            C[:, LOW, B_] = C[:, LOW, C_] = 0.1 + h2 * Km / 90.0 - h3 * Kz / 120.0
            C[:, UPP, B_] = C[:, UPP, C_] = 0.1 + h2 * Kp / 90.0 + h3 * Kz / 120.0
            C[:, LOW, D_] = 7.0 / 15.0 - h2 * Km / 90.0 - (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Km / 6.0)
            C[:, UPP, D_] = 7.0 / 15.0 - h2 * Kp / 90.0 + (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Kp / 6.0)
            C[:, MID, A_] = 0.1 + h2 * K / 90.0
            C[:, MID, B_] = C[:, MID, C_] = 7.0 / 15.0 - h2 * K / 90.0
            C[:, MID, D_] = -64.0 / 15.0 + 14.0 * h2 * K / 15.0 - h4 * K * K / 20.0 + h4 * Kzz / 20.0
        else:
            raise ValueError("order must be 2, 4 or 6")
    elif equation == CONVDIFF:                           # Section 3.5
        if order != 4:
            raise ValueError("convection-diffusion scheme is 4th order")
        g = c0[1:-1]
        for nu, s in ((LOW, -1.0), (UPP, 1.0)):
            C[:, nu, B_] = (1.0 + Rzx) * (2.0 + s * g * hz) / 24.0
            C[:, nu, C_] = (1.0 + Rzy) * (2.0 + s * g * hz) / 24.0
            C[:, nu, D_] = (2.0 / 3.0 - (Rzx + Rzy) / 6.0
                            + s * (hz * g / 12.0) * (4.0 - Rzx - Rzy + s * hz * g))
        C[:, MID, A_] = (Rzx + Rzy) / 12.0
        C[:, MID, B_] = (4.0 * Rzx - Rzy - 1.0) / 6.0
        C[:, MID, C_] = (4.0 * Rzy - Rzx - 1.0) / 6.0
        C[:, MID, D_] = -4.0 * (1.0 + Rzx + Rzy) / 3.0 - hz * hz * g * g / 6.0
        if cd_variant == CD_CORRECTED:
            g1 = np.zeros(Nz) if c1 is None else np.asarray(c1, dtype=np.float64)[1:-1]
            g2 = np.zeros(Nz) if c2 is None else np.asarray(c2, dtype=np.float64)[1:-1]
            t3 = hz ** 3 * (g2 + g * g1) / 24.0
            t2 = hz * hz * g1 / 6.0
            C[:, UPP, D_] += t3 + t2
            C[:, LOW, D_] += -t3 + t2
            C[:, MID, D_] += -hz * hz * g1 / 3.0
    else:
        raise ValueError("unknown equation")
    return C


# --------------------------------------------------------------------------
# right-hand-side operators


def _undivided_d2(f, axis):
    """D_a f = f_{+1} - 2 f + f_{-1} along one axis, at interior nodes of that axis.

    Paper: h_a^2 delta_a^2 of Section 2."""
    n = f.shape[axis]
    lo = np.take(f, range(0, n - 2), axis=axis)
    mid = np.take(f, range(1, n - 1), axis=axis)
    hi = np.take(f, range(2, n), axis=axis)
    return lo - 2.0 * mid + hi


def _interior(f):
    return f[1:-1, 1:-1, 1:-1]


def _ghost_pad(f, axis, lo_face, hi_face, h):
    """Pad the node grid by one ghost layer on each side of `axis`.

    Ghost f_{-1} = 2 f_0 - f_1 + h^2 (f_nn)_face (and the mirror at the far
    face): second-order Taylor closure, with the face data f_nn = 0 when None.
    Paper: the face closure of the 6th-order right-hand side, eq. scheme6 (the paper leaves
    it to the compact scheme it cites).
    """
    f0 = np.take(f, [0], axis=axis)
    f1 = np.take(f, [1], axis=axis)
    n = f.shape[axis]
    fn = np.take(f, [n - 1], axis=axis)
    fn1 = np.take(f, [n - 2], axis=axis)
    glo = 2.0 * f0 - f1
    ghi = 2.0 * fn - fn1
    if lo_face is not None:
        glo = glo + h * h * np.expand_dims(lo_face, axis)
    if hi_face is not None:
        ghi = ghi + h * h * np.expand_dims(hi_face, axis)
    return np.concatenate([glo, f, ghi], axis=axis)


def rhs_operator(order, equation, h, f_nodes, c0=None, c1=None, fnn=None):
    """Assemble F (interior, shape (Nz, Ny, Nx)) from f on the node grid.

    2nd order:  F = h_z^2 f                                      (Section 3.2)
    4th order:  F = h_z^2 (1 + sum_a h_a^2/12 delta_a^2) f        (eq. scheme4)
    CD:         F = h_z^2 [f + h_x^2/12 f_xx + h_y^2/12 f_yy
                           + h_z^2/12 (gamma_l f_z + f_zz)]      (eq. cd_rhs)
    6th order:  R6 of the module docstring                        (eq. scheme6)
    fnn: six face arrays of the normal second derivative of f (x-lo, x-hi,
    y-lo, y-hi, z-lo, z-hi; None = 0), used by the 6th-order ghosts only.
    """
    hx, hy, hz = h
    f = np.asarray(f_nodes, dtype=np.float64)
    fc = _interior(f)
    Dx = _undivided_d2(f, 2)[1:-1, 1:-1, :]
    Dy = _undivided_d2(f, 1)[1:-1, :, 1:-1]
    Dz = _undivided_d2(f, 0)[:, 1:-1, 1:-1]
    if equation == CONVDIFF:
        g = np.asarray(c0, dtype=np.float64)[1:-1][:, None, None]
        dz1 = f[2:, 1:-1, 1:-1] - f[:-2, 1:-1, 1:-1]           # 2 h_z delta_z f
        return hz * hz * (fc + (Dx + Dy + Dz) / 12.0 + hz * g * dz1 / 24.0)
    if order == 2:
        return hz * hz * fc.copy()
    if order == 4:
        return hz * hz * (fc + (Dx + Dy + Dz) / 12.0)
    if order != 6:
        raise ValueError("order must be 2, 4 or 6")
    hh = hz
    fnn = [None] * 6 if fnn is None else list(fnn)
    K = np.asarray(c0, dtype=np.float64)[1:-1][:, None, None]
    Kz = np.asarray(c1, dtype=np.float64)[1:-1][:, None, None]
    # fourth undivided differences, with one ghost layer beyond each face
    gx = _ghost_pad(f, 2, fnn[0], fnn[1], hh)
    gy = _ghost_pad(f, 1, fnn[2], fnn[3], hh)
    gz = _ghost_pad(f, 0, fnn[4], fnn[5], hh)
    Dx4 = _undivided_d2(_undivided_d2(gx, 2), 2)[1:-1, 1:-1, :]
    Dy4 = _undivided_d2(_undivided_d2(gy, 1), 1)[1:-1, :, 1:-1]
    Dz4 = _undivided_d2(_undivided_d2(gz, 0), 0)[:, 1:-1, 1:-1]
    # mixed terms D_a D_b f use the 12 edge mid-points of the 3x3x3 cube
    DxDy = _undivided_d2(_undivided_d2(f, 2), 1)[1:-1, :, :]
    DxDz = _undivided_d2(_undivided_d2(f, 2), 0)[:, 1:-1, :]
    DyDz = _undivided_d2(_undivided_d2(f, 1), 0)[:, :, 1:-1]
    dz1 = f[2:, 1:-1, 1:-1] - f[:-2, 1:-1, 1:-1]
    F6 = (fc + (Dx + Dy + Dz) / 12.0 - (Dx4 + Dy4 + Dz4) / 240.0
          + (DxDy + DxDz + DyDz) / 90.0 - hh * hh * K * fc / 20.0
          + hh ** 3 * Kz * dz1 / 120.0)
    return hh * hh * F6


# --------------------------------------------------------------------------
# 27-point operator and Dirichlet lifting


def apply_stencil(C, U_nodes):
    """(A U) at interior nodes, per eq. (stencil27), for U given on the node grid."""
    U = np.asarray(U_nodes, dtype=np.float64)
    Nz = U.shape[0] - 2
    out = np.zeros((Nz, U.shape[1] - 2, U.shape[2] - 2))
    for nu, dl in ((LOW, -1), (MID, 0), (UPP, 1)):
        P = U[1 + dl:Nz + 1 + dl]
        corners = P[:, :-2, :-2] + P[:, :-2, 2:] + P[:, 2:, :-2] + P[:, 2:, 2:]
        xn = P[:, 1:-1, :-2] + P[:, 1:-1, 2:]
        yn = P[:, :-2, 1:-1] + P[:, 2:, 1:-1]
        cen = P[:, 1:-1, 1:-1]
        cf = C[:, nu, :]
        out += (cf[:, A_, None, None] * corners + cf[:, B_, None, None] * xn
                + cf[:, C_, None, None] * yn + cf[:, D_, None, None] * cen)
    return out


def boundary_nodes(shape_interior, faces):
    """Node-grid array with the Dirichlet face data on boundary nodes, zero inside.

    Faces (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi; None = 0) are written in that
    order, so on shared edges and corners the z-face value wins, then y.
    Paper: the Dirichlet data of eq. bc.
    """
    Nz, Ny, Nx = shape_interior
    G = np.zeros((Nz + 2, Ny + 2, Nx + 2))
    if faces is None:
        return G
    xl, xh, yl, yh, zl, zh = faces
    if xl is not None:
        G[:, :, 0] = xl
    if xh is not None:
        G[:, :, -1] = xh
    if yl is not None:
        G[:, 0, :] = yl
    if yh is not None:
        G[:, -1, :] = yh
    if zl is not None:
        G[0, :, :] = zl
    if zh is not None:
        G[-1, :, :] = zh
    return G


def lift(C, F, faces):
    """F - (stencil applied to the Dirichlet boundary values): moves known U to the RHS.

    Paper: Section 3.6 (known boundary values carried to the right-hand side)."""
    if faces is None or all(fc is None for fc in faces):
        return F
    return F - apply_stencil(C, boundary_nodes(F.shape, faces))


# --------------------------------------------------------------------------
# discrete sine transform (Section 3.6)


def sine_matrix(N):
    """S[p-1, i-1] = sin(pi p i / (N+1)), p, i = 1..N, with the argument reduced
    exactly as an integer modulo 2(N+1) before the FP64 sine.

    Paper: Section 3.6 (eigenvectors of the second difference)."""
    M = N + 1
    p = np.arange(1, N + 1)
    k = np.outer(p, p) % (2 * M)
    return np.sin(np.pi * k / M)


def dst2_forward(Fi, Sx=None, Sy=None):
    """Fhat[l, q, p] = sum_i sum_j sin(pi p i/(Nx+1)) sin(pi q j/(Ny+1)) F[l, j, i].

    Paper: Section 3.6 (2-D DST along x, then y)."""
    Nz, Ny, Nx = Fi.shape
    Sx = sine_matrix(Nx) if Sx is None else Sx
    Sy = sine_matrix(Ny) if Sy is None else Sy
    X = Fi @ Sx.T                      # along x (contiguous rows)
    return np.matmul(Sy, X)            # along y


def dst2_inverse(W, Sx=None, Sy=None):
    """U[l, j, i] = 4/((Nx+1)(Ny+1)) sum_p sum_q sin(.) sin(.) W[l, q, p] (V is orthonormal).

    Paper: Section 3.6 (inverse 2-D DST)."""
    Nz, Ny, Nx = W.shape
    Sx = sine_matrix(Nx) if Sx is None else Sx
    Sy = sine_matrix(Ny) if Sy is None else Sy
    return (4.0 / ((Nx + 1) * (Ny + 1))) * np.matmul(Sy.T, W @ Sx)


def mode_cosines(N):
    """cos(theta_p), theta_p = p pi / (N + 1), p = 1..N.

    Paper: Section 3.6."""
    return np.cos(np.pi * np.arange(1, N + 1) / (N + 1))


def eigenvalues(C, Nx, Ny):
    """lambda_nu(p, q) for every row: array (3, Nz, Ny, Nx) for nu = l-1, l, l+1.

    Paper: Section 3.6 (lambda_nu(p, q))."""
    cx = mode_cosines(Nx)[None, None, :]
    cy = mode_cosines(Ny)[None, :, None]
    lam = np.empty((3, C.shape[0], Ny, Nx))
    for nu in range(3):
        cf = C[:, nu, :]
        lam[nu] = (4.0 * cf[:, A_, None, None] * cx * cy + 2.0 * cf[:, B_, None, None] * cx
                   + 2.0 * cf[:, C_, None, None] * cy + cf[:, D_, None, None])
    return lam


def thomas(lower, diag, upper, rhs):
    """Textbook tridiagonal LU (no pivoting), vectorised over trailing axes.

    Row l: lower[l] w[l-1] + diag[l] w[l] + upper[l] w[l+1] = rhs[l]; lower[0] and
    upper[-1] are ignored.  Returns (w, min |pivot| / max |diag|).
    Paper: Section 3.6 (one tridiagonal system in z per mode).
    """
    n = rhs.shape[0]
    cp = np.empty_like(rhs)
    dp = np.empty_like(rhs)
    piv = diag[0]
    minpiv = np.abs(piv).copy()
    cp[0] = upper[0] / piv
    dp[0] = rhs[0] / piv
    for l in range(1, n):
        piv = diag[l] - lower[l] * cp[l - 1]
        minpiv = np.minimum(minpiv, np.abs(piv))
        cp[l] = upper[l] / piv
        dp[l] = (rhs[l] - lower[l] * dp[l - 1]) / piv
    w = np.empty_like(rhs)
    w[n - 1] = dp[n - 1]
    for l in range(n - 2, -1, -1):
        w[l] = dp[l] - cp[l] * w[l + 1]
    ratio = float(np.min(minpiv) / np.max(np.abs(diag)))
    return w, ratio


def solve_assembled(C, F):
    """U = A^{-1} F by Section 3.6: 2-D DST, N_x N_y tridiagonals in z, inverse DST."""
    Nz, Ny, Nx = F.shape
    Sx, Sy = sine_matrix(Nx), sine_matrix(Ny)
    Fhat = dst2_forward(F, Sx, Sy)
    lam = eigenvalues(C, Nx, Ny)
    W, ratio = thomas(lam[LOW], lam[MID], lam[UPP], Fhat)
    U = dst2_inverse(W, Sx, Sy)
    return U, {"min_pivot_ratio": ratio}


def assemble_rhs(order, equation, h, f_nodes, C, c0=None, c1=None, faces=None, fnn=None):
    """Lifted right-hand side: R_h f minus the boundary contributions.

    Paper: Sections 2 and 3.6."""
    F = rhs_operator(order, equation, h, f_nodes, c0, c1, fnn)
    return lift(C, F, faces)


def solve(prob, cd_variant=CD_CORRECTED, return_all=False):
    """Full oracle solve of a workloads.Problem-like object (NODAL right-hand side).

    Paper: Section 3.6 (transforms, z-solves, inverse transforms)."""
    N = (prob.Nx, prob.Ny, prob.Nz)
    h = grid_steps(N, (prob.Lx, prob.Ly, prob.Lz))
    C = stencil_coefficients(prob.order, prob.equation, h, prob.c0, prob.c1, prob.c2, cd_variant)
    F = assemble_rhs(prob.order, prob.equation, h, prob.f_nodes, C, prob.c0, prob.c1,
                     prob.faces, prob.fnn)
    U, info = solve_assembled(C, F)
    if return_all:
        info.update(C=C, F=F, h=h)
    return U, info


# --------------------------------------------------------------------------
# separable right-hand sides: exact discrete solution without 3-D transforms


def solve_sine_modes(modes, amps, N, L, order, c0, c1=None, c2=None, sample=None):
    """Discrete solution for f = sum_m A_m sin(p_m pi x/Lx) sin(q_m pi y/Ly) sin(r_m pi z/Lz).

    Each term is separable: on the grid, sin(p pi x_i/Lx) is an eigenvector of
    the undivided second difference D_x (eigenvalue mu_p = 2 cos(p pi/(Nx+1)) - 2),
    also with the 6th-order ghosts, which for a sine mode with zero face data
    are its odd extension.  So R_h f = A sin_p sin_q phi(l) with a 1-D profile
    phi, the 2-D transform of sin_p sin_q is a single mode, and the solution
    is sin_p sin_q times the solution of the one tridiagonal system T_pq w = phi
    (Section 3.6).  Homogeneous Dirichlet data; order 6 uses zero face data.
    Returns U on the interior, or U at the points `sample` = (i, j, l) arrays
    of 1-based interior indices when given.
    """
    Nx, Ny, Nz = N
    h = grid_steps(N, L)
    hx, hy, hz = h
    C = stencil_coefficients(order, HELMHOLTZ, h, c0, c1, c2)
    K = np.asarray(c0, dtype=np.float64)
    Kz = None if c1 is None else np.asarray(c1, dtype=np.float64)
    lz = np.arange(0, Nz + 2)
    ix = np.arange(1, Nx + 1)
    jy = np.arange(1, Ny + 1)
    groups = {}
    for (p, q, r), A in zip(modes, amps):
        s = A * np.sin(np.pi * ((r * lz) % (2 * (Nz + 1))) / (Nz + 1))   # s_l, l = 0..Nz+1
        mux = 2.0 * np.cos(np.pi * p / (Nx + 1)) - 2.0
        muy = 2.0 * np.cos(np.pi * q / (Ny + 1)) - 2.0
        muz = 2.0 * np.cos(np.pi * r / (Nz + 1)) - 2.0
        si = s[1:-1]
        if order == 2:
            phi = hz * hz * si
        elif order == 4:
            phi = hz * hz * si * (1.0 + (mux + muy + muz) / 12.0)
        else:
            hh = hz
            base = (1.0 + (mux + muy + muz) / 12.0 - (mux ** 2 + muy ** 2 + muz ** 2) / 240.0
                    + (mux * muy + mux * muz + muy * muz) / 90.0)
            phi = hh * hh * (base * si - hh * hh * K[1:-1] * si / 20.0
                             + hh ** 3 * Kz[1:-1] * (s[2:] - s[:-2]) / 120.0)
        key = (int(p), int(q))
        groups[key] = groups.get(key, 0.0) + phi
    if sample is None:
        U = np.zeros((Nz, Ny, Nx))
    else:
        si_, sj_, sl_ = (np.asarray(a) for a in sample)
        U = np.zeros(si_.shape)
    for (p, q), phi in groups.items():
        cp, cq = np.cos(np.pi * p / (Nx + 1)), np.cos(np.pi * q / (Ny + 1))
        lam = (4.0 * C[:, :, A_] * cp * cq + 2.0 * C[:, :, B_] * cp + 2.0 * C[:, :, C_] * cq
               + C[:, :, D_])                                           # (Nz, 3)
        w, _ = thomas(lam[:, LOW], lam[:, MID], lam[:, UPP], phi)
        Sx = np.sin(np.pi * ((p * ix) % (2 * (Nx + 1))) / (Nx + 1))
        Sy = np.sin(np.pi * ((q * jy) % (2 * (Ny + 1))) / (Ny + 1))
        if sample is None:
            U += w[:, None, None] * Sy[None, :, None] * Sx[None, None, :]
        else:
            U += w[sl_ - 1] * Sy[sj_ - 1] * Sx[si_ - 1]
    return U


# --------------------------------------------------------------------------
# diagnostics (Section 5.1 error measures)


def solve_sine_modes_extended(modes, amps, N, c0, c1, c2, sample):
    """solve_sine_modes for the 6th-order scheme on a grid of one spacing h =
    1/(max N_a + 1) (N an int for the cube, or (Nx, Ny, Nz); the box is
    L_a = (N_a + 1) h and mode m is sin(p pi x / Lx) sin(q pi y / Ly)
    sin(r pi z / Lz)), with every step in extended precision (numpy longdouble:
    at least 64 significand bits): the Section 3.4 coefficients, the separable
    right-hand side of each mode, the cosines of the mode angles, the Thomas sweep
    of each (p, q) system (Section 3.6) and the sum over modes.  The coefficient
    samples c0..c2 are taken as exact.  Returns U at the `sample` points (i, j, l
    arrays of 1-based interior indices), rounded to FP64.

    Purpose: the exact discrete solution when the z-systems are ill conditioned,
    where any FP64 solve (this oracle's included) carries a rounding error of order
    eps / (smallest singular value ratio); an FP64 result is then measured against
    this one, not against another FP64 computation."""
    LD = np.longdouble
    if np.finfo(LD).nmant < 63:
        raise RuntimeError("extended precision (longdouble with >= 64 significand bits) needed")
    pi = LD("3.14159265358979323846264338327950288419716939937510582097494459")
    Nx, Ny, Nz = (N, N, N) if np.isscalar(N) else (int(v) for v in N)
    h = LD(1) / LD(max(Nx, Ny, Nz) + 1)
    h2, h3, h4 = h * h, h * h * h, h * h * h * h
    K = np.asarray(c0, dtype=np.float64).astype(LD)
    Kz = np.asarray(c1, dtype=np.float64).astype(LD)
    Kzz = np.asarray(c2, dtype=np.float64).astype(LD)
    Kl, Km, Kp, Kzl, Kzzl = K[1:-1], K[:-2], K[2:], Kz[1:-1], Kzz[1:-1]
    one = LD(1)
    # rows nu = l - 1, l, l + 1: (a, b = c, d), Section 3.4
    rows = ((np.full(Nz, one / 30), one / 10 + h2 * Km / 90 - h3 * Kzl / 120,
             LD(7) / 15 - h2 * Km / 90 - (h3 * Kzl / 20) * (one / 3 + h2 * Km / 6)),
            (one / 10 + h2 * Kl / 90, LD(7) / 15 - h2 * Kl / 90,
             -LD(64) / 15 + 14 * h2 * Kl / 15 - h4 * Kl * Kl / 20 + h4 * Kzzl / 20),
            (np.full(Nz, one / 30), one / 10 + h2 * Kp / 90 + h3 * Kzl / 120,
             LD(7) / 15 - h2 * Kp / 90 + (h3 * Kzl / 20) * (one / 3 + h2 * Kp / 6)))

    def sines(m, idx, n):
        return np.sin(pi * np.asarray((m * idx) % (2 * (n + 1)), dtype=LD) / LD(n + 1))

    lz = np.arange(0, Nz + 2)
    groups = {}
    for (p, q, r), A in zip(modes, amps):
        s = LD(float(A)) * sines(int(r), lz, Nz)
        mu = [2 * np.cos(pi * LD(int(v)) / LD(n + 1)) - 2 for v, n in ((p, Nx), (q, Ny), (r, Nz))]
        si = s[1:-1]
        base = (one + (mu[0] + mu[1] + mu[2]) / 12 - (mu[0] ** 2 + mu[1] ** 2 + mu[2] ** 2) / 240
                + (mu[0] * mu[1] + mu[0] * mu[2] + mu[1] * mu[2]) / 90)
        phi = h2 * (base * si - h2 * Kl * si / 20 + h3 * Kzl * (s[2:] - s[:-2]) / 120)
        key = (int(p), int(q))
        groups[key] = groups.get(key, LD(0)) + phi
    si_, sj_, sl_ = (np.asarray(a) for a in sample)
    U = np.zeros(si_.shape, dtype=LD)
    for (p, q), phi in groups.items():
        cp, cq = np.cos(pi * LD(p) / LD(Nx + 1)), np.cos(pi * LD(q) / LD(Ny + 1))
        lo, di, up = (4 * a * cp * cq + 2 * b * cp + 2 * b * cq + d for (a, b, d) in rows)
        cpr = np.empty(Nz, dtype=LD)
        dpr = np.empty(Nz, dtype=LD)
        cpr[0], dpr[0] = up[0] / di[0], phi[0] / di[0]
        for l in range(1, Nz):
            m = di[l] - lo[l] * cpr[l - 1]
            cpr[l] = up[l] / m
            dpr[l] = (phi[l] - lo[l] * dpr[l - 1]) / m
        w = np.empty(Nz, dtype=LD)
        w[Nz - 1] = dpr[Nz - 1]
        for l in range(Nz - 2, -1, -1):
            w[l] = dpr[l] - cpr[l] * w[l + 1]
        U += (w[sl_ - 1] * sines(q, np.arange(1, Ny + 1), Ny)[sj_ - 1]
              * sines(p, np.arange(1, Nx + 1), Nx)[si_ - 1])
    return U.astype(np.float64)


def pad_boundary(U, faces=None):
    """Interior U -> node grid with the Dirichlet face data on the boundary.

    Paper: eq. bc."""
    G = boundary_nodes(U.shape, faces)
    G[1:-1, 1:-1, 1:-1] = U
    return G


def residual_l2(C, U, F_lifted):
    """L2-res = ||A U - F||_2 over interior rows (un-normalised, as in Section 5.1)."""
    return float(np.linalg.norm(apply_stencil(C, pad_boundary(U)) - F_lifted))


def error_measures(U, u_nodes):
    """(max-err, L2-err) = (||u - U||_inf, ||u - U||_2 / ||u||_2) over interior nodes.

    Paper: the max-err and L2-err of Section 5.1's tables."""
    u = _interior(np.asarray(u_nodes))
    e = u - U
    return float(np.max(np.abs(e))), float(np.linalg.norm(e) / np.linalg.norm(u))


def max_rel_diff(U, V):
    """||U - V||_inf / ||V||_inf: the parity measure between two solutions.

    Paper: no paper counterpart (the parity measure of the tests)."""
    return float(np.max(np.abs(U - V)) / max(np.max(np.abs(V)), 1e-300))
