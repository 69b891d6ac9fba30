"""FP64 CPU oracle for complex k(z), Robin z-faces and Neumann side faces.

TEST INFRASTRUCTURE ONLY (same rule as hs_oracle: only the test-suite, the
smoke check and the benchmark's CPU legs may import it; the solver library
never calls it and shares no code with it).

Section 1 states the paper's general problem: k is complex and depends on z
only, u = 0 on the four side faces, and alpha u_z + beta u = g(x, y) on the two
z-faces with complex alpha, beta.  The schemes and the direct solver of
Sections 3 and 3.6 are worked out for Dirichlet data; the compact closure of a
Robin face belongs to a cited work that the paper does not reproduce.  This
module takes, for orders 2, 4 and 6:

  * interior rows l = 1..Nz: the compact rows of Sections 3.2 - 3.4 with
    complex K = k^2.  At orders 2 and 4 every coefficient is affine in K, so
    the complex table is the real table of Re K plus i times the K-part of the
    real table of Im K; the 6th-order rows (Section 3.4, uniform h) are
    polynomials in K and K_z and are evaluated in complex arithmetic as
    printed, as is the K-dependent part of the 6th-order right-hand side
    (Dirichlet side faces only);
  * a Dirichlet z-face: its plane holds g, moved into the next row's right-hand
    side through the stencil (as for the real problem);
  * a Robin z-face: its plane is unknown and its row is the second-order
    7-point scheme h_z^2 (dxx + dyy + dzz + K) u = h_z^2 f, the plane outside
    eliminated with the central difference of the face condition:
      lo face (l = 0):      alpha (u_1 - u_-1) / (2 h_z) + beta u_0 = g
      hi face (l = Nz + 1): alpha (u_Nz+2 - u_Nz) / (2 h_z) + beta u_Nz+1 = g
    (a second-order closure: the high-order one is out of this module's reach);
  * right-hand side: the real operator R_h of the order applied to Re f and
    Im f on interior rows, h_z^2 f plus the ghost's data term on Robin rows.

The unknowns are the planes l0..l1 (l0 = 0 for a Robin lo face, else 1; l1 =
Nz + 1 for a Robin hi face, else Nz).  Side faces stay Dirichlet, so Section
3.6's sine transforms in x and y still split the system into N_x N_y complex
tridiagonal systems in z; these are solved by the textbook recurrence.

Neumann side faces (the extension Section 1 names): a side axis may instead
carry u_n = g on both of its faces (g = 0 or per-face data).  Its boundary
nodes become unknowns, the operator sees the ghost of the central difference of
the face condition (the even reflection u_-1 = u_1 plus 2 h g), f is reflected
evenly, and the sine transform of that axis is replaced by the cosine
transform DCT-I over the nodes 0..N+1, whose modes cos(p pi i / (N+1)),
p = 0..N+1, diagonalise the reflected second difference with the same
eigenvalue formula (Section 3.6) -- the per-row coefficients are unchanged.
An axis with one face of each kind (SIDE_DN, SIDE_ND) takes the quarter-wave
transforms, modes of angle (2p - 1) pi / (2 (N + 1)), p = 1..N+1.

Arrays: f on the node grid [Nz+2][Ny+2][Nx+2] (complex; side-face nodes of a
Dirichlet axis are read by the 4th-order operator as given); the unknown grid
of a plane is [ny][nx] with nx = Nx + 2 for a Neumann x-axis (nodes 0..Nx+1),
Nx + 1 for an axis with one Neumann face (nodes 1..Nx+1 or 0..Nx), else Nx
(nodes 1..Nx), and likewise ny; face data g_lo, g_hi on that grid of
the z-face (complex; None = 0); the solution on all planes [Nz+2][ny][nx]
(Dirichlet planes hold g).
"""
from __future__ import annotations

import numpy as np

from . import hs_oracle as O

DIRICHLET = 0
ROBIN = 1


class ZFaces:
    """Kind (DIRICHLET / ROBIN) and Robin parameters of the two z-faces."""

    def __init__(self, lo=DIRICHLET, alpha_lo=1.0, beta_lo=0.0, hi=DIRICHLET, alpha_hi=1.0,
                 beta_hi=0.0):
        self.lo, self.hi = lo, hi
        self.alpha = (complex(alpha_lo), complex(alpha_hi))
        self.beta = (complex(beta_lo), complex(beta_hi))
        for kind, a in ((lo, self.alpha[0]), (hi, self.alpha[1])):
            if kind == ROBIN and a == 0:
                raise ValueError("a Robin face needs alpha != 0 (alpha = 0 is a Dirichlet face)")

    def unknown_planes(self, Nz):
        return (0 if self.lo == ROBIN else 1), (Nz + 1 if self.hi == ROBIN else Nz)


SIDE_DIRICHLET = 0
SIDE_NEUMANN = 1
SIDE_DN = 2   # Dirichlet on the low face, u_n = g on the high face
SIDE_ND = 3   # u_n = g on the low face, Dirichlet on the high face


def _lo_neu(kind):
    return kind in (SIDE_NEUMANN, SIDE_ND)


def _hi_neu(kind):
    return kind in (SIDE_NEUMANN, SIDE_DN)


def _nodes(N, kind):
    """First and last node index of the unknowns along a side axis of N interior nodes:
    the boundary node of a Neumann face is an unknown, that of a Dirichlet face is not.

    Paper: Section 1 (Neumann side faces, the extension it names)."""
    return (0 if _lo_neu(kind) else 1), (N + 1 if _hi_neu(kind) else N)


def _n_unknown(N, kind):
    first, last = _nodes(N, kind)
    return last - first + 1


def cosine_matrix(N):
    """DCT-I over the nodes 0..N+1 (M = N + 1): C[p, i] = w_i cos(pi p i / M), p, i = 0..M,
    w_0 = w_M = 1/2, else 1; the argument is reduced as an integer modulo 2M first.

    Paper: Section 3.6's transform for Section 1's Neumann side faces."""
    M = N + 1
    k = np.outer(np.arange(M + 1), np.arange(M + 1)) % (2 * M)
    C = np.cos(np.pi * k / M)
    C[:, 0] *= 0.5
    C[:, M] *= 0.5
    return C


def side_transform(N, kind):
    """(forward, inverse) matrices of one side axis, inverse(forward(x)) = x: DST-I of the
    interior nodes (Dirichlet faces), DCT-I of all nodes (Neumann faces), or for one face
    of each kind the quarter-wave transforms with theta_p = (2p - 1) pi / (2M), p = 1..M
    (M = N + 1): sines over nodes 1..M (Neumann high face), cosines over nodes 0..N
    (Neumann low face), weight 1/2 at the Neumann node.

    Paper: Section 3.6 with Section 1's side faces."""
    M = N + 1
    if kind == SIDE_NEUMANN:
        # the DCT-I is its own inverse up to 2/M: x_i = (2/M) sum_p w_p X_p cos(pi p i/M)
        C = cosine_matrix(N)
        return C, (2.0 / M) * C
    if kind in (SIDE_DN, SIDE_ND):
        p = np.arange(1, M + 1)
        i = np.arange(1, M + 1) if kind == SIDE_DN else np.arange(0, M)
        k = np.outer(2 * p - 1, i) % (4 * M)       # theta_p i as an integer multiple of pi/2M
        Q = np.sin(np.pi * k / (2 * M)) if kind == SIDE_DN else np.cos(np.pi * k / (2 * M))
        fwd = Q.copy()
        fwd[:, -1 if kind == SIDE_DN else 0] *= 0.5
        return fwd, (2.0 / M) * Q.T
    S = O.sine_matrix(N)
    return S, (2.0 / M) * S.T


def side_cosines(N, kind):
    """cos(theta_p) of the modes of one side axis.

    Paper: Section 3.6 with Section 1's side faces."""
    if kind == SIDE_NEUMANN:
        return np.cos(np.pi * np.arange(0, N + 2) / (N + 1))
    if kind in (SIDE_DN, SIDE_ND):
        M = N + 1
        return np.cos(np.pi * (2 * np.arange(1, M + 1) - 1) / (2 * M))
    return O.mode_cosines(N)


def _span(N, kind):
    """Node indices covered by a padded unknown grid along a side axis (one node beyond
    the unknowns on each side), nodes beyond a Neumann face folded back by the even
    reflection (-1 -> 1, N + 2 -> N).

    Paper: Section 1 (even reflection beyond a Neumann face)."""
    first, last = _nodes(N, kind)
    idx = np.arange(first - 1, last + 2)
    if _lo_neu(kind):
        idx[0] = 1
    if _hi_neu(kind):
        idx[-1] = N
    return idx


def _axis_n(n_unknown, kind):
    return n_unknown - int(_lo_neu(kind)) - int(_hi_neu(kind))


def reflect_pad(U, sides, side_data=None, h=None):
    """Pad a field on the unknown grid [..., ny, nx] by one node per side: beyond a
    Dirichlet face its boundary node (u = 0), beyond a Neumann face the ghost of the
    central difference of u_n = g, i.e. the even reflection plus 2 h g (outward normal).
    side_data = (x-lo, x-hi, y-lo, y-hi) arrays of u_n on the face node grids
    ([planes][Ny+2] for x-faces, [planes][Nx+2] for y-faces; None = 0, read on Neumann
    faces only), reflected evenly beyond their own edges; x-ghosts are set first, so a
    corner ghost carries the data of both faces.

    Paper: Section 1 (u_n = g faces, central-difference ghost)."""
    U = np.asarray(U)
    pad = [(0, 0)] * (U.ndim - 2) + [(1, 1), (1, 1)]
    P = np.pad(U, pad)
    sd = [None] * 4 if side_data is None else list(side_data)
    Ny = _axis_n(P.shape[-2] - 2, sides[1])
    Nx = _axis_n(P.shape[-1] - 2, sides[0])
    rows = _span(Ny, sides[1])
    for k, col, src, neu in ((0, 0, 2, _lo_neu(sides[0])), (1, -1, -3, _hi_neu(sides[0]))):
        if neu:
            P[..., :, col] = P[..., :, src]
            if sd[k] is not None:
                P[..., :, col] = P[..., :, col] + 2.0 * h[0] * np.asarray(sd[k])[..., rows]
    cols = _span(Nx, sides[0])
    for k, row, src, neu in ((2, 0, 2, _lo_neu(sides[1])), (3, -1, -3, _hi_neu(sides[1]))):
        if neu:
            P[..., row, :] = P[..., src, :]
            if sd[k] is not None:
                P[..., row, :] = P[..., row, :] + 2.0 * h[1] * np.asarray(sd[k])[..., cols]
    return P


def complex_coefficients6(h, K, Kz, Kzz):
    """6th-order rows (Section 3.4, uniform h) for complex K, K_z, K_zz (length Nz + 2):
    the printed coefficients are polynomials in K (K^2 in d_l, K_z K in d_{l+-1}), so they
    are evaluated in complex arithmetic as written."""
    hh = h[2]
    K = np.asarray(K, dtype=np.complex128)
    Kz = np.asarray(Kz, dtype=np.complex128)[1:-1]
    Kzz = np.asarray(Kzz, dtype=np.complex128)[1:-1]
    Km, Kc, Kp = K[:-2], K[1:-1], K[2:]
    h2, h3, h4 = hh ** 2, hh ** 3, hh ** 4
    C = np.zeros((K.shape[0] - 2, 3, 4), dtype=np.complex128)
    C[:, O.LOW, O.A_] = C[:, O.UPP, O.A_] = 1.0 / 30.0
    C[:, O.LOW, O.B_] = C[:, O.LOW, O.C_] = 0.1 + h2 * Km / 90.0 - h3 * Kz / 120.0
    C[:, O.UPP, O.B_] = C[:, O.UPP, O.C_] = 0.1 + h2 * Kp / 90.0 + h3 * Kz / 120.0
    C[:, O.LOW, O.D_] = 7.0 / 15.0 - h2 * Km / 90.0 - (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Km / 6.0)
    C[:, O.UPP, O.D_] = 7.0 / 15.0 - h2 * Kp / 90.0 + (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Kp / 6.0)
    C[:, O.MID, O.A_] = 0.1 + h2 * Kc / 90.0
    C[:, O.MID, O.B_] = C[:, O.MID, O.C_] = 7.0 / 15.0 - h2 * Kc / 90.0
    C[:, O.MID, O.D_] = -64.0 / 15.0 + 14.0 * h2 * Kc / 15.0 - h4 * Kc * Kc / 20.0 + h4 * Kzz / 20.0
    return C


def complex_coefficients(order, h, K, Kz=None, Kzz=None):
    """C[l-1, nu, m] (complex) for interior rows l = 1..Nz; K complex, length Nz + 2
    (order 6 also needs K_z and K_zz).

    Paper: Sections 3.2-3.4 with complex K."""
    if order == 6:
        return complex_coefficients6(h, K, Kz, Kzz)
    if order not in (2, 4):
        raise ValueError("complex coefficients: orders 2, 4 and 6")
    K = np.asarray(K, dtype=np.complex128)
    zero = np.zeros(K.shape)
    base = O.stencil_coefficients(order, O.HELMHOLTZ, h, zero)
    re = O.stencil_coefficients(order, O.HELMHOLTZ, h, K.real)
    im = O.stencil_coefficients(order, O.HELMHOLTZ, h, K.imag)
    return re + 1j * (im - base)


def robin_row(h, K_l, alpha, beta, side):
    """3 x 4 block (nu = l-1, l, l+1; a, b, c, d) of a Robin face's row (side -1: lo, +1: hi).

    Paper: Section 1's Robin face (eq. bc); a second-order closure, the paper gives none."""
    hx, hy, hz = h
    Rzx, Rzy = hz * hz / (hx * hx), hz * hz / (hy * hy)
    R = np.zeros((3, 4), dtype=np.complex128)
    R[O.MID, O.B_] = Rzx
    R[O.MID, O.C_] = Rzy
    # d_zz u with the outside plane replaced by the face condition
    R[O.MID, O.D_] = -2.0 * (Rzx + Rzy + 1.0) + hz * hz * K_l - side * 2.0 * hz * beta / alpha
    R[O.UPP if side < 0 else O.LOW, O.D_] = 2.0
    return R


def row_table(order, h, K, zf, Kz=None, Kzz=None):
    """Coefficient blocks of the unknown rows l0..l1: array (Nu, 3, 4) complex.

    Paper: Sections 3.2-3.4 and Section 1."""
    K = np.asarray(K, dtype=np.complex128)
    Nz = K.shape[0] - 2
    Ci = complex_coefficients(order, h, K, Kz, Kzz)
    rows = []
    if zf.lo == ROBIN:
        rows.append(robin_row(h, K[0], zf.alpha[0], zf.beta[0], -1))
    rows.extend(Ci)
    if zf.hi == ROBIN:
        rows.append(robin_row(h, K[Nz + 1], zf.alpha[1], zf.beta[1], +1))
    return np.array(rows)


def _face(g, Ny, Nx):
    return np.zeros((Ny, Nx), dtype=np.complex128) if g is None else np.asarray(g, np.complex128)


def _plane_part(block, P):
    """One plane's part of a row: block (4,) applied to a padded plane P [Ny+2][Nx+2].

    Paper: eq. stencil27 (one plane's part)."""
    corners = P[:-2, :-2] + P[:-2, 2:] + P[2:, :-2] + P[2:, 2:]
    xn = P[1:-1, :-2] + P[1:-1, 2:]
    yn = P[:-2, 1:-1] + P[2:, 1:-1]
    return (block[O.A_] * corners + block[O.B_] * xn + block[O.C_] * yn
            + block[O.D_] * P[1:-1, 1:-1])


def _pad2(g):
    Ny, Nx = g.shape
    P = np.zeros((Ny + 2, Nx + 2), dtype=np.complex128)
    P[1:-1, 1:-1] = g
    return P


def _f_on_unknowns(f, sides):
    """f on [Nz+2][ny+2][nx+2]: the unknown grid of every plane plus one node per side
    (beyond a Dirichlet face its boundary node as given, beyond a Neumann face the even
    reflection).

    Paper: Section 1 (even reflection beyond a Neumann face)."""
    Ny, Nx = f.shape[1] - 2, f.shape[2] - 2
    xs = _span(Nx, sides[0])
    ys = _span(Ny, sides[1])
    # every padded node is either a node of the grid or folded back onto one
    return f[:, ys][:, :, xs]


def _interior_rhs(order, h, fu, K, Kz=None, fnn=None):
    """R_h f on the interior planes for complex f (padded unknown grid fu).  Orders 2 and 4:
    the real operator on Re f and Im f.  Order 6 (R6, Dirichlet sides): the K-free part
    likewise (with the face data f_nn split the same way) plus the complex terms
    h^2 (-h^2 K f / 20 + h^3 K_z (f_{l+1} - f_{l-1}) / 120).

    Paper: eqs. scheme4 and scheme6."""
    if order != 6:
        return (O.rhs_operator(order, O.HELMHOLTZ, h, fu.real)
                + 1j * O.rhs_operator(order, O.HELMHOLTZ, h, fu.imag))
    hh = h[2]
    zero = np.zeros(fu.shape[0])
    fnn = [None] * 6 if fnn is None else list(fnn)
    part = lambda g: [None if a is None else g(np.asarray(a, dtype=np.complex128)) for a in fnn]
    F = (O.rhs_operator(6, O.HELMHOLTZ, h, fu.real, zero, zero, part(np.real))
         + 1j * O.rhs_operator(6, O.HELMHOLTZ, h, fu.imag, zero, zero, part(np.imag)))
    Kc = np.asarray(K, dtype=np.complex128)[1:-1][:, None, None]
    Kzc = np.asarray(Kz, dtype=np.complex128)[1:-1][:, None, None]
    fc = fu[1:-1, 1:-1, 1:-1]
    dz1 = fu[2:, 1:-1, 1:-1] - fu[:-2, 1:-1, 1:-1]
    return F + hh * hh * (-hh * hh * Kc * fc / 20.0 + hh ** 3 * Kzc * dz1 / 120.0)


def rhs(order, h, K, zf, f_nodes, g_lo=None, g_hi=None, sides=(SIDE_DIRICHLET, SIDE_DIRICHLET),
        side_data=None, Kz=None, Kzz=None, fnn=None):
    """Right-hand side of the unknown rows: array (Nu, ny, nx) complex.

    Paper: Sections 2 and 3.6."""
    if order == 6 and sides != (SIDE_DIRICHLET, SIDE_DIRICHLET):
        raise ValueError("6th-order complex rows: Dirichlet side faces")
    hz = h[2]
    f = np.asarray(f_nodes, dtype=np.complex128)
    Nz = f.shape[0] - 2
    fu = _f_on_unknowns(f, sides)
    ny, nx = fu.shape[1] - 2, fu.shape[2] - 2
    glo, ghi = _face(g_lo, ny, nx), _face(g_hi, ny, nx)
    # R_h of the order on the padded unknown grid (interior planes 1..Nz)
    Fi = _interior_rhs(order, h, fu, K, Kz, fnn)
    Ci = complex_coefficients(order, h, K, Kz, Kzz)
    # Dirichlet faces: their known plane leaves rows 1 / Nz through the stencil
    if zf.lo == DIRICHLET:
        Fi[0] -= _plane_part(Ci[0, O.LOW], reflect_pad(glo, sides))
    if zf.hi == DIRICHLET:
        Fi[-1] -= _plane_part(Ci[-1, O.UPP], reflect_pad(ghi, sides))
    rows = []
    if zf.lo == ROBIN:
        # u_-1 = u_1 - 2 h (g - beta u_0) / alpha: the data part enters the row with weight 1
        rows.append(hz * hz * fu[0, 1:-1, 1:-1] + 2.0 * hz * glo / zf.alpha[0])
    rows.extend(Fi)
    if zf.hi == ROBIN:
        rows.append(hz * hz * fu[Nz + 1, 1:-1, 1:-1] - 2.0 * hz * ghi / zf.alpha[1])
    F = np.array(rows)
    if side_data is not None and any(d is not None for d in side_data):
        # Neumann data: the stencil weights of the ghost nodes times their data parts
        zero = np.zeros((Nz + 2, ny, nx), dtype=np.complex128)
        F = F - apply_operator(order, h, K, zf, zero, None, None, sides, side_data, Kz, Kzz)
    return F


def eigenvalues(R, Nx, Ny, sides=(SIDE_DIRICHLET, SIDE_DIRICHLET)):
    """lambda_nu(p, q) of every unknown row: complex array (3, Nu, ny, nx).

    Paper: Section 3.6 (lambda_nu(p, q))."""
    cx = side_cosines(Nx, sides[0])[None, None, :]
    cy = side_cosines(Ny, sides[1])[None, :, None]
    lam = np.empty((3, R.shape[0], cy.shape[1], cx.shape[2]), dtype=np.complex128)
    for nu in range(3):
        cf = R[:, nu, :]
        lam[nu] = (4.0 * cf[:, O.A_, None, None] * cx * cy + 2.0 * cf[:, O.B_, None, None] * cx
                   + 2.0 * cf[:, O.C_, None, None] * cy + cf[:, O.D_, None, None])
    return lam


def solve_rows(R, F, Nx, Ny, sides=(SIDE_DIRICHLET, SIDE_DIRICHLET)):
    """U (Nu, ny, nx) = A^-1 F by Section 3.6: 2-D side transforms, complex tridiagonals
    in z, inverse transforms."""
    Tx, Txi = side_transform(Nx, sides[0])
    Ty, Tyi = side_transform(Ny, sides[1])
    Fhat = np.matmul(Ty, F @ Tx.T)
    lam = eigenvalues(R, Nx, Ny, sides)
    W, ratio = O.thomas(lam[O.LOW], lam[O.MID], lam[O.UPP], Fhat)
    return np.matmul(Tyi, W @ Txi.T), ratio


def solve(order, h, K, zf, f_nodes, g_lo=None, g_hi=None,
          sides=(SIDE_DIRICHLET, SIDE_DIRICHLET), side_data=None, Kz=None, Kzz=None, fnn=None):
    """Solution on every plane l = 0..Nz+1 (unknown grid in x, y): complex (Nz+2, ny, nx).

    Paper: Section 3.6 (transforms, z-solves, inverse transforms)."""
    f = np.asarray(f_nodes, dtype=np.complex128)
    Nz, Ny, Nx = f.shape[0] - 2, f.shape[1] - 2, f.shape[2] - 2
    ny, nx = _n_unknown(Ny, sides[1]), _n_unknown(Nx, sides[0])
    R = row_table(order, h, K, zf, Kz, Kzz)
    F = rhs(order, h, K, zf, f, g_lo, g_hi, sides, side_data, Kz, Kzz, fnn)
    Uu, ratio = solve_rows(R, F, Nx, Ny, sides)
    l0, l1 = zf.unknown_planes(Nz)
    U = np.zeros((Nz + 2, ny, nx), dtype=np.complex128)
    U[l0:l1 + 1] = Uu
    if zf.lo == DIRICHLET:
        U[0] = _face(g_lo, ny, nx)
    if zf.hi == DIRICHLET:
        U[Nz + 1] = _face(g_hi, ny, nx)
    return U, {"min_pivot_ratio": ratio}


# --------------------------------------------------------------------------
# direct definitions (for the pins): the operator evaluated from the scheme
# itself, the face condition imposed through an explicit ghost plane


def apply_operator(order, h, K, zf, U_all, g_lo=None, g_hi=None,
                   sides=(SIDE_DIRICHLET, SIDE_DIRICHLET), side_data=None, Kz=None, Kzz=None):
    """Rows l0..l1 of (A U - data terms): U_all on planes 0..Nz+1 (interior x, y).

    Interior rows: the 27-point stencil with the complex table.  Robin rows: the
    7-point second-order operator h_z^2 (dxx + dyy + dzz + K) u evaluated with an
    explicit ghost plane built from the face condition (with its data g), so that
    solving A U = F means operator(U) = rhs without the data terms.

    Paper: the scheme written out (eq. stencil27, Section 1's face conditions), for the
    pins."""
    hx, hy, hz = h
    K = np.asarray(K, dtype=np.complex128)
    U_all = np.asarray(U_all, dtype=np.complex128)
    Nz, Ny, Nx = U_all.shape[0] - 2, U_all.shape[1], U_all.shape[2]
    # beyond a Neumann side: the ghost u_-1 = u_1 + 2 h g of u_n = g, built explicitly
    P = reflect_pad(U_all, sides, side_data, h)
    Ci = complex_coefficients(order, h, K, Kz, Kzz)
    out = []
    glo, ghi = _face(g_lo, Ny, Nx), _face(g_hi, Ny, Nx)

    def seven_point(l, ghost_below, ghost_above):
        c = P[l, 1:-1, 1:-1]
        dxx = (P[l, 1:-1, :-2] - 2 * c + P[l, 1:-1, 2:]) / (hx * hx)
        dyy = (P[l, :-2, 1:-1] - 2 * c + P[l, 2:, 1:-1]) / (hy * hy)
        dzz = (ghost_below - 2 * c + ghost_above) / (hz * hz)
        return hz * hz * (dxx + dyy + dzz + K[l] * c)

    if zf.lo == ROBIN:
        a, b = zf.alpha[0], zf.beta[0]
        u1 = P[1, 1:-1, 1:-1]
        ghost = u1 - 2.0 * hz * (glo - b * P[0, 1:-1, 1:-1]) / a
        out.append(seven_point(0, ghost, u1))
    for l in range(1, Nz + 1):
        row = np.zeros((Ny, Nx), dtype=np.complex128)
        for nu, dl in ((O.LOW, -1), (O.MID, 0), (O.UPP, 1)):
            row += _plane_part(Ci[l - 1, nu], P[l + dl])
        out.append(row)
    if zf.hi == ROBIN:
        a, b = zf.alpha[1], zf.beta[1]
        uN = P[Nz, 1:-1, 1:-1]
        ghost = uN + 2.0 * hz * (ghi - b * P[Nz + 1, 1:-1, 1:-1]) / a
        out.append(seven_point(Nz + 1, uN, ghost))
    return np.array(out)


def rhs_direct(order, h, f_nodes, sides=(SIDE_DIRICHLET, SIDE_DIRICHLET), K=None, Kz=None,
               fnn=None):
    """The scheme's f-side on every plane that can be a row: R_h f on interior rows
    (f reflected beyond a Neumann side), h_z^2 f on the two face planes.

    Paper: eqs. scheme4 and scheme6 written out, for the pins."""
    hz = h[2]
    f = np.asarray(f_nodes, dtype=np.complex128)
    fu = _f_on_unknowns(f, sides)
    Fi = _interior_rhs(order, h, fu, K, Kz, fnn)
    return hz * hz * fu[0, 1:-1, 1:-1], Fi, hz * hz * fu[-1, 1:-1, 1:-1]


def solve_dense(order, h, K, zf, f_nodes, g_lo=None, g_hi=None,
                sides=(SIDE_DIRICHLET, SIDE_DIRICHLET), side_data=None, Kz=None, Kzz=None,
                fnn=None):
    """Brute force: the matrix of apply_operator (columns from unit vectors), its data
    part from the operator at U = 0, and a dense complex LU solve.

    Paper: no paper counterpart (brute-force pin)."""
    f = np.asarray(f_nodes, dtype=np.complex128)
    Nz = f.shape[0] - 2
    Ny, Nx = _n_unknown(f.shape[1] - 2, sides[1]), _n_unknown(f.shape[2] - 2, sides[0])
    l0, l1 = zf.unknown_planes(Nz)
    Nu = l1 - l0 + 1
    base = np.zeros((Nz + 2, Ny, Nx), dtype=np.complex128)
    if zf.lo == DIRICHLET:
        base[0] = _face(g_lo, Ny, Nx)
    if zf.hi == DIRICHLET:
        base[Nz + 1] = _face(g_hi, Ny, Nx)
    data = apply_operator(order, h, K, zf, base, g_lo, g_hi, sides, side_data, Kz, Kzz).ravel()
    n = Nu * Ny * Nx
    A = np.zeros((n, n), dtype=np.complex128)
    zero_faces = ZFaces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        Ue = np.zeros((Nz + 2, Ny, Nx), dtype=np.complex128)
        Ue[l0:l1 + 1] = e.reshape(Nu, Ny, Nx)
        A[:, k] = apply_operator(order, h, K, zero_faces, Ue, sides=sides, Kz=Kz, Kzz=Kzz).ravel()
    flo, Fi, fhi = rhs_direct(order, h, f, sides, K, Kz, fnn)
    rows = ([flo] if zf.lo == ROBIN else []) + list(Fi) + ([fhi] if zf.hi == ROBIN else [])
    b = np.array(rows).ravel() - data
    x = np.linalg.solve(A, b).reshape(Nu, Ny, Nx)
    U = base.copy()
    U[l0:l1 + 1] = x
    return U
