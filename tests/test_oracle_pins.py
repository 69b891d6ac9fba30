"""Pins of the CPU oracle against things other than itself (no GPU).

* the paper's printed convergence tables (Tables 4, 5, 10 digit for digit;
  Table 6 in magnitude: the paper's 6th-order right-hand side used an implicit
  derivative approximation that it does not specify),
* brute-force sparse LU of the directly assembled 27-diagonal matrix,
* observed orders 2, 4 and 6 on manufactured solutions, and the local
  truncation order of every coefficient set with its right-hand side,
* DST identities, the single-mode reduction to one 1-D tridiagonal system,
  operator symmetry, linearity,
* mutation checks: a planted mistake in the oracle makes a pin fail.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import hs_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _l2err_over_U(U, u_nodes):
    u = u_nodes[1:-1, 1:-1, 1:-1]
    return float(np.linalg.norm(u - U) / np.linalg.norm(U))


# ---------------------------------------------------------------- paper tables


@pytest.mark.parametrize("order,table", [(2, "table4_order2"), (4, "table5_order4")])
def test_paper_tables_4_5_digits(order, table):
    """Tables 4 and 5 at 125^3: max-err and L2-err reproduce to the printed 8 digits."""
    p = W.paper_helmholtz(125, order)
    U, info = O.solve(p, return_all=True)
    ref = GOLD[table]["125"]
    maxe, _ = O.error_measures(U, p.u_exact)
    assert maxe == pytest.approx(ref["max_err"], rel=2e-7)
    assert _l2err_over_U(U, p.u_exact) == pytest.approx(ref["l2_err"], rel=2e-7)
    res = O.residual_l2(info["C"], U, info["F"])
    assert res < 10 * ref["l2_res"]


def test_paper_table6_magnitude():
    """Table 6 (6th order): same magnitude; the paper's f-derivative scheme differs (unpinned digits)."""
    p = W.paper_helmholtz(125, 6)
    U, _ = O.solve(p)
    maxe, _ = O.error_measures(U, p.u_exact)
    ref = GOLD["table6_order6"]["125"]["max_err"]
    assert 0.5 * ref < maxe < 1.5 * ref


@pytest.mark.parametrize("N", [64, 128])
def test_paper_table10_convdiff_digits(N):
    """Table 10 (CD, gamma = -100, non-homogeneous z-faces): 8 printed digits."""
    p = W.paper_convdiff(N)
    U, info = O.solve(p, return_all=True)
    ref = GOLD["table10_cd"][str(N)]
    maxe, l2e = O.error_measures(U, p.u_exact)
    assert maxe == pytest.approx(ref["max_err"], rel=2e-7)
    assert l2e == pytest.approx(ref["l2_err"], rel=2e-7)


@pytest.mark.slow
def test_paper_table5_250():
    p = W.paper_helmholtz(250, 4)
    U, _ = O.solve(p)
    maxe, _ = O.error_measures(U, p.u_exact)
    assert maxe == pytest.approx(GOLD["table5_order4"]["250"]["max_err"], rel=2e-7)


# ------------------------------------------------------ brute-force sparse LU


def assemble_matrix(C, Nx, Ny, Nz):
    """The 27-diagonal matrix of eq. (stencil27), written out entry by entry.

    Returns (A_int, A_bnd, node_index): A_int acts on interior unknowns
    (row order i + Nx j + Nx Ny l, Section 3.1) and A_bnd on every node of
    the (Nz+2)(Ny+2)(Nx+2) grid (only boundary columns are non-zero).
    """
    n_int = Nx * Ny * Nz
    rows_i, cols_i, vals_i = [], [], []
    rows_b, cols_b, vals_b = [], [], []
    for l in range(1, Nz + 1):
        for j in range(1, Ny + 1):
            for i in range(1, Nx + 1):
                r = (i - 1) + Nx * (j - 1) + Nx * Ny * (l - 1)
                for dl in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        for di in (-1, 0, 1):
                            if di != 0 and dj != 0:
                                m = 0            # a: the four corners
                            elif di != 0:
                                m = 1            # b: x-neighbours
                            elif dj != 0:
                                m = 2            # c: y-neighbours
                            else:
                                m = 3            # d: centre
                            v = C[l - 1, dl + 1, m]
                            if v == 0.0:
                                continue
                            ii, jj, ll = i + di, j + dj, l + dl
                            if 1 <= ii <= Nx and 1 <= jj <= Ny and 1 <= ll <= Nz:
                                rows_i.append(r)
                                cols_i.append((ii - 1) + Nx * (jj - 1) + Nx * Ny * (ll - 1))
                                vals_i.append(v)
                            else:
                                rows_b.append(r)
                                cols_b.append(ii + (Nx + 2) * jj + (Nx + 2) * (Ny + 2) * ll)
                                vals_b.append(v)
    A_int = sp.csc_matrix((vals_i, (rows_i, cols_i)), shape=(n_int, n_int))
    A_bnd = sp.csr_matrix((vals_b, (rows_b, cols_b)),
                          shape=(n_int, (Nx + 2) * (Ny + 2) * (Nz + 2)))
    return A_int, A_bnd


def _random_faces(rs, Nx, Ny, Nz):
    return [rs.uniform(-1, 1, (Nz + 2, Ny + 2)), rs.uniform(-1, 1, (Nz + 2, Ny + 2)),
            rs.uniform(-1, 1, (Nz + 2, Nx + 2)), rs.uniform(-1, 1, (Nz + 2, Nx + 2)),
            rs.uniform(-1, 1, (Ny + 2, Nx + 2)), rs.uniform(-1, 1, (Ny + 2, Nx + 2))]


CASES = [(2, W.HELMHOLTZ, O.CD_CORRECTED), (4, W.HELMHOLTZ, O.CD_CORRECTED),
         (6, W.HELMHOLTZ, O.CD_CORRECTED), (4, W.CONVDIFF, O.CD_PAPER),
         (4, W.CONVDIFF, O.CD_CORRECTED)]


@pytest.mark.parametrize("shape", [(7, 9, 11), (8, 5, 13), (15, 15, 15)])
@pytest.mark.parametrize("order,eq,variant", CASES)
def test_solver_matches_sparse_lu(shape, order, eq, variant):
    """Separation of variables == direct LU of the assembled matrix, with random data."""
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(hash((shape, order, eq, variant)) % 2 ** 31)
    if order == 6:
        h = 1.0 / (max(shape) + 1)
        L = ((Nx + 1) * h, (Ny + 1) * h, (Nz + 1) * h)
    else:
        L = (1.0, 0.7, 1.3)
    h = O.grid_steps((Nx, Ny, Nz), L)
    c0 = rs.uniform(5.0, 40.0, Nz + 2) if eq == W.HELMHOLTZ else rs.uniform(-20, 20, Nz + 2)
    c1 = rs.uniform(-50, 50, Nz + 2)
    c2 = rs.uniform(-500, 500, Nz + 2)
    C = O.stencil_coefficients(order, eq, h, c0, c1, c2, variant)
    f = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    faces = _random_faces(rs, Nx, Ny, Nz)
    fnn = _random_faces(rs, Nx, Ny, Nz)
    F = O.rhs_operator(order, eq, h, f, c0, c1, fnn)
    U, info = O.solve_assembled(C, O.lift(C, F, faces))

    A_int, A_bnd = assemble_matrix(C, Nx, Ny, Nz)
    g = O.boundary_nodes((Nz, Ny, Nx), faces).ravel()
    rhs = F.ravel() - A_bnd @ g
    U_lu = spla.splu(A_int).solve(rhs).reshape(Nz, Ny, Nx)
    assert info["min_pivot_ratio"] > 1e-13
    assert O.max_rel_diff(U, U_lu) < 1e-11


def test_apply_stencil_matches_matrix():
    Nx, Ny, Nz = 6, 7, 5
    rs = np.random.RandomState(7)
    C = rs.uniform(-1, 1, (Nz, 3, 4))
    A_int, A_bnd = assemble_matrix(C, Nx, Ny, Nz)
    Un = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    g = Un.copy()
    g[1:-1, 1:-1, 1:-1] = 0
    ref = A_int @ Un[1:-1, 1:-1, 1:-1].ravel() + A_bnd @ g.ravel()
    assert np.allclose(O.apply_stencil(C, Un).ravel(), ref, rtol=0, atol=1e-13)


# ----------------------------------------------------- convergence and consistency


@pytest.mark.parametrize("order,expect", [(2, 4.0), (4, 16.0), (6, 64.0)])
def test_observed_order_helmholtz(order, expect):
    """Max-error ratio on halving h (N = 15, 31, 63) approaches 2^order."""
    errs = []
    for N in (15, 31, 63):
        p = W.manufactured_cube(N, order, W.k_10_5sin())
        U, _ = O.solve(p)
        errs.append(O.error_measures(U, p.u_exact)[0])
    r = errs[1] / errs[2]
    assert 0.85 * expect < r < 1.2 * expect, errs


def _cd_problem(N, gamma_prof):
    """Manufactured CD problem: u = sin(pi x) sin(pi y) sin(2 pi z) e^z, f = Lap u + gamma u_z."""
    s = complex(1.0, 2.0 * np.pi)

    def zf(z, n=0):
        return np.imag(s ** n * np.exp(s * z))

    def u(x, y, z):
        return np.sin(np.pi * x) * np.sin(np.pi * y) * zf(z)

    def f(x, y, z):
        return np.sin(np.pi * x) * np.sin(np.pi * y) * (
            zf(z, 2) - 2 * np.pi ** 2 * zf(z) + gamma_prof.f0(z) * zf(z, 1))

    return W.analytic_problem(u, f, gamma_prof, (N, N + 2, N), (1.0, 1.3, 1.0), 4,
                              equation=W.CONVDIFF)


def test_observed_order_convdiff_variants():
    """Variable gamma(z): the corrected coefficients converge at order 4, the frozen ones at 2."""
    g0 = W.gamma_2_sin2pi()
    gp = W.Profile(lambda z: 8.0 * g0.f0(z), lambda z: 8.0 * g0.f1(z), lambda z: 8.0 * g0.f2(z))
    ratios = {}
    for variant in (O.CD_PAPER, O.CD_CORRECTED):
        errs = []
        for N in (15, 31, 63):
            p = _cd_problem(N, gp)
            U, _ = O.solve(p, cd_variant=variant)
            errs.append(O.error_measures(U, p.u_exact)[0])
        ratios[variant] = errs[1] / errs[2]
    assert 13.0 < ratios[O.CD_CORRECTED] < 19.0, ratios
    assert 3.0 < ratios[O.CD_PAPER] < 5.5, ratios


def _truncation(order, eq, N, kprof, variant=O.CD_CORRECTED):
    if eq == W.HELMHOLTZ:
        p = W.manufactured_cube(N, order, kprof)
    else:
        p = _cd_problem(N, kprof)
    h = p.h
    C = O.stencil_coefficients(order, eq, h, p.c0, p.c1, p.c2, variant)
    F = O.rhs_operator(order, eq, h, p.f_nodes, p.c0, p.c1, p.fnn)
    tau = O.apply_stencil(C, p.u_exact) - F
    # away from the faces: the 6th-order ghost closure is local to one layer
    return np.max(np.abs(tau[2:-2, 2:-2, 2:-2]))


@pytest.mark.parametrize("order,eq,expo", [(2, W.HELMHOLTZ, 4), (4, W.HELMHOLTZ, 6),
                                           (6, W.HELMHOLTZ, 8), (4, W.CONVDIFF, 6)])
def test_local_truncation_order(order, eq, expo):
    """A u - F = O(h^(order+2)) (F carries the factor h^2): coefficients and RHS operator agree."""
    prof = W.k_10_5sin() if eq == W.HELMHOLTZ else W.gamma_2_sin2pi()
    t1 = _truncation(order, eq, 31, prof)
    t2 = _truncation(order, eq, 63, prof)
    r = t1 / t2
    assert 0.7 * 2 ** expo < r < 1.3 * 2 ** expo, (t1, t2, r)


def test_sixth_order_face_data_matters():
    """Dropping the face second-derivative data (zero ghosts) degrades the 6th-order error."""
    p = W.manufactured_cube(31, 6, W.k_10_5sin())
    U, _ = O.solve(p)
    e_with = O.error_measures(U, p.u_exact)[0]
    p.fnn = [None] * 6
    U0, _ = O.solve(p)
    e_without = O.error_measures(U0, p.u_exact)[0]
    assert e_without > 3 * e_with


# ------------------------------------------------------------ transform identities


@pytest.mark.parametrize("N", [1, 2, 7, 31, 32, 95])
def test_sine_matrix_orthogonality(N):
    """S S = (N+1)/2 I: the DST-I is its own inverse up to 2/(N+1)."""
    S = O.sine_matrix(N)
    assert np.allclose(S @ S, (N + 1) / 2.0 * np.eye(N), atol=1e-12 * N)
    ref = np.sin(np.pi * np.outer(np.arange(1, N + 1), np.arange(1, N + 1)) / (N + 1))
    assert np.allclose(S, ref, atol=1e-13)


def test_dst2_roundtrip():
    rs = np.random.RandomState(3)
    F = rs.standard_normal((3, 9, 14))
    assert np.allclose(O.dst2_inverse(O.dst2_forward(F)), F, atol=1e-13)


def test_dst2_forward_is_the_library_dst():
    """The plane transform against scipy's unnormalised DST-I (2 sum x_n sin(...)) along
    the two last axes, for non-square planes (a transposed pair of sine matrices fails)."""
    sfft = pytest.importorskip("scipy.fft")
    rs = np.random.RandomState(5)
    F = rs.standard_normal((3, 11, 6))
    ref = sfft.dstn(F, type=1, axes=(1, 2)) / 4.0
    assert np.max(np.abs(O.dst2_forward(F) - ref)) <= 1e-12


def test_thomas_is_the_library_banded_solve():
    """The textbook tridiagonal LU against LAPACK's banded solver (partial pivoting) on
    diagonally dominant rows, several right-hand sides; and its pivot ratio."""
    sla = pytest.importorskip("scipy.linalg")
    rs = np.random.RandomState(8)
    n, m = 17, 4
    lower = rs.uniform(-1, 1, (n, m))
    upper = rs.uniform(-1, 1, (n, m))
    diag = 2.5 + rs.uniform(0, 1, (n, m))
    rhs = rs.standard_normal((n, m))
    w, ratio = O.thomas(lower, diag, upper, rhs)
    for j in range(m):
        ab = np.zeros((3, n))
        ab[0, 1:] = upper[:-1, j]
        ab[1] = diag[:, j]
        ab[2, :-1] = lower[1:, j]
        ref = sla.solve_banded((1, 1), ab, rhs[:, j])
        assert np.max(np.abs(w[:, j] - ref)) <= 1e-13 * max(1.0, np.abs(ref).max())
    assert 0 < ratio <= 1


def test_single_mode_reduces_to_1d_system():
    """F = sin(p pi x) sin(q pi y) phi(z): U = same mode times T_pq^{-1} phi (dense 1-D solve)."""
    Nx, Ny, Nz = 12, 9, 10
    rs = np.random.RandomState(11)
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 1.0, 1.0))
    c0 = rs.uniform(10, 30, Nz + 2)
    C = O.stencil_coefficients(4, W.HELMHOLTZ, h, c0)
    p, q = 3, 7
    sx = np.sin(np.pi * p * np.arange(1, Nx + 1) / (Nx + 1))
    sy = np.sin(np.pi * q * np.arange(1, Ny + 1) / (Ny + 1))
    phi = rs.standard_normal(Nz)
    F = phi[:, None, None] * sy[None, :, None] * sx[None, None, :]
    U, _ = O.solve_assembled(C, F)
    cp, cq = np.cos(np.pi * p / (Nx + 1)), np.cos(np.pi * q / (Ny + 1))
    lam = 4 * C[:, :, 0] * cp * cq + 2 * C[:, :, 1] * cp + 2 * C[:, :, 2] * cq + C[:, :, 3]
    T = np.diag(lam[:, 1]) + np.diag(lam[1:, 0], -1) + np.diag(lam[:-1, 2], 1)
    w = np.linalg.solve(T, phi)
    ref = w[:, None, None] * sy[None, :, None] * sx[None, None, :]
    assert O.max_rel_diff(U, ref) < 1e-12


# --------------------------------------------------------------- structure


def test_symmetry_constant_k_and_asymmetry_variable_k():
    Nx, Ny, Nz = 5, 6, 7
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 1.2, 0.9))
    for order in (2, 4):
        C = O.stencil_coefficients(order, W.HELMHOLTZ, h, np.full(Nz + 2, 300.0))
        A, _ = assemble_matrix(C, Nx, Ny, Nz)
        assert abs(A - A.T).max() < 1e-15
    hu = 1.0 / 8
    C6 = O.stencil_coefficients(6, W.HELMHOLTZ, (hu, hu, hu), np.full(Nz + 2, 300.0),
                                np.zeros(Nz + 2), np.zeros(Nz + 2))
    A6, _ = assemble_matrix(C6, Nx, Ny, Nz)
    assert abs(A6 - A6.T).max() < 1e-15
    c0 = np.linspace(100, 400, Nz + 2)
    C = O.stencil_coefficients(4, W.HELMHOLTZ, h, c0)
    A, _ = assemble_matrix(C, Nx, Ny, Nz)
    assert abs(A - A.T).max() > 1e-6


def test_linearity():
    p = W.manufactured_cube(11, 6, W.k_10_5sin())
    h = p.h
    C = O.stencil_coefficients(6, W.HELMHOLTZ, h, p.c0, p.c1, p.c2)
    rs = np.random.RandomState(5)
    F1, F2 = rs.standard_normal((2, 11, 11, 11))
    U1, _ = O.solve_assembled(C, F1)
    U2, _ = O.solve_assembled(C, F2)
    U3, _ = O.solve_assembled(C, 2.0 * F1 - 3.0 * F2)
    assert O.max_rel_diff(U3, 2.0 * U1 - 3.0 * U2) < 1e-12


# ----------------------------------------------------------------- mutations


def test_planted_mistake_is_caught(monkeypatch):
    """Flipping the sign of the h^3 K_z/120 term in the 6th-order b_{l+1} breaks order 6."""
    orig = O.stencil_coefficients

    def mutated(order, equation, h, c0, c1=None, c2=None, cd_variant=O.CD_CORRECTED):
        C = orig(order, equation, h, c0, c1, c2, cd_variant)
        if order == 6:
            hz = h[2]
            Kz = np.asarray(c1)[1:-1]
            C[:, 2, 1] -= 2 * hz ** 3 * Kz / 120.0
        return C

    monkeypatch.setattr(O, "stencil_coefficients", mutated)
    t1 = _truncation(6, W.HELMHOLTZ, 31, W.k_10_5sin())
    t2 = _truncation(6, W.HELMHOLTZ, 63, W.k_10_5sin())
    assert t1 / t2 < 0.7 * 2 ** 8


def test_planted_transposed_eigen_index_is_caught(monkeypatch):
    """Using cos(theta_q) for the x-neighbour term (b and c swapped) breaks the LU pin."""
    orig = O.eigenvalues

    def mutated(C, Nx, Ny):
        C2 = C.copy()
        C2[:, :, [1, 2]] = C[:, :, [2, 1]]
        return orig(C2, Nx, Ny)

    monkeypatch.setattr(O, "eigenvalues", mutated)
    Nx, Ny, Nz = 7, 9, 11
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 0.7, 1.3))
    rs = np.random.RandomState(1)
    C = O.stencil_coefficients(4, W.HELMHOLTZ, h, rs.uniform(5, 40, Nz + 2))
    F = rs.standard_normal((Nz, Ny, Nx))
    U, _ = O.solve_assembled(C, F)
    A_int, _ = assemble_matrix(C, Nx, Ny, Nz)
    U_lu = spla.splu(A_int).solve(F.ravel()).reshape(Nz, Ny, Nx)
    assert O.max_rel_diff(U, U_lu) > 1e-3


# ------------------------------------------------- separable right-hand sides


@pytest.mark.parametrize("order", [2, 4, 6])
def test_sine_mode_solution_matches_full_oracle(order):
    """The 1-D reduction for sums of sine modes equals the full 3-D oracle solve."""
    N = (20, 17, 23) if order != 6 else (23, 23, 23)
    L = (1.0, 0.9, 1.2) if order != 6 else (1.0, 1.0, 1.0)
    rs = np.random.RandomState(order)
    modes = rs.randint(1, 12, size=(6, 3))
    amps = rs.standard_normal(6)

    def f(x, y, z):
        out = 0.0 * (x + y + z)
        for (p, q, r), A in zip(modes, amps):
            out = out + A * (np.sin(p * np.pi * x / L[0]) * np.sin(q * np.pi * y / L[1])
                             * np.sin(r * np.pi * z / L[2]))
        return out

    K = W.k_profile_to_k2(W.k_tanh(20.0, 10.0))
    c0, c1, c2 = K.sample(N[2], L[2])
    fn = W.sample_nodes(f, *N, *L)
    p = W.Problem(*N, *L, order, W.HELMHOLTZ, c0, c1, c2, fn)
    U, _ = O.solve(p)
    U2 = O.solve_sine_modes(modes, amps, N, L, order, c0, c1, c2)
    assert O.max_rel_diff(U2, U) < 1e-12
    pts = (np.array([1, 5, N[0]]), np.array([2, N[1], 7]), np.array([N[2], 3, 1]))
    Us = O.solve_sine_modes(modes, amps, N, L, order, c0, c1, c2, sample=pts)
    assert np.allclose(Us, U[pts[2] - 1, pts[1] - 1, pts[0] - 1], rtol=0, atol=1e-12 * np.abs(U).max())


def test_sine_mode_solution_in_extended_precision():
    """solve_sine_modes_extended (the exact discrete solution for ill-conditioned
    z-systems) is pinned twice:
    * where the problem is well conditioned (31^3) it equals the FP64 sine-mode
      solution, itself pinned against the full oracle, to FP64 rounding;
    * on a tiny grid (7^3) it equals an independent 40-digit computation: mpmath
      arithmetic, the z-systems solved by dense LU (not Thomas), the sine modes
      built as full 3-D fields and projected, so only the Section 3.4 rows are
      shared; agreement to the FP64 rounding of the output."""
    mp = pytest.importorskip("mpmath")
    N = 31
    modes, amps = W.sine_modes(N, 16, 4)
    c = W.k_profile_to_k2(W.k_tanh()).sample(N, 1.0)
    rs = np.random.RandomState(0)
    pts = tuple(rs.randint(1, N + 1, size=2000) for _ in range(3))
    ex = O.solve_sine_modes_extended(modes, amps, N, *c, sample=pts)
    f64 = O.solve_sine_modes(modes, amps, (N, N, N), (1.0, 1.0, 1.0), 6, *c, sample=pts)
    assert np.abs(ex - f64).max() <= 1e-12 * np.abs(ex).max()

    mp.mp.dps = 40
    n = 7
    modes = np.array([[1, 2, 3], [3, 1, 2], [1, 2, 5], [7, 7, 1]])
    amps = np.array([1.0, -0.5, 0.25, 2.0])
    k = W.k_profile_to_k2(W.k_tanh(40.0, 20.0))
    c0, c1, c2 = k.sample(n, 1.0)
    idx = np.arange(1, n + 1)
    grid = np.meshgrid(idx, idx, idx, indexing="ij")   # (i, j, l)
    ex = O.solve_sine_modes_extended(modes, amps, n, c0, c1, c2,
                                     sample=(grid[0].ravel(), grid[1].ravel(), grid[2].ravel()))
    h = mp.mpf(1) / (n + 1)
    m = lambda v: mp.mpf(float(v))
    K = [m(v) for v in c0]
    Kz = [m(v) for v in c1]
    Kzz = [m(v) for v in c2]

    def rows(l):   # (a, b, d) for nu = l-1, l, l+1 of row l (1-based), Section 3.4
        return ((mp.mpf(1) / 30, mp.mpf(1) / 10 + h**2 * K[l - 1] / 90 - h**3 * Kz[l] / 120,
                 mp.mpf(7) / 15 - h**2 * K[l - 1] / 90 - (h**3 * Kz[l] / 20) * (mp.mpf(1) / 3 + h**2 * K[l - 1] / 6)),
                (mp.mpf(1) / 10 + h**2 * K[l] / 90, mp.mpf(7) / 15 - h**2 * K[l] / 90,
                 -mp.mpf(64) / 15 + 14 * h**2 * K[l] / 15 - h**4 * K[l]**2 / 20 + h**4 * Kzz[l] / 20),
                (mp.mpf(1) / 30, mp.mpf(1) / 10 + h**2 * K[l + 1] / 90 + h**3 * Kz[l] / 120,
                 mp.mpf(7) / 15 - h**2 * K[l + 1] / 90 + (h**3 * Kz[l] / 20) * (mp.mpf(1) / 3 + h**2 * K[l + 1] / 6)))

    # f = sum of modes on the node grid; F by the explicit 25-point operator R6
    # written point by point; projected on each (p, q) sine mode, solved by dense LU
    S = lambda a, i: mp.sin(mp.pi * a * i / (n + 1))
    f = {}
    for i in range(-1, n + 3):
        for j in range(-1, n + 3):
            for l in range(-1, n + 3):
                f[i, j, l] = sum(mp.mpf(float(A)) * S(p, i) * S(q, j) * S(r, l)
                                 for (p, q, r), A in zip(modes, amps))
    U = np.zeros((n, n, n))   # [i, j, l]
    Ump = {}
    for (p, q) in sorted({(int(a), int(b)) for a, b, _ in modes}):
        rhs = mp.matrix(n, 1)
        for l in range(1, n + 1):
            acc = mp.mpf(0)
            for i in range(1, n + 1):
                for j in range(1, n + 1):
                    c = f[i, j, l]
                    s1 = sum(f[i + a, j + b, l + g] for a, b, g in
                             ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)))
                    s2 = sum(f[i + a, j + b, l + g] for a, b, g in
                             ((2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)))
                    e = sum(f[i + a, j + b, l + g] for a, b, g in
                            ((1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0), (1, 0, 1), (1, 0, -1),
                             (-1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)))
                    F6 = h**2 * ((mp.mpf(67) / 120 - h**2 * K[l] / 20) * c + s1 / 18 - s2 / 240 + e / 90
                                 + h**3 * Kz[l] * (f[i, j, l + 1] - f[i, j, l - 1]) / 120)
                    acc += F6 * S(p, i) * S(q, j)
            rhs[l - 1] = acc * 4 / (n + 1) ** 2     # coefficient of sin_p sin_q
        T = mp.matrix(n, n)
        cp, cq = mp.cos(mp.pi * p / (n + 1)), mp.cos(mp.pi * q / (n + 1))
        for l in range(1, n + 1):
            for nu, (a, b, d) in enumerate(rows(l)):
                ll = l - 1 + nu
                if 1 <= ll <= n:
                    T[l - 1, ll - 1] = 4 * a * cp * cq + 2 * b * cp + 2 * b * cq + d
        w = mp.lu_solve(T, rhs)
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                for l in range(1, n + 1):
                    Ump[i, j, l] = Ump.get((i, j, l), mp.mpf(0)) + w[l - 1] * S(p, i) * S(q, j)
    ref = np.array([float(Ump[i, j, l]) for i, j, l in
                    zip(grid[0].ravel(), grid[1].ravel(), grid[2].ravel())])
    assert np.abs(ex - ref).max() <= 4e-16 * np.abs(ref).max()
