"""Pins of the complex-k / Robin z-face oracle (oracle/hs_complex_oracle.py), CPU only.

What fixes it, independently of its own code paths:
  (a) the complex coefficient table rests on every coefficient being affine in K
      (checked on the real table, which tests/test_oracle_pins.py pins to the paper);
  (b) the separated solve (2-D DST, complex tridiagonals) equals a dense LU solve of
      the matrix assembled from the scheme itself, with the Robin face imposed by an
      explicit ghost plane (not the folded row), for every face combination;
  (c) Dirichlet faces, real K and real data reduce it to the real oracle;
  (d) alpha -> 0 turns a Robin face into the Dirichlet face u = g / beta;
  (e) mirroring z maps a Robin face (alpha, beta) on one side to (-alpha, beta) on
      the other, and the solution mirrors with it;
  (f) on a manufactured complex solution the error falls at least like h^2 with
      Robin faces, and like h^4 (4th order) with Dirichlet faces;
  (g) Neumann side axes: the DCT-I pair inverts, and it diagonalises the reflected
      second difference with eigenvalues 2 cos(theta_p) - 2, theta_p = p pi/(N+1),
      p = 0..N+1; the separated solve equals the dense solve of the operator built
      with explicit reflected ghosts; swapping x and y swaps the solution; a
      manufactured cos-cos solution converges;
  (h) the side transforms equal scipy's DST-I, DCT-I, DST-III and DCT-III;
  (i) mutations: a mistake planted in the oracle (Robin term sign, quarter-wave
      weight, Neumann data sign, mode angle, 6th-order K_z sign) makes a pin fail.
"""
import numpy as np
import pytest

from oracle import hs_oracle as O
from oracle import hs_complex_oracle as CX

D, R = CX.DIRICHLET, CX.ROBIN


def _crand(rs, shape, scale=1.0):
    return scale * (rs.uniform(-1, 1, shape) + 1j * rs.uniform(-1, 1, shape))


def _random_case(shape, seed, order):
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    h = O.grid_steps(shape, (1.0, 0.9, 1.1))
    K = (30.0 + 10.0 * rs.uniform(size=Nz + 2)) * (1.0 + 0.3j * rs.uniform(size=Nz + 2))
    f = _crand(rs, (Nz + 2, Ny + 2, Nx + 2))
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    g_lo, g_hi = _crand(rs, (Ny, Nx)), _crand(rs, (Ny, Nx))
    return h, K, f, g_lo, g_hi, rs


@pytest.mark.parametrize("order", [2, 4])
def test_coefficients_affine_in_K(order):
    rs = np.random.RandomState(order)
    h = (0.11, 0.13, 0.09)
    K1, K2 = rs.uniform(-50, 50, 9), rs.uniform(-50, 50, 9)
    C = lambda K: O.stencil_coefficients(order, O.HELMHOLTZ, h, K)
    assert np.max(np.abs(C(K1 + K2) - C(K1) - C(K2) + C(np.zeros(9)))) <= 1e-13
    assert np.array_equal(CX.complex_coefficients(order, h, K1), C(K1).astype(complex))
    Kc = K1 + 1j * K2
    t = 0.37
    assert np.allclose(CX.complex_coefficients(order, h, Kc),
                       C(K1) + 1j * (C(K2) - C(np.zeros(9))), rtol=0, atol=1e-14)
    # the imaginary part enters exactly where K does
    assert np.allclose(CX.complex_coefficients(order, h, K1 + 1j * t * K2).imag,
                       t * (C(K2) - C(np.zeros(9))), rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("faces", [(R, R), (R, D), (D, R), (D, D)])
def test_separated_solve_equals_dense_solve(order, faces):
    shape = (5, 4, 6)
    h, K, f, g_lo, g_hi, rs = _random_case(shape, 7 + order + 2 * faces[0] + faces[1], order)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    U, info = CX.solve(order, h, K, zf, f, g_lo, g_hi)
    Ud = CX.solve_dense(order, h, K, zf, f, g_lo, g_hi)
    assert O.max_rel_diff(U, Ud) <= 1e-11
    # and it satisfies the scheme: operator(U) reproduces the f-side row by row
    res = CX.apply_operator(order, h, K, zf, U, g_lo, g_hi)
    flo, Fi, fhi = CX.rhs_direct(order, h, f)
    rows = ([flo] if faces[0] == R else []) + list(Fi) + ([fhi] if faces[1] == R else [])
    want = np.array(rows)
    assert np.max(np.abs(res - want)) <= 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("order", [2, 4])
def test_dirichlet_real_case_is_the_real_oracle(order):
    Nx, Ny, Nz = 7, 6, 5
    rs = np.random.RandomState(20 + order)
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 0.8, 1.2))
    K = 20.0 + 10.0 * rs.uniform(size=Nz + 2)
    f = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    g_lo, g_hi = rs.uniform(-1, 1, (Ny, Nx)), rs.uniform(-1, 1, (Ny, Nx))
    U, _ = CX.solve(order, h, K, CX.ZFaces(), f, g_lo, g_hi)
    zl = np.zeros((Ny + 2, Nx + 2))
    zh = np.zeros((Ny + 2, Nx + 2))
    zl[1:-1, 1:-1], zh[1:-1, 1:-1] = g_lo, g_hi
    C = O.stencil_coefficients(order, O.HELMHOLTZ, h, K)
    F = O.assemble_rhs(order, O.HELMHOLTZ, h, f, C, K, None, (None, None, None, None, zl, zh))
    Ur, _ = O.solve_assembled(C, F)
    assert np.max(np.abs(U.imag)) == 0.0
    assert O.max_rel_diff(U[1:-1].real, Ur) <= 1e-13
    assert np.array_equal(U[0], g_lo) and np.array_equal(U[-1], g_hi)


@pytest.mark.parametrize("order", [2, 4])
def test_robin_face_tends_to_dirichlet_as_alpha_vanishes(order):
    shape = (6, 5, 7)
    h, K, f, g_lo, g_hi, rs = _random_case(shape, 31, order)
    beta = 2.0 + 0.5j
    Ud, _ = CX.solve(order, h, K, CX.ZFaces(D, 1, 0, D, 1, 0), f, g_lo / beta, g_hi / beta)
    prev = None
    for a in (1e-3, 1e-5, 1e-7):
        Ur, _ = CX.solve(order, h, K, CX.ZFaces(R, a, beta, R, a * (1 - 1j), beta), f, g_lo, g_hi)
        d = O.max_rel_diff(Ur, Ud)
        if prev is not None:
            assert d <= 0.02 * prev + 1e-12   # O(alpha)
        prev = d
    assert prev <= 1e-5


@pytest.mark.parametrize("order", [2, 4])
def test_z_mirror_swaps_the_faces(order):
    shape = (5, 6, 7)
    h, K, f, g_lo, g_hi, rs = _random_case(shape, 41, order)
    a_lo, b_lo, a_hi, b_hi = 1.0 - 0.3j, 0.5 + 1.0j, 0.8 + 0.1j, -1.0 + 0.4j
    U, _ = CX.solve(order, h, K, CX.ZFaces(R, a_lo, b_lo, R, a_hi, b_hi), f, g_lo, g_hi)
    # z -> Lz - z: d/dz changes sign, the faces swap
    Um, _ = CX.solve(order, h, K[::-1], CX.ZFaces(R, -a_hi, b_hi, R, -a_lo, b_lo),
                     f[::-1], g_hi, g_lo)
    assert O.max_rel_diff(Um[::-1], U) <= 1e-12


def _manufactured(N, order, zf_kind, kappa=2.5, c=(40.0, 8.0)):
    h = (1.0 / (N + 1),) * 3
    x = np.arange(N + 2) * h[0]
    z = x.copy()
    K = (c[0] + 1j * c[1]) * (1.0 + 0.5 * z)
    sxy = np.sin(np.pi * x)[None, None, :] * np.sin(2 * np.pi * x)[None, :, None]
    ez = np.exp(1j * kappa * z)[:, None, None]
    u = sxy * ez                                      # u = sin(pi x) sin(2 pi y) e^{i kappa z}
    f = (-5.0 * np.pi ** 2 - kappa ** 2 + K[:, None, None]) * u
    alpha, beta = 1.0 + 0.5j, 3.0 - 1.0j
    if zf_kind == R:
        zf = CX.ZFaces(R, alpha, beta, R, alpha, beta)
        gfun = (1j * kappa * alpha + beta) * u        # alpha u_z + beta u
    else:
        zf = CX.ZFaces()
        gfun = u
    g_lo, g_hi = gfun[0, 1:-1, 1:-1], gfun[-1, 1:-1, 1:-1]
    U, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi)
    return np.max(np.abs(U - u[:, 1:-1, 1:-1]))


@pytest.mark.parametrize("order,kind,lo_ratio", [(2, R, 3.5), (4, R, 3.5), (2, D, 3.5), (4, D, 12.0)])
def test_manufactured_complex_solution_converges(order, kind, lo_ratio):
    e = [_manufactured(N, order, kind) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= lo_ratio, e


NEU, DIR = CX.SIDE_NEUMANN, CX.SIDE_DIRICHLET


@pytest.mark.parametrize("N", [1, 6, 15])
def test_dct_pair_and_reflected_second_difference(N):
    C, Ci = CX.side_transform(N, NEU)
    assert np.max(np.abs(Ci @ C - np.eye(N + 2))) <= 1e-13
    # second difference over nodes 0..N+1 with the reflected ghosts u_-1 = u_1
    n = N + 2
    D = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    D[0, 1] = 2.0
    D[-1, -2] = 2.0
    lam = 2.0 * CX.side_cosines(N, NEU) - 2.0
    assert np.max(np.abs(C @ D @ Ci - np.diag(lam))) <= 1e-12
    # and the sine pair for comparison (Dirichlet axis)
    S, Si = CX.side_transform(N, DIR)
    assert np.max(np.abs(Si @ S - np.eye(N))) <= 1e-13


def _neumann_case(shape, seed):
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    h = O.grid_steps(shape, (1.0, 0.9, 1.1))
    K = (30.0 + 10.0 * rs.uniform(size=Nz + 2)) * (1.0 + 0.3j * rs.uniform(size=Nz + 2))
    f = _crand(rs, (Nz + 2, Ny + 2, Nx + 2))
    return h, K, f, rs


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIR), (DIR, NEU), (NEU, NEU)])
@pytest.mark.parametrize("faces", [(R, R), (D, D), (R, D)])
def test_neumann_sides_separated_equals_dense(order, sides, faces):
    shape = (5, 4, 5)
    h, K, f, rs = _neumann_case(shape, 50 + order + 3 * sides[0] + sides[1] + 7 * faces[1])
    nx = shape[0] + 2 if sides[0] == NEU else shape[0]
    ny = shape[1] + 2 if sides[1] == NEU else shape[1]
    g_lo, g_hi = _crand(rs, (ny, nx)), _crand(rs, (ny, nx))
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    U, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides)
    Ud = CX.solve_dense(order, h, K, zf, f, g_lo, g_hi, sides)
    assert U.shape == (shape[2] + 2, ny, nx)
    assert O.max_rel_diff(U, Ud) <= 1e-11


def test_neumann_x_y_swap():
    N, Nz = 6, 5
    rs = np.random.RandomState(61)
    h = O.grid_steps((N, N, Nz), (1.0, 1.0, 1.2))
    K = (25.0 + 5.0 * rs.uniform(size=Nz + 2)) * (1.0 + 0.1j)
    f = _crand(rs, (Nz + 2, N + 2, N + 2))
    zf = CX.ZFaces(R, 1.0 - 0.5j, 0.5 + 1.0j, D)
    g_lo = _crand(rs, (N, N + 2))           # unknown grid of (NEU x, DIR y): ny = N, nx = N + 2
    U1, _ = CX.solve(4, h, K, zf, f, g_lo, None, (NEU, DIR))
    U2, _ = CX.solve(4, h, K, zf, f.transpose(0, 2, 1), g_lo.T, None, (DIR, NEU))
    assert O.max_rel_diff(U2.transpose(0, 2, 1), U1) <= 1e-12


def _manufactured_neumann(N, order, zkind, kappa=2.0):
    h = (1.0 / (N + 1),) * 3
    x = np.arange(N + 2) * h[0]
    z = x.copy()
    K = (35.0 + 6.0j) * (1.0 + 0.5 * z)
    u = (np.cos(np.pi * x)[None, None, :] * np.cos(2 * np.pi * x)[None, :, None]
         * np.exp(1j * kappa * z)[:, None, None])
    f = (-5.0 * np.pi ** 2 - kappa ** 2 + K[:, None, None]) * u
    alpha, beta = 1.0 + 0.5j, 3.0 - 1.0j
    if zkind == R:
        zf = CX.ZFaces(R, alpha, beta, R, alpha, beta)
        gfun = (1j * kappa * alpha + beta) * u
    else:
        zf = CX.ZFaces()
        gfun = u
    U, _ = CX.solve(order, h, K, zf, f, gfun[0], gfun[-1], (NEU, NEU))
    return np.max(np.abs(U - u))


@pytest.mark.parametrize("order,kind,lo_ratio", [(2, R, 3.5), (4, R, 3.5), (4, D, 12.0)])
def test_neumann_manufactured_converges(order, kind, lo_ratio):
    e = [_manufactured_neumann(N, order, kind) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= lo_ratio, e


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIR), (DIR, NEU), (NEU, NEU)])
@pytest.mark.parametrize("faces", [(R, R), (D, D)])
def test_neumann_data_separated_equals_dense(order, sides, faces):
    """u_n = g on the Neumann faces: the separated solve (data moved to the right-hand
    side through the ghost nodes' stencil weights) equals the dense solve of the operator
    whose ghosts carry the data explicitly."""
    shape = (5, 4, 4)
    Nx, Ny, Nz = shape
    h, K, f, rs = _neumann_case(shape, 70 + order + 3 * sides[0] + sides[1] + 7 * faces[1])
    nx = Nx + 2 if sides[0] == NEU else Nx
    ny = Ny + 2 if sides[1] == NEU else Ny
    g_lo, g_hi = _crand(rs, (ny, nx)), _crand(rs, (ny, nx))
    sd = (_crand(rs, (Nz + 2, Ny + 2)), _crand(rs, (Nz + 2, Ny + 2)),
          _crand(rs, (Nz + 2, Nx + 2)), _crand(rs, (Nz + 2, Nx + 2)))
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    U, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    Ud = CX.solve_dense(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    assert O.max_rel_diff(U, Ud) <= 1e-11
    U0, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides)
    assert O.max_rel_diff(U, U0) > 1e-3          # the data matter


def _manufactured_neumann_data(N, order, kappa=2.0):
    """u = sin(pi x / 2) cos(2 pi y) e^{i kappa z}: u_n = -pi/2 cos(2 pi y) e^{i kappa z}
    on x = 0, 0 on x = 1 and on both y-faces; Dirichlet z-faces."""
    h = (1.0 / (N + 1),) * 3
    x = np.arange(N + 2) * h[0]
    z = x.copy()
    K = (35.0 + 6.0j) * (1.0 + 0.5 * z)
    ez = np.exp(1j * kappa * z)
    u = (np.sin(0.5 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * x)[None, :, None]
         * ez[:, None, None])
    f = (-0.25 * np.pi ** 2 - 4 * np.pi ** 2 - kappa ** 2 + K[:, None, None]) * u
    gx_lo = -0.5 * np.pi * np.cos(2 * np.pi * x)[None, :] * ez[:, None]   # [Nz+2][Ny+2]
    sd = (gx_lo, None, None, None)
    U, _ = CX.solve(order, h, K, CX.ZFaces(), f, u[0], u[-1], (NEU, NEU), sd)
    return np.max(np.abs(U - u))


@pytest.mark.parametrize("order", [2, 4])
def test_neumann_data_manufactured_converges(order):
    e = [_manufactured_neumann_data(N, order) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= 3.5, e


def _manufactured_neumann_ydata(N, order, kappa=2.0, Ly=1.3):
    """u = cos(pi x) sin(pi y / (2 Ly)) e^{i kappa z} on [0,1] x [0,Ly] x [0,1] (h_x != h_y):
    u_n = -pi/(2 Ly) cos(pi x) e^{i kappa z} on y = 0, 0 on the other side faces."""
    h = (1.0 / (N + 1), Ly / (N + 1), 1.0 / (N + 1))
    x = np.arange(N + 2) * h[0]
    y = np.arange(N + 2) * h[1]
    z = np.arange(N + 2) * h[2]
    K = (35.0 + 6.0j) * (1.0 + 0.5 * z)
    ez = np.exp(1j * kappa * z)
    u = (np.cos(np.pi * x)[None, None, :] * np.sin(0.5 * np.pi * y / Ly)[None, :, None]
         * ez[:, None, None])
    f = (-np.pi ** 2 - (0.5 * np.pi / Ly) ** 2 - kappa ** 2 + K[:, None, None]) * u
    gy_lo = -(0.5 * np.pi / Ly) * np.cos(np.pi * x)[None, :] * ez[:, None]   # [Nz+2][Nx+2]
    U, _ = CX.solve(order, h, K, CX.ZFaces(), f, u[0], u[-1], (NEU, NEU),
                    (None, None, gy_lo, None))
    return np.max(np.abs(U - u))


@pytest.mark.parametrize("order", [2, 4])
def test_neumann_ydata_anisotropic_converges(order):
    e = [_manufactured_neumann_ydata(N, order) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= 3.5, e


DN, ND = CX.SIDE_DN, CX.SIDE_ND


@pytest.mark.parametrize("kind", [DN, ND])
@pytest.mark.parametrize("N", [1, 6, 15])
def test_quarter_wave_pair_and_second_difference(kind, N):
    """One Dirichlet and one Neumann face on an axis: the quarter-wave pair inverts and
    diagonalises the second difference over the M = N + 1 unknown nodes with the
    Dirichlet neighbour 0 at one end and the reflected ghost at the other."""
    M = N + 1
    T, Ti = CX.side_transform(N, kind)
    assert T.shape == (M, M)
    assert np.max(np.abs(Ti @ T - np.eye(M))) <= 1e-13
    D = -2.0 * np.eye(M) + np.eye(M, k=1) + np.eye(M, k=-1)
    if kind == DN:
        D[-1, -2] = 2.0          # node M (Neumann): ghost M + 1 = node M - 1
    else:
        D[0, 1] = 2.0            # node 0 (Neumann): ghost -1 = node 1
    lam = 2.0 * CX.side_cosines(N, kind) - 2.0
    assert np.max(np.abs(T @ D @ Ti - np.diag(lam))) <= 1e-12


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(DN, DIR), (ND, NEU), (DN, ND), (NEU, DN)])
@pytest.mark.parametrize("faces", [(R, R), (D, D)])
def test_mixed_sides_separated_equals_dense(order, sides, faces):
    shape = (5, 4, 4)
    Nx, Ny, Nz = shape
    h, K, f, rs = _neumann_case(shape, 80 + order + 4 * sides[0] + sides[1] + 7 * faces[1])
    nx, ny = CX._n_unknown(Nx, sides[0]), CX._n_unknown(Ny, sides[1])
    g_lo, g_hi = _crand(rs, (ny, nx)), _crand(rs, (ny, nx))
    sd = (_crand(rs, (Nz + 2, Ny + 2)), _crand(rs, (Nz + 2, Ny + 2)),
          _crand(rs, (Nz + 2, Nx + 2)), _crand(rs, (Nz + 2, Nx + 2)))
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    U, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    Ud = CX.solve_dense(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    assert U.shape == (Nz + 2, ny, nx)
    assert O.max_rel_diff(U, Ud) <= 1e-11


def _manufactured_mixed(N, order, kind, kappa=2.0):
    """x-profile sin(pi x/2) (u = 0 at x = 0, u_x = 0 at x = 1: kind DN) or cos(pi x/2)
    (u_x = 0 at x = 0, u = 0 at x = 1: kind ND), times cos(2 pi y) (Neumann y) and
    e^{i kappa z} (Dirichlet z-faces)."""
    h = (1.0 / (N + 1),) * 3
    x = np.arange(N + 2) * h[0]
    z = x.copy()
    K = (35.0 + 6.0j) * (1.0 + 0.5 * z)
    px = np.sin(0.5 * np.pi * x) if kind == DN else np.cos(0.5 * np.pi * x)
    u = (px[None, None, :] * np.cos(2 * np.pi * x)[None, :, None]
         * np.exp(1j * kappa * z)[:, None, None])
    f = (-0.25 * np.pi ** 2 - 4 * np.pi ** 2 - kappa ** 2 + K[:, None, None]) * u
    x0, x1 = CX._nodes(N, kind)
    ue = u[:, :, x0:x1 + 1]                     # every y node (Neumann y), the unknown x nodes
    U, _ = CX.solve(order, h, K, CX.ZFaces(), f, ue[0], ue[-1], (kind, NEU))
    return np.max(np.abs(U - ue))


@pytest.mark.parametrize("kind", [DN, ND])
def test_mixed_sides_manufactured_converges(kind):
    e = [_manufactured_mixed(N, 4, kind) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= 12.0, e


def _case6(shape, seed):
    """Uniform h (6th order): box ((N_a + 1) h); complex K with K_z, K_zz; f and the six
    face arrays f_nn complex."""
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    hh = 1.0 / (max(shape) + 1)
    h = (hh, hh, hh)
    z = np.arange(Nz + 2) * hh
    c = (30.0 + 5.0 * rs.uniform()) * (1.0 + 0.2j)
    K = c * (1.0 + 0.5 * z + 0.3 * z * z)
    Kz = c * (0.5 + 0.6 * z)
    Kzz = c * 0.6 + 0.0 * z
    f = _crand(rs, (Nz + 2, Ny + 2, Nx + 2))
    fnn = [_crand(rs, (Nz + 2, Ny + 2)), _crand(rs, (Nz + 2, Ny + 2)),
           _crand(rs, (Nz + 2, Nx + 2)), _crand(rs, (Nz + 2, Nx + 2)),
           _crand(rs, (Ny + 2, Nx + 2)), _crand(rs, (Ny + 2, Nx + 2))]
    return h, K, Kz, Kzz, f, fnn, rs


def test_complex_coefficients6_reduce_to_real():
    rs = np.random.RandomState(3)
    h = (0.1, 0.1, 0.1)
    K, Kz, Kzz = rs.uniform(10, 50, 9), rs.uniform(-20, 20, 9), rs.uniform(-50, 50, 9)
    C = O.stencil_coefficients(6, O.HELMHOLTZ, h, K, Kz, Kzz)
    Cc = CX.complex_coefficients(6, h, K, Kz, Kzz)
    assert np.max(np.abs(Cc.imag)) == 0.0
    assert np.max(np.abs(Cc.real - C)) <= 1e-15 * np.max(np.abs(C))


@pytest.mark.parametrize("faces", [(R, R), (D, D), (R, D)])
def test_order6_separated_equals_dense(faces):
    shape = (5, 4, 6)
    h, K, Kz, Kzz, f, fnn, rs = _case6(shape, 90 + 2 * faces[0] + faces[1])
    Nx, Ny, Nz = shape
    g_lo, g_hi = _crand(rs, (Ny, Nx)), _crand(rs, (Ny, Nx))
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    U, _ = CX.solve(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    Ud = CX.solve_dense(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    assert O.max_rel_diff(U, Ud) <= 1e-11


def test_order6_real_case_is_the_real_oracle():
    shape = (7, 6, 5)
    Nx, Ny, Nz = shape
    h, K, Kz, Kzz, f, fnn, rs = _case6(shape, 97)
    K, Kz, Kzz, f = K.real, Kz.real, Kzz.real, f.real
    fnn = [a.real for a in fnn]
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    g_lo, g_hi = rs.uniform(-1, 1, (Ny, Nx)), rs.uniform(-1, 1, (Ny, Nx))
    U, _ = CX.solve(6, h, K, CX.ZFaces(), f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    zl, zh = np.zeros((Ny + 2, Nx + 2)), np.zeros((Ny + 2, Nx + 2))
    zl[1:-1, 1:-1], zh[1:-1, 1:-1] = g_lo, g_hi
    C = O.stencil_coefficients(6, O.HELMHOLTZ, h, K, Kz, Kzz)
    F = O.assemble_rhs(6, O.HELMHOLTZ, h, f, C, K, Kz, (None, None, None, None, zl, zh), fnn)
    Ur, _ = O.solve_assembled(C, F)
    assert np.max(np.abs(U.imag)) == 0.0
    assert O.max_rel_diff(U[1:-1].real, Ur) <= 1e-12


def _manufactured6(N, kappa=2.5, c=(40.0, 8.0)):
    """u = sin(pi x) sin(2 pi y) e^{i kappa z}, K = c (1 + z/2) (complex): f and its
    normal second derivatives on the z-faces analytic (zero on the x and y faces)."""
    hh = 1.0 / (N + 1)
    h = (hh, hh, hh)
    x = np.arange(N + 2) * hh
    z = x.copy()
    cc = c[0] + 1j * c[1]
    K, Kz, Kzz = cc * (1.0 + 0.5 * z), cc * 0.5 + 0.0 * z, 0.0 * z + 0.0j
    s = np.sin(np.pi * x)[None, None, :] * np.sin(2 * np.pi * x)[None, :, None]
    ez = np.exp(1j * kappa * z)
    u = s * ez[:, None, None]
    q = -5.0 * np.pi ** 2 - kappa ** 2
    f = (q + K[:, None, None]) * u
    # f = g(z) s(x, y) with g = (q + K) e^{i kappa z}: g'' = (2 i kappa K' - kappa^2 (q + K)) e^{..}
    g2 = (2j * kappa * Kz - kappa ** 2 * (q + K)) * ez
    sxy = s[0]
    fnn = [None, None, None, None, g2[0] * sxy, g2[-1] * sxy]
    U, _ = CX.solve(6, h, K, CX.ZFaces(), f, u[0, 1:-1, 1:-1], u[-1, 1:-1, 1:-1],
                    Kz=Kz, Kzz=Kzz, fnn=fnn)
    return np.max(np.abs(U - u[:, 1:-1, 1:-1]))


def test_order6_manufactured_complex_solution_converges():
    e = [_manufactured6(N) for N in (7, 15, 31)]
    assert e[2] < e[1] < e[0]
    assert e[1] / e[2] >= 40.0, e


@pytest.mark.parametrize("N", [1, 6, 15, 31])
def test_side_transforms_are_the_library_dst_dct(N):
    """The four side-axis transforms against scipy's unnormalised trigonometric
    transforms (an independent implementation): Dirichlet faces = DST-I / 2 over the
    interior nodes, Neumann faces = DCT-I / 2 over all nodes, Dirichlet low with
    Neumann high = DST-III / 2 over nodes 1..M, Neumann low with Dirichlet high =
    DCT-III / 2 over nodes 0..N.  The quarter-wave transform is also the odd outputs
    of a DST-I of length 2M over the line extended evenly about the Neumann node."""
    sfft = pytest.importorskip("scipy.fft")
    M = N + 1
    g = np.random.default_rng(N)
    x = g.standard_normal(N)
    T, _ = CX.side_transform(N, DIR)
    assert np.max(np.abs(T @ x - sfft.dst(x, type=1) / 2)) <= 1e-12
    x = g.standard_normal(M + 1)
    T, _ = CX.side_transform(N, NEU)
    assert np.max(np.abs(T @ x - sfft.dct(x, type=1) / 2)) <= 1e-12
    x = g.standard_normal(M)
    T, _ = CX.side_transform(N, DN)
    assert np.max(np.abs(T @ x - sfft.dst(x, type=3) / 2)) <= 1e-12
    ext = np.concatenate([x, x[-2::-1]])              # nodes 1..2M-1, even about node M
    assert ext.size == 2 * M - 1
    assert np.max(np.abs(T @ x - sfft.dst(ext, type=1)[0::2] / 4)) <= 1e-12
    T, _ = CX.side_transform(N, ND)
    assert np.max(np.abs(T @ x - sfft.dct(x, type=3) / 2)) <= 1e-12
    # ND is DN of the reversed line (node i -> M - i) with alternating signs
    TDN, _ = CX.side_transform(N, DN)
    sign = (-1.0) ** np.arange(M)
    assert np.max(np.abs(T @ x - sign * (TDN @ x[::-1]))) <= 1e-12


# ----------------------------------------------------------------- mutations
# A plausible mistake planted in the oracle (on the CPU, through monkeypatch) must make
# one of the pins above fail.


def test_planted_robin_sign_is_caught(monkeypatch):
    """Robin row with the sign of the eliminated face term flipped."""
    orig = CX.robin_row

    def mutated(h, K_l, alpha, beta, side):
        Rb = orig(h, K_l, alpha, beta, side)
        Rb[O.MID, O.D_] += side * 4.0 * h[2] * beta / alpha
        return Rb

    monkeypatch.setattr(CX, "robin_row", mutated)
    with pytest.raises(AssertionError):
        test_separated_solve_equals_dense_solve(4, (R, R))


def test_planted_quarter_wave_weight_is_caught(monkeypatch):
    """Quarter-wave forward transform without the weight 1/2 at the Neumann node."""
    orig = CX.side_transform

    def mutated(N, kind):
        fwd, inv = orig(N, kind)
        if kind == DN:
            fwd = fwd.copy()
            fwd[:, -1] *= 2.0
        return fwd, inv

    monkeypatch.setattr(CX, "side_transform", mutated)
    with pytest.raises(AssertionError):
        test_quarter_wave_pair_and_second_difference(DN, 6)
    with pytest.raises(AssertionError):
        test_mixed_sides_separated_equals_dense(4, (DN, DIR), (R, R))


def test_planted_neumann_data_sign_is_caught(monkeypatch):
    """Ghost of u_n = g built with the inward normal (data sign flipped) in every code
    path: the separated and dense solves still agree, the manufactured solution does
    not converge."""
    orig = CX.reflect_pad

    def mutated(U, sides, side_data=None, h=None):
        if side_data is not None:
            side_data = [None if d is None else -np.asarray(d) for d in side_data]
        return orig(U, sides, side_data, h)

    monkeypatch.setattr(CX, "reflect_pad", mutated)
    test_neumann_data_separated_equals_dense(4, (NEU, NEU), (D, D))
    with pytest.raises(AssertionError):
        test_neumann_data_manufactured_converges(4)


def test_planted_mode_angle_is_caught(monkeypatch):
    """Eigenvalues from cos(p pi / (N + 2)) instead of cos(p pi / (N + 1))."""
    orig = CX.side_cosines

    def mutated(N, kind):
        c = orig(N, kind)
        return orig(N + 1, kind)[:c.size] if kind == DIR else c

    monkeypatch.setattr(CX, "side_cosines", mutated)
    with pytest.raises(AssertionError):
        test_separated_solve_equals_dense_solve(2, (D, D))


def test_planted_order6_kz_sign_is_caught(monkeypatch):
    """6th-order rows with the sign of the K_z terms flipped."""
    orig = CX.complex_coefficients6

    def mutated(h, K, Kz, Kzz):
        return orig(h, K, -np.asarray(Kz), Kzz)

    monkeypatch.setattr(CX, "complex_coefficients6", mutated)
    with pytest.raises(AssertionError):
        test_order6_real_case_is_the_real_oracle()
    with pytest.raises(AssertionError):
        test_order6_manufactured_complex_solution_converges()
