"""Complex k(z) and Robin z-faces on the GPU (hs_zplan / hs_zsolve), against the oracle.

Parity bar: the FP64 path's 1e-12 (max relative error over the whole complex field),
on ragged sizes (runtime-sized and compiled transform lengths), every face
combination, orders 2 and 4, absent face data, Nz = 1, and one 255^3 case; with
Neumann side axes (cosine transform), every side combination; and with axes that
have one face of each kind (quarter-wave transforms), beside every other kind.
"""
import numpy as np
import pytest

import paper_1912_03565_gb300 as H
from oracle import hs_oracle as O
from oracle import hs_complex_oracle as CX

pytestmark = pytest.mark.gpu

D, R = CX.DIRICHLET, CX.ROBIN
TOL = 1e-12


def _torch():
    return pytest.importorskip("torch")


def _case(shape, L, seed, kscale=40.0):
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    z = np.arange(Nz + 2) / (Nz + 1)
    K = kscale * (1.0 + 0.5 * z) * (1.0 + 0.2j * (1.0 + np.sin(3.0 * z)))
    f = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2)) + 1j * rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    g_lo = rs.uniform(-1, 1, (Ny, Nx)) + 1j * rs.uniform(-1, 1, (Ny, Nx))
    g_hi = rs.uniform(-1, 1, (Ny, Nx)) + 1j * rs.uniform(-1, 1, (Ny, Nx))
    return O.grid_steps(shape, L), K, f, g_lo, g_hi


def _nu(N, kind):
    """Unknowns of a side axis: N (Dirichlet faces), N + 2 (Neumann faces), N + 1 (one
    of each)."""
    return {H.HS_SIDE_DIRICHLET: N, H.HS_SIDE_NEUMANN: N + 2}.get(kind, N + 1)


def _planar(torch, a):
    return torch.from_numpy(np.ascontiguousarray(np.stack([a.real, a.imag]))).cuda()


def _gpu(shape, L, order, K, zf, f, g_lo, g_hi, sides=(0, 0)):
    torch = _torch()
    Nx, Ny, Nz = shape
    s = H.ZSolver(Nx, Ny, Nz, *L, order)
    try:
        s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
        u = torch.full((2, Nz + 2, ny, nx), np.nan, dtype=torch.float64, device="cuda")
        s.solve(_planar(torch, f), u, None if g_lo is None else _planar(torch, g_lo),
                None if g_hi is None else _planar(torch, g_hi))
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        return uc[0] + 1j * uc[1]
    finally:
        s.close()


FACES = [(R, R), (R, D), (D, R), (D, D)]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("shape", [(13, 9, 7), (31, 20, 17), (63, 40, 12)])
def test_complex_solve_matches_oracle(order, faces, shape):
    L = (1.0, 0.9, 1.2)
    h, K, f, g_lo, g_hi = _case(shape, L, sum(shape) + order)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi)
    got = _gpu(shape, L, order, K, zf, f, g_lo, g_hi)
    assert O.max_rel_diff(got, ref) <= TOL


@pytest.mark.parametrize("faces", FACES)
def test_absent_face_data_and_one_plane(faces):
    """g = NULL (zero face data) and Nz = 1: one interior plane, up to three unknown rows."""
    shape, L = (15, 11, 1), (1.0, 1.0, 0.3)
    h, K, f, _, _ = _case(shape, L, 5)
    zf = CX.ZFaces(faces[0], 0.5 - 1.0j, 1.0 + 0.0j, faces[1], 2.0 + 0.0j, -0.5 + 1.5j)
    ref, _ = CX.solve(4, h, K, zf, f, None, None)
    got = _gpu(shape, L, 4, K, zf, f, None, None)
    assert O.max_rel_diff(got, ref) <= TOL


def test_dirichlet_real_data_equals_real_solver():
    """Dirichlet faces, real K, real f and g: the complex solver gives the real FP64
    solver's answer in the real part and exactly zero imaginary part."""
    torch = _torch()
    shape, L = (33, 27, 21), (1.0, 1.0, 1.0)
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(3)
    K = 25.0 + 10.0 * rs.uniform(size=Nz + 2)
    f = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    g_lo, g_hi = rs.uniform(-1, 1, (Ny, Nx)), rs.uniform(-1, 1, (Ny, Nx))
    got = _gpu(shape, L, 4, K.astype(complex), CX.ZFaces(), f.astype(complex),
               g_lo.astype(complex), g_hi.astype(complex))
    assert np.max(np.abs(got.imag)) == 0.0
    s = H.Solver(Nx, Ny, Nz, *L, 4, H.HS_HELMHOLTZ, H.HS_FP64)
    try:
        s.set_coeff(K)
        zl = np.zeros((Ny + 2, Nx + 2))
        zh = np.zeros((Ny + 2, Nx + 2))
        zl[1:-1, 1:-1], zh[1:-1, 1:-1] = g_lo, g_hi
        u = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device="cuda")
        faces = [None, None, None, None, torch.from_numpy(zl).cuda(), torch.from_numpy(zh).cuda()]
        s.solve(torch.from_numpy(f).cuda(), u, H.HS_F64, H.HS_RHS_NODAL, faces, None)
        torch.cuda.synchronize()
        assert O.max_rel_diff(got[1:-1].real, u.cpu().numpy()) <= TOL
    finally:
        s.close()


def test_complex_255_robin_matches_oracle():
    """The benchmark's size: 255^3, 4th order, Robin on both z-faces."""
    shape, L = (255, 255, 255), (1.0, 1.0, 1.0)
    h, K, f, g_lo, g_hi = _case(shape, L, 11)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, R, 1.0 + 0.5j, 3.0 - 1.0j)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi)
    got = _gpu(shape, L, 4, K, zf, f, g_lo, g_hi)
    assert O.max_rel_diff(got, ref) <= TOL


def test_errors():
    torch = _torch()
    with pytest.raises(H.HsError) as e:
        H.ZSolver(8, 8, 8, 1.0, 1.0, 1.0, 5)
    assert e.value.status == H.HS_ERR_INVALID_ARG
    with pytest.raises(H.HsError) as e:   # order 6 needs one step in every direction
        H.ZSolver(8, 8, 8, 1.0, 1.0, 1.2, 6)
    assert e.value.status == H.HS_ERR_INVALID_ARG
    s = H.ZSolver(8, 7, 6, 1.0, 1.0, 1.0, 4)
    try:
        f = torch.zeros((2, 8, 9, 10), dtype=torch.float64, device="cuda")
        u = torch.zeros((2, 8, 7, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(H.HsError) as e:
            s.solve(f, u)
        assert e.value.status == H.HS_ERR_NO_COEFF
        s.set_coeff(np.full(8, 30.0 + 1.0j))
        with pytest.raises(H.HsError) as e:
            s.set_faces(H.HS_ZFACE_ROBIN, 0.0, 1.0, H.HS_ZFACE_DIRICHLET)
        assert e.value.status == H.HS_ERR_INVALID_ARG
        with pytest.raises(H.HsError) as e:
            s.solve(f.cpu(), u)
        assert e.value.status == H.HS_ERR_INVALID_ARG
        s.solve(f, u)
        torch.cuda.synchronize()
        assert torch.count_nonzero(u).item() == 0
    finally:
        s.close()


NEU, DIRS = CX.SIDE_NEUMANN, CX.SIDE_DIRICHLET


def _neumann_case(shape, L, sides, seed):
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    z = np.arange(Nz + 2) / (Nz + 1)
    K = 40.0 * (1.0 + 0.5 * z) * (1.0 + 0.2j * (1.0 + np.cos(2.0 * z)))
    f = rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2)) + 1j * rs.uniform(-1, 1, (Nz + 2, Ny + 2, Nx + 2))
    nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
    g_lo = rs.uniform(-1, 1, (ny, nx)) + 1j * rs.uniform(-1, 1, (ny, nx))
    g_hi = rs.uniform(-1, 1, (ny, nx)) + 1j * rs.uniform(-1, 1, (ny, nx))
    return O.grid_steps(shape, L), K, f, g_lo, g_hi


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIRS), (DIRS, NEU), (NEU, NEU)])
@pytest.mark.parametrize("faces", [(R, R), (D, D), (R, D)])
@pytest.mark.parametrize("shape", [(31, 63, 9), (63, 31, 4)])
def test_neumann_sides_match_oracle(order, sides, faces, shape):
    L = (1.0, 0.8, 1.1)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, sum(shape) + 3 * sides[0] + sides[1])
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides)
    got = _gpu(shape, L, order, K, zf, f, g_lo, g_hi, sides)
    assert O.max_rel_diff(got, ref) <= TOL


def test_neumann_beside_runtime_sized_sine_axis():
    """A Neumann x-axis (compiled cosine transform, 127 + 1 points) beside a Dirichlet
    y-axis whose length has no compiled transform (runtime-sized sine transform)."""
    shape, L = (127, 20, 11), (1.0, 1.0, 1.0)
    sides = (NEU, DIRS)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 77)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 2.0 - 1.0j, D)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi, sides)
    got = _gpu(shape, L, 4, K, zf, f, g_lo, g_hi, sides)
    assert O.max_rel_diff(got, ref) <= TOL


def test_neumann_255():
    shape, L = (255, 255, 127), (1.0, 1.0, 0.5)
    sides = (NEU, NEU)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 88)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, R, 1.0 + 0.5j, 3.0 - 1.0j)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi, sides)
    got = _gpu(shape, L, 4, K, zf, f, g_lo, g_hi, sides)
    assert O.max_rel_diff(got, ref) <= TOL


def test_side_kinds_and_invalid_kinds():
    """Lengths without a compiled FFT are accepted (runtime-sized transforms); an
    unknown kind is refused and leaves the previous kinds in effect."""
    s = H.ZSolver(30, 31, 5, 1.0, 1.0, 1.0, 4)
    try:
        s.set_sides(H.HS_SIDE_NEUMANN, H.HS_SIDE_DIRICHLET)   # 31 + 1 nodes: direct sums
        s.set_sides(H.HS_SIDE_DN, H.HS_SIDE_ND)               # extended lines of 61 and 63
        with pytest.raises(H.HsError) as e:
            s.set_sides(4, 0)
        assert e.value.status == H.HS_ERR_INVALID_ARG
    finally:
        s.close()


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIRS), (DIRS, NEU), (NEU, NEU), (CX.SIDE_DN, NEU),
                                   (NEU, CX.SIDE_ND), (CX.SIDE_ND, CX.SIDE_DN)])
@pytest.mark.parametrize("shape", [(30, 20, 6), (21, 44, 5)])
def test_runtime_sized_side_transforms(order, sides, shape):
    """Side axes whose transform length has no compiled FFT: the cosine transform by
    direct sums (N + 1 = 31, 21, 45, ...) and the quarter-wave transforms through the
    runtime-sized sine transform of the extended line (2 (N + 1) = 62, 42, 90), with
    face data on every Neumann face, against the oracle at the FP64 bar."""
    torch = _torch()
    L = (1.0, 0.8, 1.1)
    Nx, Ny, Nz = shape
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 3 * sum(shape) + order)
    rs = np.random.RandomState(order + sides[0])
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    neu = [sides[0] in (NEU, CX.SIDE_ND), sides[0] in (NEU, CX.SIDE_DN),
           sides[1] in (NEU, CX.SIDE_ND), sides[1] in (NEU, CX.SIDE_DN)]
    sd = [cr(Nz + 2, (Ny if k < 2 else Nx) + 2) if neu[k] else None for k in range(4)]
    zf = CX.ZFaces(R, 1.0 + 0.5j, 2.0 - 1.0j, D)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    s = H.ZSolver(Nx, Ny, Nz, *L, order)
    try:
        s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
        u = torch.full((2, Nz + 2, ny, nx), np.nan, dtype=torch.float64, device="cuda")
        s.solve(_planar(torch, f), u, _planar(torch, g_lo), _planar(torch, g_hi),
                side_data=[None if a is None else _planar(torch, a) for a in sd])
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
    finally:
        s.close()
    assert O.max_rel_diff(uc[0] + 1j * uc[1], ref) <= TOL


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIRS), (DIRS, NEU), (NEU, NEU)])
@pytest.mark.parametrize("faces", [(R, R), (D, D), (R, D)])
def test_neumann_face_data_match_oracle(order, sides, faces):
    """u_n = g on the Neumann faces (hs_zsolve_ex): every face with its own data, the
    corner ghosts carrying two faces' data."""
    torch = _torch()
    shape, L = (31, 63, 7), (1.0, 1.3, 0.9)
    Nx, Ny, Nz = shape
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 91 + order + 3 * sides[0] + sides[1])
    rs = np.random.RandomState(5 + order)
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    sd = [cr(Nz + 2, Ny + 2) if sides[0] == NEU else None,
          cr(Nz + 2, Ny + 2) if sides[0] == NEU else None,
          cr(Nz + 2, Nx + 2) if sides[1] == NEU else None,
          cr(Nz + 2, Nx + 2) if sides[1] == NEU else None]
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    s = H.ZSolver(Nx, Ny, Nz, *L, order)
    try:
        s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
        u = torch.full((2, Nz + 2, ny, nx), np.nan, dtype=torch.float64, device="cuda")
        sdd = [None if a is None else _planar(torch, a) for a in sd]
        s.solve(_planar(torch, f), u, _planar(torch, g_lo), _planar(torch, g_hi), side_data=sdd)
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        got = uc[0] + 1j * uc[1]
        with pytest.raises(H.HsError):   # data on a Dirichlet axis' faces
            bad = [None, None, None, None]
            k = 0 if sides[0] == DIRS else (2 if sides[1] == DIRS else None)
            if k is None:
                raise H.HsError(H.HS_ERR_INVALID_ARG, "no Dirichlet axis here")
            bad[k] = _planar(torch, cr(Nz + 2, (Ny if k < 2 else Nx) + 2))
            s.solve(_planar(torch, f), u, side_data=bad)
    finally:
        s.close()
    assert O.max_rel_diff(got, ref) <= TOL


DN, ND = CX.SIDE_DN, CX.SIDE_ND
MIXED = [(DN, DIRS), (ND, DIRS), (DIRS, DN), (DIRS, ND), (DN, ND), (ND, DN), (DN, NEU),
         (NEU, ND)]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", MIXED)
@pytest.mark.parametrize("faces", [(R, R), (D, D), (D, R)])
@pytest.mark.parametrize("shape", [(31, 63, 9), (63, 31, 4)])
def test_mixed_sides_match_oracle(order, sides, faces, shape):
    """One Dirichlet and one Neumann face on an axis: quarter-wave transforms (the
    extended lines of 2N + 1 points: 127 and 63 here) beside every other kind."""
    L = (1.0, 0.8, 1.1)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, sum(shape) + 5 * sides[0] + sides[1])
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides)
    got = _gpu(shape, L, order, K, zf, f, g_lo, g_hi, sides)
    assert O.max_rel_diff(got, ref) <= TOL


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(DN, ND), (ND, NEU), (NEU, DN), (DIRS, ND)])
def test_mixed_face_data_match_oracle(order, sides):
    """u_n = g on the Neumann face of each mixed axis (the high face of DN, the low face
    of ND) with data; data on its Dirichlet face are rejected."""
    torch = _torch()
    shape, L = (31, 63, 7), (1.0, 1.3, 0.9)
    Nx, Ny, Nz = shape
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 17 + order + 5 * sides[0] + sides[1])
    rs = np.random.RandomState(9 + order)
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    neu_face = [sides[0] in (NEU, ND), sides[0] in (NEU, DN), sides[1] in (NEU, ND),
                sides[1] in (NEU, DN)]
    sd = [cr(Nz + 2, (Ny if k < 2 else Nx) + 2) if neu_face[k] else None for k in range(4)]
    zf = CX.ZFaces(R, 1.0 + 0.5j, 2.0 - 1.0j, D)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides, sd)
    s = H.ZSolver(Nx, Ny, Nz, *L, order)
    try:
        s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
        u = torch.full((2, Nz + 2, ny, nx), np.nan, dtype=torch.float64, device="cuda")
        sdd = [None if a is None else _planar(torch, a) for a in sd]
        s.solve(_planar(torch, f), u, _planar(torch, g_lo), _planar(torch, g_hi), side_data=sdd)
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        got = uc[0] + 1j * uc[1]
        for k in range(4):   # every Dirichlet face rejects data
            if neu_face[k]:
                continue
            bad = [None, None, None, None]
            bad[k] = _planar(torch, cr(Nz + 2, (Ny if k < 2 else Nx) + 2))
            with pytest.raises(H.HsError) as e:
                s.solve(_planar(torch, f), u, side_data=bad)
            assert e.value.status == H.HS_ERR_INVALID_ARG
    finally:
        s.close()
    assert O.max_rel_diff(got, ref) <= TOL


def test_mixed_255():
    """255 x 255 x 127 with a DN x-axis and an ND y-axis (extended lines of 511 points),
    Robin z-faces, face data on both Neumann faces."""
    torch = _torch()
    shape, L = (255, 255, 127), (1.0, 1.0, 0.5)
    Nx, Ny, Nz = shape
    sides = (DN, ND)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 99)
    rs = np.random.RandomState(12)
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    sd = [None, cr(Nz + 2, Ny + 2), cr(Nz + 2, Nx + 2), None]
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, R, 1.0 + 0.5j, 3.0 - 1.0j)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi, sides, sd)
    s = H.ZSolver(Nx, Ny, Nz, *L, 4)
    try:
        s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        u = torch.full((2, Nz + 2, Ny + 1, Nx + 1), np.nan, dtype=torch.float64, device="cuda")
        s.solve(_planar(torch, f), u, _planar(torch, g_lo), _planar(torch, g_hi),
                side_data=[None if a is None else _planar(torch, a) for a in sd])
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
    finally:
        s.close()
    assert O.max_rel_diff(uc[0] + 1j * uc[1], ref) <= TOL



def _case6(shape, seed):
    """Order 6 (uniform h): box ((N_a + 1) h); complex K(z) with its derivatives K_z,
    K_zz; complex f and six face arrays f_nn."""
    Nx, Ny, Nz = shape
    rs = np.random.RandomState(seed)
    hh = 1.0 / (max(shape) + 1)
    L = tuple((n + 1) * hh for n in shape)
    z = np.arange(Nz + 2) * hh
    c = (30.0 + 5.0 * rs.uniform()) * (1.0 + 0.2j)
    K = c * (1.0 + 0.5 * z + 0.3 * z * z)
    Kz = c * (0.5 + 0.6 * z)
    Kzz = c * 0.6 + 0.0 * z
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    f = cr(Nz + 2, Ny + 2, Nx + 2)
    fnn = [cr(Nz + 2, Ny + 2), cr(Nz + 2, Ny + 2), cr(Nz + 2, Nx + 2), cr(Nz + 2, Nx + 2),
           cr(Ny + 2, Nx + 2), cr(Ny + 2, Nx + 2)]
    return (hh, hh, hh), L, K, Kz, Kzz, f, fnn, cr


def _gpu6(shape, L, K, Kz, Kzz, zf, f, g_lo, g_hi, fnn):
    torch = _torch()
    Nx, Ny, Nz = shape
    s = H.ZSolver(Nx, Ny, Nz, *L, 6)
    try:
        s.set_coeff6(K, Kz, Kzz)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        u = torch.full((2, Nz + 2, Ny, Nx), np.nan, dtype=torch.float64, device="cuda")
        s.solve(_planar(torch, f), u, _planar(torch, g_lo), _planar(torch, g_hi),
                fnn=None if fnn is None else [None if a is None else _planar(torch, a) for a in fnn])
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        return uc[0] + 1j * uc[1]
    finally:
        s.close()


@pytest.mark.parametrize("faces", [(R, R), (D, D), (R, D), (D, R)])
@pytest.mark.parametrize("shape", [(15, 15, 15), (31, 23, 13), (9, 40, 27)])
def test_order6_complex_matches_oracle(faces, shape):
    """6th-order rows (Section 3.4) in complex arithmetic, R6 with the complex K terms
    and f_nn ghosts on all six faces, Robin or Dirichlet z-faces: GPU vs oracle."""
    h, L, K, Kz, Kzz, f, fnn, cr = _case6(shape, sum(shape) + 7 * faces[0] + faces[1])
    Nx, Ny, Nz = shape
    g_lo, g_hi = cr(Ny, Nx), cr(Ny, Nx)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    got = _gpu6(shape, L, K, Kz, Kzz, zf, f, g_lo, g_hi, fnn)
    assert O.max_rel_diff(got, ref) <= TOL


def test_order6_complex_without_face_data_and_errors():
    """fnn absent (zero face data) at 63 x 63 x 31 with Robin faces; the order-6 plan
    refuses K without its derivatives and Neumann side faces."""
    torch = _torch()
    shape = (63, 63, 31)
    h, L, K, Kz, Kzz, f, _, cr = _case6(shape, 5)
    Nx, Ny, Nz = shape
    g_lo, g_hi = cr(Ny, Nx), cr(Ny, Nx)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, R, 1.0 + 0.5j, 3.0 - 1.0j)
    ref, _ = CX.solve(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz)
    got = _gpu6(shape, L, K, Kz, Kzz, zf, f, g_lo, g_hi, None)
    assert O.max_rel_diff(got, ref) <= TOL
    s = H.ZSolver(Nx, Ny, Nz, *L, 6)
    try:
        with pytest.raises(H.HsError) as e:
            s.set_coeff(K)
        assert e.value.status == H.HS_ERR_INVALID_ARG
        with pytest.raises(H.HsError) as e:
            s.set_sides(H.HS_SIDE_NEUMANN, H.HS_SIDE_DIRICHLET)
        assert e.value.status == H.HS_ERR_UNSUPPORTED
    finally:
        s.close()


def test_order6_complex_127():
    """127^3, 6th order, Robin faces, face data on all six faces."""
    shape = (127, 127, 127)
    h, L, K, Kz, Kzz, f, fnn, cr = _case6(shape, 127)
    g_lo, g_hi = cr(127, 127), cr(127, 127)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, D)
    ref, _ = CX.solve(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    got = _gpu6(shape, L, K, Kz, Kzz, zf, f, g_lo, g_hi, fnn)
    assert O.max_rel_diff(got, ref) <= TOL



MIXTOL = 1e-10


def _gpu_mixed(shape, L, order, K, zf, f, g_lo, g_hi, sweeps, Kz=None, Kzz=None, fnn=None,
               sides=(0, 0), sd=None):
    torch = _torch()
    Nx, Ny, Nz = shape
    s = H.ZSolver(Nx, Ny, Nz, *L, order)
    try:
        if order == 6:
            s.set_coeff6(K, Kz, Kzz)
        else:
            s.set_coeff(K)
        s.set_faces(zf.lo, zf.alpha[0], zf.beta[0], zf.hi, zf.alpha[1], zf.beta[1])
        s.set_sides(*sides)
        s.set_precision(H.HS_MIXED, sweeps)
        nx, ny = _nu(Nx, sides[0]), _nu(Ny, sides[1])
        u = torch.full((2, Nz + 2, ny, nx), np.nan, dtype=torch.float64, device="cuda")
        s.solve(_planar(torch, f), u, None if g_lo is None else _planar(torch, g_lo),
                None if g_hi is None else _planar(torch, g_hi),
                fnn=None if fnn is None else [None if a is None else _planar(torch, a) for a in fnn],
                side_data=None if sd is None else [None if a is None else _planar(torch, a)
                                                   for a in sd])
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        return uc[0] + 1j * uc[1]
    finally:
        s.close()


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("shape", [(31, 20, 17), (63, 40, 12), (127, 95, 33)])
def test_mixed_precision_complex_matches_oracle(order, faces, shape):
    """HS_MIXED: FP32 solves refined with FP64 residuals; one sweep reaches the mixed
    bar against the oracle, and the unrefined solve is FP32-accurate (printed)."""
    L = (1.0, 0.9, 1.2)
    h, K, f, g_lo, g_hi = _case(shape, L, sum(shape) + order + 11)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi)
    e0 = O.max_rel_diff(_gpu_mixed(shape, L, order, K, zf, f, g_lo, g_hi, 0), ref)
    e1 = O.max_rel_diff(_gpu_mixed(shape, L, order, K, zf, f, g_lo, g_hi, 1), ref)
    print(f"mixed complex {shape} order {order} faces {faces}: unrefined {e0:.2e}, one sweep {e1:.2e}")
    assert e0 <= 1e-4
    assert e1 <= MIXTOL


@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("Nz", [1, 2, 3, 4])
def test_mixed_precision_complex_thin(faces, Nz):
    """Thin boxes, where the mixed plan's right-hand side has no rows away from both
    z ends (those rows are formed in pair arithmetic, the two rows at each end in
    FP64): one sweep still meets the mixed bar against the oracle."""
    shape, L = (15, 12, Nz), (1.0, 0.9, 0.3)
    h, K, f, g_lo, g_hi = _case(shape, L, 7 * Nz + faces[0] + 2 * faces[1])
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi)
    got = _gpu_mixed(shape, L, 4, K, zf, f, g_lo, g_hi, 1)
    assert O.max_rel_diff(got, ref) <= MIXTOL


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sides", [(NEU, DIRS), (DIRS, NEU), (NEU, NEU)])
@pytest.mark.parametrize("faces", [(R, R), (D, R)])
@pytest.mark.parametrize("shape", [(31, 63, 9), (63, 31, 4)])
def test_mixed_precision_neumann_sides(order, sides, faces, shape):
    """HS_MIXED with u_n = 0 on Neumann side faces: FP32 cosine tiles for those axes
    and even reflection in the pair residual; one sweep meets the mixed bar against
    the oracle."""
    L = (1.0, 0.8, 1.1)
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, sum(shape) + 3 * sides[0] + sides[1] + order)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(order, h, K, zf, f, g_lo, g_hi, sides)
    got = _gpu_mixed(shape, L, order, K, zf, f, g_lo, g_hi, 1, sides=sides)
    assert O.max_rel_diff(got, ref) <= MIXTOL


@pytest.mark.parametrize("M", [32, 64, 96, 128, 192, 256, 384, 512, 768, 1024])
def test_mixed_precision_cosine_lengths(M):
    """Every length the FP32 cosine tile serves (N + 1 <= 256), along x and along y
    (thin boxes, Neumann on the long axis): the refined mixed solve equals the FP64
    plan's to the mixed bar, and the unrefined error grows no faster than (N + 1) eps
    (both printed).  Longer Neumann axes are refused in mixed precision: the tile's
    running sum lets the unrefined error grow past what one sweep corrects."""
    torch = _torch()
    if M > 256:
        s = H.ZSolver(M - 1, 9, 3, 1.0, 0.9, 0.4, 4)
        try:
            s.set_sides(H.HS_SIDE_NEUMANN, H.HS_SIDE_DIRICHLET)
            with pytest.raises(H.HsError) as e:
                s.set_precision(H.HS_MIXED, 1)
            assert e.value.status == H.HS_ERR_UNSUPPORTED
        finally:
            s.close()
        return
    for shape, sides in (((M - 1, 9, 3), (NEU, DIRS)), ((7, M - 1, 3), (DIRS, NEU))):
        L = (1.0, 0.9, 0.4)
        h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, M + sides[0])
        zf = CX.ZFaces(R, 1.0 + 0.5j, 2.0 - 1.0j, D)
        ref = _gpu(shape, L, 4, K, zf, f, g_lo, g_hi, sides)
        e0 = O.max_rel_diff(_gpu_mixed(shape, L, 4, K, zf, f, g_lo, g_hi, 0, sides=sides), ref)
        e1 = O.max_rel_diff(_gpu_mixed(shape, L, 4, K, zf, f, g_lo, g_hi, 1, sides=sides), ref)
        print(f"cosine M={M} shape={shape}: unrefined {e0:.2e}, one sweep {e1:.2e}")
        assert e0 <= 40 * M * 2.0 ** -24
        assert e1 <= MIXTOL


@pytest.mark.parametrize("sides", [(NEU, DIRS), (NEU, NEU)])
def test_mixed_precision_neumann_face_data(sides):
    """HS_MIXED with u_n = g data on the Neumann side faces (the data enter F in FP64;
    the refinement's residual reflects U): one sweep meets the mixed bar."""
    shape, L = (31, 63, 7), (1.0, 1.3, 0.9)
    Nx, Ny, Nz = shape
    h, K, f, g_lo, g_hi = _neumann_case(shape, L, sides, 23 + 5 * sides[0] + sides[1])
    rs = np.random.RandomState(29)
    cr = lambda *sh: rs.uniform(-1, 1, sh) + 1j * rs.uniform(-1, 1, sh)
    neu_face = [sides[0] == NEU, sides[0] == NEU, sides[1] == NEU, sides[1] == NEU]
    sd = [cr(Nz + 2, (Ny if k < 2 else Nx) + 2) if neu_face[k] else None for k in range(4)]
    zf = CX.ZFaces(R, 1.0 + 0.5j, 2.0 - 1.0j, D)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi, sides, sd)
    got = _gpu_mixed(shape, L, 4, K, zf, f, g_lo, g_hi, 1, sides=sides, sd=sd)
    assert O.max_rel_diff(got, ref) <= MIXTOL


@pytest.mark.parametrize("faces", [(R, R), (D, R)])
def test_mixed_precision_complex_order6(faces):
    shape = (31, 23, 13)
    h, L, K, Kz, Kzz, f, fnn, cr = _case6(shape, 41 + faces[0])
    Nx, Ny, Nz = shape
    g_lo, g_hi = cr(Ny, Nx), cr(Ny, Nx)
    zf = CX.ZFaces(faces[0], 1.0 + 0.5j, 2.0 - 1.0j, faces[1], -0.7 + 0.2j, 1.5 + 0.4j)
    ref, _ = CX.solve(6, h, K, zf, f, g_lo, g_hi, Kz=Kz, Kzz=Kzz, fnn=fnn)
    got = _gpu_mixed(shape, L, 6, K, zf, f, g_lo, g_hi, 2, Kz, Kzz, fnn)
    assert O.max_rel_diff(got, ref) <= MIXTOL


def test_mixed_precision_complex_255_and_errors():
    """255^3 Robin (the zrobin255_o4 recipe's shape) with one sweep; mixed precision
    refuses mixed side axes (no FP32 quarter-wave tile) and Neumann axes whose
    length has no compiled cosine tile, and those side kinds refuse mixed precision."""
    shape, L = (255, 255, 255), (1.0, 1.0, 1.0)
    h, K, f, g_lo, g_hi = _case(shape, L, 12)
    zf = CX.ZFaces(R, 1.0 + 0.5j, 3.0 - 1.0j, R, 1.0 + 0.5j, 3.0 - 1.0j)
    ref, _ = CX.solve(4, h, K, zf, f, g_lo, g_hi)
    got = _gpu_mixed(shape, L, 4, K, zf, f, g_lo, g_hi, 1)
    assert O.max_rel_diff(got, ref) <= MIXTOL
    s = H.ZSolver(31, 30, 7, 1.0, 1.0, 1.0, 4)
    try:
        s.set_sides(H.HS_SIDE_DN, H.HS_SIDE_DIRICHLET)
        with pytest.raises(H.HsError) as e:
            s.set_precision(H.HS_MIXED, 1)
        assert e.value.status == H.HS_ERR_UNSUPPORTED
        s.set_sides(H.HS_SIDE_DIRICHLET, H.HS_SIDE_NEUMANN)   # 31 + 1 points: no cosine tile
        with pytest.raises(H.HsError) as e:
            s.set_precision(H.HS_MIXED, 1)
        assert e.value.status == H.HS_ERR_UNSUPPORTED
        s.set_sides(H.HS_SIDE_NEUMANN, H.HS_SIDE_DIRICHLET)   # 32 + 1 points: compiled
        s.set_precision(H.HS_MIXED, 1)
        with pytest.raises(H.HsError) as e:
            s.set_sides(H.HS_SIDE_DIRICHLET, H.HS_SIDE_NEUMANN)
        assert e.value.status == H.HS_ERR_UNSUPPORTED
        s.set_sides(H.HS_SIDE_DIRICHLET, H.HS_SIDE_DIRICHLET)
        with pytest.raises(H.HsError) as e:
            s.set_sides(H.HS_SIDE_DN, H.HS_SIDE_DIRICHLET)
        assert e.value.status == H.HS_ERR_UNSUPPORTED
        with pytest.raises(H.HsError) as e:
            s.set_precision(H.HS_MIXED, 9)
        assert e.value.status == H.HS_ERR_INVALID_ARG
    finally:
        s.close()
