"""The lifted right-hand side F as the solver forms it (hs_rhs_apply) against the oracle.

F is the first stage of every solve (eqs. scheme4, scheme6, cd_rhs and the
Dirichlet lifting of eq. (bc)).  The mixed path forms it as an FP32 pair
(hi + lo) in error-free pair arithmetic; the FP64 path in FP64.  Both are
compared element by element with oracle.assemble_rhs on the same input:

* FP64 plan: max |F_gpu - F_oracle| <= 1e-14 max |F_oracle| (FP64 rounding of
  a 25-point sum);
* mixed plan: max |(hi + lo) - F_oracle| <= 2e-13 max |F_oracle| (the pair
  arithmetic rounds at about 2^-46 of its largest intermediate, which is a few
  times max |F|).

Shapes are ragged against the mixed kernel's 32 x 8 x 32 tiles and include
tiles that touch no face (the kernel's plain-load path) as well as face tiles
(ghost nodes, boundary values).  Inputs: f ~ U[-1, 1] on every node, random
Dirichlet faces and (6th order) random face second derivatives, or none.
"""
import numpy as np
import pytest

import paper_1912_03565_gb300 as H
import workloads as W
from oracle import hs_oracle as O

pytestmark = pytest.mark.gpu

SHAPES = [(37, 13, 70), (70, 20, 33), (70, 40, 9), (5, 4, 3), (1, 2, 1)]
CASES = [(6, W.HELMHOLTZ), (4, W.HELMHOLTZ), (2, W.HELMHOLTZ), (4, W.CONVDIFF)]


def _problem(shape, order, eq, seed, faces):
    rs = np.random.RandomState(seed)
    Nx, Ny, Nz = shape
    if order == 6:
        h = 1.0 / (max(shape) + 1)
        L = ((Nx + 1) * h, (Ny + 1) * h, (Nz + 1) * h)
    else:
        L = (1.0, 0.8, 1.2)
    if eq == W.HELMHOLTZ:
        prof = W.k_profile_to_k2(W.k_linear(rs.uniform(10, 60), rs.uniform(0, 1)))
    else:
        g = rs.uniform(-30, 30)
        prof = W.Profile(lambda z: g + 3 * np.sin(2 * np.pi * z),
                         lambda z: 6 * np.pi * np.cos(2 * np.pi * z),
                         lambda z: -12 * np.pi ** 2 * np.sin(2 * np.pi * z))
    p = W.random_interior_problem(shape, L, order, eq, prof, seed)
    p.f_nodes = rs.uniform(-1, 1, p.f_nodes.shape)
    if faces:
        p.faces = W.faces_from_nodes(rs.uniform(-1, 1, p.f_nodes.shape))
        if order == 6:
            p.fnn = W.faces_from_nodes(rs.uniform(-1, 1, p.f_nodes.shape))
    return p


def _gpu_rhs(p, precision, f_dtype):
    import torch
    eq = H.HS_CONVDIFF if p.equation == W.CONVDIFF else H.HS_HELMHOLTZ
    npdt = np.float64 if f_dtype == H.HS_F64 else np.float32
    tdev = lambda a: None if a is None else torch.from_numpy(
        np.ascontiguousarray(a.astype(npdt))).cuda()
    s = H.Solver(p.Nx, p.Ny, p.Nz, p.Lx, p.Ly, p.Lz, p.order, eq, precision)
    try:
        s.set_coeff(p.c0, p.c1, p.c2, H.HS_CD_CORRECTED)
        f = tdev(p.f_nodes)
        faces = [tdev(a) for a in p.faces]
        fnn = [tdev(a) for a in p.fnn]
        b = H.make_boundary(faces, fnn)
        shape = (p.Nz, p.Ny, p.Nx)
        if precision == H.HS_MIXED:
            F = torch.full((2,) + shape, np.nan, dtype=torch.float32, device="cuda")
        else:
            F = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
        H.hs_rhs_apply(s.plan, f, f_dtype, H.HS_RHS_NODAL, b, F)
        torch.cuda.synchronize()
        if precision == H.HS_MIXED:
            return F[0].double().cpu().numpy() + F[1].double().cpu().numpy()
        return F.cpu().numpy()
    finally:
        s.close()


def _oracle_rhs(p, f_dtype):
    rd = (lambda a: a) if f_dtype == H.HS_F64 else (
        lambda a: None if a is None else a.astype(np.float32).astype(np.float64))
    C = O.stencil_coefficients(p.order, p.equation, p.h, p.c0, p.c1, p.c2,
                               cd_variant=O.CD_CORRECTED)
    faces = [rd(a) for a in p.faces]
    fnn = [rd(a) for a in p.fnn]
    return O.assemble_rhs(p.order, p.equation, p.h, rd(p.f_nodes), C, p.c0, p.c1,
                          faces, fnn)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("order,eq", CASES)
@pytest.mark.parametrize("f_dtype", [H.HS_F64, H.HS_F32])
@pytest.mark.parametrize("faces", [True, False])
def test_rhs_matches_oracle(shape, order, eq, f_dtype, faces):
    p = _problem(shape, order, eq, 17 + order + 3 * eq, faces)
    ref = _oracle_rhs(p, f_dtype)
    scale = np.abs(ref).max()
    for precision, tol in ((H.HS_FP64, 1e-14), (H.HS_MIXED, 2e-13)):
        got = _gpu_rhs(p, precision, f_dtype)
        assert np.isfinite(got).all(), precision
        err = np.abs(got - ref).max() / scale
        assert err <= tol, (precision, err)


def test_rhs_apply_rejects_host_pointers_and_missing_coefficients():
    import torch
    s = H.Solver(8, 8, 8, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_MIXED)
    try:
        f = torch.zeros((10, 10, 10), dtype=torch.float64, device="cuda")
        F = torch.zeros((2, 8, 8, 8), dtype=torch.float32, device="cuda")
        with pytest.raises(H.HsError) as e:
            H.hs_rhs_apply(s.plan, f, H.HS_F64, H.HS_RHS_NODAL, None, F)
        assert e.value.status == H.HS_ERR_NO_COEFF
        s.set_coeff(np.full(10, 25.0))
        with pytest.raises(H.HsError) as e:
            H.hs_rhs_apply(s.plan, f.cpu().numpy(), H.HS_F64, H.HS_RHS_NODAL, None, F)
        assert e.value.status == H.HS_ERR_INVALID_ARG
    finally:
        s.close()
