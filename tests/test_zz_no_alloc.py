"""hs_residual_static, the entry point that allocates nothing, against hs_residual (GPU).

Callers that cannot call cudaMalloc (their device memory belongs to a pool
allocator or framework, or they may only touch the buffers they are handed)
use hs_residual_static to get ||F - A U||_2 and ||F||_2 without a plan.  Its
scratch is a fixed file-scope device array shared by every call, so the test
makes two calls in a row (the second sees the first call's leftovers) and
compares both with the plan-based hs_residual at the FP64 tolerance of the
other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle.hs_oracle as O
import paper_1912_03565_gb300 as H
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _case(shape, order, equation, seed):
    rs = np.random.RandomState(seed)
    Nx, Ny, Nz = shape
    if order == 6:
        h = 1.0 / (max(shape) + 1)
        L = ((Nx + 1) * h, (Ny + 1) * h, (Nz + 1) * h)
        prof = W.k_profile_to_k2(W.k_linear(rs.uniform(5, 30), rs.uniform(0, 1)))
    elif equation == H.HS_CONVDIFF:
        L = (1.0, 0.9, 1.1)
        prof = W.gamma_2_sin2pi()
    else:
        L = (1.0, 0.9, 1.1)
        prof = W.k_profile_to_k2(W.k_10_5sin())
    c0, c1, c2 = prof.sample(Nz, L[2])
    F = rs.standard_normal((Nz, Ny, Nx))
    u = rs.standard_normal((Nz, Ny, Nx))
    return dict(shape=shape, L=L, order=order, eq=equation, c=(c0, c1, c2), F=F, u=u)


def _plan_residual(cs, Fd, ud):
    Nx, Ny, Nz = cs["shape"]
    s = H.Solver(Nx, Ny, Nz, *cs["L"], cs["order"], cs["eq"], H.HS_FP64)
    try:
        s.set_coeff(*cs["c"], H.HS_CD_CORRECTED)
        return H.hs_residual(s.plan, Fd, H.HS_F64, H.HS_RHS_ASSEMBLED, None, ud)
    finally:
        s.close()


def _oracle_residual(cs):
    """||A U - F||_2 and ||F||_2 from the FP64 CPU oracle (zero Dirichlet data)."""
    Nx, Ny, Nz = cs["shape"]
    h = O.grid_steps((Nx, Ny, Nz), cs["L"])
    C = O.stencil_coefficients(cs["order"], cs["eq"], h, *cs["c"], cd_variant=O.CD_CORRECTED)
    return O.residual_l2(C, cs["u"], cs["F"]), float(np.linalg.norm(cs["F"]))


def _static_residual(cs, Fd, ud):
    Nx, Ny, Nz = cs["shape"]
    return H.hs_residual_static(Nx, Ny, Nz, *cs["L"], cs["order"], cs["eq"], H.HS_CD_CORRECTED,
                                *cs["c"], Fd, ud)


def test_static_residual_matches_plan_residual_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    cases = [_case((40, 33, 27), 6, H.HS_HELMHOLTZ, 1),
             _case((17, 29, 9), 4, H.HS_CONVDIFF, 2)]
    dev = []
    for cs in cases:
        Fd = torch.from_numpy(cs["F"]).cuda()
        ud = torch.from_numpy(cs["u"]).cuda()
        dev.append((Fd, ud, _plan_residual(cs, Fd, ud)))
    torch.cuda.synchronize()
    # first call on this device (sets up the scratch address), then two more
    # calls in a row that must not change the device's free memory
    _static_residual(cases[0], dev[0][0], dev[0][1])
    for k, (cs, (Fd, ud, ref)) in enumerate(zip(cases, dev)):
        free0 = torch.cuda.mem_get_info()[0]
        res, fn = _static_residual(cs, Fd, ud)
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, f"call {k} changed free device memory"
        assert res == pytest.approx(ref[0], rel=TOL64)
        assert fn == pytest.approx(ref[1], rel=TOL64)
        ores, ofn = _oracle_residual(cs)
        assert res == pytest.approx(ores, rel=TOL64)
        assert fn == pytest.approx(ofn, rel=TOL64)
        assert res > 0.1 * fn  # u is not a solution: the residual is O(1)
    # the first case again, after the second one left its data in the scratch
    res, fn = _static_residual(cases[0], dev[0][0], dev[0][1])
    assert res == pytest.approx(dev[0][2][0], rel=TOL64)
    assert fn == pytest.approx(dev[0][2][1], rel=TOL64)


def test_static_residual_of_a_solution_is_small():
    torch = pytest.importorskip("torch")
    cs = _case((31, 31, 31), 6, H.HS_HELMHOLTZ, 3)
    Nx, Ny, Nz = cs["shape"]
    Fd = torch.from_numpy(cs["F"]).cuda()
    ud = torch.zeros_like(Fd)
    s = H.Solver(Nx, Ny, Nz, *cs["L"], 6, H.HS_HELMHOLTZ, H.HS_FP64)
    try:
        s.set_coeff(*cs["c"])
        s.solve(Fd, ud, H.HS_F64, H.HS_RHS_ASSEMBLED)
        torch.cuda.synchronize()
    finally:
        s.close()
    res, fn = _static_residual(cs, Fd, ud)
    assert res < 1e-12 * fn


@pytest.mark.parametrize("order,eq", [(6, H.HS_HELMHOLTZ), (4, H.HS_CONVDIFF)])
def test_static_residual_across_coefficient_chunks(order, eq):
    """Nz = 300: the coefficient table is built in chunks of 128 rows, so rows
    128/129 and 256/257 straddle chunk boundaries (each chunk starts its profile
    arrays at its own first row)."""
    torch = pytest.importorskip("torch")
    cs = _case((5, 4, 300), order, eq, 7)
    Fd = torch.from_numpy(cs["F"]).cuda()
    ud = torch.from_numpy(cs["u"]).cuda()
    ref = _plan_residual(cs, Fd, ud)
    for _ in range(2):
        res, fn = _static_residual(cs, Fd, ud)
        assert res == pytest.approx(ref[0], rel=TOL64)
        assert fn == pytest.approx(ref[1], rel=TOL64)
    ores, _ = _oracle_residual(cs)
    assert res == pytest.approx(ores, rel=TOL64)


def test_static_residual_rejects_what_it_cannot_hold():
    torch = pytest.importorskip("torch")
    Fd = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    big = torch.zeros((H.HS_STATIC_MAX_NZ + 1, 2, 2), dtype=torch.float64, device="cuda")
    c = np.full(H.HS_STATIC_MAX_NZ + 3, 25.0)
    with pytest.raises(H.HsError) as e:
        H.hs_residual_static(2, 2, H.HS_STATIC_MAX_NZ + 1, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ,
                             H.HS_CD_CORRECTED, c, None, None, big, big)
    assert e.value.status == H.HS_ERR_UNSUPPORTED
    # order 6 needs one spacing on all axes, as a plan does
    c4 = np.full(4, 25.0)
    with pytest.raises(H.HsError) as e:
        H.hs_residual_static(2, 2, 2, 1.0, 1.1, 1.0, 6, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             c4, np.zeros(4), np.zeros(4), Fd, Fd)
    assert e.value.status == H.HS_ERR_INVALID_ARG
    # non-finite coefficients
    bad = c4.copy()
    bad[2] = np.nan
    with pytest.raises(H.HsError) as e:
        H.hs_residual_static(2, 2, 2, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             bad, None, None, Fd, Fd)
    assert e.value.status == H.HS_ERR_NONFINITE
    # sizes and types the bare pointers cannot carry are checked by the binding
    with pytest.raises(ValueError):
        H.hs_residual_static(2, 2, 2, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             c4[:3], None, None, Fd, Fd)
    with pytest.raises(ValueError):
        H.hs_residual_static(2, 2, 2, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             c4, None, None, Fd.float(), Fd)
    with pytest.raises(ValueError):
        H.hs_residual_static(2, 2, 3, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             np.full(5, 25.0), None, None, Fd, Fd)
    host = np.zeros((2, 2, 2))
    with pytest.raises(H.HsError) as e:
        H.hs_residual_static(2, 2, 2, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                             c[:4], None, None, host, host)
    assert e.value.status == H.HS_ERR_INVALID_ARG


def test_static_residual_refuses_a_capturing_stream():
    """Every call copies from host memory and synchronises, which a stream
    capture cannot hold: a capturing stream is refused before any of that."""
    torch = pytest.importorskip("torch")
    cs = _case((9, 8, 7), 4, H.HS_HELMHOLTZ, 4)
    Fd = torch.from_numpy(cs["F"]).cuda()
    ud = torch.from_numpy(cs["u"]).cuda()
    _static_residual(cs, Fd, ud)   # the device's scratch address is set up outside capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(side):
        g.capture_begin(capture_error_mode="relaxed")
        try:
            H.hs_residual_static(*cs["shape"], *cs["L"], 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                                 *cs["c"], Fd, ud, stream=side)
        except H.HsError as e:
            status = e.status
        finally:
            g.capture_end()
    assert status == H.HS_ERR_INVALID_ARG
    res, _ = _static_residual(cs, Fd, ud)   # the library is still usable
    assert res > 0
