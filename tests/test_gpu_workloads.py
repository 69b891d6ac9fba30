"""GPU parity at the full sizes of the large workloads (one GPU).

* 1023^3, 6th order, k = 40 + 20 tanh(10 (z - 1/2)), f = 16 random sine modes:
  the exact discrete solution is known mode by mode (oracle.solve_sine_modes,
  itself pinned against the full oracle), so the FP64 and mixed paths are
  checked at 200k sampled points; with FP32-stored f the two GPU paths are
  compared with each other everywhere (the input rounding is common to both).
* 511^3, 4th-order convection-diffusion, gamma = 2 + sin(2 pi z), 8 right-hand
  sides U[-1, 1] stored in FP32, one multi-RHS solve per path: the first RHS
  against the full oracle, all eight between the two paths.
"""
import numpy as np
import pytest

import paper_1912_03565_gb300 as H
import workloads as W
from oracle import hs_oracle as O

pytestmark = pytest.mark.gpu


def _solve(torch, N, L, order, eq, precision, c, f, f_dtype, nrhs=1, sweeps=2,
           cd_variant=H.HS_CD_CORRECTED):
    s = H.Solver(N, N, N, L[0], L[1], L[2], order, eq, precision, max_rhs=nrhs)
    try:
        s.set_coeff(*c, cd_variant)
        if precision == H.HS_MIXED:
            H.hs_set_refinement(s.plan, sweeps)
        shape = (N, N, N) if nrhs == 1 else (nrhs, N, N, N)
        u = torch.empty(shape, dtype=torch.float64, device="cuda")
        s.solve(f, u, f_dtype, H.HS_RHS_NODAL, nrhs=nrhs)
        torch.cuda.synchronize()
        return u
    finally:
        s.close()


def _sine_mode_refs(N, modes, amps, c, pts):
    """The exact discrete solution at the sample points (extended precision) and
    the FP64 sine-mode solution's distance from it: the rounding any FP64 solve
    of this problem carries (its z-systems are ill conditioned)."""
    ext = O.solve_sine_modes_extended(modes, amps, N, *c, sample=pts)
    f64 = O.solve_sine_modes(modes, amps, (N, N, N), (1.0, 1.0, 1.0), 6, *c, sample=pts)
    scale = float(np.abs(ext).max())
    return ext, float(np.abs(f64 - ext).max()) / scale


def test_cube1023_sine_modes():
    """Parity bars against the exact discrete solution (extended precision): FP64
    path max(1e-12, 4 delta), refined mixed path max(1e-10, 4 delta), with delta the
    measured distance of the FP64 sine-mode solution from it -- the FP64 rounding
    floor of this problem (3.1e-11 on x86: the z-systems are ill conditioned, and the
    mixed path's FP64 residual refines towards an FP64-rounded solution too)."""
    torch = pytest.importorskip("torch")
    N = 1023
    modes, amps = W.sine_modes(N, 16, 4)
    K = W.k_profile_to_k2(W.k_tanh())
    c = K.sample(N, 1.0)
    rs = np.random.RandomState(0)
    pts = tuple(rs.randint(1, N + 1, size=200000) for _ in range(3))
    ref, delta = _sine_mode_refs(N, modes, amps, c, pts)
    idx = tuple(torch.from_numpy(a - 1).cuda() for a in (pts[2], pts[1], pts[0]))

    f64 = W.sine_mode_nodes_torch(N, modes, amps)
    errs, rho = {}, None
    for prec in (H.HS_FP64, H.HS_MIXED):
        s = H.Solver(N, N, N, 1.0, 1.0, 1.0, 6, H.HS_HELMHOLTZ, prec)
        try:
            s.set_coeff(*c)
            if prec == H.HS_MIXED:
                H.hs_set_refinement(s.plan, 2)
            u = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
            _, inf = s.solve(f64, u, H.HS_F64, H.HS_RHS_NODAL, info=True)
            torch.cuda.synchronize()
        finally:
            s.close()
        rho = inf["min_pivot_ratio"]
        scale = float(u.abs().max())
        got = u[idx].cpu().numpy()
        errs[prec] = float(np.max(np.abs(got - ref)) / scale)
        del u
    tol64 = max(1e-12, 4 * delta)
    msg = (f"1023^3: FP64 path {errs[H.HS_FP64]:.3e}, mixed {errs[H.HS_MIXED]:.3e} vs the "
           f"extended-precision solution; FP64 rounding floor delta {delta:.3e}; "
           f"min pivot ratio {rho:.3e}")
    print(msg)
    assert errs[H.HS_FP64] <= tol64, msg
    assert errs[H.HS_MIXED] <= max(1e-10, 4 * delta), msg

    # FP32-stored f (the workload as specified): both paths see the same input
    f32 = f64.float()
    del f64
    torch.cuda.empty_cache()
    u64 = _solve(torch, N, (1.0, 1.0, 1.0), 6, H.HS_HELMHOLTZ, H.HS_FP64, c, f32, H.HS_F32)
    umx = _solve(torch, N, (1.0, 1.0, 1.0), 6, H.HS_HELMHOLTZ, H.HS_MIXED, c, f32, H.HS_F32)
    scale = float(u64.abs().max())
    assert float((umx - u64).abs().max()) / scale <= 1e-10
    got = u64[idx].cpu().numpy()
    assert float(np.max(np.abs(got - ref)) / scale) <= 1e-5   # FP32 input rounding only


def test_sine_modes_255_near_singular():
    """The 1023^3 recipe at 255^3 (k = 40 + 20 tanh(10 (z - 1/2)): min pivot ratio
    1.9e-4), where the full O(N^4) oracle is affordable: the FP64 GPU path against
    the oracle and against the exact discrete solution, both at max(1e-12, 2 delta)
    with delta the FP64 sine-mode solution's distance from the exact one (measured
    here, 1.3e-12 on x86: two FP64 solves of this problem differ by that much);
    the refined mixed path at 1e-10."""
    torch = pytest.importorskip("torch")
    N = 255
    modes, amps = W.sine_modes(N, 16, 4)
    p = W.sine_mode_problem(N, 6, W.k_tanh(), nmodes=16, seed=4, dtype=np.float64)
    c = (p.c0, p.c1, p.c2)
    rs = np.random.RandomState(0)
    pts = tuple(rs.randint(1, N + 1, size=200000) for _ in range(3))
    ext, delta = _sine_mode_refs(N, modes, amps, c, pts)
    full, info = O.solve(p)
    f = torch.from_numpy(p.f_nodes).cuda()
    tol = max(1e-12, 2 * delta)
    for prec, bar in ((H.HS_FP64, tol), (H.HS_MIXED, 1e-10)):
        u = _solve(torch, N, (1.0, 1.0, 1.0), 6, H.HS_HELMHOLTZ, prec, c, f, H.HS_F64).cpu().numpy()
        e_full = O.max_rel_diff(u, full)
        got = u[pts[2] - 1, pts[1] - 1, pts[0] - 1]
        e_ext = float(np.max(np.abs(got - ext)) / np.abs(ext).max())
        msg = (f"255^3 precision {prec}: vs oracle {e_full:.3e}, vs exact {e_ext:.3e}, "
               f"delta {delta:.3e}, min pivot ratio {info['min_pivot_ratio']:.2e}")
        print(msg)
        assert e_full <= bar and e_ext <= bar, msg


def test_convdiff511_eight_rhs():
    torch = pytest.importorskip("torch")
    N, R = 511, 8
    probs = [W.workload_convdiff511(r) for r in range(R)]
    c = (probs[0].c0, probs[0].c1, probs[0].c2)
    f = torch.from_numpy(np.stack([p.f_nodes.astype(np.float32) for p in probs])).cuda()
    L = (1.0, 1.0, 1.0)
    u64 = _solve(torch, N, L, 4, H.HS_CONVDIFF, H.HS_FP64, c, f, H.HS_F32, nrhs=R)
    umx = _solve(torch, N, L, 4, H.HS_CONVDIFF, H.HS_MIXED, c, f, H.HS_F32, nrhs=R)
    for r in range(R):
        scale = float(u64[r].abs().max())
        assert float((umx[r] - u64[r]).abs().max()) / scale <= 1e-10, r
    ref, _ = O.solve(probs[0])   # f already FP32-valued
    assert O.max_rel_diff(u64[0].cpu().numpy(), ref) <= 1e-12
    assert O.max_rel_diff(umx[0].cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("pid", [0, 60])
def test_batch64_ill_conditioned_problems(pid):
    """The batch64 problems closest to singular (problem ids 0 and 60 of the seeded
    workload: min pivot ratio 3.7e-5 and 1.2e-5), right-hand side 0 with FP32 f.
    Two FP64 solvers -- the GPU FP64 path and the oracle -- differ here by delta
    (measured in the test; 8.9e-10 and 6.1e-12 when first measured): the FP64
    rounding floor of these problems.  The refined mixed path (automatic residual
    precision: FP64 residuals only after a pair residual stopped shrinking; stop at
    ||r|| / ||F|| <= 1e-11, at most 4 sweeps) is held to max(1e-10, 4 delta)
    against the oracle."""
    torch = pytest.importorskip("torch")
    spec = W.workload_batch_specs(64, 3)[pid]
    p = W.batch_problem(spec, 0)
    ref, oinfo = O.solve(p)
    f = torch.from_numpy(p.f_nodes.astype(np.float32)).cuda()
    out = {}
    for prec in (H.HS_FP64, H.HS_MIXED):
        s = H.Solver(p.Nx, p.Ny, p.Nz, p.Lx, p.Ly, p.Lz, 6, H.HS_HELMHOLTZ, prec)
        try:
            s.set_coeff(p.c0, p.c1, p.c2)
            if prec == H.HS_MIXED:
                H.hs_set_refinement(s.plan, 4)
                H.hs_set_refinement_tol(s.plan, 1e-11)
            u = torch.zeros((p.Nz, p.Ny, p.Nx), dtype=torch.float64, device="cuda")
            s.solve(f, u, H.HS_F32, H.HS_RHS_NODAL)
            torch.cuda.synchronize()
            out[prec] = u.cpu().numpy()
        finally:
            s.close()
    delta = O.max_rel_diff(out[H.HS_FP64], ref)
    e_mix = O.max_rel_diff(out[H.HS_MIXED], ref)
    msg = (f"batch64 problem {pid} {spec['N']}: FP64 GPU vs oracle {delta:.3e}, mixed vs "
           f"oracle {e_mix:.3e}, min pivot ratio {oinfo['min_pivot_ratio']:.2e}")
    print(msg)
    assert oinfo["min_pivot_ratio"] < 1e-4, msg
    assert e_mix <= max(1e-10, 4 * delta), msg
    assert delta <= 1e-8, msg   # a gross FP64 error would still show
