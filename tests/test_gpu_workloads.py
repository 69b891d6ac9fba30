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


def test_cube1023_sine_modes():
    torch = pytest.importorskip("torch")
    N = 1023
    modes, amps = W.sine_modes(N, 16, 4)
    K = W.k_profile_to_k2(W.k_tanh())
    c = K.sample(N, 1.0)
    rs = np.random.RandomState(0)
    pts = tuple(rs.randint(1, N + 1, size=200000) for _ in range(3))
    ref = O.solve_sine_modes(modes, amps, (N, N, N), (1.0, 1.0, 1.0), 6, *c, sample=pts)
    idx = tuple(torch.from_numpy(a - 1).cuda() for a in (pts[2], pts[1], pts[0]))

    f64 = W.sine_mode_nodes_torch(N, modes, amps)
    errs = {}
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
    # FP64 bar: 1e-12, or the rounding limit of a transform-based FP64 solve when
    # the z-systems are closer to singular: 4 eps log2(M) / (min pivot ratio)
    tol64 = max(1e-12, 4 * np.finfo(np.float64).eps * np.log2(N + 1) / rho)
    assert errs[H.HS_FP64] <= tol64, (errs, tol64)
    assert errs[H.HS_MIXED] <= 1e-10, errs

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
