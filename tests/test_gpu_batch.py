"""The batched persistent launch (hs_batch_*) on the GPU.

Uneven 6th-order problems with their own k(z) and 1-3 right-hand sides each,
FP32 f, solved in one graph launch; every (problem, RHS) result is compared
with the stand-alone mixed solve of the same problem (same tile code, so the
results agree to rounding) and, for some, with the CPU oracle.  A forced
stall (a dependency that can never be met) must end the launch with
HS_ERR_TIMEOUT inside the wait limit and leave the context usable.
"""
import numpy as np
import pytest

import paper_1912_03565_gb300 as H
import workloads as W
from oracle import hs_oracle as O

pytestmark = pytest.mark.gpu


def _specs(seed=11, n=6, sizes=(31, 63, 95)):
    return W.workload_batch_specs(nprob=n, seed=seed, sizes=sizes, max_rhs=3)


def _make(torch, specs, f_dtype=np.float32):
    probs, hosts = [], []
    for sp in specs:
        rhs = [W.batch_problem(sp, r, dtype=f_dtype) for r in range(sp["nrhs"])]
        p0 = rhs[0]
        f = torch.from_numpy(np.stack([q.f_nodes.astype(f_dtype) for q in rhs])).cuda()
        u = torch.full((sp["nrhs"], p0.Nz, p0.Ny, p0.Nx), np.nan, dtype=torch.float64,
                       device="cuda")
        probs.append(dict(N=(p0.Nx, p0.Ny, p0.Nz), L=(p0.Lx, p0.Ly, p0.Lz), order=6,
                          c0=p0.c0, c1=p0.c1, c2=p0.c2, nrhs=sp["nrhs"], f=f, u=u))
        hosts.append(rhs)
    return probs, hosts


def _single(torch, pr, r, sweeps):
    s = H.Solver(*pr["N"], *pr["L"], 6, H.HS_HELMHOLTZ, H.HS_MIXED)
    try:
        s.set_coeff(pr["c0"], pr["c1"], pr["c2"])
        H.hs_set_refinement(s.plan, sweeps)
        u = torch.empty(pr["u"].shape[1:], dtype=torch.float64, device="cuda")
        s.solve(pr["f"][r].contiguous(), u, H.HS_F32, H.HS_RHS_NODAL)
        torch.cuda.synchronize()
        return u
    finally:
        s.close()


@pytest.mark.parametrize("sweeps", [0, 1, 2])
def test_batch_matches_single_solves(sweeps):
    torch = pytest.importorskip("torch")
    specs = _specs()
    probs, hosts = _make(torch, specs)
    b = H.hs_batch_create(probs, H.HS_F32, sweeps)
    try:
        H.hs_batch_solve(b, sync=True)
        H.hs_batch_solve(b, sync=True)      # replay of the captured graph
        for k, pr in enumerate(probs):
            for r in range(pr["nrhs"]):
                ref = _single(torch, pr, r, sweeps)
                got = pr["u"][r]
                assert torch.isfinite(got).all()
                d = float((got - ref).abs().max()) / float(ref.abs().max())
                assert d <= 1e-14, (k, r, d)
        if sweeps >= 1:
            for k in (0, 3):
                ref = O.solve(hosts[k][0])[0]
                assert O.max_rel_diff(probs[k]["u"][0].cpu().numpy(), ref) <= 1e-10
    finally:
        H.hs_batch_destroy(b)


def test_batch_timeout_and_recovery():
    torch = pytest.importorskip("torch")
    specs = _specs(seed=12, n=3)
    probs, _ = _make(torch, specs)
    b = H.hs_batch_create(probs, H.HS_F32, 1)
    try:
        H.hs_batch_solve(b, sync=True)
        good = [p["u"].clone() for p in probs]
        H.hs_batch_set_wait_limit(b, 20000)          # ~2 ms per wait
        H.hs_batch_debug_stall(b, True)
        with pytest.raises(H.HsError) as e:
            H.hs_batch_solve(b, sync=True)
        assert e.value.status == H.HS_ERR_TIMEOUT
        H.hs_batch_debug_stall(b, False)
        H.hs_batch_set_wait_limit(b, 20000000)
        for p in probs:
            p["u"].fill_(0.0)
        assert H.hs_batch_solve(b, sync=True) == H.HS_OK
        for p, g in zip(probs, good):
            assert torch.equal(p["u"], g)
        # new output buffers through set_io
        u2 = torch.zeros_like(probs[1]["u"])
        H.hs_batch_set_io(b, 1, probs[1]["f"], u2)
        H.hs_batch_solve(b, sync=True)
        assert torch.equal(u2, good[1])
    finally:
        H.hs_batch_destroy(b)


def test_batch_rejects_unsupported_lengths():
    torch = pytest.importorskip("torch")
    f = torch.zeros((1, 12, 12, 12), dtype=torch.float32, device="cuda")
    u = torch.zeros((1, 10, 10, 10), dtype=torch.float64, device="cuda")
    c = np.full(12, 100.0)
    with pytest.raises(H.HsError) as e:
        H.hs_batch_create([dict(N=(10, 10, 10), L=(1, 1, 1), order=4, c0=c, nrhs=1, f=f, u=u)],
                          H.HS_F32, 1)
    assert e.value.status == H.HS_ERR_UNSUPPORTED


def test_batch_fp64_factor_path_odd_sizes():
    """Problems whose z-systems need FP64 factors (min pivot ratio < 1e-4), odd unknown
    counts and several right-hand sides: the per-RHS FP64 scratch of the batch."""
    torch = pytest.importorskip("torch")
    specs = [dict(id=0, N=(31, 31, 63), k0=60.0, a=1.0, nrhs=3),
             dict(id=1, N=(63, 31, 31), k0=55.0, a=0.9, nrhs=2),
             dict(id=2, N=(95, 31, 63), k0=45.0, a=1.0, nrhs=2)]
    probs, _ = _make(torch, specs)
    b = H.hs_batch_create(probs, H.HS_F32, 1)
    try:
        H.hs_batch_solve(b, sync=True)
        for k, pr in enumerate(probs):
            for r in range(pr["nrhs"]):
                ref = _single(torch, pr, r, 1)
                d = float((pr["u"][r] - ref).abs().max()) / float(ref.abs().max())
                assert d <= 1e-14, (k, r, d)
    finally:
        H.hs_batch_destroy(b)


def _single_info(torch, pr, r, sweeps):
    s = H.Solver(*pr["N"], *pr["L"], 6, H.HS_HELMHOLTZ, H.HS_MIXED)
    try:
        s.set_coeff(pr["c0"], pr["c1"], pr["c2"])
        H.hs_set_refinement(s.plan, sweeps)
        u = torch.empty(pr["u"].shape[1:], dtype=torch.float64, device="cuda")
        _, inf = s.solve(pr["f"][r].contiguous(), u, H.HS_F32, H.HS_RHS_NODAL, info=True)
        torch.cuda.synchronize()
        return inf["rel_residual"]
    finally:
        s.close()


def test_batch_tolerance_stops_each_problem():
    """With a tolerance every (problem, RHS) stops refining on its own once
    ||F - A U|| / ||F|| <= tol: its result equals the stand-alone solve with the
    sweep count its own residual history implies."""
    torch = pytest.importorskip("torch")
    specs = _specs(seed=13, n=5)
    probs, _ = _make(torch, specs)
    tol = 1e-9
    b = H.hs_batch_create(probs, H.HS_F32, 4)
    try:
        H.hs_batch_set_tol(b, tol)
        H.hs_batch_solve(b, sync=True)
        H.hs_batch_solve(b, sync=True)
        counts = set()
        for k, pr in enumerate(probs):
            for r in range(pr["nrhs"]):
                rr = _single_info(torch, pr, r, 4)
                need = next((m for m in range(5) if rr[m] <= tol), 4)
                counts.add(need)
                ref = _single(torch, pr, r, need)
                got = pr["u"][r]
                d = float((got - ref).abs().max()) / float(ref.abs().max())
                assert d <= 1e-14, (k, r, need, d)
        # a tolerance never met runs every sweep
        H.hs_batch_set_tol(b, 1e-30)
        H.hs_batch_solve(b, sync=True)
        pr = probs[2]
        ref = _single(torch, pr, 0, 4)
        d = float((pr["u"][0] - ref).abs().max()) / float(ref.abs().max())
        assert d <= 1e-14, d
        with pytest.raises(H.HsError):
            H.hs_batch_set_tol(b, -1.0)
    finally:
        H.hs_batch_destroy(b)


def test_batch_residual_precision_auto():
    """The batch takes the automatic residual decision per (problem, RHS): an
    ill-conditioned problem next to well-conditioned ones gives, for each, the
    stand-alone solve's result in the same mode."""
    torch = pytest.importorskip("torch")
    allspecs = W.workload_batch_specs(nprob=64, seed=3)
    specs = [dict(sp, nrhs=1) for sp in allspecs if sp["id"] == 0]
    specs += [dict(id=1, N=(63, 31, 95), k0=20.0, a=0.5, nrhs=2)]
    probs, _ = _make(torch, specs)
    for mode in (H.HS_RESID_AUTO, H.HS_RESID_F64):
        b = H.hs_batch_create(probs, H.HS_F32, 4)
        try:
            H.hs_batch_set_residual_precision(b, mode)
            H.hs_batch_solve(b, sync=True)
            for k, pr in enumerate(probs):
                for r in range(pr["nrhs"]):
                    s = H.Solver(*pr["N"], *pr["L"], 6, H.HS_HELMHOLTZ, H.HS_MIXED)
                    try:
                        s.set_coeff(pr["c0"], pr["c1"], pr["c2"])
                        H.hs_set_refinement(s.plan, 4)
                        H.hs_set_residual_precision(s.plan, mode)
                        ref = torch.empty(pr["u"].shape[1:], dtype=torch.float64, device="cuda")
                        s.solve(pr["f"][r].contiguous(), ref, H.HS_F32, H.HS_RHS_NODAL)
                        torch.cuda.synchronize()
                    finally:
                        s.close()
                    d = float((pr["u"][r] - ref).abs().max()) / float(ref.abs().max())
                    assert d <= 1e-14, (mode, k, r, d)
        finally:
            H.hs_batch_destroy(b)


def test_batch_graph_mode_all_rhs_and_tolerance():
    """The graph execution (variant 4) solves every RHS of every problem like the
    stand-alone solver, also with a tolerance, and after new output buffers."""
    torch = pytest.importorskip("torch")
    specs = _specs(seed=15, n=5)
    probs, _ = _make(torch, specs)
    b = H.hs_batch_create(probs, H.HS_F32, 2)
    try:
        H.hs_batch_set_variant(b, 4)
        H.hs_batch_solve(b, sync=True)
        H.hs_batch_solve(b, sync=True)
        nsolves = sum(pr["nrhs"] for pr in probs)
        assert H.hs_batch_graph_kernels(b) >= 12 * nsolves   # >= 12 kernels per 2-sweep solve
        for k, pr in enumerate(probs):
            for r in range(pr["nrhs"]):
                ref = _single(torch, pr, r, 2)
                d = float((pr["u"][r] - ref).abs().max()) / float(ref.abs().max())
                assert d <= 1e-14, (k, r, d)
        u2 = torch.zeros_like(probs[0]["u"])
        H.hs_batch_set_io(b, 0, probs[0]["f"], u2)
        H.hs_batch_solve(b, sync=True)
        assert torch.equal(u2, probs[0]["u"])
    finally:
        H.hs_batch_destroy(b)


def test_batch_kernel_variants_and_autotune():
    """Every execution variant (persistent kernel with register caps for 2 and 3
    CTAs per SM, staged or fused transform tiles; or the graph of stand-alone
    solves) gives the stand-alone results; the autotuner times them and keeps
    one."""
    torch = pytest.importorskip("torch")
    specs = _specs(seed=14, n=4)
    probs, _ = _make(torch, specs)
    b = H.hs_batch_create(probs, H.HS_F32, 1)
    try:
        outs = []
        for v in (0, 1, 2, 3, 4):
            H.hs_batch_set_variant(b, v)
            assert H.hs_batch_get_variant(b)[0] == v
            assert H.hs_batch_get_variant(b)[1] >= 1
            for p in probs:
                p["u"].fill_(np.nan)
            H.hs_batch_solve(b, sync=True)
            if v < 4:
                assert H.hs_batch_graph_kernels(b) == 1   # the persistent kernel
            outs.append([p["u"].clone() for p in probs])
        for k, pr in enumerate(probs):
            ref = _single(torch, pr, 0, 1)
            for v in range(5):
                x = outs[v][k]
                d = float((x[0] - ref).abs().max()) / float(ref.abs().max())
                assert d <= 1e-14, (v, k, d)
        ms = H.hs_batch_autotune(b, reps=1)
        assert ms > 0
        assert H.hs_batch_get_variant(b)[0] in (0, 1, 2, 3, 4)
        with pytest.raises(H.HsError):
            H.hs_batch_set_variant(b, 5)
    finally:
        H.hs_batch_destroy(b)
