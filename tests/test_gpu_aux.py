"""Auxiliary subsystems on the GPU: the non-finite check of f (a device reduction
whose count is exact), the synchronous solve refusing NaN / infinite input, and the
autotune cache (a second plan of the same class takes the first plan's choices
without timing; a cache file written by one process is read by another).
"""
import numpy as np
import pytest

import paper_1912_03565_gb300 as H
import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    return pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_check_finite_counts_exactly(dtype):
    torch = _torch()
    s = H.Solver(15, 14, 13, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_FP64)
    try:
        n = 3_000_001   # ragged: not a multiple of any block size
        x = torch.rand(n, dtype=getattr(torch, dtype), device="cuda")
        assert H.hs_check_finite(s.plan, x) == 0
        rs = np.random.RandomState(1)
        idx = rs.choice(n, 37, replace=False)
        vals = [np.nan, np.inf, -np.inf]
        for k, i in enumerate(idx):
            x[int(i)] = vals[k % 3]
        assert H.hs_check_finite(s.plan, x) == 37
        assert H.hs_check_finite(s.plan, x[:0]) == 0
        big = torch.full((n,), 3e38 if dtype == "float32" else 1e308, dtype=x.dtype, device="cuda")
        assert H.hs_check_finite(s.plan, big) == 0   # large but finite
    finally:
        s.close()


@pytest.mark.parametrize("precision", [H.HS_FP64, H.HS_MIXED])
def test_solve_with_info_refuses_nonfinite_f(precision):
    torch = _torch()
    p = W.workload_cube31_order4()
    s = H.Solver(p.Nx, p.Ny, p.Nz, p.Lx, p.Ly, p.Lz, p.order, H.HS_HELMHOLTZ, precision)
    try:
        s.set_coeff(p.c0, p.c1, p.c2)
        f = torch.from_numpy(p.f_nodes).cuda()
        f[3, 4, 5] = float("nan")
        u = torch.full((p.Nz, p.Ny, p.Nx), 7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(H.HsError) as e:
            s.solve(f, u, info=True)
        assert e.value.status == H.HS_ERR_NONFINITE
        assert "NaN" in str(e.value)
        torch.cuda.synchronize()
        assert bool((u == 7.0).all())   # u untouched
        fh = f.cpu().numpy().copy()     # host f: scanned on the host
        with pytest.raises(H.HsError) as e:
            s.solve(fh, u, info=True)
        assert e.value.status == H.HS_ERR_NONFINITE
        f[3, 4, 5] = 0.0
        st, inf = s.solve(f, u, info=True)
        assert st >= 0 and inf is not None
    finally:
        s.close()


def test_autotune_cache_reuses_choices(tmp_path):
    torch = _torch()
    H.hs_autotune_cache_clear()
    p = W.workload_cube255_order6(N=127)

    def plan():
        s = H.Solver(p.Nx, p.Ny, p.Nz, p.Lx, p.Ly, p.Lz, 6, H.HS_HELMHOLTZ, H.HS_MIXED)
        s.set_coeff(p.c0, p.c1, p.c2)
        return s

    a = plan()
    try:
        mx, my = H.hs_autotune(a.plan, reps=2)
        assert H.hs_autotune_cache_count() == 1
        chosen = (H.hs_get_transform_variant(a.plan, H.HS_AXIS_X),
                  H.hs_get_transform_variant(a.plan, H.HS_AXIS_Y), H.hs_get_thomas_variant(a.plan))
    finally:
        a.close()
    b = plan()
    try:
        mx2, my2 = H.hs_autotune(b.plan, reps=2)   # taken from the cache: same times
        assert (mx2, my2) == (mx, my)
        assert (H.hs_get_transform_variant(b.plan, H.HS_AXIS_X),
                H.hs_get_transform_variant(b.plan, H.HS_AXIS_Y),
                H.hs_get_thomas_variant(b.plan)) == chosen
        path = tmp_path / "tune.txt"
        H.hs_autotune_cache_save(str(path))
        H.hs_autotune_cache_clear()
        H.hs_autotune_cache_load(str(path))
        assert H.hs_autotune_cache_count() == 1
        mx3, _ = H.hs_autotune(b.plan, reps=2)
        assert abs(mx3 - mx) <= 1e-5 * mx   # printed with 6 significant digits
    finally:
        b.close()
    H.hs_autotune_cache_clear()
