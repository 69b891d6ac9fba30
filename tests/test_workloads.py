"""The seeded input generators shared by the tests, the oracle runs and the bench:
same seed, same bytes; another seed, other data; shapes and boundary values as
each generator's docstring states (CPU, small sizes)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import workloads as W  # noqa: E402


def _same(a, b):
    return a.shape == b.shape and a.dtype == b.dtype and np.array_equal(a, b)


def test_random_interior_problem_seeded():
    K = W.k_profile_to_k2(W.k_linear(10.0, 0.5))
    a = W.random_interior_problem((9, 7, 5), (1.0, 0.8, 0.6), 4, W.HELMHOLTZ, K, 11)
    b = W.random_interior_problem((9, 7, 5), (1.0, 0.8, 0.6), 4, W.HELMHOLTZ, K, 11)
    c = W.random_interior_problem((9, 7, 5), (1.0, 0.8, 0.6), 4, W.HELMHOLTZ, K, 12)
    assert a.f_nodes.shape == (7, 9, 11)
    assert _same(a.f_nodes, b.f_nodes)
    assert not np.array_equal(a.f_nodes, c.f_nodes)
    inner = a.f_nodes[1:-1, 1:-1, 1:-1]
    assert inner.min() >= -1.0 and inner.max() <= 1.0 and np.abs(inner).min() > 0
    shell = a.f_nodes.copy()
    shell[1:-1, 1:-1, 1:-1] = 0
    assert not shell.any()
    # FP32-stored variant: every value representable in FP32
    d = W.random_interior_problem((9, 7, 5), (1.0, 0.8, 0.6), 4, W.HELMHOLTZ, K, 11,
                                  dtype=np.float32)
    assert np.array_equal(d.f_nodes, d.f_nodes.astype(np.float32).astype(np.float64))


def test_noise_interior_keeps_boundary():
    p = W.manufactured_cube(7, 4, W.k_10_5sin())
    q = W.noise_interior(p, 3)
    r = W.noise_interior(p, 3)
    assert _same(q.f_nodes, r.f_nodes)
    d = q.f_nodes - p.f_nodes
    assert np.abs(d[1:-1, 1:-1, 1:-1]).min() > 0 and np.abs(d).max() <= 1.0
    d[1:-1, 1:-1, 1:-1] = 0
    assert not d.any()
    assert q.u_exact is None and p.u_exact is not None


def test_sine_mode_problem_seeded():
    a = W.sine_mode_problem(15, 6, W.k_tanh(), nmodes=4, seed=4)
    b = W.sine_mode_problem(15, 6, W.k_tanh(), nmodes=4, seed=4)
    c = W.sine_mode_problem(15, 6, W.k_tanh(), nmodes=4, seed=5)
    assert _same(a.f_nodes, b.f_nodes) and not np.array_equal(a.f_nodes, c.f_nodes)
    # sines vanish on every face (up to the sin(n pi) rounding)
    f = a.f_nodes
    for face in (f[0], f[-1], f[:, 0], f[:, -1], f[:, :, 0], f[:, :, -1]):
        assert np.abs(face).max() < 1e-12 * max(1.0, np.abs(f).max())


def test_batch_specs_seeded():
    s1 = W.workload_batch_specs(16, seed=3)
    s2 = W.workload_batch_specs(16, seed=3)
    s3 = W.workload_batch_specs(16, seed=4)
    assert s1 == s2 and s1 != s3
    for s in s1:
        assert all(n in W.BATCH_SIZES for n in s["N"])
        assert 5.0 <= s["k0"] <= 60.0 and 0.0 <= s["a"] <= 1.0 and 1 <= s["nrhs"] <= 4
    # each right-hand side of a problem is its own stream of numbers
    spec = dict(id=0, N=(9, 7, 5), k0=10.0, a=0.5, nrhs=2)
    r0 = W.batch_problem(spec, 0)
    r1 = W.batch_problem(spec, 1)
    assert not np.array_equal(r0.f_nodes, r1.f_nodes)
    assert _same(r0.f_nodes, W.batch_problem(spec, 0).f_nodes)


def test_complex_workloads_seeded():
    a = W.workload_zrobin(7)
    b = W.workload_zrobin(7)
    c = W.workload_zrobin(7, seed=99)
    assert _same(a["f"], b["f"]) and not np.array_equal(a["f"], c["f"])
    f = a["f"]
    assert f.shape == (9, 9, 9) and f.dtype == np.complex128
    inner = f[1:-1, 1:-1, 1:-1]
    assert np.abs(inner.real).max() <= 1 and np.abs(inner.imag).max() <= 1
    shell = f.copy()
    shell[1:-1, 1:-1, 1:-1] = 0
    assert not shell.any()
    # absorbing faces: beta = +-i k at z = 0 and z = 1
    assert np.isclose(a["beta_lo"] ** 2, -a["K"][0])
    assert np.isclose(a["beta_hi"] ** 2, -a["K"][-1])
    n = W.workload_zneumann(7)
    assert n["sides"] == (1, 1) and a["sides"] == (0, 0)
