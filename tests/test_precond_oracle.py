"""Pins of the preconditioner-mode oracle (oracle/hs_precond_oracle.py), CPU only.

The paper gives no formula for a coefficient that varies in x and y (it names
the preconditioner use in Section 1); the general-coefficient operator is the
compact scheme with K U averaged like f in the right-hand side.  What pins it:
  (a) for K = K(z) it equals the 27-point operator with the Section 3.3
      coefficients, which tests/test_oracle_pins.py pins against the paper;
  (b) K enters locally: a coefficient nonzero at one node changes A U only at
      that node (weight h_z^2 K U_m / 2) and its six face neighbours (h_z^2 K U_m / 12);
  (c) on a uniform grid the operator commutes with every permutation of the axes;
  (d) with K = K(z) the preconditioner is exact: BiCGStab converges in one step;
  (e) BiCGStab's answer equals a direct solve of the assembled matrix, and its
      iterates equal those of scipy's BiCGStab;
  (f) mutations: K U taken pointwise, or the preconditioner left out, makes a pin fail.
"""
import itertools

import numpy as np
import pytest

from oracle import hs_oracle as O
from oracle import hs_precond_oracle as PC


def _field(shape, seed, scale=1.0):
    return np.random.RandomState(seed).uniform(-1, 1, shape) * scale


@pytest.mark.parametrize("order", [2, 4])
def test_general_operator_reduces_to_stencil27_for_kz(order):
    Nz, Ny, Nx = 7, 6, 9
    h = (0.11, 0.13, 0.09)
    rs = np.random.RandomState(1)
    Kz = 30.0 + 20.0 * rs.uniform(size=Nz + 2)
    K = np.broadcast_to(Kz[1:-1, None, None], (Nz, Ny, Nx))
    U = rs.uniform(-1, 1, (Nz, Ny, Nx))
    C = O.stencil_coefficients(order, O.HELMHOLTZ, h, Kz)
    ref = O.apply_stencil(C, O.pad_boundary(U))
    got = PC.apply_general(order, K, U, h)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("order,centre,face", [(4, 0.5, 1.0 / 12.0), (2, 1.0, 0.0)])
def test_coefficient_enters_locally(order, centre, face):
    Nz, Ny, Nx = 6, 7, 8
    h = (0.1, 0.12, 0.08)
    U = _field((Nz, Ny, Nx), 2)
    m = (3, 2, 4)
    c = 17.0
    K = np.zeros((Nz, Ny, Nx))
    K[m] = c
    d = PC.apply_general(order, K, U, h) - PC.apply_general(order, np.zeros_like(K), U, h)
    expect = np.zeros_like(U)
    w = h[2] ** 2 * c * U[m]
    expect[m] = centre * w
    for ax in range(3):
        for s in (-1, 1):
            q = list(m)
            q[ax] += s
            expect[tuple(q)] += face * w
    assert np.max(np.abs(d - expect)) <= 1e-13 * abs(w)


def test_general_operator_commutes_with_axis_permutations():
    N = 7
    h = (0.1, 0.1, 0.1)
    K = 40.0 + _field((N, N, N), 3, 10.0)
    U = _field((N, N, N), 4)
    base = PC.apply_general(4, K, U, h)
    for perm in itertools.permutations(range(3)):
        got = PC.apply_general(4, K.transpose(perm), U.transpose(perm), h)
        assert np.max(np.abs(got - base.transpose(perm))) <= 1e-12 * np.max(np.abs(base))


def test_preconditioner_exact_for_z_only_coefficient():
    Nz, Ny, Nx = 9, 7, 8
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 0.9, 1.1))
    Kz = 50.0 + 30.0 * np.sin(np.linspace(0, 3, Nz + 2))
    K = np.broadcast_to(Kz[1:-1, None, None], (Nz, Ny, Nx)).copy()
    F = _field((Nz, Ny, Nx), 5)
    x, hist = PC.precond_solve(4, K, F, h, Kz, tol=1e-12)
    assert len(hist) == 1 and hist[0] <= 1e-12


@pytest.mark.parametrize("order", [2, 4])
def test_bicgstab_matches_direct_solve(order):
    Nz, Ny, Nx = 5, 6, 7
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 1.0, 1.0))
    rs = np.random.RandomState(6)
    K = 20.0 * (1.0 + 0.3 * rs.uniform(-1, 1, (Nz, Ny, Nx)))
    F = rs.uniform(-1, 1, (Nz, Ny, Nx))
    n = K.size
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = PC.apply_general(order, K, e.reshape(K.shape), h).ravel()
    direct = np.linalg.solve(A, F.ravel()).reshape(K.shape)
    x, hist = PC.precond_solve(order, K, F, h, PC.reference_from_field(K), tol=1e-13,
                               maxit=200)
    assert hist[-1] <= 1e-13
    assert O.max_rel_diff(x, direct) <= 1e-10
    true_res = np.linalg.norm(PC.apply_general(order, K, x, h) - F) / np.linalg.norm(F)
    assert true_res <= 1e-12



def test_bicgstab_steps_are_the_library_bicgstab():
    """The right-preconditioned BiCGStab of van der Vorst against scipy's implementation
    of the same recurrence, with the same operator and preconditioner: the iterates after
    1, 2, 3 and 5 iterations agree (a wrong step of the recurrence changes them)."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    Nz, Ny, Nx = 5, 6, 7
    h = O.grid_steps((Nx, Ny, Nz), (1.0, 1.0, 1.0))
    rs = np.random.RandomState(6)
    K = 20.0 * (1.0 + 0.3 * rs.uniform(-1, 1, (Nz, Ny, Nx)))
    F = rs.uniform(-1, 1, (Nz, Ny, Nx))
    C = O.stencil_coefficients(4, O.HELMHOLTZ, h, PC.reference_from_field(K))
    op = lambda u: PC.apply_general(4, K, u, h)
    pre = lambda r: O.solve_assembled(C, r)[0]
    n = K.size
    A = spla.LinearOperator((n, n), matvec=lambda v: op(v.reshape(K.shape)).ravel())
    M = spla.LinearOperator((n, n), matvec=lambda v: pre(v.reshape(K.shape)).ravel())
    for it in (1, 2, 3, 5):
        ref, _ = spla.bicgstab(A, F.ravel(), x0=np.zeros(n), rtol=1e-300, atol=0.0,
                               maxiter=it, M=M)
        x, hist = PC.bicgstab(op, pre, F, tol=0.0, maxit=it)
        assert len(hist) == it
        assert np.max(np.abs(x.ravel() - ref)) <= 1e-12 * np.max(np.abs(ref))

# ----------------------------------------------------------------- mutations
# A plausible mistake planted in the oracle (on the CPU, through monkeypatch) must make
# one of the pins above fail.


def test_planted_pointwise_coefficient_is_caught(monkeypatch):
    """K U taken pointwise in the 4th-order operator (not averaged like f)."""
    orig = PC.apply_general

    def mutated(order, K, U, h):
        K = np.asarray(K, dtype=np.float64)
        return orig(order, np.zeros_like(K), U, h) + h[2] ** 2 * K * np.asarray(U)

    monkeypatch.setattr(PC, "apply_general", mutated)
    with pytest.raises(AssertionError):
        test_general_operator_reduces_to_stencil27_for_kz(4)
    with pytest.raises(AssertionError):
        test_coefficient_enters_locally(4, 0.5, 1.0 / 12.0)


def test_planted_missing_preconditioner_is_caught(monkeypatch):
    """BiCGStab run without applying the separable solve."""
    orig = PC.bicgstab

    def mutated(apply_A, apply_Minv, F, tol=1e-12, maxit=100, x0=None):
        return orig(apply_A, lambda r: r, F, tol, maxit, x0)

    monkeypatch.setattr(PC, "bicgstab", mutated)
    with pytest.raises(AssertionError):
        test_preconditioner_exact_for_z_only_coefficient()
