"""Seeded, synthetic inputs for the compact-stencil Helmholtz / convection-diffusion solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It only
*generates inputs*: analytic manufactured solutions, coefficient profiles k(z)
or gamma(z) with their derivatives, noise and random sine modes.  It holds none
of the solver's arithmetic (no stencil coefficients, no right-hand-side
operator, no transform, no tridiagonal solve).

Array conventions (shared with the solver's interface):
  * node grid of one problem: shape (Nz+2, Ny+2, Nx+2), index [l, j, i], with
    x_i = i * Lx / (Nx + 1), i = 0..Nx+1 (nodes 0 and Nx+1 lie on the faces);
  * interior grid: shape (Nz, Ny, Nx);
  * coefficient profile: arrays of length Nz+2 sampled at z_l, l = 0..Nz+1;
  * x-face data: shape (Nz+2, Ny+2) [l, j]; y-face: (Nz+2, Nx+2) [l, i];
    z-face: (Ny+2, Nx+2) [j, i].  Order of the six faces: x-lo, x-hi, y-lo,
    y-hi, z-lo, z-hi.

The problems follow the paper's experiments (Section 5: the variable-k test
u = sin(beta x) sin(gamma y) exp(-k(z)/c) on [0, pi]^3, and the
convection-diffusion test with gamma = -100) and the synthetic workloads the
solver is benchmarked on (a 31^3 4th-order manufactured problem, a 255^3
6th-order problem with noise, a batch of uneven 6th-order problems, a 1023^3
sum-of-sine-modes problem and a 511^3 convection-diffusion batch).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

HELMHOLTZ = 0
CONVDIFF = 1


# --------------------------------------------------------------------------
# grids and sampling


def node_coords(N: int, L: float) -> np.ndarray:
    """Node coordinates x_i = i * L / (N + 1), i = 0..N+1 (Section 2)."""
    return np.arange(N + 2, dtype=np.float64) * (L / (N + 1))


def sample_nodes(fun: Callable, Nx: int, Ny: int, Nz: int,
                 Lx: float, Ly: float, Lz: float) -> np.ndarray:
    """Evaluate fun(x, y, z) on the full node grid, shape (Nz+2, Ny+2, Nx+2)."""
    x = node_coords(Nx, Lx)[None, None, :]
    y = node_coords(Ny, Ly)[None, :, None]
    z = node_coords(Nz, Lz)[:, None, None]
    return np.ascontiguousarray(np.broadcast_to(fun(x, y, z), (Nz + 2, Ny + 2, Nx + 2)),
                                dtype=np.float64)


def second_derivative_fd(g: Callable[[np.ndarray], np.ndarray], t: np.ndarray,
                         eta: float = 1e-3) -> np.ndarray:
    """Fourth-order central difference of a smooth analytic function g at t.

    Used only to produce face data (the normal second derivative of f on a face)
    for inputs whose closed form would be long; relative error ~1e-9.
    """
    return (-g(t + 2 * eta) + 16 * g(t + eta) - 30 * g(t) + 16 * g(t - eta)
            - g(t - 2 * eta)) / (12 * eta * eta)


# --------------------------------------------------------------------------
# coefficient profiles: k(z) with k', k'' (Helmholtz) or gamma(z) with gamma', gamma''


@dataclass
class Profile:
    """A function of z with its first two derivatives (vectorised callables)."""
    f0: Callable
    f1: Callable
    f2: Callable

    def sample(self, Nz: int, Lz: float):
        z = node_coords(Nz, Lz)
        return self.f0(z), self.f1(z), self.f2(z)


def k_profile_to_k2(k: Profile) -> Profile:
    """K = k^2 with K' = 2 k k' and K'' = 2 (k'^2 + k k'') (chain rule)."""
    return Profile(lambda z: k.f0(z) ** 2,
                   lambda z: 2.0 * k.f0(z) * k.f1(z),
                   lambda z: 2.0 * (k.f1(z) ** 2 + k.f0(z) * k.f2(z)))


def k_sine(a: float, b: float, c: float) -> Profile:
    """k(z) = a - b sin(c z): the paper's test coefficient (Section 5.1)."""
    return Profile(lambda z: a - b * np.sin(c * z),
                   lambda z: -b * c * np.cos(c * z),
                   lambda z: b * c * c * np.sin(c * z))


def k_10_5sin() -> Profile:
    """k(z) = 10 + 5 sin(pi z)."""
    return Profile(lambda z: 10.0 + 5.0 * np.sin(np.pi * z),
                   lambda z: 5.0 * np.pi * np.cos(np.pi * z),
                   lambda z: -5.0 * np.pi ** 2 * np.sin(np.pi * z))


def k_quadratic(k0: float = 20.0, q: float = 0.5) -> Profile:
    """k(z) = k0 (1 + q z^2)."""
    return Profile(lambda z: k0 * (1.0 + q * z * z),
                   lambda z: 2.0 * k0 * q * z,
                   lambda z: 2.0 * k0 * q + 0.0 * z)


def k_linear(k0: float, a: float) -> Profile:
    """k(z) = k0 (1 + a z)."""
    return Profile(lambda z: k0 * (1.0 + a * z),
                   lambda z: k0 * a + 0.0 * z,
                   lambda z: 0.0 * z)


def k_tanh(k0: float = 40.0, amp: float = 20.0, s: float = 10.0, z0: float = 0.5) -> Profile:
    """k(z) = k0 + amp tanh(s (z - z0))."""
    def t(z):
        return np.tanh(s * (z - z0))
    return Profile(lambda z: k0 + amp * t(z),
                   lambda z: amp * s * (1.0 - t(z) ** 2),
                   lambda z: -2.0 * amp * s * s * t(z) * (1.0 - t(z) ** 2))


def gamma_const(g: float) -> Profile:
    return Profile(lambda z: g + 0.0 * z, lambda z: 0.0 * z, lambda z: 0.0 * z)


def gamma_2_sin2pi() -> Profile:
    """gamma(z) = 2 + sin(2 pi z)."""
    w = 2.0 * np.pi
    return Profile(lambda z: 2.0 + np.sin(w * z),
                   lambda z: w * np.cos(w * z),
                   lambda z: -w * w * np.sin(w * z))


# --------------------------------------------------------------------------
# one problem instance


@dataclass
class Problem:
    """Everything the solver's interface takes for one right-hand side.

    f_nodes : (Nz+2, Ny+2, Nx+2) float64, f on the node grid.
    faces   : six Dirichlet face arrays (None = homogeneous).
    fnn     : six arrays of the normal second derivative of f on each face
              (None = 0); only the sixth-order right-hand side reads them.
    c0,c1,c2: coefficient profile (K, K', K'' for Helmholtz; gamma, gamma',
              gamma'' for convection-diffusion), length Nz+2.
    u_exact : exact solution on the node grid when known, else None.
    """
    Nx: int
    Ny: int
    Nz: int
    Lx: float
    Ly: float
    Lz: float
    order: int
    equation: int
    c0: np.ndarray
    c1: np.ndarray
    c2: np.ndarray
    f_nodes: np.ndarray
    faces: list = field(default_factory=lambda: [None] * 6)
    fnn: list = field(default_factory=lambda: [None] * 6)
    u_exact: Optional[np.ndarray] = None
    name: str = ""

    @property
    def h(self):
        return (self.Lx / (self.Nx + 1), self.Ly / (self.Ny + 1), self.Lz / (self.Nz + 1))


def faces_from_nodes(a: np.ndarray):
    """Six face arrays cut from a node-grid array (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi)."""
    return [np.ascontiguousarray(a[:, :, 0]), np.ascontiguousarray(a[:, :, -1]),
            np.ascontiguousarray(a[:, 0, :]), np.ascontiguousarray(a[:, -1, :]),
            np.ascontiguousarray(a[0, :, :]), np.ascontiguousarray(a[-1, :, :])]


def _face_second_derivatives(f: Callable, Nx, Ny, Nz, Lx, Ly, Lz):
    """Normal second derivative of an analytic f on the six faces (face array shapes)."""
    x = node_coords(Nx, Lx)
    y = node_coords(Ny, Ly)
    z = node_coords(Nz, Lz)
    out = []
    for xv in (0.0, Lx):
        Z, Y = np.meshgrid(z, y, indexing="ij")
        out.append(second_derivative_fd(lambda t: f(t, Y, Z), np.full_like(Z, xv)))
    for yv in (0.0, Ly):
        Z, X = np.meshgrid(z, x, indexing="ij")
        out.append(second_derivative_fd(lambda t: f(X, t, Z), np.full_like(Z, yv)))
    for zv in (0.0, Lz):
        Y, X = np.meshgrid(y, x, indexing="ij")
        out.append(second_derivative_fd(lambda t: f(X, Y, t), np.full_like(Y, zv)))
    return [np.ascontiguousarray(a) for a in out]


def analytic_problem(u: Callable, f: Callable, coef: Profile, N, L, order: int,
                     equation: int = HELMHOLTZ, name: str = "",
                     with_fnn: bool = True) -> Problem:
    """Sample an analytic (u, f) pair; Dirichlet faces come from u."""
    Nx, Ny, Nz = N
    Lx, Ly, Lz = L
    un = sample_nodes(u, Nx, Ny, Nz, Lx, Ly, Lz)
    fn = sample_nodes(f, Nx, Ny, Nz, Lx, Ly, Lz)
    c0, c1, c2 = coef.sample(Nz, Lz)
    faces = faces_from_nodes(un)
    faces = [None if not np.any(fc) else fc for fc in faces]
    fnn = (_face_second_derivatives(f, Nx, Ny, Nz, Lx, Ly, Lz) if (with_fnn and order == 6)
           else [None] * 6)
    return Problem(Nx, Ny, Nz, Lx, Ly, Lz, order, equation, c0, c1, c2, fn, faces, fnn,
                   un, name)


# --------------------------------------------------------------------------
# the paper's Helmholtz test (Section 5.1): u = sin(bx) sin(gy) exp(-k(z)/c)


def paper_helmholtz(N: int, order: int, a=10.0, b=9.0, c=10.0, beta=10.0, gamma=9.0) -> Problem:
    """Variable-k test of Section 5 on [0, pi]^3 with k = a - b sin(c z).

    The right-hand side is f = -b (2a + c) sin(cz) exp(-k/c) sin(beta x) sin(gamma y),
    valid when beta^2 + gamma^2 = a^2 + b^2.
    """
    k = k_sine(a, b, c)

    def u(x, y, z):
        return np.sin(beta * x) * np.sin(gamma * y) * np.exp(-k.f0(z) / c)

    def f(x, y, z):
        return (-b * (2 * a + c) * np.sin(c * z) * np.exp(-k.f0(z) / c)
                * np.sin(beta * x) * np.sin(gamma * y))

    return analytic_problem(u, f, k_profile_to_k2(k), (N, N, N), (np.pi,) * 3, order,
                            name=f"paper_helmholtz_{order}_{N}")


# --------------------------------------------------------------------------
# manufactured solution on the unit cube: u = sin(pi x) sin(2 pi y) sin(3 pi z) e^z


def manufactured_cube(N, order: int, k: Profile, name="manufactured") -> Problem:
    """u = sin(pi x) sin(2 pi y) sin(3 pi z) e^z, f = Laplacian(u) + k^2 u (analytic).

    u vanishes on every face, so the Dirichlet data are homogeneous.
    """
    if isinstance(N, int):
        N = (N, N, N)
    s = complex(1.0, 3.0 * np.pi)       # sin(3 pi z) e^z = Im(exp(s z))
    K = k_profile_to_k2(k)

    def zf(z, n=0):
        return np.imag(s ** n * np.exp(s * z))

    def u(x, y, z):
        return np.sin(np.pi * x) * np.sin(2 * np.pi * y) * zf(z)

    def f(x, y, z):
        return (np.sin(np.pi * x) * np.sin(2 * np.pi * y)
                * (zf(z, 2) + (K.f0(z) - 5.0 * np.pi ** 2) * zf(z)))

    return analytic_problem(u, f, K, N, (1.0, 1.0, 1.0), order, name=name)


# --------------------------------------------------------------------------
# the paper's convection-diffusion test (Section 5.2.3)


def paper_convdiff(N: int, gamma: float = -100.0) -> Problem:
    """Laplacian(u) + gamma u_z = 0 on [0, sqrt2]^2 x [0, 1] with the closed-form u."""
    r2 = math.sqrt(2.0)
    sig = math.sqrt(np.pi ** 2 + gamma ** 2 / 4.0)

    def u(x, y, z):
        zz = (2.0 * np.exp(gamma / 2.0) * np.sinh(sig * z) + np.sinh(sig * (1.0 - z))) / np.sinh(sig)
        return (np.sin(np.pi * x / r2) * np.sin(np.pi * y / r2) * np.exp(-gamma * z / 2.0) * zz)

    def f(x, y, z):
        return 0.0 * (x + y + z)

    return analytic_problem(u, f, gamma_const(gamma), (N, N, N), (r2, r2, 1.0), 4,
                            equation=CONVDIFF, name=f"paper_convdiff_{N}")


# --------------------------------------------------------------------------
# seeded synthetic workloads


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def noise_interior(prob: Problem, seed: int, amp: float = 1.0, dtype=np.float64) -> Problem:
    """Add seeded uniform[-amp, amp] noise to f at interior nodes (boundary nodes untouched)."""
    g = rng(seed)
    fn = prob.f_nodes.copy()
    fn[1:-1, 1:-1, 1:-1] += g.uniform(-amp, amp, size=(prob.Nz, prob.Ny, prob.Nx))
    fn = fn.astype(dtype).astype(np.float64) if dtype != np.float64 else fn
    out = Problem(**{**prob.__dict__})
    out.f_nodes = fn
    out.u_exact = None
    out.name = prob.name + f"+noise{seed}"
    return out


def random_interior_problem(N, L, order, equation, coef: Profile, seed: int,
                            dtype=np.float64, name="random") -> Problem:
    """f ~ U[-1, 1] at interior nodes, 0 on boundary nodes, homogeneous Dirichlet faces."""
    Nx, Ny, Nz = N
    Lx, Ly, Lz = L
    g = rng(seed)
    fn = np.zeros((Nz + 2, Ny + 2, Nx + 2))
    fn[1:-1, 1:-1, 1:-1] = g.uniform(-1.0, 1.0, size=(Nz, Ny, Nx)).astype(dtype)
    c0, c1, c2 = coef.sample(Nz, Lz)
    return Problem(Nx, Ny, Nz, Lx, Ly, Lz, order, equation, c0, c1, c2, fn, [None] * 6,
                   [None] * 6, None, name)


def sine_modes(N: int, nmodes: int, seed: int, pmax: int = 16):
    """Mode integers (p, q, r) uniform in [1, pmax] and amplitudes N(0, 1)."""
    g = rng(seed)
    pqr = g.integers(1, pmax + 1, size=(nmodes, 3))
    amp = g.standard_normal(nmodes)
    return pqr, amp


def sine_mode_problem(N: int, order: int, k: Profile, nmodes=16, seed=4, dtype=np.float32,
                      name="sine_modes") -> Problem:
    """f = sum_m A_m sin(p_m pi x) sin(q_m pi y) sin(r_m pi z) on the unit cube (FP32 stored)."""
    pqr, amp = sine_modes(N, nmodes, seed)
    x = node_coords(N, 1.0)
    fn = np.zeros((N + 2, N + 2, N + 2))
    for (p, q, r), A in zip(pqr, amp):
        fn += A * (np.sin(p * np.pi * x)[None, None, :] * np.sin(q * np.pi * x)[None, :, None]
                   * np.sin(r * np.pi * x)[:, None, None])
    fn = fn.astype(dtype).astype(np.float64)
    K = k_profile_to_k2(k)
    c0, c1, c2 = K.sample(N, 1.0)
    return Problem(N, N, N, 1.0, 1.0, 1.0, order, HELMHOLTZ, c0, c1, c2, fn, [None] * 6,
                   [None] * 6, None, name)


# --------------------------------------------------------------------------
# the named workloads


def workload_cube31_order4() -> Problem:
    """4th order, 31^3 interior on the unit cube, k = 10 + 5 sin(pi z), manufactured u."""
    return manufactured_cube(31, 4, k_10_5sin(), name="cube31_o4")


def workload_cube255_order6(seed: int = 2, N: int = 255) -> Problem:
    """6th order, N^3 (default 255^3), k = 20 (1 + z^2/2), manufactured f plus U[-1,1] noise."""
    p = manufactured_cube(N, 6, k_quadratic(20.0, 0.5), name=f"cube{N}_o6")
    return noise_interior(p, seed)


BATCH_SIZES = (63, 95, 127, 191, 255, 383)


def workload_batch_specs(nprob: int = 64, seed: int = 3, sizes=BATCH_SIZES, max_rhs: int = 4):
    """Seeded descriptions of a batch of uneven 6th-order problems.

    Each entry: (Nx, Ny, Nz), uniform h = 1/(max N + 1) with L_a = (N_a + 1) h,
    k(z) = k0 (1 + a z) with k0 ~ U[5, 60], a ~ U[0, 1], and nrhs ~ U{1..max_rhs}.
    """
    g = rng(seed)
    specs = []
    for idx in range(nprob):
        n = tuple(int(v) for v in g.choice(sizes, size=3))
        k0 = float(g.uniform(5.0, 60.0))
        a = float(g.uniform(0.0, 1.0))
        nrhs = int(g.integers(1, max_rhs + 1))
        specs.append(dict(id=idx, N=n, k0=k0, a=a, nrhs=nrhs))
    return specs


def batch_problem(spec: dict, rhs_index: int, seed: int = 3, dtype=np.float32) -> Problem:
    Nx, Ny, Nz = spec["N"]
    h = 1.0 / (max(spec["N"]) + 1)
    L = ((Nx + 1) * h, (Ny + 1) * h, (Nz + 1) * h)
    K = k_profile_to_k2(k_linear(spec["k0"], spec["a"]))
    sub = seed * 1_000_003 + spec["id"] * 16 + rhs_index
    return random_interior_problem((Nx, Ny, Nz), L, 6, HELMHOLTZ, K, sub, dtype,
                                   name=f"batch{spec['N']}r{rhs_index}")


def sine_mode_nodes_torch(N: int, modes, amps, dtype=None, device="cuda"):
    """The sum of sine modes on the node grid, built on a torch device (the
    1023^3 FP64 grid is 8.6 GB, too slow to fill with numpy).  Input generation
    only: f(x,y,z) = sum_m A_m sin(p pi x) sin(q pi y) sin(r pi z) on [0,1]^3.

    The result equals sine_mode_problem's FP64 f bit for bit: the 1-D sine
    factors are the same numpy values, and the products and sums are taken in
    the same order with correctly rounded FP64 operations (no fused
    multiply-add), so a GPU solve and the oracle see the same input."""
    import torch
    x = node_coords(N, 1.0)
    f = torch.zeros((N + 2, N + 2, N + 2), dtype=torch.float64, device=device)
    t = torch.empty_like(f)
    for (p, q, r), A in zip(modes, amps):
        sx = torch.from_numpy(np.sin(p * np.pi * x)).to(device)
        sy = torch.from_numpy(np.sin(q * np.pi * x)).to(device)
        sz = torch.from_numpy(np.sin(r * np.pi * x)).to(device)
        torch.mul(sx[None, None, :] * sy[None, :, None], sz[:, None, None], out=t)
        t.mul_(float(A))
        f.add_(t)
    del t
    return f if dtype is None else f.to(dtype)


def workload_cube1023_order6(seed: int = 4, N: int = 1023) -> Problem:
    """6th order, N^3 (default 1023^3), k = 40 + 20 tanh(10 (z - 1/2)), 16 sine modes, FP32 f."""
    return sine_mode_problem(N, 6, k_tanh(), nmodes=16, seed=seed, dtype=np.float32,
                             name=f"cube{N}_o6_modes")


def workload_convdiff511(rhs_index: int, seed: int = 5, N: int = 511) -> Problem:
    """CD 4th order, N^3 (default 511^3), gamma(z) = 2 + sin(2 pi z), U[-1,1] FP32 f."""
    return random_interior_problem((N, N, N), (1.0, 1.0, 1.0), 4, CONVDIFF, gamma_2_sin2pi(),
                                   seed * 1000 + rhs_index, np.float32,
                                   name=f"cd{N}r{rhs_index}")


def workload_zrobin(N: int = 255, seed: int = 12) -> dict:
    """Complex k(z) with first-order absorbing z-faces on the unit cube (N^3 interior).

    k(z) = 20 (1 + z^2 / 2) (1 + 0.02 i) (a weakly absorbing medium), K = k^2 at
    the nodes z_l; z-faces Robin u_z + i k u = 0 at z = 0 and u_z - i k u = 0 at
    z = 1 (alpha = 1, beta = +-i k at the face, zero data); side faces zero;
    f = U[-1,1] + i U[-1,1] at interior nodes (seeded), zero on the faces.
    Returns the plan parameters and the arrays (numpy complex)."""
    z = node_coords(N, 1.0)
    k = 20.0 * (1.0 + 0.5 * z ** 2) * (1.0 + 0.02j)
    rs = np.random.RandomState(seed)
    f = np.zeros((N + 2, N + 2, N + 2), dtype=np.complex128)
    f[1:-1, 1:-1, 1:-1] = (rs.uniform(-1, 1, (N, N, N)) + 1j * rs.uniform(-1, 1, (N, N, N)))
    return dict(N=N, L=(1.0, 1.0, 1.0), order=4, K=k * k,
                alpha_lo=1.0, beta_lo=1j * k[0], alpha_hi=1.0, beta_hi=-1j * k[-1], f=f,
                sides=(0, 0))


def workload_zneumann(N: int = 255, seed: int = 13) -> dict:
    """workload_zrobin's medium and z-faces with u_n = 0 on the four side faces
    (the side axes' boundary nodes are unknowns; side kinds (1, 1) = Neumann)."""
    w = workload_zrobin(N, seed)
    w["sides"] = (1, 1)
    return w
