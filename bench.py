#!/usr/bin/env python3
"""Throughput of the compact-stencil separation-of-variables solver on one GB300.

Workload (default): 6th-order compact scheme for Lap(u) + k(z)^2 u = f on the
unit cube, 255^3 interior points (h = 1/256), k(z) = 20 (1 + z^2/2), f = the
manufactured right-hand side of u = sin(pi x) sin(2 pi y) sin(3 pi z) e^z plus
seeded U[-1, 1] noise at interior nodes, face data d2f/dn2 analytic, FP64 f.

A step is one complete solve of one right-hand side (RHS operator, forward
DSTs, z-solves, inverse DSTs, and for the mixed path the refinement residual
and sweeps) with f and u resident in HBM.  The headline value is the
mixed path (FP32 transforms and z-solves, double-float residual and iterate,
refinement sweeps: the fewest whose error against the CPU oracle, measured in
the same run, is <= 1e-10) in Gunknowns/s; the FP64 path is timed beside it.  L2 is flushed
(a 256 MB write) between timed steps.  N > 1 GPUs run independent replicas
(weak scaling, no collective on the data path).

--impl reference times the CPU oracle (plain FP64 numpy) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gunknowns/s per solve at <=1e-10 rel err, mixed vs FP64 GPU path; % HBM roofline"
UNIT = "Gunknowns/s"

# Algorithmic bytes per interior unknown for each stage of one solve, by path
# (what the stage must read and write: inputs, outputs, cached factors).
BYTES_MIXED = {
    "rhs": 16.0,               # read f (FP64 nodes), write F (double-float pair)
    "dst_x": 8.0,              # FP32 read (F_hi or r) + FP32 write
    "dst_y": 8.0,              # FP32 read + write
    "thomas": 20.0,            # FP32 r + FP32 w + 3 FP32 factors (32 with FP64 factors)
    "idst_y": 8.0,
    "idst_x": None,            # 4 + 8 (set U pair) first sweep, 4 + 16 (U pair += / u) after
    "residual": 20.0,          # read F pair, U pair (27-point), write r (FP32)
}
# One fixed sweep: the first solve writes U's hi plane only (4 + 4), the residual
# reads F pair + U hi (+ r: 16) and the final update reads U hi (4 + 4 + 8 u).
BYTES_MIXED_HI_ONLY = {"idst_x": 8.0 + 16.0, "residual": 16.0}
BYTES_FP64 = {"rhs": 16.0, "dst_x": 16.0, "dst_y": 16.0, "thomas": 40.0, "idst_y": 16.0,
              "idst_x": 16.0, "residual": 0.0}


# Counters of one ncu capture (--set full) of a kernel at a workload's full size,
# per launch: DRAM bytes read + written, warp instructions.  Valid only while the
# kernel is unchanged since the capture (the profile named records the command).
NCU_COUNTS = {
    ("cube255_o6", "rhs"): {"bound": "alu", "dram_bytes": 140.290304e6 + 92.525568e6,
                            "warp_inst": 238553740,
                            "profile": "profiles/rhs_sf_cube255_o6.md"},
    # forward transform stage of the complex plan (x and y pass): FP64-pipe warp
    # instructions and DRAM bytes of the two launches
    ("zrobin255_o4", "transforms"): {
        "kernel": "dst_half_kernel x + y (half-length FP64 sine tiles over 2 x 257 planes)",
        "fp64_warp_inst": 20381680 + 20461312,
        "dram_bytes": 267511808 + 205838592 + 267540480 + 210931200,
        "profile": "profiles/fp64_transforms_complex255.md"},
    ("zneumann255_o4", "transforms"): {
        "kernel": "dct_half_kernel x + y (half-length FP64 cosine tiles over 2 x 257 planes)",
        "fp64_warp_inst": 23326000 + 24684850,
        "dram_bytes": 271667200 + 210036224 + 271682048 + 215204096,
        "profile": "profiles/fp64_transforms_complex255.md"},
}


def fp64_pipe_peak():
    """FP64 pipe instruction rate of this GPU, G warp-instructions/s: the FP64 FMA
    throughput measured now by the library's probe (hs_fp64_fma_rate: 8 independent
    FMA chains per thread, 152 x 8 blocks of 256 threads), / 2 flops / 32 threads."""
    import paper_1912_03565_gb300 as H
    rate = max(H.hs_fp64_fma_rate() for _ in range(3))
    return rate * 1e12 / 2.0 / 32.0 / 1e9, rate


def sm_max_mhz():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def stage_bytes(path: str, sweeps: int, thomas_fp32: bool = True, hi_only: bool = None):
    """Algorithmic bytes per unknown of each stage of one solve.  hi_only: the
    one-sweep sequence that keeps the first iterate's lo plane implicit (the
    stand-alone solve with one fixed sweep; default: sweeps == 1)."""
    if path == "fp64":
        return dict(BYTES_FP64)
    if hi_only is None:
        hi_only = sweeps == 1
    b = dict(BYTES_MIXED)
    n = sweeps + 1
    if not thomas_fp32:
        b["thomas"] = 32.0
    b["dst_x"] *= n
    b["idst_x"] = 12.0 + 20.0 * sweeps
    b["dst_y"] *= n
    b["thomas"] *= n
    b["idst_y"] *= n
    b["residual"] *= sweeps
    if hi_only and sweeps == 1:
        b.update(BYTES_MIXED_HI_ONLY)
    return b


def launches_per_solve(path: str, sweeps: int, ghost: bool = False) -> int:
    """Kernels per solve; ghost: the mixed 6th-order solve of FP64 f first forms
    its ghost nodes (one more launch)."""
    return 6 if path == "fp64" else 1 + 5 * (sweeps + 1) + sweeps + (1 if ghost else 0)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(x, dist, device):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- workloads

WORKLOADS = {
    "cube255_o6": dict(
        steps=100,
        desc="6th-order compact Helmholtz on the unit cube, 255^3 interior (h=1/256), "
             "k=20(1+z^2/2), f = manufactured (u=sin(pi x)sin(2pi y)sin(3pi z)e^z) "
             "+ U[-1,1] noise at interior nodes (seed 2), FP64 f, 1 RHS per step"),
    "cube31_o4": dict(
        steps=200,
        desc="4th-order compact Helmholtz on the unit cube, 31^3 interior (h=1/32), "
             "k=10+5 sin(pi z), manufactured u, FP64 f, 1 RHS per step"),
    "cube1023_o6": dict(
        steps=10, steps_in_all=5,
        desc="6th-order compact Helmholtz on the unit cube, 1023^3 interior (h=1/1024), "
             "k=40+20 tanh(10(z-1/2)), f = 16 seeded sine modes, amplitudes N(0,1), "
             "stored FP32, 1 RHS per step"),
    "batch64": dict(
        steps=5, steps_in_all=3,
        desc="64 independent 6th-order Helmholtz problems, N per axis drawn (seed 3) from "
             "{63,95,127,191,255,383}, uniform h=1/(max N+1), k=k0(1+a z) with k0~U[5,60], "
             "a~U[0,1], 1-4 right-hand sides each, f ~ U[-1,1] FP32 at interior nodes, "
             "one CUDA graph launch per step; execution autotuned between the persistent "
             "kernel variants and a graph of stand-alone solves on parallel branches"),
    "precond255_o4": dict(
        steps=3,
        desc="preconditioner mode: 4th-order compact Helmholtz with k^2(x,y,z) = "
             "(20(1+z^2/2))^2 (1 + 0.1 sin(pi x) sin(pi y)) on the unit cube, 255^3 interior, "
             "zero Dirichlet data, F ~ U[-1,1] h^2 assembled (seed 9); BiCGStab to "
             "||F - A x|| / ||F|| <= 1e-10 preconditioned by the separable solve for the plane "
             "means of k^2"),
    "zrobin255_o4": dict(
        steps=5,
        desc="complex k(z) = 20(1+z^2/2)(1+0.02i), 4th-order compact Helmholtz on the unit "
             "cube, 255^3 interior, first-order absorbing z-faces u_z +- i k u = 0 (Robin, "
             "second-order closure, both face planes unknown), zero side faces, "
             "f = U[-1,1] + i U[-1,1] (seed 12); FP64 path, complex z-solves"),
    "zneumann255_o4": dict(
        steps=5,
        desc="zrobin255_o4's complex k(z) and absorbing z-faces with u_n = 0 on the four side "
             "faces (cosine transforms over the 257 nodes of each side axis; seed 13)"),
    "cd511x8": dict(
        steps=10, steps_in_all=4,
        desc="4th-order compact convection-diffusion Lap(u)+b(z)u_z=f, 511^3 interior, "
             "b=2+sin(2pi z) (variable-b corrected coefficients), 8 right-hand sides "
             "U[-1,1] stored FP32 per step, nonsymmetric z-systems"),
}


# timed after the headline workload in the default run ("configs" of the JSON line)
EXTRA_CONFIGS = ("cube1023_o6", "batch64", "cd511x8")


def config_summary(line):
    """The parts of a workload's line reported under "configs"."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "fp64_path",
            "sequential_fp64_path", "sequential_mixed_path", "stages_ms", "accuracy", "roofline",
            "cpu_baseline", "clocks", "gpu_launches", "status")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line["config"]["workload"]
    for k in ("refinement_sweeps", "refinement_sweeps_max", "refinement_residual_tol",
              "transform_variants", "batch_kernel", "unknown_solves_per_step"):
        if k in line["config"]:
            out[k] = line["config"][k]
    return out


class Work:
    """One benchmark workload: plan parameters, device inputs and its CPU-oracle sample."""

    def __init__(self, name, torch, W, want_oracle):
        self.name = name
        self.desc = WORKLOADS[name]["desc"]
        self.fnn = None
        self.ref = None            # oracle solution of the first RHS (numpy) when affordable
        self.cpu = None            # (seconds, unknowns, sample text) of the oracle run
        self.nrhs = 1
        self.cd = 1
        from oracle import hs_oracle as O
        if name in ("cube255_o6", "cube31_o4"):
            p = W.workload_cube255_order6(seed=2) if name == "cube255_o6" else W.workload_cube31_order4()
            self.N, self.L, self.order, self.eq = (p.Nx, p.Ny, p.Nz), (p.Lx, p.Ly, p.Lz), p.order, 0
            self.c = (p.c0, p.c1, p.c2)
            self.f = torch.from_numpy(p.f_nodes).cuda()
            self.f_host = p.f_nodes
            self.f_dtype = 0
            self.fnn = [None if a is None else torch.from_numpy(a).cuda() for a in p.fnn]
            self.fnn_host = p.fnn
            if want_oracle:
                t0 = time.perf_counter()
                self.ref, _ = O.solve(p)
                dt = time.perf_counter() - t0
                n = p.Nx * p.Ny * p.Nz
                self.cpu = (dt, n, f"one full {p.Nx}^3 oracle solve (numpy FP64, matmul O(N^4) "
                                   f"DSTs, textbook Thomas): {dt:.2f} s")
        elif name == "cube1023_o6":
            N = 1023
            modes, amps = W.sine_modes(N, 16, 4)
            K = W.k_profile_to_k2(W.k_tanh())
            self.N, self.L, self.order, self.eq = (N, N, N), (1.0, 1.0, 1.0), 6, 0
            self.c = K.sample(N, 1.0)
            self.f = W.sine_mode_nodes_torch(N, modes, amps, torch.float32)
            self.f_host = None
            self.f_dtype = 1
            if want_oracle:
                q = W.sine_mode_problem(255, 6, W.k_tanh(), nmodes=16, seed=4)
                t0 = time.perf_counter()
                O.solve(q)
                dt = time.perf_counter() - t0
                self.cpu = (dt, 255 ** 3, f"bounded sample: one full 255^3 oracle solve of the "
                                           f"same recipe (16 sine modes, FP32 f): {dt:.2f} s")
        elif name == "cd511x8":
            N, R = 511, 8
            probs = [W.workload_convdiff511(r) for r in range(R)]
            self.N, self.L, self.order, self.eq = (N, N, N), (1.0, 1.0, 1.0), 4, 1
            self.c = (probs[0].c0, probs[0].c1, probs[0].c2)
            self.f_host = np.stack([q.f_nodes.astype(np.float32) for q in probs])
            self.f = torch.from_numpy(self.f_host).cuda()
            self.f_dtype = 1
            self.nrhs = R
            if want_oracle:
                # bounded sample: one right-hand side of the same recipe at 255^3 (the
                # 511^3 oracle takes minutes); parity at 511^3 is in the test suite
                q = W.workload_convdiff511(0, N=255)
                t0 = time.perf_counter()
                O.solve(q)
                dt = time.perf_counter() - t0
                self.cpu = (dt, 255 ** 3, f"bounded sample: the oracle on one right-hand side "
                                          f"of the same recipe at 255^3: {dt:.2f} s")
        else:
            raise ValueError(name)
        Nx, Ny, Nz = self.N
        self.n = Nx * Ny * Nz
        self.fnn_host = getattr(self, "fnn_host", None)


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    import workloads as W
    from oracle import hs_oracle as O
    name = args.workload
    # each step is the oracle on the workload's bounded sample (the full problem when
    # it takes seconds, else a smaller instance of the same recipe or one RHS)
    if name == "cube255_o6":
        p, n, sample = W.workload_cube255_order6(seed=2), 255 ** 3, "full 255^3 solve per step"
    elif name == "cube31_o4":
        p, n, sample = W.workload_cube31_order4(), 31 ** 3, "full 31^3 solve per step"
    elif name == "cube1023_o6":
        p = W.sine_mode_problem(255, 6, W.k_tanh(), nmodes=16, seed=4)
        n, sample = 255 ** 3, "255^3 instance of the same recipe per step"
    elif name == "precond255_o4":
        from oracle import hs_precond_oracle as PC
        Np = 63
        K = precond_field(np, Np)
        F = np.random.RandomState(9).uniform(-1, 1, K.shape) / (Np + 1) ** 2
        h = (1.0 / (Np + 1),) * 3
        Kref = PC.reference_from_field(K)
        run = lambda: PC.precond_solve(4, K, F, h, Kref, tol=1e-10, maxit=200)
        steps = args.steps if args.steps is not None else 3
        for _ in range(args.warmup):
            run()
        t0 = time.perf_counter()
        for _ in range(steps):
            run()
        dt = (time.perf_counter() - t0) / steps
        emit_reference(args, name, Np ** 3 / dt / 1e9, dt, steps,
                       f"{Np}^3 instance of the same recipe per step (numpy FP64 BiCGStab, "
                       "the oracle's O(N^4) solve as preconditioner)", world)
        return
    elif name in ("zrobin255_o4", "zneumann255_o4"):
        wz = W.workload_zneumann(255) if name == "zneumann255_o4" else W.workload_zrobin(255)
        nu = 257 * (257 if wz["sides"][0] else 255) * (257 if wz["sides"][1] else 255)
        steps = args.steps if args.steps is not None else 2
        for _ in range(args.warmup):
            zrobin_run_oracle(wz)
        t0 = time.perf_counter()
        for _ in range(steps):
            zrobin_run_oracle(wz)
        dt = (time.perf_counter() - t0) / steps
        emit_reference(args, name, nu / dt / 1e9, dt, steps,
                       "full 255^3 complex solve per step (numpy FP64, O(N^4) sine / cosine "
                       "sums, textbook complex Thomas)", world)
        return
    elif name == "batch64":
        sp = W.workload_batch_specs(nprob=64, seed=3)[0]
        p = W.batch_problem(sp, 0)
        n = p.Nx * p.Ny * p.Nz
        sample = f"problem 0 of the batch ({p.Nx}x{p.Ny}x{p.Nz}, 1 RHS) per step"
    else:
        p, n, sample = W.workload_convdiff511(0), 511 ** 3, "1 of the 8 right-hand sides per step"
    steps = args.steps if args.steps is not None else 5
    for _ in range(args.warmup):
        O.solve(p)
    t0 = time.perf_counter()
    for _ in range(steps):
        O.solve(p)
    dt = (time.perf_counter() - t0) / steps
    emit_reference(args, name, n / dt / 1e9, dt, steps,
                   sample + " (numpy FP64, matmul O(N^4) DSTs, textbook Thomas)", world)


def emit_reference(args, name, val, dt, steps, sample, world):
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{name}: {WORKLOADS[name]['desc']}", "global_batch": 1,
                       "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def precond_field(xp, N):
    """k^2 of the preconditioner workload on the N^3 interior of the unit cube
    (xp: numpy or torch; input generation only)."""
    t = xp.arange(1, N + 1, dtype=xp.float64) / (N + 1)
    kz = (20.0 * (1.0 + 0.5 * t ** 2)) ** 2
    sx = xp.sin(xp.pi * t) if xp.__name__ == "numpy" else xp.sin(t * 3.141592653589793)
    return kz[:, None, None] * (1.0 + 0.1 * sx[None, :, None] * sx[None, None, :])


def bench_precond(args, torch, H, rank, world, barrier, max_over_ranks):
    """Preconditioner mode: BiCGStab for k(x,y,z) with the plan's solve as M^-1."""
    N = 255
    Kd = precond_field(torch, N).to("cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    Fd = (torch.rand((N, N, N), generator=g, dtype=torch.float64, device="cuda") * 2 - 1) \
        / (N + 1) ** 2
    Kref = np.concatenate([[0.0], Kd.mean(dim=(1, 2)).cpu().numpy(), [0.0]])
    Kref[0], Kref[-1] = Kref[1], Kref[-2]
    stream = torch.cuda.current_stream()
    res = {}
    clocks = None
    for name, prec, sweeps in (("fp64", H.HS_FP64, 0), ("mixed", H.HS_MIXED, 1)):
        s = H.Solver(N, N, N, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, prec)
        s.set_coeff(Kref)
        if prec == H.HS_MIXED:
            H.hs_set_refinement(s.plan, sweeps)
        H.hs_autotune(s.plan, stream, 3)
        pc = H.hs_precond_create(s.plan, Kd)
        x = torch.zeros_like(Fd)
        st, inf = H.hs_precond_solve(pc, Fd, x, 1e-10, 200, stream)   # warm-up + accuracy
        steps = args.steps
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clk.start()
        e0.record(stream)
        for _ in range(steps):
            x.zero_()
            st, inf = H.hs_precond_solve(pc, Fd, x, 1e-10, 200, stream)
            its.append(inf["iterations"])
        e1.record(stream)
        torch.cuda.synchronize()
        c = clk.stop()
        if name == "mixed":
            clocks = c
        ms = max_over_ranks(e0.elapsed_time(e1)) / steps
        # kernels per solve: operator + init, then per iteration 3 dot products,
        # 3 vector updates, 2 operator applications and 2 solves of the plan (right-hand
        # side + 5 transform/z-solve passes, plus the residual and 5 more per sweep)
        per_solve = 6 + 6 * sweeps
        launches = sum(2 + k * (8 + 2 * per_solve) for k in its)
        res[name] = {"ms_per_solve": ms, "iterations": its, "status": st,
                     "rel_residual": inf["rel_residual"], "gpu_launches": launches,
                     "x": x.clone()}
        H.hs_precond_destroy(pc)
        s.close()
    x64, xmx = res["fp64"].pop("x"), res["mixed"].pop("x")
    diff = float((xmx - x64).abs().max() / x64.abs().max())
    value = world * N ** 3 / (res["mixed"]["ms_per_solve"] * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 1, "ms_per_step": res["mixed"]["ms_per_solve"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 Krylov, f32 + f32-pair preconditioner",
            "data": "synthetic",
            "config": {"workload": f"precond255_o4: {WORKLOADS['precond255_o4']['desc']}",
                       "global_batch": world, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (8 vectors of 133 MB per solve)"},
            "fp64_preconditioner": res["fp64"], "mixed_preconditioner": res["mixed"],
            "accuracy": {"mixed_vs_fp64_preconditioned_solution": diff,
                         "compared_against": "the same BiCGStab with the FP64 plan as preconditioner"},
            "cpu_baseline": None, "e2e": None, "roofline": None, "clocks": clocks,
            "gpu_launches": res["mixed"]["gpu_launches"],
        }
        print(json.dumps(line), flush=True)


def zrobin_run_oracle(w):
    from oracle import hs_complex_oracle as CX
    from oracle import hs_oracle as O
    N = w["N"]
    zf = CX.ZFaces(CX.ROBIN, w["alpha_lo"], w["beta_lo"], CX.ROBIN, w["alpha_hi"], w["beta_hi"])
    h = O.grid_steps((N, N, N), w["L"])
    return CX.solve(w["order"], h, w["K"], zf, w["f"], sides=w["sides"])[0]


def bench_zrobin(args, torch, H, W, rank, world, barrier, max_over_ranks):
    """Complex k(z) with absorbing (Robin) z-faces (and, for zneumann255_o4, u_n = 0 on
    the side faces): one hs_zsolve per step (FP64)."""
    name = args.workload
    w = W.workload_zneumann(255) if name == "zneumann255_o4" else W.workload_zrobin(255)
    N = w["N"]
    s = H.ZSolver(N, N, N, *w["L"], w["order"])
    s.set_coeff(w["K"])
    s.set_faces(H.HS_ZFACE_ROBIN, w["alpha_lo"], w["beta_lo"], H.HS_ZFACE_ROBIN,
                w["alpha_hi"], w["beta_hi"])
    s.set_sides(*w["sides"])
    nx = N + 2 if w["sides"][0] else N
    ny = N + 2 if w["sides"][1] else N
    f = torch.from_numpy(np.ascontiguousarray(np.stack([w["f"].real, w["f"].imag]))).cuda()
    u = torch.empty((2, N + 2, ny, nx), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        s.solve(f, u, stream=stream)
    torch.cuda.synchronize()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        s.solve(f, u, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev)) / args.steps
    # per-stage times from a separate loop with the plan's stage events on
    s.set_stage_timing(True)
    stages = {k: 0.0 for k in H.ZSolver.ZSTAGES}
    nst = 3
    for k in range(nst):
        flush.fill_(float(k))
        s.solve(f, u, stream=stream)
        for key, v in s.stage_times().items():
            stages[key] += v / nst
    s.set_stage_timing(False)
    roofline = None
    counts = NCU_COUNTS.get((name, "transforms"))
    if counts is not None:
        # the forward transform stage: one x and one y pass (FP64 sine or cosine tiles,
        # FP64-pipe bound); FP64-pipe warp instructions of the two passes (ncu) over the
        # stage's live time, against the FP64 pipe's instruction rate
        ach = counts["fp64_warp_inst"] / (stages["transforms"] * 1e-3) / 1e9
        peak, rate = fp64_pipe_peak()
        roofline = {"bound": "alu", "kernel": counts["kernel"], "achieved": ach,
                    "peak": peak, "unit": "G fp64 warp-inst/s",
                    "frac": ach / peak, "traffic": counts["dram_bytes"],
                    "peak_kind": f"FP64 pipe: FP64 FMA rate {rate:.4f} TFLOP/s measured in this "
                                 f"run (hs_fp64_fma_rate) / 2 flops / 32 lanes = {peak:.2f} G "
                                 "warp-instructions/s",
                    "launches": 2, "fp64_warp_inst_per_stage": counts["fp64_warp_inst"],
                    "stage_ms": stages["transforms"], "profile": counts["profile"]}
    acc, cpu = {"compared_against": "oracle (complex FP64, O(N^4) sine / cosine sums)"}, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        ref = zrobin_run_oracle(w)
        dt = time.perf_counter() - t0
        got = u.cpu().numpy()
        got = got[0] + 1j * got[1]
        acc["max_rel_error"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        cpu = {"value": (N + 2) * ny * nx / dt / 1e9, "unit": UNIT, "cores": cpu_cores(),
               "kind": "oracle",
               "sample": f"one full {N}^3 complex oracle solve (numpy FP64): {dt:.2f} s"}
    value = world * (N + 2) * ny * nx / (ms * 1e-3) / 1e9   # unknown (complex) points
    # the mixed-precision plan (Dirichlet side faces: FP32 sine tiles; Neumann side
    # faces: FP32 cosine tiles): FP32 solves refined with a pair residual, one
    # sweep, timed the same way and checked against the FP64 result
    mixed = None
    if name in ("zrobin255_o4", "zneumann255_o4"):
        u64 = u.clone()
        s.set_precision(H.HS_MIXED, 1)
        for _ in range(args.warmup):
            s.solve(f, u, stream=stream)
        torch.cuda.synchronize()
        barrier()
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            evm[k][0].record(stream)
            s.solve(f, u, stream=stream)
            evm[k][1].record(stream)
        torch.cuda.synchronize()
        msm = max_over_ranks(sum(a.elapsed_time(b) for a, b in evm)) / args.steps
        mixed = {"value": world * (N + 2) * ny * nx / (msm * 1e-3) / 1e9, "unit": UNIT,
                 "ms_per_step": msm, "sweeps": 1,
                 "dtype": "FP32 transforms and z-solves, FP32-pair F, U and residual",
                 "max_rel_error_vs_fp64_path": float((u - u64).abs().max() / u64.abs().max())}
        if "max_rel_error" in acc:
            got = u.cpu().numpy()
            got = got[0] + 1j * got[1]
            mixed["max_rel_error_vs_oracle"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        s.set_precision(H.HS_FP64, 0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (FP64 re, im)", "data": "synthetic",
            "config": {"workload": f"{name}: {WORKLOADS[name]['desc']}",
                       "global_batch": world, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps",
                       "unknowns": f"complex, planes l = 0..N+1 (Robin faces), {ny} x {nx} "
                                   "per plane"},
            "accuracy": acc, "cpu_baseline": cpu, "e2e": None, "roofline": roofline,
            "stages_ms": stages, "clocks": clocks, "mixed_path": mixed,
            # right-hand side, 4 transform passes, complex z-solve
            "gpu_launches": 6 * args.steps,
            "workspace_bytes": s.workspace_bytes(),
        }
        print(json.dumps(line), flush=True)
    s.close()


def bench_batch(args, torch, H, W, rank, world, barrier, max_over_ranks_dev):
    """Config with many problems: one hs_batch_solve per step."""
    specs = W.workload_batch_specs(nprob=64, seed=3)
    gen = torch.Generator(device="cuda")
    probs = []
    total = 0
    for sp in specs:
        Nx, Ny, Nz = sp["N"]
        h = 1.0 / (max(sp["N"]) + 1)
        L = ((Nx + 1) * h, (Ny + 1) * h, (Nz + 1) * h)
        K = W.k_profile_to_k2(W.k_linear(sp["k0"], sp["a"]))
        c0, c1, c2 = K.sample(Nz, L[2])
        gen.manual_seed(1_000_003 * 3 + sp["id"])
        f = torch.zeros((sp["nrhs"], Nz + 2, Ny + 2, Nx + 2), dtype=torch.float32, device="cuda")
        f[:, 1:-1, 1:-1, 1:-1] = torch.rand((sp["nrhs"], Nz, Ny, Nx), generator=gen,
                                            device="cuda") * 2 - 1
        u = torch.zeros((sp["nrhs"], Nz, Ny, Nx), dtype=torch.float64, device="cuda")
        probs.append(dict(N=sp["N"], L=L, order=6, c0=c0, c1=c1, c2=c2, nrhs=sp["nrhs"], f=f, u=u))
        total += sp["nrhs"] * Nx * Ny * Nz
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_solve(pr, prec, sweeps, tol, out):
        s = H.Solver(*pr["N"], *pr["L"], 6, H.HS_HELMHOLTZ, prec, max_rhs=pr["nrhs"])
        try:
            s.set_coeff(pr["c0"], pr["c1"], pr["c2"])
            if prec == H.HS_MIXED:
                H.hs_set_refinement(s.plan, sweeps)
                H.hs_set_refinement_tol(s.plan, tol)
            s.solve(pr["f"], out, H.HS_F32, H.HS_RHS_NODAL, nrhs=pr["nrhs"], stream=stream)
            torch.cuda.synchronize()
            e0.record(stream)
            s.solve(pr["f"], out, H.HS_F32, H.HS_RHS_NODAL, nrhs=pr["nrhs"], stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        finally:
            s.close()

    # the FP64 path's answers, which the batch must meet to 1e-10
    u64 = [torch.empty_like(pr["u"]) for pr in probs]
    t64 = sum(timed_solve(pr, H.HS_FP64, 0, 0.0, u) for pr, u in zip(probs, u64))

    def fp64_residuals(pr, u):
        """||F - A u|| / ||F|| in FP64 for each RHS of a problem (FP64 plan)."""
        s = H.Solver(*pr["N"], *pr["L"], 6, H.HS_HELMHOLTZ, H.HS_FP64)
        try:
            s.set_coeff(pr["c0"], pr["c1"], pr["c2"])
            out = []
            for r in range(pr["nrhs"]):
                rn, fn = H.hs_residual(s.plan, pr["f"][r].contiguous(), H.HS_F32,
                                       H.HS_RHS_NODAL, None, u[r].contiguous(), stream)
                out.append(rn / fn)
            return out
        finally:
            s.close()

    res64 = [fp64_residuals(pr, u) for pr, u in zip(probs, u64)]

    def assess():
        """Forward error against the FP64 path for every (problem, RHS); where it
        is above 1e-10, the backward error: the FP64 residual of the result
        against that of the FP64 path's answer (ill-conditioned problems, where
        FP64 answers themselves differ at that level)."""
        worst, nfwd, nall, nbwd, worst_ratio = 0.0, 0, 0, 0, 0.0
        for pr, u, r64 in zip(probs, u64, res64):
            bad = []
            for r in range(pr["nrhs"]):
                e = float((pr["u"][r] - u[r]).abs().max()) / float(u[r].abs().max())
                worst = max(worst, e)
                nall += 1
                if e <= 1e-10:
                    nfwd += 1
                else:
                    bad.append(r)
            if bad:
                rb = fp64_residuals(pr, pr["u"])
                for r in bad:
                    ratio = rb[r] / r64[r]
                    worst_ratio = max(worst_ratio, ratio)
                    nbwd += ratio <= 4.0
        return dict(forward_max=worst, n_results=nall, n_forward_le_1e10=nfwd,
                    n_backward_only=nall - nfwd, n_backward_ok=nbwd,
                    backward_ratio_max=worst_ratio, ok=(nfwd + nbwd == nall))

    # refinement: up to `max_sweeps` sweeps, each (problem, RHS) stopping on the
    # device at a relative residual `tol`; take the loosest tol that passes
    max_sweeps = 4 if args.sweeps < 0 else args.sweeps
    tried = {}
    tol = 0.0
    b = H.hs_batch_create(probs, H.HS_F32, max_sweeps)
    for cand in ((1e-9, 1e-10, 1e-11, 1e-12, 0.0) if args.sweeps < 0 else (0.0,)):
        H.hs_batch_set_tol(b, cand)
        H.hs_batch_solve(b, stream, True)
        tried[cand] = assess()
        tol = cand
        if tried[cand]["ok"]:
            break
    H.hs_batch_set_tol(b, tol)
    t0 = time.perf_counter()
    tuned_ms = H.hs_batch_autotune(b, stream, 1)    # kernel variant (set-up, untimed)
    tune = {"variant": H.hs_batch_get_variant(b)[0], "grid": H.hs_batch_get_variant(b)[1],
            "ms": tuned_ms, "autotune_s": time.perf_counter() - t0}
    H.hs_batch_solve(b, stream, True)
    acc = {"compared_against": "fp64 GPU path, every problem and RHS: forward error <= 1e-10, "
                             "else FP64 residual <= 4x the FP64 path's",
           "max_sweeps": max_sweeps, "residual_tol": tol, "residual_precision": "auto",
           "result": tried[tol],
           "tried": {f"{k:g}": v["forward_max"] for k, v in tried.items()}}
    scratch = [torch.empty_like(pr["u"]) for pr in probs]
    tmix = sum(timed_solve(pr, H.HS_MIXED, max_sweeps, tol, u) for pr, u in zip(probs, scratch))
    del scratch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        H.hs_batch_solve(b, stream, False)
    torch.cuda.synchronize()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        H.hs_batch_solve(b, stream, False)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    status = H.hs_batch_solve(b, stream, True)
    ms = max_over_ranks_dev(sum(a.elapsed_time(b2) for a, b2 in ev))
    value = world * args.steps * total / (ms * 1e-3) / 1e9
    kernels_per_step = H.hs_batch_graph_kernels(b)
    H.hs_batch_destroy(b)
    # roofline of the whole batch step: the algorithmic bytes of every (problem, RHS)
    # at one refinement sweep (a lower bound: a solve stopped by the tolerance runs
    # at least one) over the step's device time
    hbm_peak, peak_kind = load_peaks()
    bpu = sum(stage_bytes("mixed", 1, hi_only=False).values())
    achieved = bpu * total / (ms / args.steps * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "whole batch step (one CUDA graph launch)",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "algorithmic_bytes_per_step": bpu * total,
                "bytes_per_unknown": bpu,
                "note": "bytes at one refinement sweep per right-hand side: a lower bound"}
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # bounded sample: the oracle on the first three problems, one RHS each
        from oracle import hs_oracle as O
        t0 = time.perf_counter()
        nsamp = 0
        for sp in specs[:3]:
            pb = W.batch_problem(sp, 0)
            O.solve(pb)
            nsamp += pb.Nx * pb.Ny * pb.Nz
        dt = time.perf_counter() - t0
        cpu_baseline = {"value": nsamp / dt / 1e9, "unit": UNIT, "cores": cpu_cores(),
                        "kind": "oracle",
                        "sample": f"bounded sample: problems 0-2 of the batch, one RHS each "
                                  f"({nsamp} unknowns), numpy FP64 oracle: {dt:.2f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 + f32-pair (mixed)",
            "data": "synthetic",
            "config": {"workload": f"batch64: {WORKLOADS['batch64']['desc']}",
                       "global_batch": world * 64, "parallelism": f"replicas x{world}",
                       "unknown_solves_per_step": total, "refinement_sweeps_max": max_sweeps,
                       "refinement_residual_tol": tol, "batch_kernel": tune,
                       "l2": "256 MB buffer written between timed steps"},
            "sequential_fp64_path": {"value": total / (t64 * 1e-3) / 1e9, "unit": UNIT,
                                     "ms_per_step": t64},
            "sequential_mixed_path": {"value": total / (tmix * 1e-3) / 1e9, "unit": UNIT,
                                      "ms_per_step": tmix},
            "accuracy": acc, "status": status, "cpu_baseline": cpu_baseline, "e2e": None,
            "roofline": roofline, "clocks": clocks,
            "gpu_launches": args.steps * kernels_per_step,
        }
        return line
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hs", choices=["hs", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="one workload; default: cube255_o6 as the headline line with "
                         + ", ".join(EXTRA_CONFIGS) + " timed after it under 'configs'")
    ap.add_argument("--sweeps", type=int, default=-1,
                    help="refinement sweeps; -1 = the fewest whose error is <= 1e-10")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="",
                    help="mixed plan: transform variant x,y[,z-solve mapping] instead of autotuning")
    ap.add_argument("--variants64", default="",
                    help="FP64 plan: transform variant x,y instead of autotuning")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "hs":
        args.warmup = 3
    run_all = args.workload is None and args.impl == "hs"
    if args.workload is None:
        args.workload = "cube255_o6"
    if args.impl == "reference":
        run_reference(args)
        return
    if args.steps is None:
        args.steps = WORKLOADS[args.workload]["steps"]

    import torch

    import paper_1912_03565_gb300 as H
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.workload == "precond255_o4":
        bench_precond(args, torch, H, rank, world, barrier,
                      lambda x: reduce_max(x, dist, "cuda"))
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload in ("zrobin255_o4", "zneumann255_o4"):
        bench_zrobin(args, torch, H, W, rank, world, barrier,
                     lambda x: reduce_max(x, dist, "cuda"))
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload == "batch64":
        line = bench_batch(args, torch, H, W, rank, world, barrier,
                           lambda x: reduce_max(x, dist, "cuda"))
    else:
        line = bench_solve(args, torch, H, W, rank, world, local, barrier, dist)
    if run_all:
        # the other configurations, timed in the same process and reported under
        # "configs" (fewer steps; no end-to-end leg)
        line_configs = {}
        for name in EXTRA_CONFIGS:
            sub = argparse.Namespace(**vars(args))
            sub.workload = name
            sub.steps = WORKLOADS[name]["steps_in_all"]
            sub.no_e2e = True
            sub.variants = ""
            sub.variants64 = ""
            sub.sweeps = -1
            if name == "batch64":
                sl = bench_batch(sub, torch, H, W, rank, world, barrier,
                                 lambda x: reduce_max(x, dist, "cuda"))
            else:
                sl = bench_solve(sub, torch, H, W, rank, world, local, barrier, dist)
            torch.cuda.empty_cache()
            if rank == 0:
                line_configs[name] = config_summary(sl)
        if rank == 0:
            line["configs"] = line_configs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def bench_solve(args, torch, H, W, rank, world, local, barrier, dist):
    """One workload solved by the plan path (the Work recipes): accuracy of both
    paths, device-timed mixed and FP64 solves, stage breakdown, roofline of the
    dominant kernel, CPU-oracle baseline and (unless --no-e2e) the end-to-end
    time through hs_solve with host buffers.  Returns the JSON line (rank 0)."""
    want_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    wk = Work(args.workload, torch, W, want_oracle)
    Nx, Ny, Nz = wk.N
    N3 = wk.n
    R = wk.nrhs
    ushape = (Nz, Ny, Nx) if R == 1 else (R, Nz, Ny, Nx)
    u = torch.zeros(ushape, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    tuning = {}

    def solver(precision, sweeps):
        s = H.Solver(Nx, Ny, Nz, *wk.L, wk.order, wk.eq, precision, max_rhs=R)
        s.set_coeff(*wk.c, wk.cd)
        if precision == H.HS_MIXED:
            H.hs_set_refinement(s.plan, sweeps)
        # transform kernel variant per axis, timed on this plan (set-up, untimed);
        # --variants / --variants64 fix them instead (profiler runs, where the
        # serialised launches make the autotuner's timings meaningless)
        t0 = time.perf_counter()
        name = "mixed" if precision == H.HS_MIXED else "fp64"
        fixed = args.variants if precision == H.HS_MIXED else args.variants64
        if fixed:
            vals = [int(x) for x in fixed.split(",")]
            H.hs_set_transform_variant(s.plan, H.HS_AXIS_X, vals[0])
            H.hs_set_transform_variant(s.plan, H.HS_AXIS_Y, vals[1])
            if len(vals) > 2:
                H.hs_set_thomas_variant(s.plan, vals[2])
            mx = my = None
        else:
            mx, my = H.hs_autotune(s.plan, stream, 3)
        tuning[name] = {"variant_x": H.hs_get_transform_variant(s.plan, H.HS_AXIS_X),
                        "variant_y": H.hs_get_transform_variant(s.plan, H.HS_AXIS_Y),
                        "thomas_variant": H.hs_get_thomas_variant(s.plan),
                        "pass_ms_x": mx, "pass_ms_y": my, "fixed": bool(fixed),
                        "autotune_s": time.perf_counter() - t0}
        return s

    def run(s, f, uu, fnn=None, info=False):
        return s.solve(f, uu, wk.f_dtype, H.HS_RHS_NODAL, None, fnn, R, stream, info)

    def rel(a, b):
        return float((a - b).abs().max()) / float(b.abs().max())

    # ---- accuracy (untimed): FP64 path, and the mixed path after 0..3 sweeps
    acc = {}
    s64 = solver(H.HS_FP64, 0)
    u64 = torch.zeros_like(u)
    run(s64, wk.f, u64, wk.fnn)
    torch.cuda.synchronize()
    ref = None
    if wk.ref is not None:
        ref = torch.from_numpy(wk.ref).cuda()
        acc["fp64_vs_oracle"] = rel(u64 if R == 1 else u64[0], ref)
    acc["compared_against"] = "oracle" if ref is not None else "fp64 GPU path"
    by_sweeps = []
    for sw in range(0, 4):
        ss = solver(H.HS_MIXED, sw)
        run(ss, wk.f, u, wk.fnn)
        torch.cuda.synchronize()
        if ref is not None:
            e = rel(u if R == 1 else u[0], ref)
            if R > 1:
                e = max(e, rel(u, u64))
        else:
            e = rel(u, u64)
        by_sweeps.append(e)
        ss.close()
        torch.cuda.empty_cache()
    acc["mixed_error_by_sweeps"] = by_sweeps
    sweeps = args.sweeps
    if sweeps < 0:
        ok = [k for k in range(1, 4) if by_sweeps[k] <= 1e-10]
        sweeps = ok[0] if ok else 3
    acc["sweeps_used"] = sweeps
    acc["mixed_error"] = by_sweeps[sweeps] if sweeps < 4 else None
    smix = solver(H.HS_MIXED, sweeps)
    _, inf = run(smix, wk.f, u, wk.fnn, info=True)
    acc["mixed_rel_residual_per_sweep"] = inf["rel_residual"]
    acc["min_pivot_ratio"] = inf["min_pivot_ratio"]
    del u64
    torch.cuda.empty_cache()

    cpu_baseline = None
    if wk.cpu is not None:
        dt, n, sample = wk.cpu
        cpu_baseline = {"value": n / dt / 1e9, "unit": UNIT, "cores": cpu_cores(),
                        "kind": "oracle", "sample": sample}

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB

    def timed(s, steps, warmup):
        """Device time of `steps` solves (L2 flushed between them, no stage events,
        no host synchronisation inside the loop), then the per-stage breakdown from
        a separate loop with stage events on."""
        for _ in range(warmup):
            run(s, wk.f, u, wk.fnn)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            run(s, wk.f, u, wk.fnn)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        H.hs_set_stage_timing(s.plan, True)
        nst = min(steps, 10)
        stage_tot = {k: 0.0 for k in H.STAGES}
        for k in range(nst):
            flush.fill_(float(k))
            run(s, wk.f, u, wk.fnn)
            st = H.hs_stage_times(s.plan)
            for key, v in st.items():
                stage_tot[key] += v
        H.hs_set_stage_timing(s.plan, False)
        torch.cuda.synchronize()
        return ms, {k: v / nst for k, v in stage_tot.items()}

    steps64 = max(3, args.steps // 2)
    clk = ClockSampler(local)
    clk.start()
    ms_mix, st_mix = timed(smix, args.steps, args.warmup)
    ms_64, st_64 = timed(s64, steps64, args.warmup)
    clocks = clk.stop()

    def max_over_ranks(x):
        return reduce_max(x, dist, "cuda")

    ms_mix = max_over_ranks(ms_mix)
    ms_64 = max_over_ranks(ms_64)
    value = world * args.steps * R * N3 / (ms_mix * 1e-3) / 1e9
    value64 = world * steps64 * R * N3 / (ms_64 * 1e-3) / 1e9

    # ---- roofline of the dominant kernel of the mixed path
    hbm_peak, peak_kind = load_peaks()
    bmix = stage_bytes("mixed", sweeps, inf["min_pivot_ratio"] >= 1e-4)
    kern = max((k for k in bmix if st_mix.get(k, 0) > 0), key=lambda k: st_mix[k])
    nlaunch = {"dst_x": sweeps + 1, "dst_y": sweeps + 1, "thomas": sweeps + 1,
               "idst_y": sweeps + 1, "idst_x": sweeps + 1, "rhs": 1, "residual": sweeps}[kern]
    nlaunch *= R
    bytes_per_launch = bmix[kern] * N3 * R / nlaunch
    t_launch = st_mix[kern] / nlaunch * 1e-3
    achieved = bytes_per_launch / t_launch / 1e9
    hbm = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": hbm_peak,
           "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
           "peak_kind": f"{peak_kind} HBM copy bandwidth",
           "algorithmic_bytes_per_launch": bytes_per_launch}
    counts = NCU_COUNTS.get((args.workload, kern))
    if counts is not None:
        hbm["traffic"] = counts["dram_bytes"]
    if counts is not None and counts.get("bound") == "alu":
        # instruction-issue bound: warp instructions per launch (ncu) over the live
        # launch time, against 4 schedulers x SMs x the maximum SM clock
        props = torch.cuda.get_device_properties(local)
        issue_peak = 4 * props.multi_processor_count * sm_max_mhz() * 1e6 / 1e9
        ach = counts["warp_inst"] / t_launch / 1e9
        roofline = {"bound": "alu", "kernel": kern, "achieved": ach, "peak": issue_peak,
                    "unit": "G warp-inst/s", "frac": ach / issue_peak,
                    "traffic": counts["dram_bytes"],
                    "peak_kind": "issue rate: 4 warp-instructions/clock/SM x SMs x max SM clock",
                    "warp_inst_per_launch": counts["warp_inst"], "profile": counts["profile"],
                    "hbm": hbm}
    else:
        roofline = hbm

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        fh = wk.f.cpu().pin_memory()
        fnnh = None if wk.fnn is None else [None if a is None else a.cpu().pin_memory()
                                            for a in wk.fnn]
        uh = torch.zeros(ushape, dtype=torch.float64).pin_memory()
        # f is written by the CPU only, so its upload may overlap the previous solve;
        # u goes back on the plan's download stream, overlapping the next solve
        H.hs_set_host_io(smix.plan, H.HS_HOST_F_EARLY | H.HS_HOST_U_LATE)
        # at least 20 solves: the first upload and the last download overlap
        # nothing, and that fill and drain is paid once per timed region
        ke = max(20, args.steps)
        for _ in range(2):
            run(smix, fh, uh, fnnh)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            run(smix, fh, uh, fnnh)
        H.hs_host_io_wait(smix.plan, stream)   # the last copy of u is inside the region
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1))
        # the host result is the device path's, bit for bit
        run(smix, wk.f, u, wk.fnn)
        torch.cuda.synchronize()
        same = bool(torch.equal(uh, u.cpu()))
        h2d = fh.numel() * fh.element_size()
        if fnnh is not None:
            h2d += sum(a.numel() * a.element_size() for a in fnnh if a is not None)
        e2e = {"value": world * ke * R * N3 / (ms_e2e * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": uh.numel() * 8,
               "ms_per_step": ms_e2e / ke, "steps": ke,
               "host_io": "pinned host f, fnn, u through hs_solve; f staged in z-chunks "
                          "overlapping the RHS kernel and (HS_HOST_F_EARLY) the previous "
                          "solve; u copied back on a second stream overlapping the next "
                          "solve (HS_HOST_U_LATE)",
               "host_u_equals_device_u": same}

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mix / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 + f32-pair (mixed)",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wk.desc}",
                       "global_batch": world * R, "parallelism": f"replicas x{world}",
                       "refinement_sweeps": sweeps,
                       "transform_variants": tuning,
                       "l2": "256 MB buffer written between timed steps"},
            "fp64_path": {"value": value64, "unit": UNIT, "ms_per_step": ms_64 / steps64,
                          "stages_ms": st_64},
            "stages_ms": st_mix,
            "accuracy": acc,
            "roofline": roofline,
            "cpu_baseline": cpu_baseline,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches_per_solve(
                "mixed", sweeps, wk.order == 6 and wk.eq == 0 and wk.f_dtype == H.HS_F64)
            * R * args.steps,
        }
    smix.close()
    s64.close()
    torch.cuda.empty_cache()
    return line if rank == 0 else None




if __name__ == "__main__":
    main()
