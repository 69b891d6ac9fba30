"""Host-side logic of bench.py on CPU: the multi-rank reductions (gloo, 2 ranks),
the reference arm under torchrun, and the bookkeeping helpers."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.reduce_max(10.0 * (rank + 1), dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_reduce_max_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, 29531, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 20.0, 1: 20.0}
    assert bench.reduce_max(3.5, None, "cpu") == 3.5


def test_reference_arm_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29533", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "cube31_o4", "--steps", "1", "--warmup", "1",
           "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"


def test_stage_bytes_and_launch_counts():
    b = bench.stage_bytes("mixed", 1, hi_only=False)
    assert b["residual"] == 20.0 and b["dst_x"] == 16.0 and b["idst_x"] == 32.0
    # one fixed sweep: the first iterate's lo plane is never stored
    h = bench.stage_bytes("mixed", 1)
    assert h["residual"] == 16.0 and h["idst_x"] == 24.0
    assert sum(b.values()) - sum(h.values()) == 12.0
    assert bench.stage_bytes("mixed", 2)["residual"] == 40.0
    assert bench.stage_bytes("mixed", 1, thomas_fp32=False)["thomas"] == 64.0
    assert bench.launches_per_solve("mixed", 1) == 12
    assert bench.launches_per_solve("fp64", 0) == 6
    assert bench.launches_per_solve("mixed", 1, ghost=True) == 13
    assert set(bench.WORKLOADS) >= {"cube255_o6", "cube1023_o6", "cd511x8"}


def test_complex_workloads_and_fp64_pipe_peak():
    """The complex-plan workloads, their counters and the FP64 pipe's rate the bench uses;
    the oracle leg on a small instance of the Neumann recipe (every plane and side node
    is an unknown: Robin z-faces, Neumann x and y)."""
    assert {"zrobin255_o4", "zneumann255_o4"} <= set(bench.WORKLOADS)
    assert callable(bench.fp64_pipe_peak)   # measured on the GPU by hs_fp64_fma_rate
    for name in ("zrobin255_o4", "zneumann255_o4"):
        c = bench.NCU_COUNTS[(name, "transforms")]
        assert c["fp64_warp_inst"] > 0 and c["dram_bytes"] > 0
        assert os.path.exists(os.path.join(ROOT, c["profile"]))
    import numpy as np
    import workloads as W
    w = W.workload_zneumann(7)
    U = bench.zrobin_run_oracle(w)
    assert U.shape == (9, 9, 9) and np.all(np.isfinite(U))
    w = W.workload_zrobin(7)
    assert bench.zrobin_run_oracle(w).shape == (9, 7, 7)
