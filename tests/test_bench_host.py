"""Host-side logic of bench.py without a GPU: the max-over-ranks timing of the N > 1 path
(two gloo ranks on the CPU) and the reference arm's rank layout and JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 3.5 * rank, dist, "cpu")
        dist.barrier()
        with open(os.path.join(out, f"rank{rank}.txt"), "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    vals = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert vals == [13.5, 13.5]          # every rank sees the slowest rank's time


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, None, "cpu") == 7.25


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], capture_output=True, text=True, env=env, timeout=900)


def test_reference_arm_other_ranks_exit_without_output():
    r = _run_reference(1, 2)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_line():
    # the oracle as it stands on a bounded sample of the 128^3 workload (about 10-20 s of CPU)
    r = _run_reference(0, 2)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("diffusion3d-7pt-128^3")
    # what was timed is stated: a sample per step, extrapolated to a whole solve, on all cores
    cb = d["cpu_baseline"]
    assert d["extrapolated"] is True and cb["extrapolated"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["timed_iters"] == cb["timed_iters"] > 0
    assert d["scaled_to_iters"] == cb["scaled_to_iters"] > 1000
    assert cb["threads"] == cb["cores"] == os.cpu_count() and cb["cpu_model"]
    # ms_per_step is the wall time of the sample that ran, far below the extrapolated value
    assert 0 < d["ms_per_step"] < d["value"]
    assert abs(d["value"] - (1e3 * cb["setup_s"] + cb["ms_per_iter"] * cb["scaled_to_iters"])) <= 1e-3 * d["value"]


def test_openmp_oracle_build_gives_the_checker_bits():
    # the timing build (OpenMP over rows, blocks and vector entries) against the checker
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    from paper_2407_15973_gb300 import problems as PB
    pr = PB.make_problem("voronoi3d", seed=4, m=14)
    b = O.spmv(pr.A, pr.x_star)
    out = {}
    for par in (False, True):
        old = O.use_parallel(par)
        try:
            assert O.threads() == (os.cpu_count() if par else 1)
            P = O.Preconditioner(pr.A, pr.block_ptr, fmt=O.BF16)
            r1 = O.pcg(pr.A, P, b, tol=1e-10, maxit=500, policy=O.POLICY_FMP, mode=1)
            r0 = O.pcg(pr.A, P, b, tol=1e-10, maxit=500, policy=O.POLICY_UNIFORM)
            out[par] = (P.G, P.pool, r1["x"], r1["hist"], r0["x"], r0["hist"])
        finally:
            O.use_parallel(old)
    for a, c in zip(out[False], out[True]):
        assert np.array_equal(a, c)


def test_host_cpu_reports_model_and_cores():
    sys.path.insert(0, ROOT)
    import bench
    model, cores = bench.host_cpu()
    assert isinstance(model, str) and model and cores == os.cpu_count()


def test_algorithmic_bytes_of_the_128_cube_workload():
    # per-launch bytes the roofline divides by (values read or written once): the SpMV moves
    # A (12 B per nonzero), row pointers, p and q; the fused BF16 apply the inverses, the block
    # scales and r, q in / r, z out; the x/p update x, p, z in and x, p out
    sys.path.insert(0, ROOT)
    import bench
    n, nnz, nb, bs = 128 ** 3, 7 * 128 ** 3 - 6 * 128 ** 2, 128 ** 3 // 32, 32
    assert nnz == 14581760                                  # Table 4.1
    got = bench.algorithmic_bytes(n, nnz, nb, bs, 2)
    assert got == {"spmv": 174981120 + 8388612 + 33554432, "apply": 134217728 + 262144 + 67108864,
                   "update_xp": 83886080}
    assert bench.algorithmic_bytes(n, nnz, nb, bs, 4)["apply"] == 268435456 + 67108864      # FP32: no scales
