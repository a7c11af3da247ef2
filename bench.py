"""Benchmark: time-to-solution of mixed-precision BJAC-PCG vs uniform binary64 BJAC-PCG.

Workload: 3D 7-point variable-coefficient diffusion on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760, Table 4.1 size), coefficient log-uniform in [1e-3, 1e3] constant on 8^3
subcubes, harmonic-mean faces, diagonal shift 1/dt = 100; x* ~ U[-1, 1] (seeded), b = A x*,
x0 = 0, tol 1e-10 on ||r||/||b||. A step is one bjac_setup + pcg_solve + bjac_destroy of
that system with the chosen policy (every kernel of the hot path runs in it). The
matrix (175 MB) and the block inverses (134-537 MB) are larger than the 129 MB L2, so no
explicit L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank solves its own system (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-solution at ||r||/||b||≤1e-10: mixed vs FP64 BJAC on 1 GB300; HBM GB/s"
TOL = 1e-10
MAXIT = 5000
FMT = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16s": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=128, help="grid side (128 = the named workload)")
    ap.add_argument("--bs", type=int, default=32)
    ap.add_argument("--fmt", default="bf16", choices=list(FMT))
    ap.add_argument("--temporal", default="none", choices=["none", "hl", "lh"],
                    help="aMP switching for the headline policy (adp_tol 10 for hl, 1e-5 for lh)")
    ap.add_argument("--flexible", action="store_true", help="flexible-CG beta for the headline policy")
    ap.add_argument("--no-modes", action="store_true", help="skip the per-mode table")
    ap.add_argument("--cpu-iters", type=int, default=16,
                    help="oracle PCG iterations in the all-core CPU sample (a quarter of them single-threaded)")
    ap.add_argument("--ref-iters", type=int, default=12,
                    help="oracle PCG iterations per step of the reference arm (after the full setup)")
    ap.add_argument("--spmv-kernel", default="auto", choices=["auto", "tma", "warp"],
                    help="pin the SpMV kernel instead of the timed choice (for profiler runs)")
    ap.add_argument("--spmv-layout", default="auto", choices=["auto", "csr", "sell", "sell-pf"],
                    help="pin the loop SpMV's matrix layout instead of the timed choice")
    ap.add_argument("--apply-kernel", default="auto", choices=["auto", "generic", "tma", "reg", "mix"],
                    help="pin the low-precision apply kernel instead of the timed choice")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven loop instead of the CUDA graph (the profiler sees every kernel)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workload configurations (27-point anisotropic 160^3, 256 batched "
                         "2D systems, Voronoi 256^3)")
    ap.add_argument("--profile-kt", action="store_true",
                    help="with --profile-iters: profile fMP BJAC(2, 2) with 32 blocks on the 128^3 Diff3D-Const "
                         "system instead of the headline policy")
    ap.add_argument("--l2-residency", default="on", choices=["on", "off"],
                    help="evict_last L2 policy on the PCG vectors in the loop kernels (default on)")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="only set up the headline policy and run this many eager PCG iterations "
                         "(a short, fixed launch sequence for ncu)")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="only set up a batch of this many 2D systems of the batched workload's law twice "
                         "(the first setup times the kernel variants) and solve each time for at most "
                         "--profile-iters iterations (200 if unset): a short launch sequence for ncu")
    return ap.parse_args()


def workload_config(args):
    return {"workload": f"diffusion3d-7pt-{args.m}^3-subcube8-logU[1e-3,1e3]-dt1e-2",
            "n": args.m ** 3, "block_size": args.bs, "mixed_format": args.fmt, "tol": TOL,
            "step": "bjac_setup + pcg_solve + bjac_destroy", "l2": "inputs larger than L2 (no flush)",
            "l2_residency": args.l2_residency, "temporal": args.temporal, "flexible": args.flexible}


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        self.out.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
def algorithmic_bytes(n, nnz, nb, bs, fmt_bytes):
    """Bytes each kernel of one PCG iteration must move (values read or written once)."""
    spmv = 12 * nnz + 4 * (n + 1) + 8 * n + 8 * n                 # A, rowptr, p, q
    apply_fused = nb * bs * bs * fmt_bytes + 4 * nb * (fmt_bytes == 2) + 8 * n * 4   # Q, scales, r, q in; r, z out
    update_xp = 8 * n * 5                                          # x, p, z in; x, p out
    return {"spmv": spmv, "apply": apply_fused, "update_xp": update_xp}


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel, {}).get(workload_key)
    if not e:
        return None
    if e.get("source_hash") != source_hash(e.get("sources", [])):
        return None
    return e.get("bytes_per_launch")


# ------------------------------------------------------------------------------------------
def max_over_ranks(value, dist, device):
    """The slowest rank's value (the job's time); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, dist):
    import torch
    from paper_2407_15973_gb300 import binding as B
    from paper_2407_15973_gb300 import problems as PB

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    B.lib()
    pr = PB.make_problem("subcube3d", seed=rank, m=args.m, bs=args.bs)
    A, n, nnz, nb = pr.A, pr.A.n, pr.A.nnz, pr.nb
    dA = B.DeviceCSR(A)
    xs = torch.as_tensor(pr.x_star).cuda()
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)                       # input construction, not timed (also times the SpMV kernels)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def step(pol, want_stats=False):
        x.zero_()
        pol = dict(pol)
        bp = pol.pop("block_ptr", pr.block_ptr)
        h = B.bjac_setup(dA, bp, **pol)
        st = h.solve(b, x, tol=TOL, maxit=MAXIT)
        h.close()
        return st

    def timed(pol, k, w):
        for _ in range(w):
            st = step(pol)
        barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        stats = []
        ev[0].record(stream)
        for i in range(k):
            stats.append(step(pol))
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev[0].elapsed_time(ev[k]) / k
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(k)]
        ms = max_over_ranks(ms, dist, "cuda")
        timed.last_steps = per
        return ms, stats

    spmv_pin = {"auto": 0, "tma": 1, "warp": 2}[args.spmv_kernel]
    B.bjac_spmv_kernel(spmv_pin)
    B.bjac_l2_residency(1 if args.l2_residency == "on" else 0)
    apply_pin = {"auto": 0, "generic": 1, "tma": 2, "reg": 3, "mix": 4}[args.apply_kernel]
    layout_pin = {"auto": 0, "csr": 1, "sell": 2, "sell-pf": 3}[args.spmv_layout]
    head = dict(select=B.SELECT_FIXED, fixed_fmt=FMT[args.fmt], apply_variant=apply_pin,
                graph_mode=1 if args.eager else 0, spmv_format=layout_pin, flexible=args.flexible,
                temporal={"none": B.TEMPORAL_NONE, "hl": B.TEMPORAL_HL, "lh": B.TEMPORAL_LH}[args.temporal],
                adp_tol={"none": 10.0, "hl": 10.0, "lh": 1e-5}[args.temporal])
    if args.profile_iters:
        if args.profile_kt:
            pk = PB.make_problem("diff3d-const", seed=0, m=args.m)
            dK = B.DeviceCSR(pk.A)
            bk = torch.empty(pk.A.n, dtype=torch.float64, device="cuda")
            B.bjac_spmv(dK, torch.as_tensor(pk.x_star).cuda(), bk)
            xk = torch.zeros(pk.A.n, dtype=torch.float64, device="cuda")
            h = B.bjac_setup(dK, np.linspace(0, pk.A.n, 33).astype(np.int32), select=B.SELECT_KT,
                             fixed_fmt=FMT["fp32"], graph_mode=head["graph_mode"])
            prof = h.profile(bk, xk, tol=TOL, maxit=args.profile_iters)
        else:
            h = B.bjac_setup(dA, pr.block_ptr, **head)
            prof = h.profile(b, x, tol=TOL, maxit=args.profile_iters)
        h.close()
        return {"profile": prof}
    with ClockSampler(dev) as clk:
        ms_mixed, st_mixed = timed(head, args.steps, args.warmup)
    clocks = clk.summary()
    step_ms = list(timed.last_steps)
    ms_fp64, st_fp64 = timed(dict(select=B.SELECT_UNIFORM, graph_mode=head["graph_mode"],
                                  spmv_format=layout_pin), args.steps, args.warmup)
    sm = st_mixed[-1]
    s64 = st_fp64[-1]
    err_x = float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))

    # per-mode table (setup + solve, one warm-up, two timed)
    modes = {}
    if not args.no_modes:
        table = {"uniform-fp64": dict(select=B.SELECT_UNIFORM)}
        for f in ("fp32", "bf16", "fp16s"):
            table[f"fmp-{f}"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT[f])
        table["amp-hl10-bf16"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT["bf16"], temporal=B.TEMPORAL_HL,
                                      adp_tol=10.0)
        table["amp-lh1e-5-bf16"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT["bf16"], temporal=B.TEMPORAL_LH,
                                        adp_tol=1e-5)
        table["fmp-bf16-flexible"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT["bf16"], flexible=True)
        table["amp-hl10-bf16-flexible"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT["bf16"],
                                               temporal=B.TEMPORAL_HL, adp_tol=10.0, flexible=True)
        table["rule"] = dict(select=B.SELECT_RULE)
        from paper_2407_15973_gb300 import selector as SEL
        if os.path.exists(SEL.DEFAULT_WEIGHTS):
            table["mlp"] = dict(select=B.SELECT_MLP, mlp_params=SEL.load(), safety_theta=SEL.load_safety_theta())
        # the 128^3 workload is also measured with blocks of 64 rows
        bp64 = PB.uniform_blocks(n, 64)
        table["uniform-fp64-bs64"] = dict(select=B.SELECT_UNIFORM, block_ptr=bp64)
        for f in ("fp32", "bf16"):
            table[f"fmp-{f}-bs64"] = dict(select=B.SELECT_FIXED, fixed_fmt=FMT[f], block_ptr=bp64)
        for name, pol in table.items():
            ms, sts = timed(pol, 2, 1)
            s = sts[-1]
            bsz = 64 if "block_ptr" in pol else args.bs
            pbytes = sum(cnt * bsz * bsz * {0: 8, 1: 4, 2: 2, 3: 2}[f] for f, cnt in enumerate(s["blocks_per_fmt"]))
            modes[name] = {"ms": round(ms, 3), "solve_ms": round(s["solve_ms"], 3), "setup_ms": round(s["setup_ms"], 3),
                           "iters": s["iters"], "true_relres": s["true_relres"], "converged": s["converged"],
                           "blocks_per_fmt": s["blocks_per_fmt"], "block_size": bsz,
                           "precond_bytes": int(pbytes)}

    # per-kernel device times of one iteration (eager launches, CUDA events on the stream)
    h = B.bjac_setup(dA, pr.block_ptr, **head)
    apply_kernel, tune_ms = h.apply_kernel()
    layout = h.spmv_format()
    x.zero_()
    prof = h.profile(b, x, tol=TOL, maxit=MAXIT)
    h.close()
    fb = {0: 8, 1: 4, 2: 2, 3: 2}[FMT[args.fmt]]
    alg = algorithmic_bytes(n, nnz, nb, args.bs, fb)
    shares = {k: prof[k] for k in ("spmv", "apply", "update_xp")}
    dom = max(shares, key=shares.get)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            peak = float(json.load(f)["hbm_gbs"])
        peak_src = "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    achieved = alg[dom] / (prof[dom] * 1e-3) / 1e9
    wl_key = f"m{args.m}_bs{args.bs}_{args.fmt}"
    # both SpMV kernels on this matrix, y = A x with the dot (standalone launches)
    spmv_var = {}
    xy = torch.zeros(1, dtype=torch.float64, device="cuda")
    yv = torch.empty(n, dtype=torch.float64, device="cuda")
    for v, name in ((1, "tma"), (2, "warp")):
        old = B.bjac_spmv_kernel(v)
        for _ in range(3):
            B.bjac_spmv(dA, xs, yv, xy)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(20):
            B.bjac_spmv(dA, xs, yv, xy)
        ev1.record(stream)
        torch.cuda.synchronize()
        B.bjac_spmv_kernel(old)
        spmv_var[name] = round(ev0.elapsed_time(ev1) / 20, 5)
    # the loop SpMV in both layouts through handles (y = A x with the dot, standalone launches)
    layout_ms = {}
    for name, fmt_pin in (("csr", 1), ("sell32", 2), ("sell32-prefetch", 3)):
        hl = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=FMT[args.fmt], spmv_format=fmt_pin)
        for _ in range(3):
            hl.spmv(xs, yv, xy)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(20):
            hl.spmv(xs, yv, xy)
        ev1.record(stream)
        torch.cuda.synchronize()
        hl.close()
        layout_ms[name] = round(ev0.elapsed_time(ev1) / 20, 5)
    apply_name = {"generic": "k_apply_generic", "tma": "k_apply_tma", "register": "k_apply_reg",
                  "mixed": "k_apply_mix32"}[apply_kernel]
    csr_name = {"tma": "k_spmv", "warp": "k_spmv_warp"}[B.bjac_spmv_tuning(dA)[0]]
    spmv_name = {"sell32": "k_spmv_sell", "sell32-prefetch": "k_spmv_sell_pf"}.get(layout["format"], csr_name)
    kernel_name = {"spmv": spmv_name, "apply": apply_name, "update_xp": "k_update_xp"}[dom]
    roofline = {"kernel": kernel_name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": committed_traffic(kernel_name, wl_key), "algorithmic_bytes": alg[dom],
                "launch_ms": round(prof[dom], 5),
                "per_kernel_ms": {k: round(v, 5) for k, v in shares.items()},
                "per_kernel_gbs": {k: round(alg[k] / (shares[k] * 1e-3) / 1e9, 1) for k in shares},
                "apply_kernel": apply_name,
                "spmv_kernel_name": spmv_name,
                "spmv_layout": {"format": layout["format"], "stored_entries": layout["entries"],
                                "setup_timing_ms": dict(zip(("csr", "sell32", "sell32-prefetch"),
                                                            [round(t, 4) for t in layout["ms"]])),
                                "standalone_ms": layout_ms},
                "spmv_variant_ms": spmv_var,
                "spmv_kernel": B.bjac_spmv_tuning(dA)[0],
                "spmv_autotune_ms": dict(zip(("tma", "warp"),
                                             [round(t, 4) for t in B.bjac_spmv_tuning(dA)[1]])),
                "apply_autotune_ms": dict(zip(("generic", "tma", "register"), [round(t, 4) for t in tune_ms]))}

    # end to end through the public API with host buffers: upload A and b from pinned host
    # memory, set up, solve, read x back
    hA = [torch.as_tensor(np.asarray(a)).pin_memory() for a in (A.rowptr, A.colidx, A.val)]
    hb = b.cpu().pin_memory()
    hx = torch.empty(n, dtype=torch.float64).pin_memory()

    def e2e_step():
        t = [a.to("cuda", non_blocking=True) for a in hA]
        d = B.DeviceCSR.__new__(B.DeviceCSR)
        d.n, d.rowptr, d.colidx, d.val, d.nnz = n, t[0], t[1], t[2], nnz
        d.c = B.bjac_csr(n, nnz, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr())
        bd = hb.to("cuda", non_blocking=True)
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        h = B.bjac_setup(d, pr.block_ptr, **head)
        h.solve(bd, xd, tol=TOL, maxit=MAXIT)
        h.close()
        hx.copy_(xd, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / args.steps
    h2d = sum(a.numel() * a.element_size() for a in hA) + n * 8
    d2h = n * 8

    setup_kernels = 2 + (0 if head["select"] in (B.SELECT_FIXED, B.SELECT_UNIFORM) else 1)
    setup_kernels += 3 if layout["format"] != "csr" else 0       # slice lengths, scan, fill
    per_step = [setup_kernels + s["kernel_launches"] for s in st_mixed]     # setup + the solve's own count
    out = {
        "metric": METRIC, "value": round(ms_mixed, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_mixed, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (block apply), bf16/fp16/fp32 storage",
        "data": "synthetic (seeded generator, b = A x*)",
        "config": workload_config(args),
        "iters": sm["iters"], "true_relres": sm["true_relres"], "x_rel_err": err_x,
        "setup_ms": round(sm["setup_ms"], 3), "solve_ms": round(sm["solve_ms"], 3),
        "fp64_uniform": {"ms": round(ms_fp64, 4), "iters": s64["iters"], "true_relres": s64["true_relres"],
                         "setup_ms": round(s64["setup_ms"], 3), "solve_ms": round(s64["solve_ms"], 3)},
        "speedup_vs_fp64": round(ms_fp64 / ms_mixed, 3),
        "step_ms": {"median": round(statistics.median(step_ms), 4), "min": round(min(step_ms), 4),
                    "max": round(max(step_ms), 4)},
        "modes": modes,
        "roofline": roofline,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(sum(per_step)),
        "clocks": clocks,
    }
    return out


# ------------------------------------------------------------------------------------------
def other_configs():
    """One measured step per policy (after a warm-up step that runs the autotuners for the
    shape) on the other workload configurations; the batched one against the same systems
    solved one after another by the single-system solver."""
    import torch
    from paper_2407_15973_gb300 import binding as B
    from paper_2407_15973_gb300 import problems as PB
    from paper_2407_15973_gb300 import selector as SEL
    stream = torch.cuda.current_stream()
    params = SEL.load() if os.path.exists(SEL.DEFAULT_WEIGHTS) else None
    theta_s = SEL.load_safety_theta() if params is not None else 0.5

    def timed_step(dA, bp, b, pol):
        x = torch.zeros(dA.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = B.bjac_setup(dA, bp, **pol)
        st = h.solve(b, x, tol=TOL, maxit=20000)
        h.close()
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": round(e0.elapsed_time(e1), 3), "setup_ms": round(st["setup_ms"], 3),
                "solve_ms": round(st["solve_ms"], 3), "iters": st["iters"], "true_relres": st["true_relres"],
                "converged": st["converged"], "blocks_per_fmt": st["blocks_per_fmt"],
                "fallback_used": st["fallback_used"]}, x

    out = {}
    for key, name, modes in (
            ("aniso27-q1-160^3-lognormal2-z1e4-bs64", "aniso27",
             ("uniform-fp64", "fmp-fp32", "fmp-bf16", "rule", "mlp")),
            ("voronoi7pt-256^3-5mat-1e6-uneven16..128", "voronoi3d",
             ("uniform-fp64", "fmp-fp32", "fmp-bf16", "fmp-fp16s", "rule", "mlp+fp64-fallback")),
            ("mscore7pt-96^3-rand1e10core-rand1e2-bs32", "mscore3d",
             ("uniform-fp64", "fmp-fp32", "fmp-bf16", "rule", "mlp", "mlp+fp64-fallback"))):
        t0 = time.time()
        pr = PB.make_problem(name, seed=0, m=96 if name == "mscore3d" else None)
        gen = time.time() - t0
        dA = B.DeviceCSR(pr.A)
        xs = torch.as_tensor(pr.x_star).cuda()
        b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, xs, b)
        pols = {"uniform-fp64": dict(select=B.SELECT_UNIFORM),
                "fmp-fp32": dict(select=B.SELECT_FIXED, fixed_fmt=FMT["fp32"]),
                "fmp-bf16": dict(select=B.SELECT_FIXED, fixed_fmt=FMT["bf16"]),
                "fmp-fp16s": dict(select=B.SELECT_FIXED, fixed_fmt=FMT["fp16s"]),
                "rule": dict(select=B.SELECT_RULE)}
        if params is not None:
            pols["mlp"] = dict(select=B.SELECT_MLP, mlp_params=params, safety_theta=theta_s)
            pols["mlp+fp64-fallback"] = dict(select=B.SELECT_MLP, mlp_params=params, safety_theta=theta_s,
                                             fp64_fallback=True)
        timed_step(dA, pr.block_ptr, b, pols["fmp-fp32"])          # warm-up: autotuners for this shape
        res = {}
        bsz = np.diff(pr.block_ptr).astype(np.int64)
        for m in modes:
            if m in pols:
                res[m], x = timed_step(dA, pr.block_ptr, b, pols[m])
                res[m]["x_rel_err"] = float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))
                # preconditioner bytes from the formats the setup chose
                h = B.bjac_setup(dA, pr.block_ptr, **pols[m])
                fm = h.formats()
                h.close()
                res[m]["precond_bytes"] = int(np.sum(bsz * bsz * np.array([8, 4, 2, 2])[fm]))
        base = res.get("uniform-fp64", {}).get("ms")
        out[key] = {"n": pr.A.n, "nnz": pr.A.nnz, "blocks": pr.nb, "generate_s": round(gen, 1),
                    "modes": res,
                    "speedup_vs_fp64": {m: round(base / r["ms"], 3) for m, r in res.items() if base}}
        del dA, b, xs

    # the paper's own configuration: BJAC(k = 2, t = 2) of Eq. 3-2 / 3-3 with 32 blocks on the
    # Diff3D laws of Section 4.1.1 (Table 4.2 / Figure 4.3 report 148 -> 165 iterations for
    # Const and 185 -> 211 for Dis(1000), uniform -> fp32 fMP, on CPUs with an unstated b)
    paper = {}
    for law in ("const", "ani", "dis", "rand"):
        pr = PB.make_problem(f"diff3d-{law}", seed=0, m=128)
        bp = np.linspace(0, pr.A.n, 33).astype(np.int32)
        dA = B.DeviceCSR(pr.A)
        xs = torch.as_tensor(pr.x_star).cuda()
        b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, xs, b)
        pols = {"uniform-fp64": dict(select=B.SELECT_KT, fixed_fmt=FMT["fp64"]),
                "fmp-fp32": dict(select=B.SELECT_KT, fixed_fmt=FMT["fp32"]),
                "amp-hl10-fp32": dict(select=B.SELECT_KT, fixed_fmt=FMT["fp32"], temporal=B.TEMPORAL_HL,
                                      adp_tol=10.0)}
        timed_step(dA, bp, b, pols["fmp-fp32"])
        res = {m: timed_step(dA, bp, b, p)[0] for m, p in pols.items()}
        paper[f"diff3d-{law}-128^3"] = {m: {k: r[k] for k in ("ms", "setup_ms", "solve_ms", "iters", "true_relres",
                                                             "converged")} for m, r in res.items()}
        paper[f"diff3d-{law}-128^3"]["speedup_fmp_vs_fp64"] = round(res["uniform-fp64"]["ms"] / res["fmp-fp32"]["ms"], 3)
        del dA, b, xs
    out["paper_bjac_k2t2_32blocks"] = paper

    # 256 independent 2D systems in one persistent launch vs one after another
    t0 = time.time()
    systems = PB.batch2d(256, seed=0)
    gen = time.time() - t0
    dAs = [B.DeviceCSR(p.A) for p in systems]
    bs = []
    for d, p in zip(dAs, systems):
        bv = torch.empty(p.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(d, torch.as_tensor(p.x_star).cuda(), bv)
        bs.append(bv)
    pol = dict(select=B.SELECT_FIXED, fixed_fmt=FMT["fp32"])

    def batched_step():
        xs_ = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in systems]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt = B.Batch(dAs, [p.block_ptr for p in systems], **pol)
        rc, st = bt.solve(bs, xs_, tol=TOL, maxit=20000)
        info = bt.info()
        bt.close()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), rc, st, info

    batched_step()
    ms_b, rc, st, info = batched_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    seq_it = []
    for d, p, bv in zip(dAs, systems, bs):
        h = B.bjac_setup(d, p.block_ptr, **pol)
        xv = torch.zeros(p.A.n, dtype=torch.float64, device="cuda")
        seq_it.append(h.solve(bv, xv, tol=TOL, maxit=20000)["iters"])
        h.close()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    its = [s["iters"] for s in st]
    out["batched2d-256-sides32..512-fp32-bs16/32"] = {
        "systems": len(systems), "rows": int(sum(p.A.n for p in systems)),
        "nnz": int(sum(p.A.nnz for p in systems)), "generate_s": round(gen, 1),
        "batched": {"ms": round(ms_b, 3), "setup_ms": round(st[0]["setup_ms"], 3),
                    "solve_ms": round(st[0]["solve_ms"], 3), "status": rc,
                    "all_converged": all(s["converged"] for s in st),
                    "worst_true_relres": max(s["true_relres"] for s in st),
                    "iters_max": max(its), "iters_mean": round(float(np.mean(its)), 1),
                    "tile_rows": info["tile_rows"], "grid": info["grid"], "tiles": info["ntiles"]},
        "sequential_single_solver": {"ms": round(ms_s, 3),
                                     "max_iter_diff_vs_batched": int(np.max(np.abs(np.array(seq_it) - np.array(its))))},
        "speedup_batched_vs_sequential": round(ms_s / ms_b, 3)}
    return out


# ------------------------------------------------------------------------------------------
def host_cpu():
    """(model name, logical cores) of this host: lscpu, else /proc/cpuinfo."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return model or platform.processor() or "unknown", os.cpu_count() or 1


def oracle_problem(args):
    import oracle as O
    from paper_2407_15973_gb300 import problems as PB
    pr = PB.make_problem("subcube3d", seed=0, m=args.m, bs=args.bs)
    return pr, O.spmv(pr.A, pr.x_star)


def oracle_iters(args, fallback=None):
    """The oracle's own iteration count for this system (a whole serial solve run once by
    oracle/reference_runs.py), else `fallback` (the GPU's count), with the source named."""
    ref = os.path.join(ROOT, "oracle", "full_size_reference.json")
    key = f"m{args.m}_bs{args.bs}_{args.fmt}"
    if os.path.exists(ref):
        with open(ref) as f:
            it = json.load(f).get(key, {}).get("iters", 0)
        if it:
            return it, "the oracle's own whole solve of this system (oracle/full_size_reference.json)"
    if fallback:
        return fallback, "the GPU solve's count (no whole oracle solve recorded for this system)"
    raise SystemExit(f"no oracle iteration count for {key}: run oracle/reference_runs.py")


def oracle_sample(pr, b, args, k, parallel):
    """The CPU oracle, unchanged, on the bench's own system: its full setup (binary64 LU
    inverse of every block, rounding to the format) and then k PCG iterations of fMP in the
    binary32-emulation mode (the GPU's arithmetic), both timed with a wall clock. parallel:
    the OpenMP build of the same source on every host core (same bits), else the
    single-threaded checker. Returns (setup seconds, seconds per iteration, threads)."""
    import oracle as O
    old = O.use_parallel(parallel)
    try:
        threads = O.threads()
        t0 = time.perf_counter()
        P = O.Preconditioner(pr.A, pr.block_ptr, fmt=FMT[args.fmt])
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.pcg(pr.A, P, b, tol=TOL, maxit=k, policy=O.POLICY_FMP, mode=1)
        t_iter = (time.perf_counter() - t0) / k
    finally:
        O.use_parallel(old)
    return t_setup, t_iter, threads


def cpu_baseline(args, gpu_iters):
    """The oracle timed on this host: all cores (the baseline) and one thread, each on a
    bounded sample (full setup + a few iterations), extrapolated to a whole solve."""
    model, cores = host_cpu()
    pr, b = oracle_problem(args)
    iters, src = oracle_iters(args, gpu_iters)
    s_all, it_all, thr = oracle_sample(pr, b, args, args.cpu_iters, True)
    s_one, it_one, _ = oracle_sample(pr, b, args, max(2, args.cpu_iters // 4), False)
    ms_all = (s_all + it_all * iters) * 1e3
    ms_one = (s_one + it_one * iters) * 1e3
    return {"value": round(ms_all, 1), "unit": "ms", "cores": thr, "threads": thr, "host_cores": cores,
            "cpu_model": model, "kind": "oracle", "extrapolated": True, "timed_iters": args.cpu_iters,
            "scaled_to_iters": iters, "iters_source": src,
            "setup_s": round(s_all, 3), "ms_per_iter": round(it_all * 1e3, 2),
            "sample": f"OpenMP build on {thr} threads: full setup ({s_all:.2f} s) + {args.cpu_iters} fMP PCG "
                      f"iterations ({it_all * 1e3:.1f} ms each) of the same {args.m}^3 system, timed; "
                      f"time to solution = setup + {iters} x per-iteration time",
            "single_thread": {"value": round(ms_one, 1), "threads": 1, "timed_iters": max(2, args.cpu_iters // 4),
                              "setup_s": round(s_one, 3), "ms_per_iter": round(it_one * 1e3, 2)}}


def run_reference(args, world):
    """The reference arm: the oracle (the paper has no code), OpenMP build on every host core.
    Each step is a bounded sample, timed (full setup + --ref-iters PCG iterations); the
    metric is that sample extrapolated to a whole solve (median over the timed steps)."""
    model, cores = host_cpu()
    pr, b = oracle_problem(args)
    iters, src = oracle_iters(args)
    k = args.ref_iters
    walls, ttx, setups, per_it = [], [], [], []
    thr = 1
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s, it, thr = oracle_sample(pr, b, args, k, True)
        wall = time.perf_counter() - t0
        if i >= args.warmup:
            walls.append(wall)
            setups.append(s)
            per_it.append(it)
            ttx.append((s + it * iters) * 1e3)
    value = statistics.median(ttx)
    cb = {"value": round(value, 1), "unit": "ms", "cores": thr, "threads": thr, "host_cores": cores,
          "cpu_model": model, "kind": "oracle", "extrapolated": True, "timed_iters": k, "scaled_to_iters": iters,
          "iters_source": src, "setup_s": round(statistics.median(setups), 3),
          "ms_per_iter": round(statistics.median(per_it) * 1e3, 2),
          "sample": f"each step: OpenMP build on {thr} threads, full setup + {k} fMP PCG iterations of the same "
                    f"{args.m}^3 system, timed; value = median over steps of setup + {iters} x per-iteration time"}
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(walls) * 1e3, 1),
            "extrapolated": True, "timed_iters": k, "scaled_to_iters": iters,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (oracle; f32-emulated block apply)", "data": "synthetic (seeded generator, b = A x*)",
            "config": workload_config(args), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_batch(args):
    """The batched kernel on a smaller batch of the 256-system workload's law, for ncu."""
    import torch
    from paper_2407_15973_gb300 import binding as B
    from paper_2407_15973_gb300 import problems as PB
    torch.cuda.init()
    systems = PB.batch2d(args.profile_batch, seed=0)
    dAs = [B.DeviceCSR(p.A) for p in systems]
    bs = []
    for d, p in zip(dAs, systems):
        bv = torch.empty(p.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(d, torch.as_tensor(p.x_star).cuda(), bv)
        bs.append(bv)
    runs = []
    for _ in range(2):
        xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in systems]
        bt = B.Batch(dAs, [p.block_ptr for p in systems], select=B.SELECT_FIXED, fixed_fmt=FMT["fp32"])
        rc, st = bt.solve(bs, xs, tol=TOL, maxit=args.profile_iters or 200)
        runs.append({"solve_ms": round(st[0]["solve_ms"], 3), "status": rc, **bt.info()})
        bt.close()
    return {"profile_batch": {"systems": len(systems), "rows": int(sum(p.A.n for p in systems)),
                              "nnz": int(sum(p.A.nnz for p in systems)), "runs": runs}}


def main():
    args = parse()
    if args.profile_batch:
        print(json.dumps(profile_batch(args)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, world)))
        return
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    out = run_ours(args, rank, world, dist)
    if rank == 0 and world == 1 and not args.profile_iters:
        if not args.no_configs:
            out["other_configs"] = other_configs()
        out["cpu_baseline"] = cpu_baseline(args, out["iters"])
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
