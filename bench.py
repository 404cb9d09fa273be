#!/usr/bin/env python3
"""AU-NMF throughput on one GB300 (or N replicas): iterations/s of Alg. 1 on a
dense 96,000 x 64,000 FP32 matrix (planted rank 50 + |N(0, 0.01^2)| noise),
k = 50, through the library's C ABI.

One step = one AU-NMF iteration (both products with A, both Gram matrices,
both local updates, the relative residual).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--algo hals] [--prec tf32]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NMF iters/s & TFLOP/s (MU/HALS/ABPP), mixed vs FP32 at matched rel. residual"
M_FULL, N_FULL, K_FULL, RANK_FULL, SEED = 96_000, 64_000, 50, 50, 1609
# --workload: the default dense case, the sparse case and the 80 GB dense case
WORKLOADS = {
    "dense": {"m": M_FULL, "n": N_FULL, "k": K_FULL, "rank": RANK_FULL},
    "sparse": {"m": 1_000_000, "n": 500_000, "k": 50, "density": 1e-4},
    "scale": {"m": 172_800, "n": 115_200, "k": 100, "rank": 100},
    # 256 problems, m and n uniform in [500, 8000], k from {8, 16, 32, 64}, ABPP
    "batched": {"m": 8000, "n": 8000, "k": 64, "count": 256},
    # the dense matrix factorised at ranks from 10 to 512 (Sec. 6.3's sweep of k,
    # carried past the rank where the products leave the HBM roof)
    # power-law sparse matrix at the size of webbase-2001 (Sec. 6, the paper's
    # largest sparse input), which is not available: synthetic stand-in
    "webbase": {"m": 118_142_155, "n": 118_142_155, "k": 50, "nnz": 1_019_903_190},
    "ksweep": {"m": M_FULL, "n": N_FULL, "k": 512, "rank": RANK_FULL,
               "ks": [10, 20, 30, 40, 50, 64, 100, 128, 192, 256, 320, 384, 448, 512]},
}
# dense tensor rate of TF32 relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def recorded_traffic(workload_key, prec, launch):
    """DRAM bytes of one product launch from a committed ncu capture, or None
    when there is none or the kernel's source changed since it was taken."""
    import hashlib

    try:
        entries = json.load(open(TRAFFIC))["entries"]
    except Exception:
        return None
    for e in entries:
        if (e["workload"], e["prec"], e["launch"]) != (workload_key, prec, launch):
            continue
        src = os.path.join(ROOT, e["source"])
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        except OSError:
            return None
        return e["dram_bytes"] if sha == e["source_sha256"] else None
    return None
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP32_LANES = 128  # FP32 FMA lanes per SM


def num_sms(device=0):
    import torch

    return torch.cuda.get_device_properties(device).multi_processor_count


def peaks():
    try:
        d = json.load(open(PEAKS))
        return d, "measured"
    except Exception:
        return FALLBACK, "fallback"


def flops_per_iter(m, n, k, algo):
    """Sec. 5.2.1: 4mnk + (m+n)k^2 for the products and Grams; MU/HALS local
    updates add 2(m+n)k^2 (Secs. 4.1, 4.2).  BPP's local work is data
    dependent and not counted."""
    f = 4.0 * m * n * k + (m + n) * k * k
    if algo in ("mu", "hals"):
        f += 2.0 * (m + n) * k * k
    return f


def product_bytes(m, n, k, prec):
    """Algorithmic bytes of one dense product launch: A once (4 B FP32/TF32,
    2 B for the BF16 copy), the fixed factor once, the output once."""
    ea = 2 if prec == "bf16" else 4
    return ea * m * n + 4 * (n * k + m * k)


def spmm_bytes(rows, cols, nnz, k):
    """Algorithmic bytes of one sparse product launch: values and column
    indices once (8 B per nonzero), row pointers, the fixed factor once, the
    output once."""
    return 8 * nnz + 8 * (rows + 1) + 4 * cols * k + 4 * rows * k


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    import torch.distributed as dist

    import datetime

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # a replica that dies or never arrives ends the others' next barrier
        # or reduction with an error after this long, instead of a hang
        timeout = datetime.timedelta(seconds=float(os.environ.get("AUNMF_PG_TIMEOUT_S", "600")))
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo", timeout=timeout)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    # NCCL reduces device tensors, gloo (CPU runs of the replica logic) host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- oracle
def oracle_sample(algo, A_slice, k, iters=1):
    """Runs the FP64 oracle on a slice of the workload; returns (seconds per
    iteration, threads)."""
    import numpy as np

    from oracle import oracle as orc
    from paper_1609_09154_gb300 import synth

    ms, ns = A_slice.shape
    W0, H0 = synth.init_factors(ms, ns, k, seed=SEED)
    t0 = time.perf_counter()
    out = orc.nmf_run(A_slice, k, algo, iters, W0, H0)
    dt = (time.perf_counter() - t0) / iters
    assert out["rc"] in (0, -5) and np.isfinite(out["relres"]).all()
    return dt, orc.num_threads()


def make_slice(ms, ns):
    """A slice with the workload's recipe (rank-50 uniform factors + noise),
    drawn on the host in FP64 and rounded to FP32."""
    import numpy as np

    from paper_1609_09154_gb300 import synth

    A, _, _ = synth.dense_lowrank(ms, ns, RANK_FULL, seed=SEED)
    return A.astype(np.float32).astype(np.float64)


SLICE = (19_200, 12_800)  # 1/25 of the rows x 1/5 of the columns: 4% of the entries


def cpu_baseline(algo, k, iters=1):
    ms, ns = SLICE
    A = make_slice(ms, ns)
    dt, threads = oracle_sample(algo, A, k, iters)
    scale = (M_FULL * N_FULL) / (ms * ns)  # the products dominate: cost ~ m n k
    return {
        "value": 1.0 / (dt * scale), "unit": "iters/s", "cores": threads, "kind": "oracle",
        "sample": (f"{iters} {algo.upper()} iteration(s) of the FP64 oracle on a {ms}x{ns} "
                   f"slice (k={k}, same recipe), {dt:.2f} s/iteration, scaled by the "
                   f"entry ratio {scale:.0f} to the {M_FULL}x{N_FULL} workload"),
    }


def run_reference(args):
    world, rank, _ = (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if rank != 0:
        return 0
    from oracle import oracle as orc

    orc.build()
    if args.oracle_full:
        return run_reference_full(args)
    ms, ns = SLICE
    A = make_slice(ms, ns)
    scale = (M_FULL * N_FULL) / (ms * ns)
    for _ in range(args.warmup):
        oracle_sample(args.algo, A[:ms // 8], args.k, 1)  # short untimed warm-up
    t0 = time.perf_counter()
    threads = 1
    for _ in range(args.steps):
        _, threads = oracle_sample(args.algo, A, args.k, 1)
    dt = (time.perf_counter() - t0) / args.steps
    value = 1.0 / (dt * scale)
    cfg = config_dict(args)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # the measured wall time of one step, i.e. of one sampled iteration;
        # value = 1 / (that time x sample_scale)
        "ms_per_step": dt * 1e3, "sample_scale": scale,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step: one {args.algo.upper()} iteration of the FP64 "
                                   f"oracle on a {ms}x{ns} slice ({dt:.2f} s measured), "
                                   f"iters/s of the {M_FULL}x{N_FULL} workload = 1 / ({dt:.2f} s"
                                   f" x {scale:.0f}), the entry ratio (the products, O(m n k), "
                                   f"dominate the oracle's iteration)"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_full(args):
    """The oracle on the whole 96,000 x 64,000 workload (A drawn on the host in
    FP64 by row blocks, 49 GB), `steps` iterations timed without scaling: a
    check of the slice-and-scale figure the default arms report.  Minutes of
    host time per iteration; not part of the default run."""
    import numpy as np

    from oracle import oracle as orc
    from paper_1609_09154_gb300 import synth

    m, n, k = M_FULL, N_FULL, args.k
    t0 = time.perf_counter()
    A, _, _ = synth.dense_lowrank_blocked(m, n, RANK_FULL, seed=SEED)
    np.copyto(A, A.astype(np.float32))  # the FP32-rounded A the GPU sees
    W0, H0 = synth.init_factors(m, n, k, seed=SEED)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    out = orc.nmf_run(A, k, args.algo, args.steps, W0, H0)
    dt = (time.perf_counter() - t0) / args.steps
    assert out["rc"] in (0, -5) and np.isfinite(out["relres"]).all()
    ms, ns = SLICE
    dt_slice, threads = oracle_sample(args.algo, make_slice(ms, ns), k, 1)
    line = {
        "impl": "reference", "oracle_full": True, "metric": METRIC, "value": 1.0 / dt,
        "unit": "iters/s", "steps": args.steps, "ms_per_step": dt * 1e3, "dtype": "f64",
        "config": config_dict(args), "cores": threads, "host_generation_s": round(t_gen, 1),
        "relres": [float(x) for x in out["relres"]],
        "slice_check": {"slice": f"{ms}x{ns}", "s_per_iter": dt_slice,
                        "scaled_s_per_iter": dt_slice * (m * n) / (ms * ns),
                        "full_over_scaled": dt / (dt_slice * (m * n) / (ms * ns))},
    }
    print(json.dumps(line))
    return 0


def config_dict(args):
    m, n = getattr(args, "m", M_FULL), getattr(args, "n", N_FULL)
    wl = getattr(args, "workload", "dense")
    if wl == "webbase":
        desc = (f"sparse CSR {m}x{n}, {args.nnz:,} nonzeros drawn with power-law row and column "
                f"degrees (stand-in for webbase-2001), values U(0,1], k={args.k}, "
                f"{args.algo.upper()}, FP32 SpMM")
        size = f"{8 * args.nnz / 1e9:.1f} GB of CSR values and indices"
    elif wl == "sparse":
        desc = (f"sparse CSR {m}x{n}, density {args.density:g} at uniform positions, values "
                f"U(0,1], k={args.k}, {args.algo.upper()}, FP32 SpMM")
        size = f"{8 * m * n * args.density / 1e9:.2f} GB of CSR values and indices"
    else:
        desc = (f"dense {m}x{n} FP32, planted rank {getattr(args, 'rank', RANK_FULL)} + "
                f"|N(0,0.01^2)|, k={args.k}, {args.algo.upper()}, products in "
                f"{args.prec.upper()}")
        size = f"A is {4 * m * n / 1e9:.1f} GB"
    return {"workload": desc, "m": m, "n": n, "k": args.k, "algo": args.algo,
            "prec": args.prec,
            "l2": f"inputs larger than the 129 MB L2 ({size}), no flush needed",
            "parallelism": f"replicas x{args.gpus}"}


def workload_key(args):
    return f"{args.workload} {args.m}x{args.n} k={args.k}"


# --------------------------------------------------------------------- batched
def run_batched(args):
    """One batched ABPP run of `steps` iterations over 256 uneven problems,
    against looping the single-problem entry point over them."""
    import numpy as np
    import torch

    from paper_1609_09154_gb300 import aunmf, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = np.random.default_rng(SEED + rank)
    count = WORKLOADS["batched"]["count"]
    dims = [(int(g.integers(500, 8001)), int(g.integers(500, 8001)), int(g.choice([8, 16, 32, 64])))
            for _ in range(count)]
    As, H0s, ks = [], [], []
    for i, (m, n, k) in enumerate(dims):
        A, _, _ = synth.dense_lowrank_torch(m, n, k, seed=SEED + 31 * i + rank, device=dev)
        _, H0 = synth.init_factors_torch(m, n, k, seed=SEED + 31 * i + rank, device=dev)
        As.append(A)
        H0s.append(H0)
        ks.append(k)
    torch.cuda.synchronize()
    h = aunmf.Handle()
    h.run_batched(As, ks, args.warmup, H0s, prec=args.prec, allow_noconverge=True)  # + autotune
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Ws, Hs, rel, info = h.run_batched(As, ks, args.steps, H0s, prec=args.prec,
                                      allow_noconverge=True)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    t_batch = max_over_ranks(e0.elapsed_time(e1), world)
    clk = clocks.stop()
    # the same work through the single-problem path, one problem after another
    torch.cuda.synchronize()
    e0.record()
    for A, k, H0 in zip(As, ks, H0s):
        h.run(A, k, "abpp", args.steps, torch.zeros((A.shape[0], k), device=dev), H0,
              prec=args.prec, allow_noconverge=True)
    e1.record()
    torch.cuda.synchronize()
    t_loop = max_over_ranks(e0.elapsed_time(e1), world)
    if rank == 0:
        sum_mn = sum(m * n for m, n, _ in dims)
        ea = 2 if args.prec == "bf16" else 4
        bytes_iter = 2 * ea * sum_mn  # each product streams one copy of every A once
        line = {
            "metric": METRIC, "value": world * args.steps / (t_batch / 1e3),
            "unit": "batch iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.prec, "data": "synthetic",
            "config": {"workload": f"batched: {count} dense problems, m, n uniform in [500, 8000], "
                                   f"k from {{8,16,32,64}}, planted rank k + noise, ABPP, products "
                                   f"in {args.prec.upper()}",
                       "sum_mn": sum_mn, "l2": "inputs larger than L2, no flush needed",
                       "parallelism": f"replicas x{world}"},
            "loop_ms_per_step": t_loop / args.steps, "speedup_vs_loop": t_loop / t_batch,
            "roofline": {"bound": "hbm", "achieved": bytes_iter / (t_batch / args.steps / 1e3) / 1e9,
                         "peak": peaks()[0]["hbm_gbs"], "unit": "GB/s",
                         "frac": bytes_iter / (t_batch / args.steps / 1e3) / 1e9 / peaks()[0]["hbm_gbs"],
                         "traffic": None,
                         "kernel": "whole batched iteration (A's bytes of both products over the step)",
                         "note": "the products stream at HBM speed; the iteration is bound by the "
                                 "BPP solves (~2.2M right-hand sides per iteration, issue- and "
                                 "latency-bound), so this fraction is the products' share of the step"},
            "relres_median_last": float(np.median(rel[:, -1])), "bpp_pivots": info["bpp_pivots"],
            "tuned_bpp_tile": [info["tuned_bpp_warps"], info["tuned_bpp_rows"]],
            "tuned_gemm_stages": [info["tuned_gemm_stages_aht"], info["tuned_gemm_stages_wta"]],
            "gpu_launches": int(info["launches"]), "clocks": clk,
        }
        print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- k sweep
def run_ksweep(args):
    """HALS on the dense matrix at each rank of the sweep, TF32 and BF16
    products: iterations/s (CUDA graph) and the product launches' average
    times (profile mode), with the fraction of the HBM roof (algorithmic
    bytes) and of the tensor roof (2 m n k flop per product) each reaches."""
    import torch

    from paper_1609_09154_gb300 import aunmf, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n = args.m, args.n
    A, _, _ = synth.dense_lowrank_torch(m, n, args.rank, seed=SEED + rank, device=dev)
    h = aunmf.Handle()
    pk, pks = peaks()
    tensor_peak = {"tf32": pk["bf16_tflops"] * TF32_PER_BF16, "bf16": pk["bf16_tflops"]}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    clocks.start()
    rows, launches = [], 0
    for k in (args.ks or WORKLOADS["ksweep"]["ks"]):
        W0, H0 = synth.init_factors_torch(m, n, k, seed=SEED + rank, device=dev)
        W, H = torch.empty_like(W0), torch.empty_like(H0)
        for prec in ("tf32", "bf16"):
            h.run(A, k, "hals", args.warmup, W0, H0, prec=prec, out=(W, H))
            barrier(world)
            torch.cuda.synchronize()
            e0.record()
            _, _, rel, inf_t = h.run(A, k, "hals", args.steps, W0, H0, prec=prec, out=(W, H))
            e1.record()
            launches += int(inf_t["launches"])
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world)
            _, _, _, inf = h.run(A, k, "hals", args.steps, W0, H0, prec=prec, out=(W, H),
                                 profile=True)
            t_aht = inf["ms_aht"] / max(1, inf["n_aht"])
            t_wta = inf["ms_wta"] / max(1, inf["n_wta"])
            t = max(t_aht, t_wta) / 1e3
            gbs = product_bytes(m, n, k, prec) / t / 1e9
            tfs = 2.0 * m * n * k / t / 1e12
            fh, ft = gbs / pk["hbm_gbs"], tfs / tensor_peak[prec]
            rows.append({"k": k, "prec": prec, "iters_per_s": world * args.steps / (ms / 1e3),
                         "relres_last": float(rel[-1]), "ms_aht": round(t_aht, 4),
                         "ms_wta": round(t_wta, 4), "product_gbs": round(gbs, 1),
                         "product_tflops": round(tfs, 1), "frac_hbm": round(fh, 4),
                         "frac_tensor": round(ft, 4), "bound": "hbm" if fh >= ft else "tensor"})
        del W0, H0, W, H
    clk = clocks.stop()
    if rank == 0:
        top = [r for r in rows if r["k"] == args.k and r["prec"] == args.prec] or rows[-1:]
        top = top[0]
        ach = top["product_tflops"]
        line = {
            "metric": METRIC, "value": top["iters_per_s"], "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": world * 1e3 / top["iters_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": top["prec"], "data": "synthetic",
            "config": {"workload": f"k sweep: dense {m}x{n} FP32, planted rank {args.rank} + "
                                   f"|N(0,0.01^2)|, HALS at k in {args.ks or WORKLOADS['ksweep']['ks']}, "
                                   f"TF32 and BF16 products; value at k={top['k']} "
                                   f"{top['prec'].upper()}",
                       "m": m, "n": n, "k": top["k"], "algo": "hals", "prec": top["prec"],
                       "l2": "inputs larger than the 129 MB L2, no flush needed",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": top["bound"], "achieved": ach,
                         "peak": round(tensor_peak[top["prec"]], 1), "unit": "TFLOP/s",
                         "frac": ach / tensor_peak[top["prec"]], "traffic": None,
                         "kernel": "k_gemm_tc (the slower product launch)",
                         "peak_note": f"bf16_tflops of {pks} peaks"
                                      + (" x 1.1/2.25 (nominal TF32/BF16 ratio)"
                                         if top["prec"] == "tf32" else "")},
            "sweep": rows, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- accuracy
def accuracy_vs_oracle(h, dev, iters=30):
    """Every local update in every precision form against the FP64 oracle on
    the small dense configuration (2,000 x 1,500, planted rank 10 + noise,
    k = 10, 30 iterations from the same (W0, H0)): the largest |relres
    difference| over the iterations, the final one, the relative difference
    of the objective 0.5 ||A - WH||^2 (= relres^2 ||A||^2 / 2), and the
    factors' relative Frobenius distance from the oracle's."""
    import numpy as np
    import torch

    from oracle import oracle as orc
    from paper_1609_09154_gb300 import synth

    m, n, k = 2000, 1500, 10
    A, _, _ = synth.dense_lowrank(m, n, k, seed=2024)
    W0, H0 = synth.init_factors(m, n, k, seed=2024)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    A, W0, H0 = r32(A), r32(W0), r32(H0)
    d = lambda x: torch.as_tensor(x.astype(np.float32), device=dev)  # noqa: E731
    out = {"workload": f"dense {m}x{n}, planted rank {k} + |N(0,0.01^2)|, k={k}, "
                       f"{iters} iterations, FP64 oracle on the same FP32-rounded inputs"}
    for algo in ("mu", "hals", "abpp"):
        ref = orc.nmf_run(A, k, algo, iters, W0, H0)
        rr = ref["relres"]
        nw, nh = np.linalg.norm(ref["W"]), np.linalg.norm(ref["H"])
        for prec in ("fp32", "tf32", "bf16"):
            W, H, rel, _ = h.run(d(A), k, algo, iters, d(W0), d(H0), prec=prec,
                                 allow_noconverge=True)
            Wh = W.cpu().numpy().astype(np.float64)
            Hh = H.cpu().numpy().astype(np.float64)
            out[f"{algo}_{prec}"] = {
                "relres_max_abs_diff": float(np.abs(rel - rr).max()),
                "relres_last_abs_diff": float(abs(rel[-1] - rr[-1])),
                "objective_rel_diff": float(abs(rel[-1] ** 2 - rr[-1] ** 2) / rr[-1] ** 2),
                "w_rel_err": float(np.linalg.norm(Wh - ref["W"]) / nw),
                "h_rel_err": float(np.linalg.norm(Hh - ref["H"]) / nh),
            }
    return out


# --------------------------------------------------------------------- gather roof
def gather_roof(aunmf, csr, m, n, k, kern, dev, reps=5):
    """The sparse products against the measured gather roof: the library's
    probe kernel loads the same rows the product gathers (the CSR's column
    indices over H^T for A H^T, the CSC's row indices over W for W^T A) and
    does nothing else; fraction = probe time / product time."""
    import torch

    rowptr, colidx, _ = csr
    counts = (rowptr[1:] - rowptr[:-1]).to(torch.int64)
    rows_of = torch.repeat_interleave(torch.arange(m, device=dev, dtype=torch.int32), counts)
    order = torch.sort(colidx, stable=True).indices
    csc_rows = rows_of[order].contiguous()
    del rows_of, order
    ld = (k + 3) // 4 * 4
    sink = torch.zeros(1, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, idx, nrows in (("aht", colidx, n), ("wta", csc_rows, m)):
        X = torch.rand((nrows, ld), device=dev)
        for _ in range(2):
            aunmf.probe_gather(idx, X, k, sink)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0.record()
            aunmf.probe_gather(idx, X, k, sink)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        sp = kern[name]["ms_avg"]
        out[name] = {"probe_ms": round(best, 4), "spmm_ms": round(sp, 4),
                     "frac_of_gather_roof": best / sp,
                     "gathered_tbs": idx.numel() * k * 4 / (best / 1e3) / 1e12,
                     "table_mb": round(nrows * k * 4 / 1e6, 1)}
        del X
    out["note"] = ("probe = the library's gather-roof kernel on the product's own index stream "
                   "(every nonzero's factor row loaded once, widest loads, no other work); "
                   "best of 5 CUDA-event timings")
    return out


# --------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    from paper_1609_09154_gb300 import aunmf, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n, k = args.m, args.n, args.k
    sparse = args.workload in ("sparse", "webbase")
    if args.workload == "webbase":
        csr = synth.sparse_powerlaw_torch(m, n, args.nnz, seed=SEED + rank, device=dev)
        torch.cuda.empty_cache()
    if sparse:
        if args.workload == "sparse":
            csr = synth.sparse_uniform_torch(m, n, args.density, seed=SEED + rank, device=dev)
        A = aunmf.csr_matrix(*csr, (m, n))
        nnz = int(csr[2].numel())
    else:
        A, _, _ = synth.dense_lowrank_torch(m, n, args.rank, seed=SEED + rank, device=dev)
        nnz = m * n
    W0, H0 = synth.init_factors_torch(m, n, k, seed=SEED + rank, device=dev)
    torch.cuda.synchronize()
    h = aunmf.Handle()
    W = torch.empty_like(W0)
    H = torch.empty_like(H0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(prec, profile=False, algo=None):
        """warm-up (untimed), then `steps` iterations from (W0, H0) timed with
        CUDA events around the call (the library's stream is the current
        stream's device; the call returns after its stream synchronises)."""
        algo = algo or args.algo
        h.run(A, k, algo, args.warmup, W0, H0, prec=prec, out=(W, H), allow_noconverge=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record()
        _, _, r, inf = h.run(A, k, algo, args.steps, W0, H0, prec=prec, out=(W, H),
                             profile=profile, allow_noconverge=True)
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world), r, inf

    # the timed region of the headline number: the whole run, as a CUDA graph
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms_total, rel, info_g = timed(args.prec)
    clk = clocks.stop()
    value = world * args.steps / (ms_total / 1e3)
    # the same run in profile mode (no graph; CUDA events around each phase on
    # the library's stream) for the per-kernel durations of the roofline
    _, _, info = timed(args.prec, profile=True)
    # the three precision forms from the same start: matched residual, the
    # factors' distance from the FP32 form's, and the time each form takes to
    # reach a residual that all of them reach
    forms = None
    if not sparse and not args.no_forms:
        forms, fac, rels = {}, {}, {}
        for pr in ("fp32", "tf32", "bf16"):
            t, r, _ = timed(pr)
            fac[pr] = (W.clone(), H.clone())
            rels[pr] = r
            forms[pr] = {"iters_per_s": world * args.steps / (t / 1e3),
                         "ms_per_step": t / args.steps, "relres_last": float(r[-1])}
        base = forms["fp32"]
        target = max(f["relres_last"] for f in forms.values())
        Wb, Hb = fac["fp32"]
        for pr, f in forms.items():
            f["speedup_vs_fp32"] = f["iters_per_s"] / base["iters_per_s"]
            f["relres_gap_vs_fp32"] = abs(f["relres_last"] - base["relres_last"])
            Wf, Hf = fac[pr]
            f["w_rel_err_vs_fp32"] = float(torch.linalg.norm(Wf - Wb) / torch.linalg.norm(Wb))
            f["h_rel_err_vs_fp32"] = float(torch.linalg.norm(Hf - Hb) / torch.linalg.norm(Hb))
            hit = int(np.argmax(rels[pr] <= target)) + 1
            f["iters_to_target"] = hit
            f["ms_to_target"] = hit * f["ms_per_step"]
        forms["target_relres"] = target
        forms["note"] = ("each form runs the same iterations from the same (W0, H0); the target "
                         "is the largest final relres of the three, which all of them reach; "
                         "factor errors are ||X_form - X_fp32||_F / ||X_fp32||_F")
        del fac

    # the paper's three local updates (Secs. 4.1-4.3) on the same input and
    # precision: iterations/s, relres, time per phase and the product roofline
    algos = None
    if not sparse and not args.no_algos:
        algos = {}
        for al in ("mu", "hals", "abpp"):
            t, r, _ = timed(args.prec, algo=al)
            _, _, inf = timed(args.prec, profile=True, algo=al)
            st = max(1, args.steps)
            ph = {p: round(inf[f"ms_{p}"] / st, 4) for p in ("aht", "wta", "update", "gram", "other")}
            t_prod = max(inf["ms_aht"] / max(1, inf["n_aht"]), inf["ms_wta"] / max(1, inf["n_wta"]))
            prod = {"ms_avg": round(t_prod, 4)}
            if args.prec != "fp32":
                gbs = product_bytes(m, n, k, args.prec) / (t_prod / 1e3) / 1e9
                prod.update({"bound": "hbm", "achieved_gbs": round(gbs, 1),
                             "frac": gbs / peaks()[0]["hbm_gbs"]})
            algos[al] = {"iters_per_s": world * args.steps / (t / 1e3),
                         "ms_per_step": t / args.steps, "relres_last": float(r[-1]),
                         "phases_ms_per_step": ph, "slower_product": prod,
                         "update_share": ph["update"] / max(1e-9, sum(ph.values())),
                         "bpp_redone": inf.get("bpp_redone", 0) if al == "abpp" else None}

    # dominant kernel: the product launch with the larger summed time
    pk, pks = peaks()
    kern = {
        "aht": {"ms_avg": info["ms_aht"] / max(1, info["n_aht"]), "launches": info["n_aht"]},
        "wta": {"ms_avg": info["ms_wta"] / max(1, info["n_wta"]), "launches": info["n_wta"]},
    }
    dom = max(kern, key=lambda x: kern[x]["ms_avg"] * kern[x]["launches"])
    t_launch = kern[dom]["ms_avg"] / 1e3
    if sparse:
        by = spmm_bytes(m, n, nnz, k) if dom == "aht" else spmm_bytes(n, m, nnz, k)
        ach = by / t_launch / 1e9
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": recorded_traffic(workload_key(args), args.prec, dom),
                "kernel": f"{dom} (CSR/CSC SpMM)",
                "peak_note": f"hbm_gbs of {pks} peaks; algorithmic bytes count each nonzero, "
                             f"the fixed factor and the output once (the k-vector gathers "
                             f"are served from L2)"}
    elif args.prec == "fp32":
        sm_mhz = (clk or {}).get("sm_mhz") or 1485.0
        sms = num_sms(local)
        peak = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        ach = 2.0 * m * n * k / t_launch / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "kernel": f"{dom} (FP32 FMA products)",
                "peak_note": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (median SM "
                             f"clock sampled during the timed region)"}
    else:
        by = product_bytes(m, n, k, args.prec)
        ach = by / t_launch / 1e9
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": recorded_traffic(workload_key(args), args.prec, dom),
                "kernel": f"{dom} (k_gemm_tc)",
                "peak_note": f"hbm_gbs of {pks} peaks"}
    if args.workload == "sparse":
        roof["gather_roof"] = gather_roof(aunmf, csr, m, n, k, kern, dev)
    for kk in kern.values():
        kk["ms_avg"] = round(kk["ms_avg"], 4)
    steps = max(1, args.steps)
    phases = {p: round(info[f"ms_{p}"] / steps, 4) for p in ("aht", "wta", "update", "gram", "other")}
    phases["setup_and_teardown_ms_total"] = round(
        info["ms_total"] - sum(info[f"ms_{p}"] for p in ("aht", "wta", "update", "gram", "other")), 3)

    # end to end through the host-buffer entry point: H2D of A, W0, H0 and the
    # D2H of W, H, relres inside the timed region
    e2e = None
    if not args.no_e2e and not sparse:
        Ah = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
        Ah.copy_(A)
        W0h = W0.cpu().pin_memory()
        H0h = H0.cpu().pin_memory()
        Wh = torch.empty((m, k), dtype=torch.float32, pin_memory=True)
        Hh = torch.empty((k, n), dtype=torch.float32, pin_memory=True)
        del A
        torch.cuda.empty_cache()
        barrier(world)
        t0 = time.perf_counter()
        h.run_host(Ah.numpy(), k, args.algo, args.steps, W0h.numpy(), H0h.numpy(),
                   prec=args.prec, W=Wh.numpy(), H=Hh.numpy())
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * args.steps / t_e2e, "unit": "iters/s",
               "h2d_bytes_per_step": (4 * m * n + 4 * m * k + 4 * k * n) / args.steps,
               "d2h_bytes_per_step": (4 * m * k + 4 * k * n + 8 * args.steps) / args.steps,
               "note": f"one aunmf_run_host call of {args.steps} iterations; copies of "
                       f"the whole input/output amortised over its steps"}
    cpu = None
    if (rank == 0 and world == 1 and not args.no_cpu and args.workload == "dense"
            and (m, n) == (M_FULL, N_FULL)):
        cpu = cpu_baseline(args.algo, k)
    accuracy = None
    if rank == 0 and not args.no_accuracy and not sparse:
        accuracy = accuracy_vs_oracle(h, dev)

    if rank == 0:
        f_it = flops_per_iter(m, n, k, args.algo)
        if sparse:  # Sec. 5.2.1: 4 nnz k for the products
            f_it = f_it - 4.0 * m * n * k + 4.0 * nnz * k
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.prec],
            "data": "synthetic", "config": config_dict(args),
            "tflops": f_it * value / 1e12,
            "relres_last": float(rel[-1]) if len(rel) else None,
            "forms": forms, "algos": algos, "accuracy_vs_fp64": accuracy,
            "roofline": roof, "kernels": kern, "phases_ms_per_step": phases,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(info_g["launches"]), "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="hals", choices=["mu", "hals", "abpp"])
    ap.add_argument("--prec", default="tf32", choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--workload", default="dense", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--m", type=int, default=None, help="rows of A (profiling cases)")
    ap.add_argument("--n", type=int, default=None, help="columns of A (profiling cases)")
    ap.add_argument("--nnz", type=int, default=None, help="nonzeros of the power-law case")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32 / TF32 / BF16 comparison runs")
    ap.add_argument("--no-algos", action="store_true",
                    help="skip the MU / HALS / ABPP runs on the same input")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison with the FP64 oracle on the small configuration")
    ap.add_argument("--ks", type=lambda v: [int(x) for x in v.split(",")], default=None,
                    help="--workload ksweep: ranks to run (comma-separated; default: the full sweep)")
    ap.add_argument("--oracle-full", action="store_true",
                    help="--impl reference: time the oracle on the whole workload, unscaled")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    args.m = args.m or wl["m"]
    args.n = args.n or wl["n"]
    args.k = args.k or wl["k"]
    args.rank = wl.get("rank", RANK_FULL)
    args.density = wl.get("density", 0.0)
    args.nnz = args.nnz or wl.get("nnz", 0)
    if args.workload in ("sparse", "webbase"):
        args.prec = "fp32"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        if args.prec == "fp32":
            args.prec = "tf32"
        return run_batched(args)
    if args.workload == "ksweep":
        if args.prec == "fp32":
            args.prec = "tf32"
        return run_ksweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
