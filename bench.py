#!/usr/bin/env python
"""Benchmark of the crossbar nodal solve on one GB300 (or N independent replicas).

Workload (default ``xbar256_mixed``): a 256 x 256 crossbar (131072 unknowns),
R_s = R_w = R_b = 1 ohm, R_sense = 10 ohm, G log-uniform in [1e-6, 1e-4] S,
8192 input vectors uniform in [0, 0.5] V; synthetic, seeded.

One step = one pass of the whole hot path over one batch, through the C ABI:
    xbar_set_conductances (assembly) -> xbar_factor -> xbar_solve
in the mixed form (FP32 factor + FP32 substitutions + FP64-residual
refinement to max |dI|/|I| <= 1e-8).  ``value`` is input vectors solved per
second (solves/s) over all ranks.  The plain FP64 block-LU path is timed on the
same GPU in the same run (``fp64_baseline``) and the CPU oracle on the host
cores (``cpu_baseline``), which also gives the measured error of this run's
currents.  Phases are timed with CUDA events recorded by the library around
each kernel launch on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xbar|reference]

Multi-GPU: the path has no exchange step; N ranks run independent replicas
(each its own map and batch, seed + rank), ``scaling`` = "weak".
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s vs plain FP64 block-LU on same GPU at ≤1e-8 rel. current error"
UNIT = "solves/s"
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xbar", choices=["xbar", "reference"])
    ap.add_argument("--workload", default="xbar256_mixed")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=64, help="vectors the CPU oracle substitutes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-factor-rates", action="store_true", help="skip the standalone factor timings")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate workload nested in the default line")
    ap.add_argument("--batch", type=int, default=0, help="override the workload's batch size (profiling runs)")
    ap.add_argument("--algorithm", default="thomas", choices=["thomas", "cr"],
                    help="factor and substitution of the pipelined step: block Thomas or block cyclic reduction "
                         "(tensor-core products)")
    ap.add_argument("--epochs", type=int, default=24, help="surrogate workload: training epochs")
    ap.add_argument("--line-passes", type=int, default=2, help="surrogate workload: line-model passes")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Dist:
    """Replicas only: a barrier and max/sum reductions of timing scalars across ranks (NCCL on the
    GPUs; gloo with CPU tensors where there is no GPU, as in the multi-process CPU tests)."""

    def __init__(self, backend="nccl"):
        import torch
        self.rank, self.world, self.local = dist_env()
        self.torch = torch
        self.pg = None
        self.dev = "cuda" if backend == "nccl" else "cpu"
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.dev)
        self.pg.all_reduce(t)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"xbar_clocks_{os.getpid()}_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Peaks of the arithmetic pipes used here, from unit counts and the maximum SM clock of a GB300
# (152 SMs; 128 FP32 lanes and 2 FP64 FMA per SM per clock); HBM from the measured copy.
def pipe_peaks(sm_max_mhz=2070.0):
    clk = sm_max_mhz * 1e6
    return {"fp32_tflops": 152 * 128 * 2 * clk / 1e12, "fp64_tflops": 152 * 2 * 2 * clk / 1e12}


def algorithmic_work(phase, M, N, B):
    """(amount, unit, bound) of the method's own work for ONE launch of a phase kernel."""
    if phase == "sweep":          # (2N-1) dense (M x M)(M x B) products
        return (2 * N - 1) * 2.0 * M * M * B, "flop"
    if phase == "resid":          # per word-line node and vector: chain fwd (3) + bwd (2) + residual (7)
        return 12.0 * M * N * B, "flop"
    if phase == "update":         # w += d (1) and the current dot (2)
        return 3.0 * M * N * B, "flop"
    if phase == "factor":         # N inversions of M x M (Gauss-Jordan 2M^3) + Schur formation
        return N * (2.0 * M ** 3 + 4.0 * M * M), "flop"
    return 0.0, "flop"


# ---------------------------------------------------------------------------------------------
# the xbar (GPU) arm
# ---------------------------------------------------------------------------------------------
def run_xbar(args):
    import torch

    from paper_2410_19993_gb300 import inputs, xbar

    d = Dist()
    rank, world, local = d.rank, d.world, d.local
    torch.cuda.set_device(local)
    w = inputs.WORKLOADS[args.workload]
    M, N, B = w.M, w.N, (args.batch or w.B)
    R = w.circuits[0].as_tuple()
    G, V = inputs.crossbar(M, N, B, seed=w.seed + rank, g_lo=w.g_lo, g_hi=w.g_hi, v_max=w.v_max)
    stream = torch.cuda.current_stream()
    Gd = torch.from_numpy(G).cuda()
    Vd = torch.from_numpy(V).cuda()
    # Two conductance maps in flight, one handle and stream each: step k sets and factors map k+1
    # on its stream, then solves map k's batch on the other.  The factor (a 16-block cluster for
    # the mixed path) runs on SMs the solve leaves free.  Both maps hold the workload's conductances.
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    xbs = [xbar.Crossbar.assemble(Gd, *R, stream=s) for s in streams]
    for xb_ in xbs:
        xb_.set_option("eager_assembly", 1)  # set_conductances assembles: see step_pipelined
        xb_.set_option("algorithm", args.algorithm)
        if args.algorithm == "cr":
            xb_.set_option("cr_products", 1)
    Is = [torch.zeros((B, N), dtype=torch.float64, device="cuda") for _ in range(2)]
    I64s = [torch.zeros((B, N), dtype=torch.float64, device="cuda") for _ in range(2)]
    info_box = {}
    pipe = {"k": 0, "prec": None, "solved": set()}

    def prime(prec):
        """Factor map 0 before a run of pipelined steps (outside any timed region)."""
        torch.cuda.synchronize()
        xbs[0].set_conductances(Gd)
        xbs[0].factor(prec)
        torch.cuda.synchronize()
        pipe["k"], pipe["prec"] = 0, prec

    def step_pipelined(V_in, outs, solve_kwargs):
        k = pipe["k"]
        cur, nxt = xbs[k % 2], xbs[(k + 1) % 2]
        nxt.set_conductances(Gd)  # map k+1: set and (eager_assembly) assembled on its own stream ...
        # map k's solve starts once that assembly is done, with the factor already queued ahead of
        # it: the factor's 16-block cluster then takes its SMs before the solve's sweep fills them
        # (a cluster needs 16 free SMs of one GPC, which a running sweep rarely leaves)
        assembled = torch.cuda.Event()
        assembled.record(streams[(k + 1) % 2])
        streams[k % 2].wait_event(assembled)
        nxt.factor(pipe["prec"])
        _, info = cur.solve(V_in, outs[k % 2], **solve_kwargs)  # ... beside map k's solve
        pipe["solved"].add((id(outs), k % 2))
        pipe["k"] = k + 1
        return info

    def step_mixed():
        info_box.update(step_pipelined(Vd, Is, {"tol": TOL, "max_iter": 10}))

    def step_fp64():
        step_pipelined(Vd, I64s, {})

    def step_mixed_sequential():
        xbs[0].set_conductances(Gd)
        xbs[0].factor("fp32_ir")
        xbs[0].solve(Vd, Is[0], tol=TOL, max_iter=10)

    def timed(fn, K):
        """Device time of K steps: both handles' streams start after and end before the events."""
        d.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s_ in streams:
            s_.wait_event(e0)
        for _ in range(K):
            fn()
        for s_ in streams:
            ev = torch.cuda.Event()
            ev.record(s_)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        d.barrier()
        return e0.elapsed_time(e1) / 1e3

    def profile(on):
        for x in xbs:
            x.profile_enable(on)

    def profile_read():
        tot = {}
        for x in xbs:
            for ph, v in x.profile_read(reset=True).items():
                t = tot.setdefault(ph, {"launches": 0, "ms": 0.0})
                t["launches"] += v["launches"]
                t["ms"] += v["ms"]
        return tot

    prime("fp32_ir")
    for _ in range(args.warmup):
        step_mixed()
    prime("fp32_ir")  # the factor of the first timed step's map precedes the timed region
    cvd = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    clocks = Clocks(int(cvd[local]) if local < len(cvd) and cvd[local].isdigit() else local)
    profile(True)
    clocks.start()
    t_mixed = timed(step_mixed, args.steps)
    clk = clocks.stop()
    prof = profile_read()
    profile(False)
    t_mixed = d.max(t_mixed)
    total_solves = d.sum(float(B * args.steps))
    value = total_solves / t_mixed
    I_mixed = Is[(args.steps - 1) % 2].cpu().numpy()
    for b_ in (0, 1):  # both maps hold the same conductances: equal currents, bit for bit
        if (id(Is), b_) in pipe["solved"]:
            assert np.array_equal(Is[b_].cpu().numpy(), I_mixed), "the two maps' solves differ"

    # the same steps one map at a time (no overlap between the factor and the solve)
    step_mixed_sequential()
    t_seq = d.max(timed(step_mixed_sequential, args.steps))
    sequential = {"value": d.sum(float(B * args.steps)) / t_seq, "unit": UNIT,
                  "ms_per_step": 1e3 * t_seq / args.steps}
    assert np.array_equal(Is[0].cpu().numpy(), I_mixed), "sequential and pipelined solves differ"

    # plain FP64 block-LU on the same GPU, same two-map schedule
    prime("fp64")
    step_fp64()
    prime("fp64")
    profile(True)
    t64 = d.max(timed(step_fp64, args.fp64_steps))
    prof64 = profile_read()
    profile(False)
    fp64_value = d.sum(float(B * args.fp64_steps)) / t64
    I_fp64 = I64s[(args.fp64_steps - 1) % 2].cpu().numpy()
    err_vs_fp64 = float(np.max(np.abs(I_mixed - I_fp64) / np.maximum(np.abs(I_fp64), 1e-300)))

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Gh = torch.from_numpy(G).pin_memory()
        Vh = torch.from_numpy(V).pin_memory()
        Ih = torch.zeros((B, N), dtype=torch.float64).pin_memory()

        def step_e2e():  # the same two-map schedule with host buffers
            k = pipe["k"]
            xbs[(k + 1) % 2].set_conductances(Gh)
            assembled = torch.cuda.Event()
            assembled.record(streams[(k + 1) % 2])
            streams[k % 2].wait_event(assembled)
            xbs[(k + 1) % 2].factor("fp32_ir")
            xbs[k % 2].solve(Vh, Ih, tol=TOL, max_iter=10)
            pipe["k"] = k + 1

        prime("fp32_ir")
        step_e2e()
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_e2e()
        torch.cuda.synchronize()
        t_e2e = d.max(time.perf_counter() - t0)
        e2e = {"value": d.sum(float(B * args.steps)) / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(G.nbytes + V.nbytes), "d2h_bytes_per_step": int(B * N * 8),
               "ms_per_step": 1e3 * t_e2e / args.steps}
        assert np.array_equal(Ih.numpy(), I_mixed), "host-buffer solve differs from device-buffer solve"

    # factorizations/s of each factor (one handle, one map at a time, nothing overlapped) and the
    # latency of one map's solve for 1 and 16 input vectors right after it (the paper's
    # decomposition/solve split at small batches)
    factorizations = factor_rates(xbar, torch, Gd, Vd, R, N, d) if not args.no_factor_rates else None

    # per-phase kernel times inside the timed region, and the roofline of the dominant kernel
    per_step = {ph: {"launches": v["launches"] / args.steps, "ms": v["ms"] / args.steps}
                for ph, v in prof.items() if v["launches"]}
    launches = int(sum(v["launches"] for v in prof.values()))
    # the dominant kernel of the critical path: the solve's phases (the next map's assembly and
    # factor run beside them on the other stream and are hidden: the step time is the solve's)
    dom = max((ph for ph in per_step if ph not in ("assemble", "factor")), key=lambda ph: per_step[ph]["ms"])
    work, _ = algorithmic_work(dom, M, N, B)
    ms_launch = prof[dom]["ms"] / prof[dom]["launches"]
    mp = measured_peaks()
    peaks = pipe_peaks(mp.get("sm_max_mhz", 2070.0))
    achieved = work / (ms_launch / 1e3) / 1e12
    if dom == "sweep" and M <= 256:
        # tensor-core sweep (tcgen05 kind::f16 with BF16 operands: six split products per algorithmic
        # multiply-add in the initial solve, three in the corrections); timed inside a seconds-long
        # step, so the sustained BF16 figure
        bf16 = mp.get("bf16_tflops_sustained", mp.get("bf16_tflops", 1704.4))
        bound, peak, note = "tensor", bf16, ("BF16 dense, measured sustained cuBLAS figure (of measured); achieved "
                                            "counts algorithmic flops only, averaged over the solve's sweep launches "
                                            "(the initial one issues six BF16 products per multiply-add, the "
                                            "corrections three)")
    elif dom in ("sweep", "factor", "update"):
        bound, peak, note = "alu", peaks["fp32_tflops"], "FP32 FMA pipe, 152 SM x 128 lanes x 2 x max SM clock"
    else:
        bound, peak, note = "alu", peaks["fp64_tflops"], "FP64 FMA pipe, 152 SM x 2 DFMA x 2 x max SM clock"
    traffic, traffic_note = None, None
    if dom == "sweep" and (M, N) == (256, 256) and bound == "tensor":
        # ncu DRAM read + write per sweep_tc_kernel launch at B = 2048 (the capture fits the size
        # rule; the full batch does not), averaged over the solve's launches (1.667 GB initial, which
        # writes the FP32 state, and 2.218 GB for each correction), scaled by B / 2048: the kernel's
        # streams are per vector, the factor blocks it re-reads come from L2
        traffic = 2.034e9 * B / 2048
        traffic_note = (f"ncu dram__bytes_read+write at B=2048 (mean of the solve's three sweep launches) "
                        f"x B/2048 = {B / 2048:g}")
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note, "peak_note": note,
                "work_per_launch": work, "ms_per_launch": ms_launch,
                "selection": "largest phase on the solve's stream (the critical path); the next map's assembly "
                             "and factor overlap it on the second stream"}
    if dom == "sweep" and bound == "tensor":
        # Above ~0.6 PF of BF16 the substitution is HBM-bound: its algorithmic bytes per input vector
        # are V and I in FP64 and the forward results written and read back in FP32,
        # 8M + 8N + 2 (2MN 4).  The HBM roof is the primary one; the tensor reading stays beside it.
        hbm_bytes = B * (8.0 * M + 8.0 * N + 2.0 * (2.0 * M * N * 4.0))
        hbm_peak = mp.get("hbm_gbs", 6780.0)
        hbm_achieved = hbm_bytes / (ms_launch / 1e3) / 1e9
        tensor = {k: roofline[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_note")}
        roofline.update({"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_achieved / hbm_peak, "bytes_per_launch": hbm_bytes,
                         "peak_note": "measured copy bandwidth (of measured)", "tensor": tensor})

    cpu = None
    err_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, Iref = cpu_baseline(M, N, G, R, V, args.cpu_sample)
        err_vs_oracle = float(np.max(np.abs(I_mixed - Iref) / np.abs(Iref)))
        cpu["fp64_gpu_err_vs_oracle"] = float(np.max(np.abs(I_fp64 - Iref) / np.abs(Iref)))

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16x3 tensor products) + f32-pair refinement", "data": "synthetic",
        "config": {"workload": args.workload + (f"_B{B}" if args.batch else ""), "M": M, "N": N, "B": B,
                   "R_s": R[0], "R_w": R[1], "R_b": R[2], "R_sense": R[3], "precision": "fp32 factor, sweeps on BF16 tensor cores (three-term split, fp32 accumulation), float-pair (~48-bit) residual/update", "tol": TOL,
                   "step": "set_conductances + factor + solve (all refinement)", "algorithm": args.algorithm,
                   "schedule": "two maps in flight: each step sets and factors the next map on a second "
                               "stream while this map's batch is solved (FP64 baseline and e2e the same)",
                   "l2": "working set per step (>6 GB) exceeds the 129 MB L2", "parallelism": f"replicas{world}"},
        "fp64_baseline": {"value": fp64_value, "unit": UNIT, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                          "steps": args.fp64_steps,
                          "phases_ms_per_step": {ph: v["ms"] / args.fp64_steps for ph, v in prof64.items() if v["launches"]}},
        "sequential": sequential,
        "speedup_vs_fp64": value / fp64_value,
        "rel_err_vs_fp64_gpu": err_vs_fp64,
        "rel_err_vs_oracle": err_vs_oracle,
        "refinement": {k: info_box.get(k) for k in ("iters", "max_rel_dI", "resid_inf", "err_est")},
        "phases_per_step": per_step,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "factorizations": factorizations,
        "gpu_launches": launches,
        "clocks": clk,
    }
    for x in xbs:
        x.destroy()
    del Is, I64s
    if world == 1 and not args.no_surrogate:
        # the learned-surrogate workload (128 x 128 maps, train, calibrate, predict 50 held-out maps
        # with exact fallback) on the same GPU after the headline's buffers are released; its full
        # line is `--workload surrogate128`
        sur = run_surrogate(argparse.Namespace(**{**vars(args), "no_cpu_baseline": True}), emit=False)
        out["surrogate128"] = {k: sur[k] for k in ("metric", "value", "unit", "ms_per_step", "speedup_vs_exact",
                                                  "exact_baseline", "fallback_vectors_per_step",
                                                  "vectors_per_step", "clocks")}
        out["surrogate128"]["rel_err_with_fallback"] = sur["rel_err"]["surrogate_with_fallback"]
        out["surrogate128"]["config"] = {k: sur["config"][k] for k in ("workload", "M", "N", "train", "test", "bound")}
    if rank == 0:
        print(json.dumps(out), flush=True)
    d.close()


def factor_rates(xbar, torch, Gd, Vd, R, N, d):
    """Standalone factor time per algorithm and precision, and the solve latency that follows.

    One handle on the current stream; each factor is timed alone (K back-to-back factors between
    CUDA events after a warm-up), so these are the absolute factorizations/s of one map, not the
    overlapped figure of the two-maps-in-flight schedule."""
    variants = [("thomas_fp32", "thomas", "fp32_ir", -1), ("cr_fp32_tensor", "cr", "fp32_ir", 1),
                ("cr_fp32_cuda_cores", "cr", "fp32_ir", 0), ("thomas_fp64", "thomas", "fp64", -1),
                ("cr_fp64", "cr", "fp64", -1)]
    out = {}
    xb = xbar.Crossbar.assemble(Gd, *R)
    stream = torch.cuda.current_stream()

    def events_ms(fn, K):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    for name, algo, prec, prod in variants:
        xb.set_option("algorithm", algo)
        xb.set_option("cr_products", prod)
        xb.factor(prec)
        xb.sync()
        K = 3 if prec == "fp64" else 10
        ms = d.max(events_ms(lambda: xb.factor(prec), K))
        rec = {"algorithm": algo, "precision": prec, "factor_ms": ms, "factorizations_per_s": 1e3 / ms,
               "products": {1: "tensor cores (tcgen05, three-term BF16)", 0: "CUDA cores"}.get(prod, "CUDA cores")}
        for Bs in (1, 16):
            Ib = torch.zeros((Bs, N), dtype=torch.float64, device="cuda")
            xb.solve(Vd[:Bs], Ib, tol=TOL, max_iter=10)
            xb.sync()
            box = {}

            def one():
                _, info = xb.solve(Vd[:Bs], Ib, tol=TOL, max_iter=10)
                box.update(info)

            rec[f"solve_ms_B{Bs}"] = d.max(events_ms(one, 3))
            rec[f"iters_B{Bs}"] = box.get("iters")
        out[name] = rec
    xb.destroy()
    out["note"] = ("one 256x256 map at a time: factor_ms = mean of back-to-back factors (CUDA events); "
                   "solve_ms_B* = one xbar_solve (all refinement) of 1 or 16 vectors after it")
    return out


def run_transfer(args):
    """Currents-only transfer-matrix mode on the 256 x 256, 8192-vector inputs: one step is
    set_conductances + factor(FP32_IR) + xbar_transfer_matrix (M unit solves) + xbar_solve_transfer
    (I = V G_eff in FP64).  A different path from the substitutions, reported on its own line."""
    import torch

    from paper_2410_19993_gb300 import inputs, xbar

    d = Dist()
    rank, world, local = d.rank, d.world, d.local
    torch.cuda.set_device(local)
    w = inputs.WORKLOADS["xbar256_mixed"]
    M, N, B = w.M, w.N, (args.batch or w.B)
    R = w.circuits[0].as_tuple()
    G, V = inputs.crossbar(M, N, B, seed=w.seed + rank, g_lo=w.g_lo, g_hi=w.g_hi, v_max=w.v_max)
    stream = torch.cuda.current_stream()
    Gd = torch.from_numpy(G).cuda()
    Vd = torch.from_numpy(V).cuda()
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    I64 = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    xb = xbar.Crossbar.assemble(Gd, *R, stream=stream)
    info_box = {}

    def step():
        xb.set_conductances(Gd)
        xb.factor("fp32_ir")
        _, info = xb.transfer_matrix(tol=TOL, max_iter=10)
        info_box.update(info)
        xb.solve_transfer(Vd, I)

    def timed(fn, K):
        d.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        d.barrier()
        return e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        step()
    cvd = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    clocks = Clocks(int(cvd[local]) if local < len(cvd) and cvd[local].isdigit() else local)
    xb.profile_enable(True)
    clocks.start()
    t_step = d.max(timed(step, args.steps))
    clk = clocks.stop()
    prof = xb.profile_read(reset=True)
    xb.profile_enable(False)
    value = d.sum(float(B * args.steps)) / t_step
    I_t = I.cpu().numpy()
    # the FP64 product alone (G_eff cached): its own roofline, FP64 pipe
    t_gemm = d.max(timed(lambda: xb.solve_transfer(Vd, I), 10)) / 10
    gemm_tflops = 2.0 * B * M * N / t_gemm / 1e12
    peaks = pipe_peaks(measured_peaks().get("sm_max_mhz", 2070.0))

    # plain FP64 substitution path on the same GPU, and the error against it
    def step_fp64():
        xb.set_conductances(Gd)
        xb.factor("fp64")
        xb.solve(Vd, I64)

    step_fp64()
    t64 = d.max(timed(step_fp64, args.fp64_steps))
    fp64_value = d.sum(float(B * args.fp64_steps)) / t64
    I_fp64 = I64.cpu().numpy()
    err_vs_fp64 = float(np.max(np.abs(I_t - I_fp64) / np.maximum(np.abs(I_fp64), 1e-300)))
    cpu, err_vs_oracle = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, Iref = cpu_baseline(M, N, G, R, V, args.cpu_sample)
        err_vs_oracle = float(np.max(np.abs(I_t - Iref) / np.abs(Iref)))
    per_step = {ph: {"launches": v["launches"] / args.steps, "ms": v["ms"] / args.steps}
                for ph, v in prof.items() if v["launches"]}
    out = {
        "metric": "solves/s, currents-only transfer-matrix mode (G_eff from M unit solves + FP64 product) at "
                  "\u22641e-8 rel. current error",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 product; G_eff from the f32 (bf16x3) + f32-pair refinement solve",
        "data": "synthetic",
        "config": {"workload": "xbar256_transfer" + (f"_B{B}" if args.batch else ""), "M": M, "N": N, "B": B,
                   "R_s": R[0], "R_w": R[1], "R_b": R[2], "R_sense": R[3], "tol": TOL,
                   "step": "set_conductances + factor(fp32_ir) + transfer_matrix (M unit solves) + FP64 product",
                   "parallelism": f"replicas{world}"},
        "fp64_baseline": {"value": fp64_value, "unit": UNIT, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                          "path": "FP64 factor + FP64 substitutions"},
        "speedup_vs_fp64": value / fp64_value,
        "rel_err_vs_fp64_gpu": err_vs_fp64,
        "rel_err_vs_oracle": err_vs_oracle,
        "refinement_of_unit_solves": {k: info_box.get(k) for k in ("iters", "max_rel_dI", "err_est")},
        "phases_per_step": per_step,
        "roofline": {"kernel": "gemm_f64 (I = V G_eff)", "bound": "alu", "achieved": gemm_tflops,
                     "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": gemm_tflops / peaks["fp64_tflops"],
                     "traffic": None, "peak_note": "FP64 FMA pipe, 152 SM x 2 DFMA x 2 x max SM clock",
                     "ms_per_launch": 1e3 * t_gemm, "work_per_launch": 2.0 * B * M * N},
        "cpu_baseline": cpu,
        "gpu_launches": int(sum(v["launches"] for v in prof.values())),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    xb.destroy()
    d.close()


def run_paper_experiments(args):
    """The paper's timing experiments (Sec. III) re-run on this implementation: simulation time of
    m x n crossbars for m, n in {2, ..., 256} (one input vector), a 256 x 256 crossbar partitioned
    into t x t tiles (all tiles in one CUDA-graph launch of the tile batch), and the decomposition /
    solve split for batches of 1, 2, 10, 100 and 1000.  Parasitic resistors 5 Ohm each (source and
    sense resistors equal to the wire segments), random conductances and voltages as elsewhere.
    Each time is the wall time of the user-visible calls with the stream synchronised, mean of 10
    runs; the FP64 path is the paper's method (LU in FP64), the mixed path is given beside it.  Each
    single-map case runs with the handle's default algorithm (block Thomas; blocks over rows, and
    there cyclic reduction, when 2n <= m in FP64) and again with block cyclic reduction over the
    blocks ('_cr' keys)."""
    import torch

    from paper_2410_19993_gb300 import inputs, xbar

    torch.cuda.set_device(0)
    R = (5.0, 5.0, 5.0, 5.0)
    runs = 10
    sizes = [2, 4, 8, 16, 32, 64, 128, 256]

    def wall(fn, n=runs):
        fn()  # warm-up (allocations, lazy setup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0) / n

    # (a) simulation time per crossbar size, one input vector
    size_sweep = []
    for m in sizes:
        for n in sizes:
            G, V = inputs.crossbar(m, n, 1, seed=0)
            Gd, Vd = torch.from_numpy(G).cuda(), torch.from_numpy(V).cuda()
            I = torch.zeros((1, n), dtype=torch.float64, device="cuda")
            xb = xbar.Crossbar.assemble(Gd, *R)
            row = {"m": m, "n": n}
            for algo in ("auto", "cr"):
                xb.set_option("algorithm", -1 if algo == "auto" else "cr")
                for prec in ("fp64", "fp32_ir"):
                    def sim():
                        xb.set_conductances(Gd)
                        xb.factor(prec)
                        xb.solve(Vd, I, tol=TOL, max_iter=10)
                    row[prec + ("_cr" if algo == "cr" else "") + "_ms"] = wall(sim)
            xb.destroy()
            size_sweep.append(row)

    # (b) 256 x 256 partitioned into t x t tiles, one input vector
    M = N = 256
    G, V = inputs.crossbar(M, N, 1, seed=0)
    partition = []
    for t in (256, 128, 64, 32, 16):
        tiles, Vs, Is = [], [], []
        for r0 in range(0, M, t):
            for c0 in range(0, N, t):
                tiles.append((torch.from_numpy(np.ascontiguousarray(G[r0:r0 + t, c0:c0 + t])).cuda(), *R))
                Vs.append(torch.from_numpy(np.ascontiguousarray(V[:, r0:r0 + t])).cuda())
                Is.append(torch.zeros((1, t), dtype=torch.float64, device="cuda"))
        b = xbar.Batch(tiles)
        row = {"tile": t, "tiles": len(tiles)}
        for prec in ("fp64", "fp32_ir"):
            row[prec + "_ms"] = wall(lambda: b.run(prec, Vs, Is, tol=TOL, max_iter=6))
        b.destroy()
        partition.append(row)

    # (c) decomposition / solve split per batch size
    split = []
    for m in (32, 128, 256):
        for B in (1, 2, 10, 100, 1000):
            G, V = inputs.crossbar(m, m, B, seed=0)
            Gd, Vd = torch.from_numpy(G).cuda(), torch.from_numpy(V).cuda()
            I = torch.zeros((B, m), dtype=torch.float64, device="cuda")
            xb = xbar.Crossbar.assemble(Gd, *R)
            row = {"m": m, "n": m, "B": B}
            for algo in ("auto", "cr"):
                xb.set_option("algorithm", -1 if algo == "auto" else "cr")
                for prec in ("fp64", "fp32_ir"):
                    def dec():
                        xb.set_conductances(Gd)
                        xb.factor(prec)
                    t_dec = wall(dec)
                    t_sol = wall(lambda: xb.solve(Vd, I, tol=TOL, max_iter=10))
                    row[prec + ("_cr" if algo == "cr" else "")] = {
                        "decompose_ms": t_dec, "solve_ms": t_sol, "solve_share": t_sol / (t_dec + t_sol),
                        "per_sample_ms": (t_dec + t_sol) / B}
            xb.destroy()
            split.append(row)

    out = {"metric": "simulation time of the paper's experiments (Sec. III), this implementation", "value": None,
           "unit": "ms", "n_gpus": 1, "data": "synthetic", "higher_is_better": False,
           "config": {"workload": "paper_experiments", "R_s": R[0], "R_w": R[1], "R_b": R[2], "R_sense": R[3],
                      "runs": runs, "tol": TOL},
           "size_sweep": size_sweep, "partition_256": partition, "batch_split": split}
    print(json.dumps(out), flush=True)


def cpu_baseline(M, N, G, R, V, sample):
    """The oracle as it stands on the host cores: one factorization plus `sample` substitutions."""
    import oracle
    B = V.shape[0]
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    f = oracle.factor(M, N, G, *R)
    t_fac = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve_factored(f, V[:sample], nthreads=threads)
    t_sol = (time.perf_counter() - t0) / sample
    value = B / (t_fac + B * t_sol)
    # exact currents of the whole batch by linearity (M unit substitutions)
    Geff = oracle.transfer_matrix(f, nthreads=threads)
    return ({"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
             "sample": f"one banded-LU factorization ({t_fac:.1f} s) + {sample} substitutions "
                       f"({1e3 * t_sol:.1f} ms each on {threads} threads); value = B/(t_factor + B*t_subst), B={B}"},
            V @ Geff)


# ---------------------------------------------------------------------------------------------
# the reference arm: the CPU oracle, timed as it stands on the host cores
# ---------------------------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2410_19993_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    M, N, B = w.M, w.N, w.B
    R = w.circuits[0].as_tuple()
    G, V = inputs.crossbar(M, N, B, seed=w.seed, g_lo=w.g_lo, g_hi=w.g_hi, v_max=w.v_max)
    threads = os.cpu_count() or 1
    per_step = max(1, min(args.cpu_sample, B))
    t0 = time.perf_counter()
    f = oracle.factor(M, N, G, *R)
    t_fac = time.perf_counter() - t0
    for k in range(args.warmup):
        oracle.solve_factored(f, V[(k * per_step) % B:][:per_step], nthreads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.solve_factored(f, V[(k * per_step) % B:][:per_step], nthreads=threads)
    t_steps = time.perf_counter() - t0
    t_sol = t_steps / (args.steps * per_step)
    value = B / (t_fac + B * t_sol)
    sample = (f"each step substitutes {per_step} vectors; one banded-LU factorization ({t_fac:.1f} s) "
              f"timed once; value = B/(t_factor + B*t_subst), B={B}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_steps / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "M": M, "N": N, "B": B, "R_s": R[0], "R_w": R[1], "R_b": R[2],
                   "R_sense": R[3], "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_tiles(args):
    """784-256-10 network mapped onto 30 ragged tiles, 4096 vectors each: one graph launch per step."""
    import torch

    from paper_2410_19993_gb300 import inputs, xbar

    d = Dist()
    torch.cuda.set_device(d.local)
    tiles = inputs.fc_tiles(B=args.batch or 4096, seed=d.rank)
    Vs = [torch.from_numpy(t.V).cuda() for t in tiles]
    Is = [torch.zeros((t.V.shape[0], t.G.shape[1]), dtype=torch.float64, device="cuda") for t in tiles]
    I64 = [torch.zeros_like(I) for I in Is]
    b = xbar.Batch([(t.G, *t.circuit.as_tuple()) for t in tiles])
    Bs = [t.V.shape[0] for t in tiles]
    t0 = time.perf_counter()
    b.autotune("fp32_ir", Bs, os.path.join(tempfile.gettempdir(), "xbar_autotune_tiles.json"))
    t_tune = time.perf_counter() - t0
    total = float(sum(Bs))

    def timed(prec, outs, K):
        for _ in range(args.warmup):
            b.run(prec, Vs, outs, tol=TOL, max_iter=4)
        torch.cuda.synchronize()
        d.barrier()
        t1 = time.perf_counter()
        infos = None
        for _ in range(K):
            _, infos = b.run(prec, Vs, outs, tol=TOL, max_iter=4)
        torch.cuda.synchronize()
        return d.max(time.perf_counter() - t1), infos

    clocks = Clocks(d.local)
    clocks.start()
    t_mixed, infos = timed("fp32_ir", Is, args.steps)
    clk = clocks.stop()
    t64, _ = timed("fp64", I64, args.fp64_steps)
    err = max(float(np.max(np.abs(a.cpu().numpy() - c.cpu().numpy()) / np.abs(c.cpu().numpy())))
              for a, c in zip(Is, I64))
    out = {
        "metric": METRIC, "value": d.sum(total * args.steps) / t_mixed, "unit": UNIT, "n_gpus": d.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_mixed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16x3 tensor products) + f32-pair refinement",
        "data": "synthetic",
        "config": {"workload": "fc784_256_10_tiles", "tiles": len(tiles),
                   "shapes": {f"{m}x{n}": sum(t.G.shape == (m, n) for t in tiles)
                              for (m, n) in sorted({t.G.shape for t in tiles})},
                   "B_per_tile": Bs[0], "step": "one CUDA-graph launch: factor + solve + refinement of all tiles",
                   "autotune_s": t_tune, "parallelism": f"replicas{d.world}"},
        "fp64_baseline": {"value": d.sum(total * args.fp64_steps) / t64, "unit": UNIT,
                          "ms_per_step": 1e3 * t64 / args.fp64_steps},
        "rel_err_vs_fp64_gpu": err,
        "refinement_iters": sorted({i["iters"] for i in infos}),
        "clocks": clk,
    }
    out["speedup_vs_fp64"] = out["value"] / out["fp64_baseline"]["value"]
    # Step-level HBM roofline: the graph runs every tile's kernels concurrently, so no single
    # kernel's launch time exists here; the algorithmic bytes of all solve phases of all tiles
    # (sweeps: 8M + 8N + 2 (2MN 4) per vector each; residuals 12 and updates 20 bytes per node and
    # vector) over the step time give the aggregate rate.  The factors' bytes are not counted.
    iters = max(i["iters"] for i in infos)
    step_bytes = 0.0
    for t, Bt in zip(tiles, Bs):
        Mt_, Nt_ = t.G.shape
        per_vec = ((1 + iters) * (8.0 * Mt_ + 8.0 * Nt_ + 2.0 * (2.0 * Mt_ * Nt_ * 4.0))
                   + iters * 12.0 * Mt_ * Nt_ + max(iters - 1, 0) * 20.0 * Mt_ * Nt_)
        step_bytes += per_vec * Bt
    hbm_peak = measured_peaks().get("hbm_gbs", 6780.0)
    achieved = step_bytes / (t_mixed / args.steps) / 1e9
    out["roofline"] = {"kernel": "all kernels of the graph step (solve phases of every tile)", "bound": "hbm",
                       "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                       "traffic": None, "bytes_per_step": step_bytes,
                       "peak_note": "measured copy bandwidth (of measured)"}
    if d.rank == 0:
        print(json.dumps(out), flush=True)
    b.destroy()
    d.close()


def run_surrogate(args, emit=True):
    """Learned surrogate on 128 x 128 maps: exact solves make the data, the GPU trains, calibrates,
    then predicts 50 held-out maps x 1000 vectors with exact fallback above 1% estimated error."""
    import torch

    from paper_2410_19993_gb300 import inputs, xbar

    d = Dist()
    torch.cuda.set_device(d.local)
    w = inputs.WORKLOADS["surrogate128"]
    x = w.extra
    M, N = w.M, w.N
    R = w.circuits[0].as_tuple()
    bound = 0.01
    stream = torch.cuda.current_stream()
    xb = xbar.Crossbar.assemble(torch.zeros((M, N), dtype=torch.float64, device="cuda") + 1e-5, *R, stream=stream)

    def exact(G, V, I):
        xb.set_conductances(G)
        xb.factor("fp32_ir")
        xb.solve(V, I, tol=TOL, max_iter=10)

    def maps(n, B, seed):
        out = []
        for G, V in inputs.maps(n, M, N, B, seed=seed + 1000 * d.rank, g_lo=w.g_lo, g_hi=w.g_hi, v_max=w.v_max):
            out.append((torch.from_numpy(G).cuda(), torch.from_numpy(V).cuda(),
                        torch.zeros((B, N), dtype=torch.float64, device="cuda")))
        return out

    train = maps(x["train_maps"], x["train_B"], x["train_seed"])
    calib = maps(x["calib_maps"], x["calib_B"], x["calib_seed"])
    test = maps(x["test_maps"], x["test_B"], x["test_seed"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for G, V, I in train + calib:
        exact(G, V, I)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0

    s = xbar.Surrogate(M, N, R, passes=args.line_passes, g_scale=w.g_hi, v_scale=w.v_max, seed=5)
    t0 = time.perf_counter()
    e1 = max(1, int(round(0.75 * args.epochs)))
    l1 = s.train([G for G, _, _ in train], [V for _, V, _ in train], [I for _, _, I in train],
                 epochs=e1, batch_rows=4096, lr=1e-3, seed=9)
    l2 = s.train([G for G, _, _ in train], [V for _, V, _ in train], [I for _, _, I in train],
                 epochs=args.epochs - e1, batch_rows=4096, lr=3e-4, seed=10)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    c = s.calibrate([G for G, _, _ in calib], [V for _, V, _ in calib], [I for _, _, I in calib], quantile=0.99)
    losses = np.concatenate([l1, l2]) if len(l2) else l1

    Iex = [torch.zeros_like(I) for _, _, I in test]
    Isur = [torch.zeros_like(I) for _, _, I in test]
    est = [torch.zeros_like(I) for _, _, I in test]
    nfb = [0]

    def step_exact():
        for (G, V, _), I in zip(test, Iex):
            exact(G, V, I)

    def step_sur():
        nfb[0] = 0
        for (G, V, _), I, e in zip(test, Isur, est):
            xb.set_conductances(G)
            _, info = s.solve(xb, V, I, bound=bound, err_est=e)
            nfb[0] += info["n_fallback"]

    def timed(fn, K):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        d.barrier()
        t1 = time.perf_counter()
        for _ in range(K):
            fn()
        torch.cuda.synchronize()
        return d.max(time.perf_counter() - t1)

    clocks = Clocks(d.local)
    clocks.start()
    t_sur = timed(step_sur, args.steps)
    clk = clocks.stop()
    t_ex = timed(step_exact, max(1, args.steps // 2))
    n_vec = sum(V.shape[0] for _, V, _ in test)
    value = d.sum(float(n_vec * args.steps)) / t_sur
    exact_value = d.sum(float(n_vec * max(1, args.steps // 2))) / t_ex

    # accuracy against the exact solves, and of the estimates the network corrects
    zero = xbar.Surrogate(M, N, R, passes=args.line_passes, g_scale=w.g_hi, v_scale=w.v_max)
    zero.set_params(np.zeros(zero.n_params(), dtype=np.float32))
    e_sur, e_net, e_line, e_ideal, acc_bad = [], [], [], [], 0
    for (G, V, _), Ie, Is_, ee in zip(test, Iex, Isur, est):
        Ie_h = Ie.cpu().numpy()
        Ip = torch.zeros_like(Ie)
        s.predict(G, V, Ip)
        Il = torch.zeros_like(Ie)
        zero.predict(G, V, Il)
        Iid = (V @ G).cpu().numpy()
        rel = lambda a: np.abs(a - Ie_h) / np.abs(Ie_h)
        e_sur.append(rel(Is_.cpu().numpy()))
        e_net.append(rel(Ip.cpu().numpy()))
        e_line.append(rel(Il.cpu().numpy()))
        e_ideal.append(rel(Iid))
        accepted = np.all(ee.cpu().numpy() <= bound, axis=1)
        acc_bad += int((e_sur[-1][accepted] > bound).sum())
    zero.destroy()
    q = lambda a: {"median": float(np.median(a)), "p99": float(np.quantile(a, 0.99)), "max": float(np.max(a))}
    cat = lambda a: np.concatenate(a).ravel()
    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        G0, V0 = inputs.maps(1, M, N, x["test_B"], seed=x["test_seed"])[0]
        cpu, _ = cpu_baseline(M, N, G0, R, V0, args.cpu_sample)
    out = {
        "metric": "surrogate solves/s (per-column MLP + exact fallback above 1% estimated error)",
        "value": value, "unit": UNIT, "n_gpus": d.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_sur / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 network, fp32 line model", "data": "synthetic",
        "config": {"workload": "surrogate128", "M": M, "N": N, "R_s": R[0], "R_w": R[1], "R_b": R[2],
                   "R_sense": R[3], "train": f"{x['train_maps']} maps x {x['train_B']} vectors",
                   "calib": f"{x['calib_maps']} maps x {x['calib_B']} vectors",
                   "test": f"{x['test_maps']} held-out maps x {x['test_B']} vectors", "bound": bound,
                   "line_passes": args.line_passes, "epochs": args.epochs, "batch_rows": 4096,
                   "step": "per test map: set_conductances + surrogate solve (line model, features, network, "
                           "fallback solves)", "parallelism": f"replicas{d.world}"},
        "exact_baseline": {"value": exact_value, "unit": UNIT,
                           "step": "per test map: set_conductances + factor(fp32_ir) + solve(tol 1e-8)"},
        "speedup_vs_exact": value / exact_value,
        "fallback_vectors_per_step": nfb[0], "vectors_per_step": n_vec,
        "accepted_columns_above_bound": acc_bad,
        "rel_err": {"surrogate_with_fallback": q(cat(e_sur)), "network": q(cat(e_net)),
                    "line_model_alone": q(cat(e_line)), "ideal_mvm": q(cat(e_ideal))},
        "training": {"datagen_s": t_data, "train_s": t_train, "rows": x["train_maps"] * x["train_B"] * N,
                     "loss_first": losses[0].tolist(), "loss_last": losses[-1].tolist(), "calibration_c": c,
                     "scaling": s.scaling()},
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    if d.rank == 0 and emit:
        print(json.dumps(out), flush=True)
    s.destroy()
    xb.destroy()
    d.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "fc784_256_10_tiles":
        run_tiles(args)
    elif args.workload == "surrogate128":
        run_surrogate(args)
    elif args.workload == "xbar256_transfer":
        run_transfer(args)
    elif args.workload == "paper_experiments":
        run_paper_experiments(args)
    else:
        run_xbar(args)


if __name__ == "__main__":
    main()
