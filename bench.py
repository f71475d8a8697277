#!/usr/bin/env python
"""Throughput of the SNAPS outlier-detection hot path on B300.

One step = the whole path over one population: normalise the resident
features (snaps_index), then both self-joins over every requested subspace,
the four metrics, their FP64-normalised forms and the top-100 rankings
(snaps_scores).  Default workload: N = 31,693 objects (seed 0, the paper's
SNAPShot1 size) in all 32,752 subspaces of 2-15 of 15 features, k = 10,
eps = 0.05 sqrt(d), plain FP32 join.

Metric: objects x subspaces scored per second, whole job (all ranks).
`value` is device-timed with inputs resident in HBM (CUDA events on the
stream the library launches on, L2 flushed before every step); `e2e` is the
same metric through the C ABI with host buffers: the features are copied in
from pinned host memory and the top-100 rankings copied back every step.

`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.  Under torchrun the subspaces are
shared out across the ranks (whole 32-subspace chunks, longest first to the
least-loaded rank, Sec. 3.8.2; no collective on the data path), so the job's
total work is fixed (strong scaling); the reported time is the max over
ranks, and rank 0 gathers every rank's top-100 lists after the timed legs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import snaps_inputs  # noqa: E402

N_DEFAULT = 31693
K_DEFAULT = 10
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2
SAMPLE_SEED = 1              # the 64-subspace oracle sample of the batching workload
COMPARES_PER_SM_CLK = 64     # FP32 compare throughput per SM per clock
MUFU_PER_SM_CLK = 16         # special-function (square root) throughput per SM per clock
FMA_LANES_PER_SM_CLK = 128   # FP32 add / FMA lane-operations per SM per clock
# DRAM bytes (read + write) per pair-subspace evaluation, from one ncu capture
# of each kernel as it stands (dram__bytes_read.sum + dram__bytes_write.sum):
# the tree join on one 32-subspace chunk at N = 31,693 (7.82 MB + 3.44 MB),
# the tensor-core join on one block of 256 subspaces at N = 31,693 (351 MB +
# 980 MB: its per-query writes scatter over 256 output rows, which the L2
# cannot hold).  Both kernels read their candidates from L2, so DRAM traffic
# grows with the evaluations only through the outputs and the row copies.
TREE_DRAM_BYTES_PER_EVAL = (7.822592e6 + 3.436544e6) / (31693 * 31692 * 32)
TC_DRAM_BYTES_PER_EVAL = (350.9632e6 + 980.276224e6) / (31693 * 31692 * 256)


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PEAKS = _load_peaks()


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--masks", default="all",
                    help="'all', a count of seeded sample subspaces, or 'chunk:H' (H = 10 binary "
                         "digits: the 32 subspaces (H << 5) | L sharing that high part)")
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--precision", choices=["fp32", "tc_f16", "tc_bf16", "tc_tf32", "both", "all"],
                    default="both",
                    help="fp32: the plain join; tc_f16 / tc_bf16 / tc_tf32: the tensor-core filtered join "
                         "with FP16 / BF16 / TF32 operands; both (default): time the plain join as the "
                         "headline and the FP16 tensor-core join beside it on the same workload; "
                         "all: the BF16 and TF32 tensor-core joins beside those two")
    ap.add_argument("--index", choices=["auto", "grid", "none"], default="auto",
                    help="grid index for subspaces of <= 4 features: the library's choice "
                         "(auto), always, or never")
    ap.add_argument("--tc-steps", type=int, default=1,
                    help="timed steps of the tensor-core leg under --precision both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving", type=int, default=0, metavar="R",
                    help="instead of the batching workload, run a Poisson stream of R scoring "
                         "requests through snaps_submit/snaps_poll and report p50/p99 latency")
    ap.add_argument("--select", type=int, default=0, metavar="M",
                    help="instead of the batching workload, time parameter selection (eps grid "
                         "of 16 values over [0.02, 0.12] sqrt(d), k grid 2..32, top-n = 1 %% of N) "
                         "on M seeded sample subspaces")
    ap.add_argument("--rubin", type=int, default=0, metavar="P",
                    help="Rubin-scale leg: P of the 105 two-feature subspaces (evenly spaced) at --rubin-n "
                         "objects through the grid index")
    ap.add_argument("--rubin-n", type=int, default=5_000_000)
    ap.add_argument("--rubin-full", action="store_true",
                    help="Rubin-scale leg on the full 15-feature subspace (brute force, one call, no "
                         "warm-up call) instead of the two-feature subspaces")
    ap.add_argument("--rubin-cells", type=int, default=0, metavar="R",
                    help="grid cells 1/R of eps wide for the Rubin leg (0: the library's choice)")
    ap.add_argument("--serving-leg", type=int, default=60, metavar="R",
                    help="after the batching legs (one GPU), a Poisson stream of R requests through "
                         "both join forms, reported as the line's `serving` object (0: skip)")
    ap.add_argument("--by-dimension", action="store_true",
                    help="instead of the batching workload, time one call over 256 seeded subspaces of each "
                         "dimension (all of them where fewer exist) through the tensor-core form and the "
                         "plain form, N = --n objects")
    ap.add_argument("--precision-config", action="store_true",
                    help="instead of the batching workload, the precision workload: N = 250,000 objects "
                         "(--precision-n), the plain FP32 join against both tensor-core forms on 256 "
                         "subspaces (eight whole 32-subspace chunks) and on 256 random subspaces")
    ap.add_argument("--precision-n", type=int, default=250_000)
    ap.add_argument("--serving-max-n", type=int, default=100000)
    ap.add_argument("--serving-max-masks", type=int, default=64)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-load", type=float, default=0.7)
    return ap.parse_args()


def workload_masks(spec: str) -> np.ndarray:
    if spec == "all":
        return snaps_inputs.all_masks()
    if spec.startswith("chunk:"):
        allm = snaps_inputs.all_masks()
        return allm[(allm >> 5) == int(spec[6:], 2)]
    return snaps_inputs.mask_sample(int(spec), SAMPLE_SEED)


def workload_name(args, n_masks):
    if args.masks == "all":
        sub = "all 32,752 subspaces"
    elif args.masks.startswith("chunk:"):
        sub = f"the {n_masks} subspaces with high features {args.masks[6:]}"
    else:
        sub = f"{n_masks} sampled subspaces"
    return (f"batched scoring: N={args.n} objects x {sub} of 2-15 of 15 features, "
            f"k={args.k}, eps=0.05*sqrt(d), seed 0")


# ---- clocks --------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- our arm -------------------------------------------------------------------------------

def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x: a job's time is its slowest rank's, and
    the job's throughput is all ranks' units over that time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, dist):
    import torch

    import paper_2405_20176_b300 as snaps

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2405_20176_b300 import shard

    x = snaps_inputs.population(args.n, 0)
    all_masks = workload_masks(args.masks)
    # this rank's share of the subspaces (all of them on one GPU)
    parts, _ = shard.partition(all_masks, args.n, world)
    positions = parts[rank]
    masks = all_masks[positions]
    m, n, k = masks.size, args.n, args.k
    m_total = all_masks.size
    index_flag = {"auto": 0, "grid": snaps.SNAPS_INDEX_GRID, "none": snaps.SNAPS_INDEX_NONE}[args.index]
    head_prec = {"tc_f16": snaps.SNAPS_TC_F16, "tc_bf16": snaps.SNAPS_TC_BF16, "tc_tf32": snaps.SNAPS_TC_TF32}.get(
        args.precision, snaps.SNAPS_FP32) | index_flag
    form_name = {snaps.SNAPS_FP32: "fp32", snaps.SNAPS_TC_F16: "tc_f16", snaps.SNAPS_TC_BF16: "tc_bf16",
                 snaps.SNAPS_TC_TF32: "tc_tf32"}
    ctx = snaps.snaps_create(local)
    stream = torch.cuda.current_stream()
    x_dev = torch.from_numpy(x).to(dev)
    scores = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
    norm = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
    top = torch.empty((m, 4, 100), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(precision):
        pop = snaps.snaps_index(ctx, x_dev, snaps.SNAPS_NORM_MINMAX, stream=stream)
        snaps.snaps_scores(pop, masks, k, precision=precision, scores=scores, norm=norm,
                           top=top, top_n=100, stream=stream)
        return pop

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_leg(precision, steps, warmup):
        """W untimed steps, then K steps bracketed by barrier + synchronize; CUDA events on
        the launch stream per step, the library's per-phase trace, clocks sampled."""
        for w in range(warmup):
            t0 = time.perf_counter()
            snaps.snaps_release(step(precision))
            torch.cuda.synchronize()
            print(f"[bench] precision {precision} warmup {w}: {time.perf_counter() - t0:.3f} s",
                  file=sys.stderr, flush=True)
        barrier()
        snaps.snaps_trace(ctx, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        pops = []
        with ClockSampler(local) as clk:
            barrier()
            for s in range(steps):
                flush.fill_(float(s))                      # evict the previous step from L2
                ev[s][0].record(stream)
                pops.append(step(precision))
                ev[s][1].record(stream)
            barrier()
        trace = snaps.snaps_trace_read(ctx)
        trace["_steps"] = snaps.snaps_trace_steps(ctx)
        snaps.snaps_trace(ctx, False)
        for p in pops:
            snaps.snaps_release(p)
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, dev)
        return total_ms, trace, clk.summary()

    total_ms, trace, clocks = timed_leg(head_prec, args.steps, args.warmup)
    units = float(n) * m_total * args.steps
    value = units / (total_ms / 1e3)
    evals_per_step = float(n) * (n - 1) * m
    props = torch.cuda.get_device_properties(local)
    max_mhz = clocks["sm_max_mhz"] or 2032.0
    launches = int(sum(v[1] for kn, v in trace.items() if not kn.startswith("_")))

    def alu_roofline(trace, steps):
        """ALU roofline of the plain path's dominant join kernel: one FP32 compare per
        (pair, subspace) evaluation is the algorithmic minimum."""
        tree_ms = trace["join_tree"][0]
        lane_ms = trace["join_lane"][0]
        dominant = "join_tree" if tree_ms >= lane_ms else "join_lane"
        dom_ms, dom_launches = trace[dominant]
        peak = props.multi_processor_count * COMPARES_PER_SM_CLK * max_mhz * 1e6 / 1e12
        achieved = evals_per_step * steps / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else None
        measured_alu = snaps.snaps_calibrate_alu(local) / 1e12
        traffic = TREE_DRAM_BYTES_PER_EVAL * evals_per_step if dominant == "join_tree" else None
        loaded, total_steps = trace["_steps"]
        executed = loaded / total_steps if (dominant == "join_tree" and total_steps) else None
        return {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak,
                "unit": "Tevals/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "executed_fraction": executed,
                "frac_executed": (achieved * executed / peak) if (achieved and executed) else None,
                "executed_basis": "64-row steps of the candidate streams loaded and evaluated over all steps "
                                  "(the rest skipped by their box bound, which proves every pair fails), "
                                  "counted by the kernel during the timed steps",
                "traffic_basis": "DRAM bytes per launch: an ncu capture of one 32-subspace chunk (11.3 MB for "
                                 "3.2e10 evaluations) scaled by the launch's evaluations",
                "peak_basis": f"{props.multi_processor_count} SMs x {COMPARES_PER_SM_CLK} FP32 "
                              f"compares/clk x {max_mhz:.0f} MHz (one compare per pair-subspace "
                              f"evaluation)",
                "kernel_ms_per_launch": dom_ms / max(dom_launches, 1),
                "measured_alu_peak": measured_alu,
                "frac_of_measured_alu": (achieved / measured_alu) if achieved else None}

    def tensor_roofline(trace, steps):
        """Tensor roofline of the tensor-core join: 2 x 32 FLOPs per (pair, subspace)
        evaluation (two K = 16 MMAs, over the high and the low parts of the squared
        differences, FP16 or BF16) against the measured dense BF16 peak (FP16 runs at
        the same rate)."""
        tc_ms, tc_launches = trace["join_tc"]
        flops = 2.0 * 32 * evals_per_step * steps
        achieved = flops / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
        peak = PEAKS.get("bf16_tflops_sustained") or PEAKS.get("bf16_tflops") or 1400.0
        return {"bound": "tensor", "kernel": "join_tc", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": TC_DRAM_BYTES_PER_EVAL * evals_per_step,
                "traffic_basis": "DRAM bytes per launch: an ncu capture of one 256-subspace block (1.33 GB "
                                 "for 2.6e11 evaluations) scaled by the launch's evaluations",
                "peak_basis": "measured dense BF16 GEMM, sustained (MEASURED_PEAKS.json); FP16 "
                              "has the same dense rate; 64 FLOPs per evaluation (two K = 16 MMAs)",
                "evals_per_s": evals_per_step * steps / (tc_ms / 1e3) if tc_ms > 0 else None,
                "kernel_ms_per_launch": tc_ms / max(tc_launches, 1)}

    roofline = tensor_roofline(trace, args.steps) if (head_prec & 0xFF) != snaps.SNAPS_FP32 else \
        alu_roofline(trace, args.steps)

    tc_legs = {}
    for form in {"both": [snaps.SNAPS_TC_F16],
                 "all": [snaps.SNAPS_TC_F16, snaps.SNAPS_TC_BF16, snaps.SNAPS_TC_TF32]}.get(
            args.precision, []):
        tc_ms, tc_trace, tc_clocks = timed_leg(form | index_flag, args.tc_steps, 1)
        tc_units = float(n) * m_total * args.tc_steps
        tc_legs[form_name[form]] = {"value": tc_units / (tc_ms / 1e3), "unit": "objects*subspaces/s",
                  "ms_per_step": tc_ms / args.tc_steps, "steps": args.tc_steps, "warmup": 1,
                  "vs_plain": (tc_units / (tc_ms / 1e3)) / value,
                  "distance_evals_per_s": float(n) * (n - 1) * m_total * args.tc_steps / (tc_ms / 1e3),
                  "roofline": tensor_roofline(tc_trace, args.tc_steps),
                  "phase_ms_per_step": {kn: v[0] / args.tc_steps for kn, v in tc_trace.items()
                                        if not kn.startswith("_")},
                  "gpu_launches": int(sum(v[1] for kn, v in tc_trace.items() if not kn.startswith("_"))),
                  "clocks": tc_clocks,
                  "exactness": (f"eps counts, kNN lists, in-degrees and kNN means bit-identical to the plain "
                                f"FP32 join; mean eps distances from the {form_name[form][3:].upper()} "
                                f"high/low accumulator, within 1e-5")}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        x_pin = torch.from_numpy(x).pin_memory()
        top_host = torch.empty((m, 4, 100), dtype=torch.int32).pin_memory()
        x_stage = torch.empty_like(x_dev)

        def e2e_step():
            x_stage.copy_(x_pin, non_blocking=True)     # H2D of this step's input
            pop = snaps.snaps_index(ctx, x_stage, snaps.SNAPS_NORM_MINMAX, stream=stream)
            snaps.snaps_scores(pop, masks, k, precision=head_prec, scores=scores, norm=norm,
                               top=top_host, top_n=100, stream=stream)   # D2H of the rankings
            snaps.snaps_release(pop)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": units / e2e_s, "unit": "objects*subspaces/s",
               "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(m * 4 * 100 * 4)}

    # every rank's top-100 lists on rank 0, in request order (after the timed legs)
    gathered = shard.gather({"top": top.cpu().numpy()}, positions, m_total, rank, world, dist)
    if rank == 0 and gathered["top"].shape[0] != m_total:
        raise RuntimeError("the gathered top lists do not cover every subspace")
    snaps.snaps_destroy(ctx)
    result = {
        "metric": "objects*subspaces/s",
        "value": value,
        "unit": "objects*subspaces/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(args, m_total), "objects": n, "subspaces": int(m_total), "k": k,
                   "precision": form_name[head_prec & 0xFF],
                   "index": args.index,
                   "l2": "flushed before every step (512 MB write)",
                   "parallelism": (f"subspaces sharded x{world}: whole 32-subspace chunks, longest first "
                                   f"to the least-loaded rank (rank 0: {m} of {m_total})")},
        "distance_evals_per_s": float(n) * (n - 1) * m_total * args.steps / (total_ms / 1e3),
        "roofline": roofline,
        "phase_ms_per_step": {kname: v[0] / args.steps for kname, v in trace.items() if not kname.startswith("_")},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    result.update(tc_legs)
    return result


# ---- serving: a Poisson stream of mixed requests ----------------------------------------------

def serving_requests(args, rng, count):
    """Populations N ~ LogUniform(1e3, max_n) (seeded per population), requests
    with 1..max_masks subspaces (d uniform in 2..15, then a uniform subset),
    k in {5, 10, 20}, eps = 0.05 sqrt(d)."""
    n_pops = 12
    pops = []
    for p in range(n_pops):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(args.serving_max_n))))
        pops.append((n, int(rng.integers(0, 1 << 30))))
    reqs = []
    for _ in range(count):
        pi = int(rng.integers(0, n_pops))
        nm = int(rng.integers(1, args.serving_max_masks + 1))
        masks = []
        for _ in range(nm):
            d = int(rng.integers(2, 16))
            feats = rng.choice(15, size=d, replace=False)
            masks.append(int(sum(1 << int(f) for f in feats)))
        reqs.append((pi, np.array(masks, dtype=np.uint16), int(rng.choice([5, 10, 20]))))
    return pops, reqs


def run_serving(args, count=None, with_tc=None):
    """The same Poisson stream of requests through the plain form and, under
    --precision both, through the tensor-core form: identical arrivals (the rate
    is set from the plain form's service time alone), p50/p99 latency for each."""
    import torch

    import paper_2405_20176_b300 as snaps

    count = args.serving if count is None else count
    with_tc = (args.precision == "both") if with_tc is None else with_tc
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20240530)
    pops, reqs = serving_requests(args, rng, count)
    ctx = snaps.snaps_create(0)
    snaps.snaps_set_slots(ctx, args.serving_slots)
    handles = [snaps.snaps_index(ctx, snaps_inputs.population(n, seed)) for n, seed in pops]
    tops = [torch.empty((m.size, 4, 100), dtype=torch.int32, device="cuda") for _, m, _ in reqs]
    torch.cuda.synchronize()
    head = {"tc_f16": snaps.SNAPS_TC_F16, "tc_bf16": snaps.SNAPS_TC_BF16}.get(args.precision, snaps.SNAPS_FP32)
    # service time of one request alone, to set the arrival rate
    n_cal = min(8, len(reqs))
    for (pi, m, k), tp in zip(reqs[:n_cal], tops[:n_cal]):   # warm-up
        snaps.snaps_scores(handles[pi], m, k, precision=head, top=tp, top_n=100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (pi, m, k), tp in zip(reqs[:n_cal], tops[:n_cal]):
        snaps.snaps_scores(handles[pi], m, k, precision=head, top=tp, top_n=100)
    torch.cuda.synchronize()
    mean_service = (time.perf_counter() - t0) / n_cal
    rate = args.serving_load / mean_service
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))

    def stream(precision):
        with ClockSampler(0) as clk:
            start = time.perf_counter()
            tickets = []
            for (pi, m, k), tp, at in zip(reqs, tops, arrivals):
                wait = start + at - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                tickets.append(snaps.snaps_submit(ctx, handles[pi], m, k, precision=precision, top=tp,
                                                  top_n=100))
            results = [snaps.snaps_poll(ctx, t, -1) for t in tickets]
            makespan = time.perf_counter() - start
        lat = np.array([r.latency_us for r in results]) / 1e3
        queue = np.array([r.queue_us for r in results]) / 1e3
        work = float(sum(r.objects_x_subspaces for r in results))
        bad = [r.status for r in results if r.status != snaps.SNAPS_OK]
        return {"value": work / makespan, "unit": "objects*subspaces/s",
                "p50_latency_ms": float(np.percentile(lat, 50)),
                "p99_latency_ms": float(np.percentile(lat, 99)),
                "p50_queue_ms": float(np.percentile(queue, 50)),
                "p99_queue_ms": float(np.percentile(queue, 99)),
                "requests": len(results), "failed": len(bad), "makespan_s": makespan,
                "clocks": clk.summary()}

    main = stream(head)
    main["fused_launches"], main["fused_requests"] = snaps.snaps_serving_stats(ctx)
    tc = stream(snaps.SNAPS_TC_F16) if with_tc else None
    for h in handles:
        snaps.snaps_release(h)
    snaps.snaps_destroy(ctx)
    out = {
        "metric": "objects*subspaces/s (serving stream)",
        "value": main["value"],
        "unit": "objects*subspaces/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "p50_latency_ms": main["p50_latency_ms"],
        "p99_latency_ms": main["p99_latency_ms"],
        "p50_queue_ms": main["p50_queue_ms"],
        "p99_queue_ms": main["p99_queue_ms"],
        "shared_launches": main["fused_launches"],
        "requests_in_shared_launches": main["fused_requests"],
        "requests": main["requests"],
        "failed": main["failed"],
        "makespan_s": main["makespan_s"],
        "arrival_rate_per_s": rate,
        "mean_service_alone_s": mean_service,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"Poisson stream of {len(reqs)} scoring requests at load "
                               f"{args.serving_load} of one request's service rate; 12 resident "
                               f"populations N ~ LogUniform(1e3, {args.serving_max_n}); 1-"
                               f"{args.serving_max_masks} subspaces (d uniform 2..15); "
                               f"k in {{5,10,20}}; eps = 0.05*sqrt(d); top-100 outputs",
                   "slots": args.serving_slots,
                   "precision": {snaps.SNAPS_TC_F16: "tc_f16", snaps.SNAPS_TC_BF16: "tc_bf16"}.get(head, "fp32")},
        "clocks": main["clocks"],
    }
    if tc is not None:
        tc["vs_plain"] = tc["value"] / main["value"]
        out["tc_f16"] = tc
    return out


# ---- parameter selection ------------------------------------------------------------------------

def run_select(args):
    """Parameter selection as Sec. 3.5.3 and 3.5.2 chain it: the eps grid ends
    from the selectivities 0.001 N and 0.15 N (sampled histogram), then one
    selection join per subspace for the eps and k grids."""
    import torch

    import paper_2405_20176_b300 as snaps

    torch.cuda.set_device(0)
    x = snaps_inputs.population(args.n, 0)
    masks = snaps_inputs.mask_sample(args.select, SAMPLE_SEED)
    # k_min = 2 .. k_max = 4096, fine at small k and coarse at large k (Sec. 3.6.2)
    k_grid = [2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128, 256, 512, 1024, 2048, 4096]
    top_n = max(1, args.n // 100)
    n_eps = 16
    ctx = snaps.snaps_create(0)
    pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
    lo, hi = snaps.snaps_eps_range(pop, args.n, masks[:2])   # warm-up
    snaps.snaps_select(pop, masks[:2], lo, hi, n_eps, k_grid, top_n)
    torch.cuda.synchronize()
    snaps.snaps_trace(ctx, True)
    t0 = time.perf_counter()
    emin, emax = snaps.snaps_eps_range(pop, args.n, masks)
    t1 = time.perf_counter()
    _, e_sel, _, k_sel = snaps.snaps_select(pop, masks, emin, emax, n_eps, k_grid, top_n)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    tr = snaps.snaps_trace_read(ctx)
    snaps.snaps_release(pop)
    snaps.snaps_destroy(ctx)
    d = np.array([bin(int(v)).count("1") for v in masks])
    return {"metric": "subspaces selected/s (eps range, eps and k grids)", "value": masks.size / (t2 - t0),
            "unit": "subspaces/s", "n_gpus": 1, "higher_is_better": True,
            "seconds": t2 - t0, "seconds_eps_range": t1 - t0, "seconds_select": t2 - t1,
            "phase_ms": {k: v[0] for k, v in tr.items() if v[1]},
            "eps_range_over_sqrt_d_median": [float(np.median(emin / np.sqrt(d))),
                                             float(np.median(emax / np.sqrt(d)))],
            "eps_select_histogram": np.bincount(e_sel.ravel(), minlength=n_eps).tolist(),
            "k_select_values": np.bincount(np.asarray(k_grid)[k_sel.ravel()]).nonzero()[0].tolist(),
            "config": {"workload": f"N={args.n} objects, {masks.size} sampled subspaces; eps range from "
                                   f"selectivity 0.001 N .. 0.15 N (1024 sampled objects, 4096 bins); eps "
                                   f"grid {n_eps} values; k grid {k_grid}; top-n {top_n}"}}


def run_by_dimension(args):
    """Device time of one call over 256 seeded subspaces of one dimension d,
    for every d, through the tensor-core form (FP16 operands) and the plain
    form (no index): where each form spends its time, by dimension."""
    import torch

    import paper_2405_20176_b300 as snaps

    torch.cuda.set_device(0)
    n = args.n
    x = snaps_inputs.population(n, 0)
    ctx = snaps.snaps_create(0)
    pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
    allm = snaps_inputs.all_masks()
    pc = np.array([bin(int(v)).count("1") for v in allm])
    rng = np.random.default_rng(SAMPLE_SEED)
    rows = []
    for d in range(2, 16):
        pool = allm[pc == d]
        ms = np.sort(rng.choice(pool, size=min(256, pool.size), replace=False)).astype(np.uint16)
        sc = torch.empty((ms.size, 4, n), device="cuda")
        row = {"d": d, "subspaces": int(ms.size)}
        for name, prec in (("tc_f16", snaps.SNAPS_TC_F16), ("fp32", snaps.SNAPS_FP32 | snaps.SNAPS_INDEX_NONE)):
            snaps.snaps_scores(pop, ms, args.k, precision=prec, scores=sc)   # warm-up
            torch.cuda.synchronize()
            snaps.snaps_trace(ctx, True)
            snaps.snaps_scores(pop, ms, args.k, precision=prec, scores=sc)
            torch.cuda.synchronize()
            tr = snaps.snaps_trace_read(ctx)
            snaps.snaps_trace(ctx, False)
            row[name + "_join_ms"] = tr["join_tc"][0] + tr["join_tree"][0] + tr["join_lane"][0]
        row["eps_neighbours_per_object"] = float(sc[:, 0].double().mean().item())
        rows.append(row)
        print(f"[bench] d={d}: {row}", file=sys.stderr, flush=True)
    snaps.snaps_release(pop)
    snaps.snaps_destroy(ctx)
    return {"metric": "join ms per call of 256 subspaces of one dimension", "n": n, "k": args.k,
            "rows": rows,
            "config": {"workload": f"N={n} objects (seed 0); per dimension d = 2..15, 256 subspaces drawn "
                                   f"with seed {SAMPLE_SEED} (all of them where fewer exist); k={args.k}, "
                                   f"eps=0.05*sqrt(d); the tensor-core form with FP16 operands and the plain "
                                   f"form without the grid index; one warm-up call, one timed call each"}}


def run_precision(args):
    """Precision workload: the plain FP32 join and both tensor-core forms on
    the same population and subspaces, two subspace sets of 256 each: eight
    whole 32-subspace chunks (the all-subspace workload's shape, where the
    plain form runs the subspace-batched tree join) and 256 random subspaces
    (where it joins each subspace on its own).  One warm-up call on a small
    population, then one timed call per form and set (library trace on the
    launch stream).  The errors against the FP64 oracle on sampled queries
    at this size come from tests/test_gpu_precision.py."""
    import torch

    import paper_2405_20176_b300 as snaps

    torch.cuda.set_device(0)
    n = args.precision_n
    x = snaps_inputs.population(n, 0)
    sets = {"chunks": snaps_inputs.chunk_sample(8, SAMPLE_SEED),
            "random": snaps_inputs.mask_sample(256, SAMPLE_SEED)}
    forms = {"fp32": snaps.SNAPS_FP32, "tc_f16": snaps.SNAPS_TC_F16, "tc_bf16": snaps.SNAPS_TC_BF16,
             "tc_tf32": snaps.SNAPS_TC_TF32}
    ctx = snaps.snaps_create(0)
    warm = snaps.snaps_index(ctx, torch.from_numpy(snaps_inputs.population(4096, 1)).cuda())
    sc = torch.empty((256, 4, 4096), device="cuda")
    for m in sets.values():
        for prec in forms.values():
            snaps.snaps_scores(warm, m, args.k, precision=prec, scores=sc)
    torch.cuda.synchronize()
    snaps.snaps_release(warm)
    pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
    sc = torch.empty((256, 4, n), device="cuda")
    top = torch.empty((256, 4, 100), dtype=torch.int32, device="cuda")
    rows = {}
    with ClockSampler(0) as clk:
        for sname, m in sets.items():
            row = {}
            for fname, prec in forms.items():
                snaps.snaps_trace(ctx, True)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                snaps.snaps_scores(pop, m, args.k, precision=prec, scores=sc[:m.size], top=top[:m.size],
                                   top_n=100)
                ev1.record()
                torch.cuda.synchronize()
                tr = snaps.snaps_trace_read(ctx)
                snaps.snaps_trace(ctx, False)
                ms = ev0.elapsed_time(ev1)
                row[fname] = {"ms": ms, "objects_x_subspaces_per_s": float(n) * m.size / (ms / 1e3),
                              "evals_per_s": float(n) * (n - 1) * m.size / (ms / 1e3),
                              "phase_ms": {k: v[0] for k, v in tr.items() if v[1]}}
                print(f"[bench] precision {sname} {fname}: {ms:.1f} ms", file=sys.stderr, flush=True)
            for fname in ("tc_f16", "tc_bf16", "tc_tf32"):
                row[fname]["vs_plain"] = row["fp32"]["ms"] / row[fname]["ms"]
            rows[sname] = row
    snaps.snaps_release(pop)
    snaps.snaps_destroy(ctx)
    return {"metric": "objects*subspaces/s, tensor-core forms vs plain FP32 (precision workload)",
            "unit": "objects*subspaces/s", "n": n, "k": args.k, "sets": rows, "clocks": clk.summary(),
            "dtype": "f32 (plain), f16 / bf16 / tf32 high+low parts with f32 accumulation (tensor-core forms)",
            "data": "synthetic",
            "config": {"workload": f"N={n} objects (seed 0); 'chunks': eight whole 32-subspace chunks "
                                   f"(seed {SAMPLE_SEED}), 'random': 256 random subspaces (seed {SAMPLE_SEED}); "
                                   f"k={args.k}, eps=0.05*sqrt(d); scores and top-100 on the device; one "
                                   f"timed call per form and set after a warm-up on 4,096 objects"}}


def run_rubin(args):
    """Rubin-scale leg: two-feature subspaces of a 5,000,000-object population
    through the grid index (sort-by-cell, Sec. 3.8.1), scores and top-100 on the
    device.  One call over the chosen subspaces is timed after a one-subspace
    warm-up call."""
    import torch

    import paper_2405_20176_b300 as snaps

    torch.cuda.set_device(0)
    n = args.rubin_n
    full = (1 << 15) - 1
    if args.rubin_full:
        masks = np.array([full], dtype=np.uint16)
    else:
        pairs = snaps_inputs.pairs_and_full()
        pairs = pairs[pairs != full]
        sel = np.linspace(0, pairs.size - 1, min(args.rubin, pairs.size)).round().astype(int)
        masks = pairs[np.unique(sel)]
    x = snaps_inputs.population(n, 0)
    ctx = snaps.snaps_create(0)
    if args.rubin_cells:
        snaps.snaps_autotune_set(ctx, n, args.k, 2, True, 1.0 / args.rubin_cells)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda(), snaps.SNAPS_NORM_MINMAX, stream=stream)
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t0
    sc = torch.empty((masks.size, 4, n), dtype=torch.float32, device="cuda")
    top = torch.empty((masks.size, 4, 100), dtype=torch.int32, device="cuda")
    if not args.rubin_full:
        snaps.snaps_scores(pop, masks[:1], args.k, scores=sc[:1], top=top[:1], top_n=100, stream=stream)
        torch.cuda.synchronize()
    snaps.snaps_trace(ctx, True)
    with ClockSampler(0) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        snaps.snaps_scores(pop, masks, args.k, scores=sc, top=top, top_n=100, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    tr = snaps.snaps_trace_read(ctx)
    held, budget = snaps.snaps_mem_info(ctx)
    # every ordered eps-neighbour pair needs one square root for the mean distance
    nbr_pairs = float(sc[:, 0].double().sum().item())
    props = torch.cuda.get_device_properties(0)
    clocks = clk.summary()
    mhz = clocks["sm_max_mhz"] or 2032.0
    if args.rubin_full:
        # brute force in one subspace of d = 15 features: per ordered pair, d
        # subtractions and d FMAs on the FP32 pipe are the algorithmic minimum
        d = 15
        join_ms = tr["join_lane"][0]
        fp32_peak = props.multi_processor_count * FMA_LANES_PER_SM_CLK * mhz * 1e6 / 1e12
        evals = float(n) * (n - 1)
        achieved = evals * 2 * d / (join_ms / 1e3) / 1e12 if join_ms > 0 else None
        roofline = {"bound": "alu", "kernel": "join_single_kernel (one subspace at a time)",
                    "achieved": achieved, "peak": fp32_peak, "unit": "T FP32 ops/s",
                    "frac": achieved / fp32_peak if achieved else None, "traffic": None,
                    "peak_basis": f"{props.multi_processor_count} SMs x {FMA_LANES_PER_SM_CLK} FP32 lane-ops/clk "
                                  f"x {mhz:.0f} MHz; {2 * d} FP32 ops ({d} subtractions, {d} FMAs) per "
                                  f"evaluated pair, {evals:.3e} pairs",
                    "evals_per_s": evals / (join_ms / 1e3) if join_ms > 0 else None,
                    "eps_neighbour_pairs": nbr_pairs}
    else:
        grid_ms = tr["grid"][0]
        mufu_peak = props.multi_processor_count * MUFU_PER_SM_CLK * mhz * 1e6 / 1e12
        achieved = nbr_pairs / (grid_ms / 1e3) / 1e12 if grid_ms > 0 else None
        roofline = {"bound": "alu", "kernel": "grid phase (index build, grid_tile_kernel, grid_ring_kernel)",
                    "achieved": achieved, "peak": mufu_peak, "unit": "T sqrt/s",
                    "frac": achieved / mufu_peak if achieved else None, "traffic": None,
                    "peak_basis": f"{props.multi_processor_count} SMs x {MUFU_PER_SM_CLK} MUFU ops/clk x "
                                  f"{mhz:.0f} MHz: one square root per ordered eps-neighbour pair "
                                  f"({nbr_pairs:.3e} in this call), the algorithmic minimum of the mean "
                                  f"eps distance",
                    "eps_neighbour_pairs": nbr_pairs}
    out_bytes = sc.numel() * 4 + top.numel() * 4
    snaps.snaps_release(pop)
    snaps.snaps_destroy(ctx)
    units = float(n) * masks.size
    what = "full 15-feature subspace, brute force" if args.rubin_full else "two-feature subspaces, grid index"
    return {"metric": f"objects*subspaces/s (Rubin scale, {what})",
            "value": units / (ms / 1e3), "unit": "objects*subspaces/s", "n_gpus": 1, "higher_is_better": True,
            "ms": ms, "ms_per_subspace": ms / masks.size, "subspaces": int(masks.size),
            "brute_force_equivalent_evals_per_s": float(n) * (n - 1) * masks.size / (ms / 1e3),
            "phase_ms": {k: v[0] for k, v in tr.items() if v[1]},
            "index_s": index_s,
            "hbm_bytes": {"library_held": held, "caller_outputs": out_bytes, "total": held + out_bytes},
            "roofline": roofline,
            "clocks": clocks, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"N={n} objects (seed 0), the full 15-feature subspace, k={args.k}, "
                                    f"eps=0.05*sqrt(15); brute force, one subspace at a time; scores and "
                                    f"top-100 on the device; one timed call, no warm-up call")
                       if args.rubin_full else
                       (f"N={n} objects (seed 0), {masks.size} of the 105 two-feature subspaces "
                        f"(evenly spaced), k={args.k}, eps=0.05*sqrt(2); grid index over both "
                        f"features, cells {'eps/3 (the library default)' if not args.rubin_cells else f'eps/{args.rubin_cells}'} "
                        f"wide; scores and top-100 on the device")}}


# ---- CPU oracle legs -------------------------------------------------------------------------

def oracle_rate(x, masks, budget_s, k):
    """Run the FP64 oracle subspace by subspace until budget_s has passed;
    returns (objects*subspaces/s, subspaces done, seconds, threads)."""
    import oracle
    xn = oracle.normalise(x)
    done, t0 = 0, time.perf_counter()
    for mask in masks:
        oracle.subspace(xn, int(mask), k)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return x.shape[0] * done / el, done, el, oracle.threads()


def cpu_baseline(args):
    x = snaps_inputs.population(args.n, 0)
    sample = snaps_inputs.mask_sample(64, SAMPLE_SEED)
    v, done, el, thr = oracle_rate(x, sample, 15.0, args.k)
    return {"value": v, "unit": "objects*subspaces/s", "cores": thr, "kind": "oracle",
            "sample": f"FP64 oracle (normalise, brute-force joins, metrics, ranks, top-100) on "
                      f"{done} of the 64 seeded sample subspaces, all {args.n} queries, "
                      f"{el:.1f} s"}


def run_reference(args):
    x = snaps_inputs.population(args.n, 0)
    sample = snaps_inputs.mask_sample(64, SAMPLE_SEED)
    per_step = 2
    import oracle
    oracle.build()
    for w in range(args.warmup):
        oracle_rate(x, sample[w * per_step:(w + 1) * per_step], 0.0, args.k)
    t_total, done_total = 0.0, 0
    for s in range(args.steps):
        ms = sample[(args.warmup + s) * per_step % 64:][:per_step]
        t0 = time.perf_counter()
        for mask in ms:
            oracle.subspace(oracle.normalise(x), int(mask), args.k)
        t_total += time.perf_counter() - t0
        done_total += len(ms)
    value = args.n * done_total / t_total
    thr = oracle.threads()
    sample_txt = (f"{per_step} of the 64 seeded sample subspaces per step, all {args.n} queries, "
                  f"FP64 oracle on {thr} host threads")
    return {
        "impl": "reference",
        "metric": "objects*subspaces/s",
        "value": value,
        "unit": "objects*subspaces/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args, 32752 if args.masks == "all" else int(args.masks)),
                   "objects": args.n, "k": args.k},
        "cpu_baseline": {"value": value, "unit": "objects*subspaces/s", "cores": thr,
                         "kind": "oracle", "sample": sample_txt},
        "e2e": {"value": value, "unit": "objects*subspaces/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return 0
    if args.serving:
        print(json.dumps(run_serving(args)))
        return 0
    if args.select:
        print(json.dumps(run_select(args)))
        return 0
    if args.rubin:
        print(json.dumps(run_rubin(args)))
        return 0
    if args.by_dimension:
        print(json.dumps(run_by_dimension(args)))
        return 0
    if args.precision_config:
        print(json.dumps(run_precision(args)))
        return 0
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    res = run_ours(args, rank, world, dist)
    if rank == 0:
        if world == 1 and args.serving_leg > 0:
            sv = run_serving(args, count=args.serving_leg, with_tc=True)
            keep = ("value", "unit", "p50_latency_ms", "p99_latency_ms", "p50_queue_ms", "p99_queue_ms",
                    "requests", "failed", "makespan_s", "arrival_rate_per_s", "mean_service_alone_s",
                    "shared_launches", "requests_in_shared_launches", "config", "clocks")
            res["serving"] = {key: sv[key] for key in keep}
            res["serving"]["tc_f16"] = {key: sv["tc_f16"][key] for key in
                                        ("value", "p50_latency_ms", "p99_latency_ms", "p50_queue_ms",
                                         "p99_queue_ms", "failed", "makespan_s", "vs_plain", "clocks")}
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(res))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
