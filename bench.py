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
bounded sample of the same workload.  Under torchrun each rank runs its own
replica (subspaces are independent; no collective on the data path) and the
reported time is the max over ranks.
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
    ap.add_argument("--precision", choices=["fp32", "tc_f16"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving", type=int, default=0, metavar="R",
                    help="instead of the batching workload, run a Poisson stream of R scoring "
                         "requests through snaps_submit/snaps_poll and report p50/p99 latency")
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

def run_ours(args, rank, world, dist):
    import torch

    import paper_2405_20176_b300 as snaps

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    x = snaps_inputs.population(args.n, 0)
    masks = workload_masks(args.masks)
    m, n, k = masks.size, args.n, args.k
    precision = snaps.SNAPS_FP32 if args.precision == "fp32" else snaps.SNAPS_TC_F16
    ctx = snaps.snaps_create(local)
    stream = torch.cuda.current_stream()
    x_dev = torch.from_numpy(x).to(dev)
    scores = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
    norm = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
    top = torch.empty((m, 4, 100), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        pop = snaps.snaps_index(ctx, x_dev, snaps.SNAPS_NORM_MINMAX, stream=stream)
        snaps.snaps_scores(pop, masks, k, precision=precision, scores=scores, norm=norm,
                           top=top, top_n=100, stream=stream)
        return pop

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(args.warmup):
        t0 = time.perf_counter()
        snaps.snaps_release(step())
        torch.cuda.synchronize()
        print(f"[bench] warmup {w}: {time.perf_counter() - t0:.3f} s", file=sys.stderr, flush=True)
    barrier()
    snaps.snaps_trace(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    pops = []
    with ClockSampler(local) as clk:
        barrier()
        for s in range(args.steps):
            flush.fill_(float(s))                      # evict the previous step from L2
            ev[s][0].record(stream)
            pops.append(step())
            ev[s][1].record(stream)
        barrier()
    trace = snaps.snaps_trace_read(ctx)
    snaps.snaps_trace(ctx, False)
    for p in pops:
        snaps.snaps_release(p)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = float(n) * m * args.steps * world
    value = units / (total_ms / 1e3)

    # roofline of the dominant kernel (the subspace-batched join)
    tree_ms, tree_launches = trace["join_tree"]
    lane_ms, _ = trace["join_lane"]
    evals_per_step = float(n) * (n - 1) * m
    props = torch.cuda.get_device_properties(local)
    clocks = clk.summary()
    max_mhz = clocks["sm_max_mhz"] or 2032.0
    peak = props.multi_processor_count * COMPARES_PER_SM_CLK * max_mhz * 1e6 / 1e12
    dominant = "join_tree" if tree_ms >= lane_ms else "join_lane"
    dom_ms = max(tree_ms, lane_ms)
    dom_launches = trace[dominant][1]
    achieved = evals_per_step * args.steps / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else None
    launches = int(sum(v[1] for v in trace.values()))
    measured_alu = snaps.snaps_calibrate_alu(local) / 1e12

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        x_pin = torch.from_numpy(x).pin_memory()
        top_host = torch.empty((m, 4, 100), dtype=torch.int32).pin_memory()
        x_stage = torch.empty_like(x_dev)

        def e2e_step():
            x_stage.copy_(x_pin, non_blocking=True)     # H2D of this step's input
            pop = snaps.snaps_index(ctx, x_stage, snaps.SNAPS_NORM_MINMAX, stream=stream)
            snaps.snaps_scores(pop, masks, k, precision=precision, scores=scores, norm=norm,
                               top=top_host, top_n=100, stream=stream)   # D2H of the rankings
            snaps.snaps_release(pop)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": units / e2e_s, "unit": "objects*subspaces/s",
               "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(m * 4 * 100 * 4)}

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
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(args, m), "objects": n, "subspaces": int(m), "k": k,
                   "precision": args.precision, "l2": "flushed before every step (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "distance_evals_per_s": evals_per_step * args.steps * world / (total_ms / 1e3),
        "roofline": {"bound": "alu", "kernel": dominant,
                     "achieved": achieved, "peak": peak, "unit": "Tevals/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "peak_basis": f"{props.multi_processor_count} SMs x {COMPARES_PER_SM_CLK} "
                                   f"FP32 compares/clk x {max_mhz:.0f} MHz (one compare per "
                                   f"pair-subspace evaluation)",
                     "kernel_ms_per_launch": dom_ms / max(dom_launches, 1),
                     "measured_alu_peak": measured_alu,
                     "frac_of_measured_alu": (achieved / measured_alu) if achieved else None},
        "phase_ms_per_step": {kname: v[0] / args.steps for kname, v in trace.items()},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    return result


# ---- serving: a Poisson stream of mixed requests ----------------------------------------------

def serving_requests(args, rng):
    """Populations N ~ LogUniform(1e3, max_n) (seeded per population), requests
    with 1..max_masks subspaces (d uniform in 2..15, then a uniform subset),
    k in {5, 10, 20}, eps = 0.05 sqrt(d)."""
    n_pops = 12
    pops = []
    for p in range(n_pops):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(args.serving_max_n))))
        pops.append((n, int(rng.integers(0, 1 << 30))))
    reqs = []
    for _ in range(args.serving):
        pi = int(rng.integers(0, n_pops))
        nm = int(rng.integers(1, args.serving_max_masks + 1))
        masks = []
        for _ in range(nm):
            d = int(rng.integers(2, 16))
            feats = rng.choice(15, size=d, replace=False)
            masks.append(int(sum(1 << int(f) for f in feats)))
        reqs.append((pi, np.array(masks, dtype=np.uint16), int(rng.choice([5, 10, 20]))))
    return pops, reqs


def run_serving(args):
    import torch

    import paper_2405_20176_b300 as snaps

    torch.cuda.set_device(0)
    rng = np.random.default_rng(20240530)
    pops, reqs = serving_requests(args, rng)
    ctx = snaps.snaps_create(0)
    snaps.snaps_set_slots(ctx, args.serving_slots)
    handles = [snaps.snaps_index(ctx, snaps_inputs.population(n, seed)) for n, seed in pops]
    tops = [torch.empty((m.size, 4, 100), dtype=torch.int32, device="cuda") for _, m, _ in reqs]
    torch.cuda.synchronize()
    # service time of one request alone, to set the arrival rate
    t0 = time.perf_counter()
    n_cal = min(8, len(reqs))
    for (pi, m, k), tp in zip(reqs[:n_cal], tops[:n_cal]):
        snaps.snaps_scores(handles[pi], m, k, top=tp, top_n=100)
    torch.cuda.synchronize()
    mean_service = (time.perf_counter() - t0) / n_cal
    rate = args.serving_load / mean_service
    gaps = rng.exponential(1.0 / rate, size=len(reqs))
    arrivals = np.cumsum(gaps)
    with ClockSampler(0) as clk:
        start = time.perf_counter()
        tickets = []
        for (pi, m, k), tp, at in zip(reqs, tops, arrivals):
            wait = start + at - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tickets.append(snaps.snaps_submit(ctx, handles[pi], m, k, top=tp, top_n=100))
        results = [snaps.snaps_poll(ctx, t, -1) for t in tickets]
        makespan = time.perf_counter() - start
    lat = np.array([r.latency_us for r in results]) / 1e3
    queue = np.array([r.queue_us for r in results]) / 1e3
    work = float(sum(r.objects_x_subspaces for r in results))
    bad = [r.status for r in results if r.status != snaps.SNAPS_OK]
    for h in handles:
        snaps.snaps_release(h)
    snaps.snaps_destroy(ctx)
    return {
        "metric": "objects*subspaces/s (serving stream)",
        "value": work / makespan,
        "unit": "objects*subspaces/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "p50_latency_ms": float(np.percentile(lat, 50)),
        "p99_latency_ms": float(np.percentile(lat, 99)),
        "p50_queue_ms": float(np.percentile(queue, 50)),
        "p99_queue_ms": float(np.percentile(queue, 99)),
        "requests": len(results),
        "failed": len(bad),
        "makespan_s": makespan,
        "arrival_rate_per_s": rate,
        "mean_service_alone_s": mean_service,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"Poisson stream of {len(reqs)} scoring requests at load "
                               f"{args.serving_load} of one request's service rate; 12 resident "
                               f"populations N ~ LogUniform(1e3, {args.serving_max_n}); 1-"
                               f"{args.serving_max_masks} subspaces (d uniform 2..15); "
                               f"k in {{5,10,20}}; eps = 0.05*sqrt(d); top-100 outputs",
                   "slots": args.serving_slots, "precision": args.precision},
        "clocks": clk.summary(),
    }


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
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    res = run_ours(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(res))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
