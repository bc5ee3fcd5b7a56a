"""Benchmark of the step-1 hot path at L = 451 (the paper's Algorithm 1 on synthetic inputs).

One step = the sieve bound over 10^6 sampled starts (labs_sample_threshold) + 65,536 skew-symmetric
self-avoiding walks of 10^5 flips each behind 256 distinct 24-element prefixes (labs_skew_search):
6.55e9 flips, each scanning 202 neighbours x 225 even lags.  Metric: flips/s (higher is better).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs its own 65,536 walks (walk ids offset by
rank), no data-path collective; value = all ranks' flips / max-over-ranks time ("weak" scaling).
The reference arm (--impl reference) is the CPU oracle timed on the host cores on a bounded sample.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import labs_inputs as inp  # noqa: E402

W1 = inp.STEP1_451
METRIC = "flips/s"
WORKLOAD = "step1_skew_walks_L451_p24_65536walks_1e5flips"
SM_MAX_MHZ = 2070.0
SMS = 152
LANES_PER_SM = 128  # 4 schedulers x 32 lanes: one lane-instruction issue slot each per cycle
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "walk_kernel_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2409_07222_gb300", "csrc", f) for f in ("walk.cu", "labs_core.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walks", type=int, default=W1["n_walks"])
    ap.add_argument("--flips", type=int, default=W1["flip_budget"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-walks", type=int, default=64)
    ap.add_argument("--cpu-flips", type=int, default=6000)
    ap.add_argument("--workload", default="step1", choices=["step1", "mixed", "pq", "pq_indep", "learned", "network", "operators", "legendre",
                             "exhaustive", "energy", "deltas", "peaks", "workflow"],
                    help="step1: L=451 walks (the headline); mixed: all lengths 450..527 in one batched launch; "
                         "pq: step-2 refinement from step-1 candidates; learned: the learned-proposal experiment; "
                         "network: the proposal network's inference alone; operators: the end-element operators; "
                         "legendre: Legendre seeds for step 2 (Table 2 lengths); pq_indep: step 2 with one queue per candidate; exhaustive: all skew sequences of L = 37 and 61; energy / deltas: the energy batch and the "
                         "neighbour scan entry points alone; workflow: Fig. 4 end to end (step 1 -> sieve -> step 2 -> "
                         "operators -> step 2 at L +- 1)")
    ap.add_argument("--L", type=int, default=451, help="pq workload: sequence length")
    ap.add_argument("--pq-expansions", type=int, default=inp.STEP2["max_expansions"])
    ap.add_argument("--pq-hlog2", type=int, default=28)
    ap.add_argument("--pq-tr", type=int, default=0, help="pq workload: MAKE_ROTATIONS per side (0: off)")
    ap.add_argument("--pq-indep-pops", type=int, default=500, help="pq_indep workload: pops per candidate")
    ap.add_argument("--pq-indep-hlog2", type=int, default=20,
                    help="pq_indep workload: log2 of each candidate's visited-set slots")
    ap.add_argument("--wf-flips", type=int, default=10000, help="workflow workload: flips per step-1 walk")
    ap.add_argument("--wf-op-expansions", type=int, default=10**6,
                    help="workflow workload: step-2 expansions at L + 1 and L - 1")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def terms_per_flip(L, p):
    k = (L - 1) // 2
    return (k - p + 1) * ((L - 1) // 2)  # free neighbours x even lags


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(n_walks):
    """DRAM bytes of one walk-kernel launch, scaled by walks from the committed ncu capture of a smaller
    launch (its traffic is the per-walk candidate records and statistics); None if the kernel changed."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d["dram_bytes_per_walk"] * n_walks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(walks, flips, threads=None):
    """The oracle (plain C over +-1 arrays) on a bounded sample of the same workload."""
    import oracle

    threads = threads or os.cpu_count() or 1
    L, p = W1["L"], W1["p"]
    pre = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"])
    n_thr = max(1, W1["n_thresh_samples"] * walks // W1["n_walks"])
    rank = min(n_thr - 1, W1["thresh_rank"] * walks // W1["n_walks"])
    t0 = time.perf_counter()
    thr = oracle.threshold(L, True, p, pre, W1["seed"], n_thr, rank)
    oracle.walk_search(L, True, p, pre, walks, flips, W1["T_i"], W1["seed"], R=W1["R"], bloom_log2=W1["bloom_log2"],
                       bloom_k=W1["bloom_k"], E_thr=thr, n_threads=threads)
    dt = time.perf_counter() - t0
    return {"value": walks * flips / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": "%d walks x %d flips of the L=451 p=24 workload (walk ids 0..%d) + sieve bound over %d "
                      "samples, %.1f s" % (walks, flips, walks - 1, n_thr, dt)}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    # each step is a bounded sample of the workload; the whole run stays within a few minutes
    walks, flips = args.cpu_walks, max(200, args.cpu_flips // 2)
    for _ in range(args.warmup):
        cpu_baseline(walks, max(50, flips // 10))
    t, vals = 0.0, []
    res = None
    for _ in range(args.steps):
        res = cpu_baseline(walks, flips)
        vals.append(res["value"])
    value = statistics.mean(vals)
    res["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": walks * flips / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": W1["L"], "p": W1["p"], "walks_timed": walks,
                       "flips_per_walk_timed": flips,
                       "sample": "each step times %d walks x %d flips of the 65,536 x 10^5 workload (walk ids 0..%d)"
                                 % (walks, flips, walks - 1)},
            "cpu_baseline": res, "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def unit_terms(L, p):
    """Neighbour-lag multiply-adds of one flip: skew walks scan k-p+1 neighbours over (L-1)/2 even lags,
    unrestricted walks L neighbours over L-1 lags."""
    if L % 2:
        return terms_per_flip(L, p)
    return L * (L - 1)


def run_mixed(args, ws, rank, local):
    """Batched step 1 over L = 450..527: per-length sieve bounds + one persistent walk launch, replayed
    from a CUDA graph; walks per length uniform in {1024..16384} (seed 2410), 10^4 flips each."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lg.load()
    MX = inp.MIXED
    counts = inp.mixed_walk_counts()
    lengths = list(counts)
    walks = [counts[L] for L in lengths]
    budget = MX["flip_budget"] if args.flips == W1["flip_budget"] else args.flips
    p = MX["p"]
    pre_h = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"])
    pre = torch.from_numpy(pre_h.view(np.int64)).to(dev)
    cfg = lg.make_batch_cfg(len(lengths), p=p, flip_budget=budget, seed=MX["count_seed"], R=W1["R"],
                            n_thresh_samples=W1["n_thresh_samples"], thresh_rank=W1["thresh_rank"], use_graph=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    out = lg.labs_batched_search(cfg, lengths, walks, pre, walk_stats=False)  # autotune + capture
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        lg.labs_batched_search(cfg, lengths, walks, pre, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        lg.labs_batched_search(cfg, lengths, walks, pre, out=out)
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = lg.stats_numpy(out[3])
        if int(st["flips"]) != sum(walks) * budget:
            raise RuntimeError("batched walks made %d flips" % int(st["flips"]))
    clk = clocks.stop()
    total_ms = sum(step_ms)
    flips = args.steps * sum(walks) * budget
    terms = sum(w * budget * unit_terms(L, p) for L, w in zip(lengths, walks))
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    achieved = terms / (statistics.mean(step_ms) * 1e-3) / 1e9
    line = {"metric": METRIC, "value": flips / (total_ms * 1e-3), "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "mixed_L450-527_walks_U1024-16384_1e4flips", "lengths": len(lengths),
                       "walks": sum(walks), "flips_per_walk": budget, "p_odd": p, "graph": True,
                       "first_call_s_incl_autotune_and_capture": first_s,
                       "l2": "flushed between timed steps (256 MB write)"},
            "gpu_launches": (4 * len(lengths) + 2) * args.steps, "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "walk_kernel (one launch, all lengths) + 78 sieve bounds",
                         "work": "per flip: (k-p+1)(L-1)/2 terms (odd L, skew) or L(L-1) terms (even L)"}}
    print(json.dumps(line))
    return 0


def run_pq(args, ws, rank, local):
    """Step 2 (Algorithm 2) at one length: 4,096 distinct seeds = the best states of a step-1 search at
    that length (16,384 walks x 5,000 flips, p = 24 for odd L), open set 2^22, B = 4,096 pops per round."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lg.load()
    S2 = inp.STEP2
    L = args.L
    skew = L % 2 == 1
    p = W1["p"] if skew else 0
    pre_h = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"]) if p else np.zeros(1, np.uint64)
    n_w, R = 16384, 4
    cfg = lg.make_walk_cfg(L, skew=skew, p=p, n_walks=n_w, flip_budget=5000, seed=W1["seed"], R=R,
                           E_thr=lg.INT32_MAX)
    out, _, _ = lg.labs_skew_search(cfg, pre_h, with_walk_stats=False)
    cand = lg.candidates_numpy(out, n_w, R).reshape(-1)
    cand = cand[cand["E"] != lg.INT32_MAX]
    order = np.lexsort((cand["fp"], cand["E"]))
    _, first = np.unique(cand["fp"][order], return_index=True)
    pick = order[np.sort(first)][: S2["n_seeds"]]
    pick = pick[np.lexsort((cand["fp"][pick], cand["E"][pick]))]
    W = (L + 63) // 64
    seeds = torch.from_numpy(np.ascontiguousarray(cand["seq"][pick][:, :W]).view(np.int64)).to(dev)
    seed_best = int(cand["E"][pick].min())
    times = []
    for it in range(max(1, args.warmup) + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, bE, st = lg.labs_pq_refine(L, seeds, B=S2["B"], cap=S2["cap"], H_log2=args.pq_hlog2,
                                         max_expansions=args.pq_expansions, T_u=S2["T_u"], T_r=args.pq_tr)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times[-args.steps:])
    s2 = lg.pq_stats_numpy(st)
    exps = int(s2["expansions"])
    terms = exps * L * (L - 1)
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    line = {"metric": "expansions/s", "value": exps / t, "unit": "expansions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "step2_pq_L%d_4096seeds_cap2^22_B4096" % L + ("_Tr%d" % args.pq_tr if args.pq_tr else ""),
                       "L": L, "seeds": int(len(pick)), "T_r": args.pq_tr,
                       "max_expansions": args.pq_expansions, "H_slots_log2": args.pq_hlog2,
                       "seed_best_E": seed_best, "best_E": int(bE.cpu()[0]), "stats": {k: int(s2[k]) for k in
                       ("expansions", "rounds", "survivors", "admitted", "evicted", "h_size", "improvements",
                        "stop_reason", "status")}},
            "neighbour_evaluations_per_s": exps * L / t,
            "roofline": {"bound": "alu", "achieved": terms / t / 1e9, "peak": peak, "unit": "Gop/s",
                         "frac": terms / t / 1e9 / peak, "traffic": None,
                         "work": "per expansion L(L-1) neighbour-lag multiply-adds (whole step timed, host-driven)"}}
    print(json.dumps(line))
    return 0


def run_workflow(args, ws, rank, local):
    """Fig. 4 end to end at L = 451 (workflow.two_step_search): step 1 over the step-1 workload's walks
    (65,536 per GPU, p = 24, sieve bound from 10^6 samples) with --wf-flips flips each, the 4,096 best
    distinct candidates, step 2 at L (B = 4,096, open set 2^22), the end-element operators, step 2 at
    L + 1 and L - 1.  Each rank runs its own walks (walk_begin = rank x walks); rank 0 merges the
    candidates and runs the step-2 stages.  Timed on the host clock around whole workflow passes."""
    import torch

    import paper_2409_07222_gb300 as lg
    from paper_2409_07222_gb300 import workflow

    torch.cuda.set_device(local)
    lg.load()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    L, p = 451, W1["p"]
    pre_h = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"])
    S2 = inp.STEP2
    times, res = [], None
    for it in range(max(1, args.warmup) + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = workflow.two_step_search(L, pre_h, p=p, n_walks=args.walks, flip_budget=args.wf_flips, seed=W1["seed"],
                                       R=W1["R"], n_thresh_samples=W1["n_thresh_samples"],
                                       thresh_rank=W1["thresh_rank"], walk_begin=rank * args.walks,
                                       K=S2["n_seeds"], B=S2["B"], cap=S2["cap"], H_log2=args.pq_hlog2,
                                       max_expansions=args.pq_expansions, op_max_expansions=args.wf_op_expansions)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    if rank != 0:
        return 0
    t = statistics.mean(times[-args.steps:])
    stages = {str(Ln): {"E": res[Ln]["E"], "F": round(res[Ln]["F"], 4), "seconds": round(res[Ln]["seconds"], 4),
                        "expansions": res[Ln]["stats"]["expansions"], "improvements": res[Ln]["stats"]["improvements"],
                        "hex": res[Ln]["hex"]} for Ln in (L, L + 1, L - 1)}
    s1 = res["step1"]
    line = {"metric": "workflow seconds", "value": t, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "fig4_workflow_L451_p24_%dwalks_x%dflips_step2_%d_ops_%d" % (
                           args.walks * ws, args.wf_flips, args.pq_expansions, args.wf_op_expansions),
                       "L": L, "walks_per_gpu": args.walks, "flips_per_walk": args.wf_flips,
                       "seeds": s1["candidates"], "E_thr": s1["E_thr"], "max_expansions": args.pq_expansions,
                       "op_max_expansions": args.wf_op_expansions, "timing": "host clock, whole workflow"},
            "step1": {"seconds": round(s1["seconds"], 4), "flips": s1["flips"], "best_E": s1["best_E"]},
            "operators": res["operators"], "stages": stages}
    print(json.dumps(line))
    return 0


def issue_peaks(local):
    """Measured lane-instructions per SM clock of each instruction class (labs_measure_issue_rates) and the
    chip peaks they imply at the maximum SM clock (SMS x rate x 2070 MHz)."""
    import paper_2409_07222_gb300 as lg

    rates = lg.labs_measure_issue_rates(local)
    return {"lanes_per_clk_per_sm": rates,
            "peak_Gops_at_max_clock": {k: SMS * v * SM_MAX_MHZ * 1e6 / 1e9 for k, v in rates.items()}}


def run_peaks(args, ws, rank, local):
    import torch

    torch.cuda.set_device(local)
    clocks = ClockSampler(local)
    pk = issue_peaks(local)
    clk = clocks.stop()
    line = {"metric": "issue rate", "unit": "lane-instructions per SM clock", "n_gpus": 1,
            "config": {"workload": "issue_rate_probe", "threads_per_sm": 1024, "chains_per_thread": 16,
                       "sms": SMS},
            "clocks": clk, **pk}
    print(json.dumps(line))
    return 0


def reduce_over_ranks(total_ms, units, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time (MAX) and the units all ranks
    processed (SUM).  Works on any initialised process group (NCCL on GPUs, gloo on CPUs); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), int(units)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([int(units)], dtype=torch.int64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def shard(rank, n_per_rank):
    """Walk ids of a rank: [rank * n, (rank + 1) * n); ranks share no walk and need no data exchange."""
    return rank * n_per_rank, n_per_rank


def peaks():
    """Measured peaks of this GPU pool (HBM copy GB/s, dense BF16 TFLOP/s burst and sustained) if the file
    is present, else {} (the caller then uses the fallback figure and says so)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def network_roofline(lg, L, n, local):
    """The network's inference (labs_policy_forward) on n walks' sequences: its FLOPs per call over the
    CUDA-event time of 10 calls on the launching stream, against the measured dense BF16 peak (burst:
    the forward is timed on its own)."""
    import ctypes

    import torch

    pol = lg.Policy(L, seed=1, device=local)
    w = torch.from_numpy(inp.random_words(n, L, seed=3).view(np.int64)).to(torch.device("cuda", local))
    out = torch.empty((n, L), dtype=torch.float32, device=w.device)
    lib = lg.load()
    st = torch.cuda.current_stream(w.device)
    args = (pol.h, ctypes.c_void_p(w.data_ptr()), n, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    for _ in range(3):
        lib.labs_policy_forward(*args)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(10):
        lib.labs_policy_forward(*args)
    e1.record(st)
    st.synchronize()
    ms = e0.elapsed_time(e1) / 10
    status = lib.labs_policy_sync_status(pol.h, ctypes.c_void_p(st.cuda_stream))
    flop = n * (2 * 64 * 2 * 9 * L + 2 * 2 * 64 * 64 * 9 * L + 2 * 256 * 64 * L + 2 * 256 * L)
    pk = peaks()
    peak = pk.get("bf16_tflops", 1900.0)
    src = "bf16_tflops burst, of measured" if "bf16_tflops" in pk else "1.9 PFLOP/s, of fallback"
    ach = flop / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "kernel": "labs_policy_forward (features, conv1, 2 x tcgen05 conv, tcgen05 dense, 256->L)",
            "work": "2*64*(2+2*64)*9*L + 2*256*65*L FLOP per sequence", "n": n, "ms_per_forward": ms,
            "status": status, "peak_source": src}


def run_operators(args, ws, rank, local):
    """The end-element operators at L=451 on 2^20 sequences (the four L+1 and two L-1 results with their
    exact energies), as results per second.  The work is the six energies: one popcount per 32 products,
    sum over k of ceil((L'-k)/32) per result; POPC issues at 16 lanes per clock per SM on this part."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    lg.load()
    L, n = W1["L"], 1 << 20
    w = torch.from_numpy(inp.random_words(n, L, seed=11).view(np.int64)).to(torch.device("cuda", local))
    st = torch.cuda.current_stream()
    for _ in range(3):
        lg.labs_sequence_operators(L, w)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(st)
    for _ in range(reps):
        lg.labs_sequence_operators(L, w)
    e1.record(st)
    st.synchronize()
    ms = e0.elapsed_time(e1) / reps
    def popc_per_energy(Lv):  # one popcount per 32 products of each lag
        return sum(-(-(Lv - k) // 32) for k in range(1, Lv))

    popc = 4 * popc_per_energy(L + 1) + 2 * popc_per_energy(L - 1)
    ach = popc * n / (ms * 1e-3) / 1e9
    peak = SMS * 16 * SM_MAX_MHZ * 1e6 / 1e9
    line = {"metric": "operator results/s", "value": 6 * n / (ms * 1e-3), "unit": "results/s", "n_gpus": 1,
            "steps": reps, "warmup": 3, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "sequence_operators_L451_2^20seq", "L": L, "n": n},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpopc/s", "frac": ach / peak,
                         "traffic": None, "kernel": "operators_kernel",
                         "work": "6 energies per sequence: sum_k ceil((L'-k)/32) popcounts each; "
                                 "peak = 152 SMs x 16 POPC/clk x 2070 MHz"}}
    print(json.dumps(line))
    return 0


def _time_calls(fn, reps=10, warm=3):
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3


def run_energy(args, ws, rank, local):
    """labs_energy_batch on 2^22 random sequences of L = 451 (the sieve sample's shape, 4x larger): all
    C_k and E; one popcount per 32 products of each lag, 268 MB of sequences read per call."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    lg.load()
    L, n = W1["L"], 1 << 22
    w = torch.from_numpy(inp.random_words(n, L, seed=21).view(np.int64)).to(torch.device("cuda", local))
    t = _time_calls(lambda: lg.labs_energy_batch(w, L))
    popc = n * sum(-(-(L - k) // 32) for k in range(1, L))
    peak = SMS * 16 * SM_MAX_MHZ * 1e6 / 1e9
    line = {"metric": "energies/s", "value": n / t, "unit": "energies/s", "n_gpus": 1, "steps": 10, "warmup": 3,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": "energy_batch_L451_2^22seq", "L": L, "n": n},
            "roofline": {"bound": "alu", "achieved": popc / t / 1e9, "peak": peak, "unit": "Gpopc/s",
                         "frac": popc / t / 1e9 / peak, "traffic": None, "kernel": "energy_batch_kernel",
                         "work": "sum_k ceil((L-k)/32) popcounts per sequence; input %.0f MB per call, "
                                 "%.2f TB/s" % (n * 64 / 1e6, n * 64 / t / 1e12)}}
    print(json.dumps(line))
    return 0


def run_deltas(args, ws, rank, local):
    """labs_flip_deltas on 2^16 skew-symmetric sequences of L = 451 with p = 24: Delta E of every free
    neighbour (202 pair flips x 225 even lags per sequence), tables built in the call."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    lg.load()
    L, p, n = W1["L"], W1["p"], 1 << 16
    pre = torch.from_numpy(inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"]).view(np.int64)).to(
        torch.device("cuda", local))
    cfg = lg.make_walk_cfg(L, skew=True, p=p, n_walks=n, flip_budget=1, seed=5, R=1, E_thr=lg.INT32_MAX)
    out, _, _ = lg.labs_skew_search(cfg, pre, with_walk_stats=False)  # skew sequences one flip from a start
    cand = lg.candidates_numpy(out, n, 1).reshape(-1)
    W = (L + 63) // 64
    seqs = torch.from_numpy(np.ascontiguousarray(cand["seq"][:, :W]).view(np.int64)).to(torch.device("cuda", local))
    t = _time_calls(lambda: lg.labs_flip_deltas(seqs, L, skew=True, p=p))
    terms = n * terms_per_flip(L, p)
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    line = {"metric": "neighbour evaluations/s", "value": n * 202 / t, "unit": "evaluations/s", "n_gpus": 1,
            "steps": 10, "warmup": 3, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "flip_deltas_skew_L451_p24_2^16seq", "L": L, "p": p, "n": n},
            "roofline": {"bound": "alu", "achieved": terms / t / 1e9, "peak": peak, "unit": "Gop/s",
                         "frac": terms / t / 1e9 / peak, "traffic": None, "kernel": "flip_deltas_kernel",
                         "work": "45450 neighbour-lag multiply-adds per sequence (as the walk's step)"}}
    print(json.dumps(line))
    return 0


def run_exhaustive(args, ws, rank, local):
    """Exhaustive skew enumeration: every skew-symmetric sequence of L = 37 (2^19 assignments, the small
    configuration) and of L = 61 (2^31), minimum energy, optimum count and argmin, as assignments per
    second.  Each assignment is evaluated from scratch in both of the kernel's passes: per even lag one
    64-bit popcount (two 32-bit ones) for L <= 64 (one word), two (four 32-bit ones) above."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    lg.load()
    res, t_tot, popc_tot, n_tot = [], 0.0, 0, 0
    for L in (inp.EXHAUSTIVE_37["L"], 61):
        k = (L - 1) // 2
        lg.labs_skew_exhaustive(L)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        minE, cnt, arg, _ = lg.labs_skew_exhaustive(L)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        n = 1 << (k + 1)
        t_tot += t
        n_tot += n
        words = 1 if L <= 64 else 2
        popc_tot += 2 * n * 2 * words * ((L - 1) // 2)  # two passes, 2 x words 32-bit popcounts per even lag
        res.append({"L": L, "assignments": n, "seconds": t, "min_E": int(minE.cpu()[0]), "count": int(cnt.cpu()[0]),
                    "argmin_free_bits": int(arg.cpu()[0]), "F": round(L * L / (2.0 * int(minE.cpu()[0])), 4)})
    peak = SMS * 16 * SM_MAX_MHZ * 1e6 / 1e9
    ach = popc_tot / t_tot / 1e9
    line = {"metric": "assignments/s", "value": n_tot / t_tot, "unit": "assignments/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": t_tot * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "exhaustive_skew_L37_L61", "lengths": [r["L"] for r in res]},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpopc/s", "frac": ach / peak,
                         "traffic": None, "kernel": "exh_min_kernel + exh_count_kernel",
                         "work": "2 passes x (L-1)/2 even lags x 2 32-bit popcounts per word of the "
                                 "sequence (1 word for L <= 64) per assignment; peak = 152 SMs x 16 POPC/clk x "
                                 "2070 MHz"},
            "per_length": res}
    print(json.dumps(line))
    return 0


def run_pq_indep(args, ws, rank, local):
    """Step 2 with one queue per candidate: the 4,096 best distinct states of a step-1 search at L (as in
    the pq workload) each refined alone, B = 1, unbounded queue, --pq-indep-pops pops each."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lg.load()
    L = args.L
    skew = L % 2 == 1
    p = W1["p"] if skew else 0
    pre_h = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"]) if p else np.zeros(1, np.uint64)
    n_w, R = 16384, 4
    cfg = lg.make_walk_cfg(L, skew=skew, p=p, n_walks=n_w, flip_budget=5000, seed=W1["seed"], R=R, E_thr=lg.INT32_MAX)
    out, _, _ = lg.labs_skew_search(cfg, pre_h, with_walk_stats=False)
    cand = lg.candidates_numpy(out, n_w, R).reshape(-1)
    cand = cand[cand["E"] != lg.INT32_MAX]
    order = np.lexsort((cand["fp"], cand["E"]))
    _, first = np.unique(cand["fp"][order], return_index=True)
    pick = order[np.sort(first)][: inp.STEP2["n_seeds"]]
    W = (L + 63) // 64
    seeds = torch.from_numpy(np.ascontiguousarray(cand["seq"][pick][:, :W]).view(np.int64)).to(dev)
    pops = args.pq_indep_pops
    times = []
    for it in range(max(1, args.warmup) + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, bE, st = lg.labs_pq_independent(L, seeds, max_expansions=pops, H_log2=args.pq_indep_hlog2)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times[-args.steps:])
    stn = st.cpu().numpy().view(lg.PQ_STATS_DTYPE).reshape(-1)
    exps = int(stn["expansions"].sum())
    terms = exps * L * (L - 1)
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    line = {"metric": "expansions/s", "value": exps / t, "unit": "expansions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "step2_independent_L%d_4096candidates_%dpops" % (L, pops), "L": L,
                       "candidates": int(len(pick)), "pops_each": pops, "H_slots_log2": args.pq_indep_hlog2,
                       "seed_best_E": int(cand["E"][pick].min()), "best_E": int(bE.min().cpu()),
                       "improved_candidates": int((stn["improvements"] > 0).sum()),
                       "status_nonzero": int((stn["status"] != 0).sum())},
            "neighbour_evaluations_per_s": exps * L / t,
            "roofline": {"bound": "alu", "achieved": terms / t / 1e9, "peak": peak, "unit": "Gop/s",
                         "frac": terms / t / 1e9 / peak, "traffic": None,
                         "work": "per expansion L(L-1) neighbour-lag multiply-adds (whole refinement timed)"}}
    print(json.dumps(line))
    return 0


def run_legendre(args, ws, rank, local):
    """Legendre seeds: the construction's throughput (every rotation of every prime with up to 30%
    appended, L = 450..527, exact energies on the device) with its POPC roofline; then, at the lengths of
    Table 2, the (0.20, 0.24, 0.1) family and step 2 (Algorithm 2, B = 4,096, open set 2^22) from all of
    its seeds, with the best constructed and refined merit factors per length (Table 2 prints 6.1976 /
    6.3088, 6.2332 / 6.2998, 6.4292 / 6.4292, 6.3240 / 6.3240: context from the paper's own search)."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lg.load()
    S2 = inp.STEP2
    # construction throughput: every rotation of every prime with up to 30% appended, L = 450..527
    fams = [(L, torch.from_numpy(lg.labs_legendre_family(L, 0.0, 1.0, 0.3)).to(dev)) for L in range(450, 528)]
    for L, fam in fams[:2]:
        lg.labs_legendre_construct(L, fam)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for L, fam in fams:
        lg.labs_legendre_construct(L, fam)
    e1.record()
    torch.cuda.synchronize()
    t_con = e0.elapsed_time(e1) * 1e-3
    n_tot = sum(int(f.shape[0]) for _, f in fams)
    popc_tot = sum(int(f.shape[0]) * sum(-(-(L - k) // 32) for k in range(1, L)) for L, f in fams)
    # Table 2 lengths: the (0.20, 0.24, 0.1) family, then step 2 from all of its seeds
    per_L = []
    for L in (450, 471, 491, 526):
        fam = torch.from_numpy(lg.labs_legendre_family(L)).to(dev)
        seqs, E = lg.labs_legendre_construct(L, fam)
        torch.cuda.synchronize()
        n = fam.shape[0]
        t0 = time.perf_counter()
        best, bE, st = lg.labs_pq_refine(L, seqs, B=S2["B"], cap=S2["cap"], H_log2=args.pq_hlog2,
                                         max_expansions=args.pq_expansions, T_u=S2["T_u"])
        torch.cuda.synchronize()
        t_pq = time.perf_counter() - t0
        s2 = lg.pq_stats_numpy(st)
        per_L.append({"L": L, "seeds": int(n), "F_construct": round(L * L / (2.0 * int(E.min())), 4),
                      "F_refined": round(L * L / (2.0 * int(bE.cpu()[0])), 4), "expansions": int(s2["expansions"]),
                      "refine_s": t_pq})
    peak = SMS * 16 * SM_MAX_MHZ * 1e6 / 1e9
    ach = popc_tot / t_con / 1e9
    line = {"metric": "seeds/s", "value": n_tot / t_con, "unit": "seeds/s", "n_gpus": 1, "steps": 1, "warmup": 2,
            "ms_per_step": t_con * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "legendre_seeds_L450-527_all_rotations", "seeds": n_tot,
                       "table2_family": "r 0.20..0.24 of L, t <= 0.1 p", "max_expansions": args.pq_expansions},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpopc/s", "frac": ach / peak,
                         "traffic": None, "kernel": "legendre_kernel",
                         "work": "sum_k ceil((L-k)/32) popcounts per seed; peak = 152 SMs x 16 POPC/clk x 2070 MHz"},
            "per_length": per_L}
    print(json.dumps(line))
    return 0


def run_network(args, ws, rank, local):
    """The proposal network's inference at L=451 on 8,192 sequences (one chunk's worth of walks), as
    sequences scored per second, with the tensor-core roofline of the forward."""
    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    lg.load()
    roof = network_roofline(lg, W1["L"], 8192, local)
    ms = roof["ms_per_forward"]
    line = {"metric": "sequences/s", "value": 8192 / (ms * 1e-3), "unit": "sequences/s", "n_gpus": 1, "steps": 10,
            "warmup": 3, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "proposal_network_forward_L451_8192seq", "L": W1["L"], "n": 8192},
            "roofline": roof}
    print(json.dumps(line))
    return 0


def run_learned(args, ws, rank, local):
    """Learned proposal at L=451: tuples from plain walks, training, lambda pre-registered on pilot seeds,
    equal-budget gain over 30 fresh seeds (rank-sum) and time to a pre-registered E*, plain vs learned."""
    import torch

    import paper_2409_07222_gb300 as lg
    from paper_2409_07222_gb300 import learn

    torch.cuda.set_device(local)
    lg.load()
    pre = inp.distinct_prefixes(W1["n_prefix"], W1["p"], seed=W1["prefix_seed"])
    t0 = time.perf_counter()
    res = learn.experiment(L=W1["L"], p=W1["p"], prefixes=pre, device=local, log=lambda m: print(m, file=sys.stderr))
    tt = res["time_to_target"]
    roof = network_roofline(lg, W1["L"], 8192, local)
    line = {"metric": "time-to-E* speedup (learned vs plain)", "value": tt["speedup_learned_vs_plain"],
            "unit": "x", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": (time.perf_counter() - t0) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+bf16/fp32",
            "data": "synthetic", "config": {"workload": "learned_proposal_L451", "L": W1["L"], "p": W1["p"]},
            "roofline": roof, "learned": res}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "mixed":
        return run_mixed(args, ws, rank, local)
    if args.workload == "pq":
        return run_pq(args, ws, rank, local)
    if args.workload == "energy":
        return run_energy(args, ws, rank, local)
    if args.workload == "deltas":
        return run_deltas(args, ws, rank, local)
    if args.workload == "exhaustive":
        return run_exhaustive(args, ws, rank, local)
    if args.workload == "pq_indep":
        return run_pq_indep(args, ws, rank, local)
    if args.workload == "legendre":
        return run_legendre(args, ws, rank, local)
    if args.workload == "operators":
        return run_operators(args, ws, rank, local)
    if args.workload == "network":
        return run_network(args, ws, rank, local)
    if args.workload == "learned":
        return run_learned(args, ws, rank, local)
    if args.workload == "peaks":
        return run_peaks(args, ws, rank, local)
    if args.workload == "workflow":
        return run_workflow(args, ws, rank, local)

    import torch

    import paper_2409_07222_gb300 as lg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    lg.load()

    L, p, R = W1["L"], W1["p"], W1["R"]
    n_walks, budget = args.walks, args.flips
    rates = issue_peaks(local)["lanes_per_clk_per_sm"] if rank == 0 else None  # before any timing
    pre_h = inp.distinct_prefixes(W1["n_prefix"], p, seed=W1["prefix_seed"])
    pre = torch.from_numpy(pre_h.view(np.int64)).to(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    thr = torch.empty(1, dtype=torch.int32, device=dev)

    def step():
        thr_t = lg.labs_sample_threshold(L, True, p, pre, W1["seed"], W1["n_thresh_samples"], W1["thresh_rank"])
        thr.copy_(thr_t)  # torch copy outside the library: stays out of the walk-kernel window below
        cfg = lg.make_walk_cfg(L, skew=True, p=p, n_walks=n_walks, flip_budget=budget, T_i=W1["T_i"],
                               seed=W1["seed"], R=R, bloom_log2=W1["bloom_log2"], bloom_k=W1["bloom_k"],
                               walk_begin=shard(rank, n_walks)[0], E_thr_dev=thr)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out, _, st = lg.labs_skew_search(cfg, pre, with_walk_stats=False)
        e1.record()
        return e0, e1, out, st

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    clocks = ClockSampler(local)
    step_ms, walk_ms = [], []
    flips_seen = 0
    launches_per_step = 4 + 2  # sample, select, histogram, select; walk init, walk
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        e0, e1, out, st = step()
        s1.record()
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        walk_ms.append(e0.elapsed_time(e1))
        flips_seen += int(lg.stats_numpy(st)["flips"])
    barrier()
    clk = clocks.stop()

    total_ms, flips_seen = reduce_over_ranks(sum(step_ms), flips_seen, dev)
    expected = args.steps * n_walks * budget * ws
    if flips_seen != expected:
        raise RuntimeError("walks made %d flips, expected %d" % (flips_seen, expected))
    value = flips_seen / (total_ms * 1e-3)

    # end to end through the public API with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e_ms = []
        cfg = lg.make_walk_cfg(L, skew=True, p=p, n_walks=n_walks, flip_budget=budget, T_i=W1["T_i"],
                               seed=W1["seed"], R=R, bloom_log2=W1["bloom_log2"], bloom_k=W1["bloom_k"],
                               E_thr=lg.LABS_AUTO_THRESHOLD, n_thresh_samples=W1["n_thresh_samples"],
                               thresh_rank=W1["thresh_rank"], walk_begin=shard(rank, n_walks)[0])
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out_h, st_h = lg.labs_skew_search_host(cfg, pre_h, device=local)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        tot, _ = reduce_over_ranks(sum(e2e_ms), 0, dev)
        e2e = {"value": args.steps * n_walks * budget * ws / (tot * 1e-3), "unit": METRIC,
               "h2d_bytes_per_step": int(pre_h.nbytes),
               "d2h_bytes_per_step": int(n_walks * R * 96 + 48)}

    # the only exchange of sharded step 1: every rank's sieved candidates reduced to the 4,096 step-2 seeds
    # (host merge after the timed region; N = 1 does the same reduction locally)
    from paper_2409_07222_gb300.merge import merge_across_ranks

    t0 = time.perf_counter()
    cand_h = lg.candidates_numpy(out, n_walks, R)
    seeds = merge_across_ranks(cand_h, inp.STEP2["n_seeds"])
    merge_ms = (time.perf_counter() - t0) * 1e3

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    flips_per_launch = n_walks * budget
    terms = flips_per_launch * terms_per_flip(L, p)
    walk_s = statistics.mean(walk_ms) * 1e-3
    achieved = terms / walk_s / 1e9
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "p": p, "walks_per_gpu": n_walks, "flips_per_walk": budget,
                   "T_i": W1["T_i"], "prefixes": W1["n_prefix"], "thresh_samples": W1["n_thresh_samples"],
                   "R": R, "bloom_bits": 1 << W1["bloom_log2"], "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "walks sharded by rank" if ws > 1 else "single GPU"},
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "candidate_merge": {"seeds": int(len(seeds)), "best_E": int(seeds["E"][0]) if len(seeds) else None,
                            "ms": merge_ms, "ranks": ws,
                            "what": "K = 4,096 smallest distinct (E, fp) over all ranks' candidates, host merge "
                                    "after the timed region"},
        "clocks": clk,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                     "traffic": traffic_per_launch(n_walks),
                     "kernel": "walk_kernel", "walk_kernel_ms": walk_s * 1e3,
                     "work": "%d neighbour-lag terms per flip (202 free x 225 even lags), one int32 multiply-add "
                             "each; peak = 152 SMs x 128 lanes x 2070 MHz (issue slots)" % terms_per_flip(L, p),
                     "measured_lanes_per_clk_per_sm": rates,
                     "dp4a_pipe": {"peak": SMS * rates["DP4A"] * 4 * SM_MAX_MHZ * 1e6 / 1e9,
                                   "frac": achieved / (SMS * rates["DP4A"] * 4 * SM_MAX_MHZ * 1e6 / 1e9),
                                   "unit": "Gop/s",
                                   "basis": "measured DP4A lane rate x 4 multiply-adds per DP4A x 152 SMs x "
                                            "2070 MHz: the ceiling of a scan made of DP4A alone"}},
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_walks, args.cpu_flips)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
