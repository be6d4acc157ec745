"""Benchmark: Mandelbrot dwell map n = 16384, dwell 2048, window
[-1.5, 0.5] x [-1, 1] (FP32, uint32 map), rendered by ASK on GB300.

One step = one ASK render of the whole map (init + one level kernel per
subdivision depth + leaf kernel) into a preallocated 1.07 GB device map.
Before timing, an untimed autotune picks (g, r, B) over the 75-point sweep
g in {2..32}, r in {2, 4, 8}, B in {16..256} and then the CUDA block shape.

Printed (rank 0, one JSON line): Gpixels/s of ASK (headline), dwell
iterations per second (executed and exhaustive-equivalent), the exhaustive
and CDP2 kernels at the same configuration, the roofline of the dominant
kernel against the FP32 pipe, the CPU reference timed on the host cores, an
end-to-end number through the C ABI with a host output buffer, and SM clocks
sampled during the timed region.

``--impl reference`` times the CPU reference instead (the plain C oracle,
all host cores, a fixed sample of initial regions per step).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpixels/s and dwell-iter/s (ASK vs exhaustive vs CDP2, 1 GB300); p50/p99 latency"
UNIT = "Gpixels/s"
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "dram_traffic_ask_n16384_d2048.json")
KERNEL_SOURCES = ["paper_2206_02255_gb300/csrc/ask_kernels.cu",
                  "paper_2206_02255_gb300/csrc/ask_work.cuh",
                  "paper_2206_02255_gb300/csrc/ask_device.cuh",
                  "paper_2206_02255_gb300/csrc/ask_internal.h"]


def recorded_traffic(kernel_key, workload):
    """DRAM bytes per launch of `kernel_key` from the committed ncu record,
    or None if the record is for another workload or the kernels changed
    since it was taken."""
    import hashlib
    try:
        rec = json.load(open(TRAFFIC_RECORD))
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["kernel_source_sha256"] or not rec["workload"].startswith(workload):
            return None
        return rec["per_launch_dram_bytes"].get(kernel_key)
    except Exception:
        return None


# FP32-pipe instructions per dwell iteration of the stepwise loop: zi*zi,
# fma(zr, zr, zi2) for the test, fma(-zi, zi, cr), fma(zr, zr, t), zr + zr,
# fma(., zi, ci): 1 FMUL + 4 FFMA + 1 FADD.  This is the roofline's unit.
FP32_OPS_PER_ITER = 6
# The kernels run updates in blocks with one test per block (escape is
# absorbing), so an update that counts costs 3 FFMA + 1 FADD: the bound on
# useful issue, reported beside the first.
FP32_OPS_PER_UPDATE = 4
# The headline's subdivision parameters (the 75-point sweep's pick on GB300;
# the sweep still runs and its pick is reported).  The reference arm renders
# the same map with the same parameters.
HEADLINE_G, HEADLINE_R, HEADLINE_B = 16, 4, 16
# The same for the n = 65536, dwell 4096 map (its sweep's pick on GB300).
LARGE_G, LARGE_R, LARGE_B = 32, 2, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ask", choices=["ask", "reference"])
    ap.add_argument("--no-tune", action="store_true", help="skip the autotune sweep")
    ap.add_argument("--tune-headline", action="store_true",
                    help="time the headline at the sweep's pick instead of --g/--r/--B")
    ap.add_argument("--g", type=int, default=HEADLINE_G)
    ap.add_argument("--r", type=int, default=HEADLINE_R)
    ap.add_argument("--B", type=int, default=HEADLINE_B)
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: skip the n=65536, batch and serving sub-results")
    ap.add_argument("--block", default="16x16")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="override n (small cases for profiling; not the headline)")
    ap.add_argument("--max-dwell", type=int, default=None)
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the exhaustive and CDP2 comparison arms")
    ap.add_argument("--workload", default="single",
                    choices=["single", "large", "batch", "serve", "deep"],
                    help="single: one n=16384 map per step (default); large: one n=65536, "
                         "dwell 4096 map (17.2 GB) per step, tuned ASK vs exhaustive; batch: "
                         "256 frames of mixed size and zoom per step; serve: Poisson render "
                         "requests; deep: one n=8192 double-precision map of a 2^-30 wide "
                         "seahorse-valley window per step")
    ap.add_argument("--frames", type=int, default=256, help="batch: frames per step")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas of the workload)
# ---------------------------------------------------------------------------
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def percentile(sorted_vals, q):
    """q-th percentile (nearest rank) of an ascending list."""
    if not sorted_vals:
        return None
    k = max(0, min(len(sorted_vals) - 1, int(round(q / 100.0 * len(sorted_vals) + 0.5)) - 1))
    return sorted_vals[k]


def finite(x):
    """x, or None for NaN (a comparison arm that was not run)."""
    return None if x != x else x


def whole_job_rate(world, units, seconds, device):
    """Units processed by all ranks / the slowest rank's time: the whole-job
    throughput of a replicated (weak-scaling) run."""
    return sum_over_ranks(world, float(units), device) / max_over_ranks(world, seconds, device)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU reference (the oracle as it stands), all host cores
# ---------------------------------------------------------------------------
def cpu_reference_sample(C, g, r, B, seconds, seed=2206, threads=None):
    """Render seeded initial regions with the CPU reference on every host
    core (or on ``threads`` of them) until about ``seconds`` of wall time;
    returns (pixels, s, cores, regions)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    from paper_2206_02255_gb300 import inputs
    orc = oracle.default()
    cores = threads or oracle.default_threads()
    order = inputs.sample_initial_regions(g, g * g, seed)
    done_px = 0
    used = 0
    t0 = time.perf_counter()

    def one(cell):
        res = orc.render_ms_region(C["window"], C["n"], C["max_dwell"], g, r, B, cell[0], cell[1])
        return 0 if res is None else res[0][2] * res[0][3]

    with ThreadPoolExecutor(cores) as ex:
        k = 0
        while k < len(order) and time.perf_counter() - t0 < seconds:
            batch = order[k:k + cores]
            k += len(batch)
            for px in ex.map(one, batch):
                done_px += px
            used += len(batch)
    return done_px, time.perf_counter() - t0, cores, used


def workload_config(C, g, r, B, block):
    """The `config` object of both arms: the workload and the subdivision
    parameters that fix its map (the block shape does not change the map)."""
    px = float(C["n"]) * C["n"]
    return {"workload": C["name"], "n": C["n"], "max_dwell": C["max_dwell"],
            "window": list(C["window"]), "g": g, "r": r, "B": B, "block": list(block),
            "l2": "output map %.2f GB > 129 MB L2, rewritten every step" % (px * 4 / 1e9)}


def measure_large(ctx, dev, local, world, steps=3, warmup=2):
    """The n = 65536, dwell 4096 map (17.2 GB) rendered by ASK at its tuned
    (g, r, B): `steps` timed renders with CUDA events, per-kernel times from
    the timing ring, executed iterations from a counting render."""
    import torch

    from paper_2206_02255_gb300 import ask, inputs

    C = inputs.C2
    win, n, M = C["window"], C["n"], C["max_dwell"]
    g, r, B = LARGE_G, LARGE_R, LARGE_B
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((n, n), dtype=torch.int32, device=dev)
    p = ask.make_params(g, r, B)
    _, cst = ctx.render("ask", win, n, M, ask.make_params(g, r, B, flags=ask.FLAG_COUNT), out=out,
                        stats=True)
    for _ in range(warmup):
        ctx.render("ask", win, n, M, p, out=out)
    ctx.timing_read()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    pt = ask.make_params(g, r, B, flags=ask.FLAG_TIMING)
    ev[0].record(stream)
    for k in range(steps):
        ctx.render("ask", win, n, M, pt, out=out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(world, ev[0].elapsed_time(ev[-1]) / steps, dev)
    per = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(steps))
    t = ctx.timing_read()
    R = max(1, t["renders"])
    del out
    torch.cuda.empty_cache()
    px = float(n) * n
    return {"workload": C["name"], "n": n, "max_dwell": M, "window": list(win),
            "g": g, "r": r, "B": B, "steps": steps, "ms_per_step": ms,
            "gpix_s": world * px / (ms / 1e3) / 1e9, "min_ms": per[0], "max_ms": per[-1],
            "dwell_iter_s_executed": cst["iterations"] / (ms / 1e3),
            "kernels_ms": {"leaf": t["ms_leaf"] / R,
                           "levels": [x / R for x in t["ms_per_level"][:cst["levels"]]]},
            "leaf_iterations": cst["leaf_iterations"], "levels": cst["levels"],
            "leaves": cst["leaves"], "gpu_launches_per_step": cst["kernel_launches"],
            "l2": "output map %.1f GB > 129 MB L2" % (4 * px / 1e9), "clocks": clk}


def run_reference(args):
    from paper_2206_02255_gb300 import inputs
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    C = inputs.C1
    g, r, B = args.g, args.r, args.B
    block = tuple(int(v) for v in args.block.split("x"))
    per_step = 4.0
    for _ in range(args.warmup):
        cpu_reference_sample(C, g, r, B, 0.5)
    px_total = 0
    t_total = 0.0
    cores = regions = 0
    for k in range(args.steps):
        px, t, cores, regions = cpu_reference_sample(C, g, r, B, per_step, seed=2206 + k)
        px_total += px
        t_total += t
    value = px_total / t_total / 1e9
    sample = ("%d seeded initial regions (of %dx%d) per step of n=%d, max_dwell=%d, g=%d r=%d B=%d"
              % (regions, g, g, C["n"], C["max_dwell"], g, r, B))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(C, g, r, B, block), "method": "oracle (CPU, all host cores)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2206_02255_gb300 import ask, build, inputs

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    large = args.workload == "large"
    C = dict(inputs.C2 if large else inputs.C1)
    if args.n or args.max_dwell:
        C["n"] = args.n or C["n"]
        C["max_dwell"] = args.max_dwell or C["max_dwell"]
        C["name"] = "mandelbrot_n%d_d%d" % (C["n"], C["max_dwell"])
    win, n, M = C["window"], C["n"], C["max_dwell"]
    ctx = ask.Context(local)
    out = torch.empty((n, n), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    bx, by = (int(v) for v in args.block.split("x"))

    def one(method, g, r, B, block, flags=0):
        return ctx.render(method, win, n, M, ask.make_params(g, r, B, block, flags), out=out)

    def time_renders(method, g, r, B, block, reps, flags=0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        one(method, g, r, B, block, flags)
        e0.record(stream)
        for _ in range(reps):
            one(method, g, r, B, block, flags)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    # ---- untimed autotune: (g, r, B) sweep, then block shape -------------
    # The headline runs at --g/--r/--B (the sweep's usual pick, shared with
    # the reference arm) unless --tune-headline; the sweep's pick is reported.
    tune = {"g": args.g, "r": args.r, "B": args.B, "block": [bx, by]}
    if large and (args.g, args.r, args.B) == (HEADLINE_G, HEADLINE_R, HEADLINE_B):
        tune.update(g=LARGE_G, r=LARGE_R, B=LARGE_B)
    sweep = []
    swept = None
    if not args.no_tune and (not large or args.tune_headline):
        best = None
        for g, r, B in inputs.c1_sweep():
            ms = time_renders("ask", g, r, B, (16, 16), 2)
            sweep.append((g, r, B, ms))
            if best is None or ms < best[3]:
                best = (g, r, B, ms)
        g, r, B = best[:3]
        bbest = None
        for blk in inputs.BLOCK_SHAPES:
            ms = time_renders("ask", g, r, B, blk, 3)
            if bbest is None or ms < bbest[1]:
                bbest = (blk, ms)
        swept = {"g": g, "r": r, "B": B, "block": list(bbest[0]), "ms": bbest[1],
                 "headline_ms_same_reps": time_renders("ask", tune["g"], tune["r"], tune["B"],
                                                       (bx, by), 3)}
        if args.tune_headline:
            tune = {k: swept[k] for k in ("g", "r", "B", "block")}
    g, r, B, blk = tune["g"], tune["r"], tune["B"], tuple(tune["block"])

    # ---- counting run (untimed): algorithmic work per kernel ---------------
    _, cst = ctx.render("ask", win, n, M, ask.make_params(g, r, B, blk, ask.FLAG_COUNT), out=out,
                        stats=True)
    ask_map = out.clone()
    _, est = ctx.render("exhaustive", win, n, M, ask.make_params(g, r, B, blk, ask.FLAG_COUNT),
                        out=out, stats=True)
    mismatch = int((ask_map != out).sum().item())
    del ask_map
    launches_per_step = cst["kernel_launches"]

    # ---- timed region: K ASK renders ---------------------------------------
    for _ in range(args.warmup):
        one("ask", g, r, B, blk)
    ctx.timing_read()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        one("ask", g, r, B, blk, ask.FLAG_TIMING)
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms_step = ev[0].elapsed_time(ev[-1]) / args.steps
    ms_step = max_over_ranks(world, ms_step, dev)
    per_step = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps))
    step_pct = {"p50_ms": percentile(per_step, 50), "p99_ms": percentile(per_step, 99),
                "min_ms": per_step[0], "max_ms": per_step[-1]}
    timing = ctx.timing_read()

    # ---- comparison arms, each tuned on its own (untimed for the headline)
    ms_ex = ms_cdp = ms_cdp_fnf = float("nan")
    ex_block = cdp_cfg = None
    if not args.no_compare:
        reps = max(3, args.steps // 4) if not large else 3
        for blkx in inputs.BLOCK_SHAPES:
            t = time_renders("exhaustive", g, r, B, blkx, 2)
            if ex_block is None or t < ex_block[1]:
                ex_block = (blkx, t)
        ms_ex = time_renders("exhaustive", g, r, B, ex_block[0], reps)
    if not args.no_compare and not large:
        # CDP2 arms: the n = 16384 comparison (the large map compares ASK with
        # the exhaustive kernel only)
        reps = max(3, args.steps // 4)
        fnf = ask.FLAG_CDP2_FIRE_AND_FORGET
        for cg in (8, 16, 32, 64):
            for cr in (2, 4):
                for cB in (16, 32, 64, 128):
                    for cblk in ((16, 16), (64, 8)):
                        t = time_renders("cdp2", cg, cr, cB, cblk, 1, fnf)
                        if cdp_cfg is None or t < cdp_cfg[4]:
                            cdp_cfg = (cg, cr, cB, cblk, t)
        cg, cr, cB, cblk = cdp_cfg[:4]
        ms_cdp_fnf = time_renders("cdp2", cg, cr, cB, cblk, reps, fnf)
        ms_cdp = time_renders("cdp2", cg, cr, cB, cblk, 1)
    # ---- the paper's SBR / MBR mappings (Sec. 4.3), each tuned on its own
    schemes = None
    if not args.no_compare and not large:
        reps = max(3, args.steps // 4)
        schemes = {"ask_default": {"ms": ms_step, "g": g, "r": r, "B": B, "block": list(blk)}}
        space = [(sg, sr, sB, sblk) for sg in (8, 16, 32, 64) for sr in (2, 4)
                 for sB in (16, 32, 64) for sblk in ((16, 16), (32, 8))]
        fnf = ask.FLAG_CDP2_FIRE_AND_FORGET
        for name, method, f in (("ask_sbr", "ask", ask.FLAG_SBR), ("ask_mbr", "ask", ask.FLAG_MBR),
                                ("dp_mbr", "cdp2", ask.FLAG_MBR | fnf)):
            bestc = None
            for sg, sr, sB, sblk in space:
                t = time_renders(method, sg, sr, sB, sblk, 1, f)
                if bestc is None or t < bestc[4]:
                    bestc = (sg, sr, sB, sblk, t)
            sg, sr, sB, sblk = bestc[:4]
            schemes[name] = {"ms": time_renders(method, sg, sr, sB, sblk, reps, f),
                             "g": sg, "r": sr, "B": sB, "block": list(sblk)}
            if method == "cdp2":
                schemes[name]["fire_and_forget"] = True
                schemes[name]["ms_tail_launch"] = time_renders(method, sg, sr, sB, sblk, 1,
                                                               ask.FLAG_MBR)
        if cdp_cfg is not None:
            schemes["dp_sbr"] = {"ms": ms_cdp_fnf, "ms_tail_launch": ms_cdp, "fire_and_forget": True,
                                 "g": cdp_cfg[0], "r": cdp_cfg[1], "B": cdp_cfg[2],
                                 "block": list(cdp_cfg[3])}

    # ---- cost model (Sec. 4) beside the tuner and the paper's configurations
    model = None
    if not args.no_compare and not large:
        from paper_2206_02255_gb300 import autotune
        mc = autotune.model_choice(ctx, win, n, M, g, r, B)
        model = {"P": mc["P"], "lambda_fit": mc["lam"], "kappa_ms": mc["kappa_ms"],
                 "q": mc["q"], "c": mc["c"], "model_speedup_vs_ex": mc["model_speedup"],
                 "model_optimum": [mc["g"], mc["r"], mc["B"]], "tuned": [g, r, B],
                 "tuned_ms": ms_step}
        try:
            model["model_optimum_ms"] = time_renders("ask", mc["g"], mc["r"], mc["B"], blk, 3)
        except ask.AskError as exc:
            model["model_optimum_ms"] = None
            model["model_optimum_error"] = str(exc)
        model["paper_configs_ms"] = {"%d,%d,%d" % pc: time_renders("ask", *pc, blk, 3)
                                     for pc in ((32, 4, 16), (64, 4, 16))}

    pixels = float(n) * n
    value = world * pixels / (ms_step / 1e3) / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # ---- roofline of the dominant kernel (FP32 pipe) ----------------------
    R = timing["renders"]
    kern = {"leaf": timing["ms_leaf"] / R}
    for i, t in enumerate(timing["ms_per_level"]):
        kern["level%d" % i] = t / R
    dom = max(kern, key=kern.get)
    it_dom = cst["leaf_iterations"] if dom == "leaf" else cst["iterations_per_level"][int(dom[5:])]
    achieved = it_dom / (kern[dom] / 1e3) / 1e9           # G dwell-iterations / s
    f_mhz = 2070.0
    try:
        f_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        pass
    # The roofline's unit is the stepwise iteration's 6 FP32-pipe instructions
    # (1 FMUL + 4 FFMA + 1 FADD); "frac_useful_4op" takes the 4 instructions
    # an update costs when the test is amortised over a block (3 FFMA +
    # 1 FADD), the bound on useful issue.  achieved = the dominant kernel's
    # dwell iterations (a counting render) / its mean CUDA-event time.
    peak = sms * 128 * f_mhz * 1e6 / FP32_OPS_PER_ITER / 1e9
    peak4 = sms * 128 * f_mhz * 1e6 / FP32_OPS_PER_UPDATE / 1e9
    key = "leaf_refill_kernel" if dom == "leaf" else "level_kernel_" + dom
    traffic = recorded_traffic(key, C["name"]) if (g, r, B) == (16, 4, 16) else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "Gdwell-iter/s", "frac": achieved / peak, "traffic": traffic,
                "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (sm_max_mhz) / %d FP32-pipe "
                              "instructions per stepwise iteration" % (sms, f_mhz, FP32_OPS_PER_ITER),
                "frac_useful_4op": achieved / peak4,
                "peak_useful_4op": peak4,
                "peak_useful_4op_basis": "%d SMs x 128 FP32 lanes x %.0f MHz / %d FP32-pipe "
                                         "instructions per blocked update (3 FFMA + 1 FADD)"
                                         % (sms, f_mhz, FP32_OPS_PER_UPDATE),
                "achieved_basis": "%d dwell iterations of the %s kernel (counting render) / "
                                  "%.4f ms mean CUDA-event time over %d timed steps"
                                  % (it_dom, dom, kern[dom], R)}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (
            sms * 128 * clk["sm_mhz"] * 1e6 / FP32_OPS_PER_ITER / 1e9)

    # ---- the deferred-fill kernel against HBM write bandwidth --------------
    # algorithmic bytes: 4 per pixel of the regions it fills (large uniform
    # regions; small ones are filled inside the level kernels).  By default
    # the leaf kernel's fill warps write these bands; ASK_FLAG_SERIAL_FILL
    # runs the fill kernel alone over every SM, so its time can be read.
    roofline_fill = None
    for _ in range(5):
        one("ask", g, r, B, blk, ask.FLAG_TIMING | ask.FLAG_SERIAL_FILL)
    tser = ctx.timing_read()
    ms_fill = tser["ms_fill"] / tser["renders"]
    if cst.get("deferred_fill_pixels") and ms_fill > 0:
        hbm = 6793.4
        try:
            hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        except Exception:
            pass
        fb = 4.0 * cst["deferred_fill_pixels"]
        roofline_fill = {"bound": "hbm", "kernel": "fill", "achieved": fb / (ms_fill / 1e3) / 1e9,
                         "peak": hbm, "unit": "GB/s", "frac": fb / (ms_fill / 1e3) / 1e9 / hbm,
                         "bytes_per_launch": fb, "ms": ms_fill,
                         "render_ms_with_serial_fill": tser["ms_total"] / tser["renders"],
                         "traffic": recorded_traffic("fill_kernel", C["name"])
                         if (g, r, B) == (16, 4, 16) else None,
                         "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}

    # ---- end to end through the C ABI with a host buffer -------------------
    # ask_render_host takes the window and parameters by value and writes
    # the map into a pinned host buffer: the call has no input array, so
    # nothing is copied host -> device.  Between calls a plain device ->
    # host copy of the same 1 GiB (no render) probes the host link, so a
    # slow call can be told apart from a slow link.
    e2e = None
    if not args.no_e2e:
        host = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
        for _ in range(3):  # warm-up calls (the host buffer's pages, the band events)
            ctx.render_host("ask", win, n, M, ask.make_params(g, r, B, blk), out=host)
        k_e2e = max(3, args.steps // 2)

        def link_probe():
            torch.cuda.synchronize(dev)
            tc = time.perf_counter()
            host.copy_(out, non_blocking=True)
            torch.cuda.synchronize(dev)
            return 1e3 * (time.perf_counter() - tc)

        barrier(world)
        calls = []
        t_calls = 0.0
        for _ in range(k_e2e):
            tc = time.perf_counter()
            ctx.render_host("ask", win, n, M, ask.make_params(g, r, B, blk), out=host)
            dt = time.perf_counter() - tc
            t_calls += dt
            calls.append(1e3 * dt)
        t_e2e = max_over_ranks(world, t_calls / k_e2e, dev)
        probes = [link_probe() for _ in range(k_e2e)]
        # the same call with the map rendered in device memory and copied after
        staged = ask.make_params(g, r, B, blk, ask.FLAG_STAGED_COPY)
        ctx.render_host("ask", win, n, M, staged, out=host)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            ctx.render_host("ask", win, n, M, staged, out=host)
        t_staged = max_over_ranks(world, (time.perf_counter() - t0) / k_e2e, dev)
        sc, sp = sorted(calls), sorted(probes)
        e2e = {"value": world * pixels / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(pixels * 4), "ms_per_step": 1e3 * t_e2e,
               "inputs": "none: window, n, max_dwell and (g, r, B) are passed by value",
               "path": "banded: each band of initial-region rows is copied while the next renders",
               "ms_per_call": calls, "p50_ms": percentile(sc, 50), "p99_ms": percentile(sc, 99),
               "value_at_p50": world * pixels / (percentile(sc, 50) / 1e3) / 1e9,
               "link_probe_ms": probes,
               "link_probe_gbs_p50": 4 * pixels / (percentile(sp, 50) / 1e3) / 1e9,
               "staged_copy_ms_per_step": 1e3 * t_staged}
        del host

    # ---- CPU reference on a bounded sample (rank 0, N = 1) -----------------
    cpu = None
    if world == 1 and not args.no_cpu:
        px, t, cores, regions = cpu_reference_sample(C, g, r, B, 12.0)
        px1, t1, _, regions1 = cpu_reference_sample(C, g, r, B, 4.0, threads=1)
        cpu = {"value": px / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d seeded initial regions of %dx%d (%d pixels) at n=%d, max_dwell=%d, "
                         "g=%d r=%d B=%d" % (regions, g, g, px, n, M, g, r, B),
               "single_thread": {"value": px1 / t1 / 1e9, "cores": 1,
                                 "sample": "%d seeded initial regions (%d pixels)" % (regions1, px1)}}

    # ---- the other configurations as compact sub-results of the same run:
    #      n = 65536 map, 256-frame batch, served requests
    subs = {}
    if args.workload == "single" and not args.headline_only and args.n is None \
            and args.max_dwell is None:
        del out
        torch.cuda.empty_cache()
        subs["large"] = measure_large(ctx, dev, local, world)
        subs["batch"] = measure_batch(ctx, dev, local, world, rank, 256, steps=1, warmup=1,
                                      probes=4, full=False)
        subs["serve"] = measure_serve(ctx, dev, local, world, rank, sat_passes=3)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(C, g, r, B, blk),
            "method": "ask", "parallelism": "replicas" if world > 1 else "single",
            "tune": swept,
            "dwell_iter_s": {"executed": cst["iterations"] / (ms_step / 1e3),
                             "exhaustive_equivalent": est["iterations"] / (ms_step / 1e3)},
            "step_ms": step_pct,
            "exhaustive": {"ms": finite(ms_ex), "gpix_s": finite(pixels / (ms_ex / 1e3) / 1e9),
                           "dwell_iter_s": finite(est["iterations"] / (ms_ex / 1e3)),
                           "block": list(ex_block[0]) if ex_block else None},
            "cdp2": ({"ms_tail_launch": ms_cdp, "ms_fire_and_forget": ms_cdp_fnf,
                      "gpix_s": pixels / (min(ms_cdp, ms_cdp_fnf) / 1e3) / 1e9,
                      "tuned": {"g": cdp_cfg[0], "r": cdp_cfg[1], "B": cdp_cfg[2],
                                "block": list(cdp_cfg[3])}} if cdp_cfg else None),
            "speedup_vs_exhaustive": finite(ms_ex / ms_step),
            "speedup_vs_cdp2": finite(min(ms_cdp, ms_cdp_fnf) / ms_step),
            "mismatch_vs_exhaustive_pixels": mismatch,
            "schemes": schemes, "cost_model": model,
            "kernels_ms": kern, "levels": cst["levels"],
            "regions_per_level": cst["regions_per_level"], "leaves": cst["leaves"],
            "fills_per_level": cst["fills_per_level"],
            "iterations_per_level": cst["iterations_per_level"],
            "leaf_iterations": cst["leaf_iterations"],
            "roofline": roofline, "roofline_fill": roofline_fill,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "tune_sweep_top5": sorted(sweep, key=lambda t: t[3])[:5],
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Batched workload: 256 frames, sides 512..8192, zoomed on boundary points
# ---------------------------------------------------------------------------
def measure_batch(ctx, dev, local, world, rank, nframes, steps, warmup, probes=6, full=True):
    """The batched workload: per-frame ASK against one batch (and its CUDA
    graph).  Returns the measured quantities as a dict; `full` adds the
    model-vs-measured comparison of the tuner's probes and the end-to-end
    pass."""
    import torch

    from paper_2206_02255_gb300 import ask, autotune, inputs

    stream = torch.cuda.current_stream(dev)
    frames = inputs.batch_frames(count=nframes, seed=0 + rank)
    sizes = [f["n"] * f["n"] for f in frames]
    pad = [(z + 3) // 4 * 4 for z in sizes]               # keep every map 16-byte aligned
    total_px = float(sum(sizes))
    big = torch.empty(sum(pad), dtype=torch.int32, device=dev)
    off = 0
    for f, z, zp in zip(frames, sizes, pad):
        f["out"] = big[off:off + z].view(f["n"], f["n"])
        off += zp

    tuner = autotune.BatchTuner(ctx, probes=probes).fit(frames)
    for f in frames:
        f["g"], f["r"], f["B"] = tuner.choose(f)
    probe_models = []
    if full:
        for pf, cfg, _ in tuner.probes:
            mc = autotune.model_choice(ctx, pf["window"], pf["n"], pf["max_dwell"], cfg["g"],
                                       cfg["r"], cfg["B"])
            try:
                scratch = torch.empty((pf["n"], pf["n"]), dtype=torch.int32, device=dev)
                model_ms = autotune.time_config(ctx, pf["window"], pf["n"], pf["max_dwell"], mc["g"],
                                                mc["r"], mc["B"], scratch)
                del scratch
            except ask.AskError:
                model_ms = None
            probe_models.append(dict(n=pf["n"], max_dwell=pf["max_dwell"],
                                     measured=(cfg["g"], cfg["r"], cfg["B"]),
                                     measured_ms=round(cfg["ms"], 3),
                                     model=(mc["g"], mc["r"], mc["B"]),
                                     model_ms=None if model_ms is None else round(model_ms, 3),
                                     P=round(mc["P"], 3), lambda_fit=round(mc["lam"], 2)))

    def per_frame():
        for f in frames:
            ctx.render("ask", f["window"], f["n"], f["max_dwell"],
                       ask.make_params(f["g"], f["r"], f["B"]), out=f["out"])

    def batched():
        ctx.render_batch(frames)

    def persistent():
        ctx.render_batch(frames, flags=ask.FLAG_PERSISTENT)

    graph = ctx.graph_batch(frames)
    pgraph = ctx.graph_batch(frames, flags=ask.FLAG_PERSISTENT)

    def timed(fn, k):
        for _ in range(max(1, warmup)):
            fn()
        barrier(world)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(world, e0.elapsed_time(e1) / k, dev)

    clocks = ClockSampler(local)
    ms_frame = timed(per_frame, steps)
    clocks.start()
    time.sleep(0.3)
    ms_batch = timed(batched, steps)
    clk = clocks.stop()
    ms_graph = timed(graph.launch, steps)
    clocks_p = ClockSampler(local)
    clocks_p.start()
    time.sleep(0.3)
    ms_pers = timed(persistent, steps)
    clk_p = clocks_p.stop()
    ms_pgraph = timed(pgraph.launch, steps)
    st = ctx.render_batch(frames, flags=ask.FLAG_COUNT, stats=True)
    launches = st["kernel_launches"]
    stp = ctx.render_batch(frames, flags=ask.FLAG_COUNT | ask.FLAG_PERSISTENT, stats=True)
    graph.close()
    pgraph.close()
    gp = lambda ms: world * total_px / (ms / 1e3) / 1e9
    res = {"frames": len(frames), "pixels": int(total_px),
           "per_frame_ask": {"ms": ms_frame, "gpix_s": gp(ms_frame)},
           "batched": {"ms": ms_batch, "gpix_s": gp(ms_batch), "launches": launches,
                       "form": "launch chain: init, one level kernel per depth, leaf kernel"},
           "graph": {"ms": ms_graph, "gpix_s": gp(ms_graph)},
           "persistent": {"ms": ms_pers, "gpix_s": gp(ms_pers), "launches": stp["kernel_launches"],
                          "form": "init kernel + one persistent kernel over a device work queue",
                          "clocks": clk_p},
           "persistent_graph": {"ms": ms_pgraph, "gpix_s": gp(ms_pgraph)},
           "speedup_batch_vs_per_frame": ms_frame / ms_batch,
           "speedup_persistent_vs_chain": ms_batch / ms_pers,
           "speedup_persistent_vs_per_frame": ms_frame / ms_pers,
           "dwell_iter_s": {"executed": st["iterations"] / (ms_batch / 1e3)},
           "tuned_probes": tuner.summary(), "clocks": clk, "steps": steps}
    if full:
        res["model_vs_measured"] = probe_models
        # end to end: the batched render plus every map copied to pinned host memory
        host = torch.empty(sum(pad), dtype=torch.int32, pin_memory=True)
        steps_e2e = max(2, steps // 2)
        batched()
        host.copy_(big, non_blocking=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            batched()
            host.copy_(big, non_blocking=True)
            torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(world, (time.perf_counter() - t0) / steps_e2e, dev)
        res["e2e"] = {"value": gp(t_e2e * 1e3), "unit": UNIT, "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": int(4 * total_px), "ms_per_step": 1e3 * t_e2e}
        del host
    for f in frames:
        f["out"] = None
    del big
    torch.cuda.empty_cache()
    return res


def run_batch(args):
    import torch

    from paper_2206_02255_gb300 import ask, build

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    ctx = ask.Context(local)
    res = measure_batch(ctx, dev, local, world, rank, args.frames, args.steps, args.warmup)
    if rank == 0:
        b = res["batched"]
        line = {
            "metric": METRIC, "value": b["gpix_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch_%d_frames_side512-8192_zoom1-1e4_dwell256-8192"
                                   % res["frames"],
                       "frames": res["frames"], "pixels": res["pixels"],
                       "l2": "%.1f GB of maps per step > 129 MB L2" % (4 * res["pixels"] / 1e9)},
            "method": "ask_batch", "parallelism": "replicas" if world > 1 else "single",
            "e2e": res.pop("e2e"), "gpu_launches": b["launches"] * args.steps,
            "clocks": res.pop("clocks"),
        }
        line.update(res)
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# Served workload: Poisson render requests, continuous batching
# ---------------------------------------------------------------------------
def measure_serve(ctx, dev, local, world, rank, sat_passes=3, count=2000):
    """The served workload: Poisson requests (lambda = 200/s, seed 7) through
    the continuous-batching server and through per-frame ASK, then the first
    600 requests all waiting at t = 0 (saturation), `sat_passes` passes of
    each, the median pass reported.  Returns a dict."""
    import torch

    from paper_2206_02255_gb300 import autotune, inputs, serve

    reqs = inputs.serving_requests(count=count, seed=7 + rank)
    tuner = autotune.BatchTuner(ctx, probes=4).fit(reqs[::20])
    cfg = {d["id"]: tuner.choose(d) for d in reqs}

    def fresh(ds, at_zero=False):
        out = []
        for d in ds:
            q = serve.Request(d, *cfg[d["id"]])
            if at_zero:
                q.t = 0.0
            out.append(q)
        return out

    # both paths share one pinned-buffer pool; results are released when
    # delivered.  Warm up (allocator caches, pinned buffers, first launches).
    pool, dpool = serve.PinnedPool(), serve.DevicePool(local)
    pool.reserve([d["n"] for d in reqs], per_class=4)
    srv = serve.Server(device=local, slots=2, budget_bytes=40 * 2 ** 30, pool=pool, keep=False,
                       dpool=dpool)
    srv.run(fresh(reqs[:64], at_zero=True))
    serve.serve_per_frame(ctx, fresh(reqs[:64], at_zero=True), pool=pool, keep=False, dpool=dpool)
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    s0, b0 = srv.single_dispatches, srv.batch_dispatches
    served = serve.summarize(srv.run(fresh(reqs)))
    dispatches = {"single_frame": srv.single_dispatches - s0, "batches": srv.batch_dispatches - b0}
    clk = clocks.stop()
    alone = serve.summarize(serve.serve_per_frame(ctx, fresh(reqs), pool=pool, keep=False,
                                                  dpool=dpool))
    # saturation: one untimed pass first fills the buffer pools to the depth
    # full batches need (a server in steady state holds them)
    srv.run(fresh(reqs[:600], at_zero=True))
    sat_s = sorted((serve.summarize(srv.run(fresh(reqs[:600], at_zero=True)))
                    for _ in range(sat_passes)), key=lambda r: r["gpix_s"])
    sat_a = sorted((serve.summarize(serve.serve_per_frame(ctx, fresh(reqs[:600], at_zero=True),
                                                          pool=pool, keep=False, dpool=dpool))
                    for _ in range(sat_passes)), key=lambda r: r["gpix_s"])
    sat_served, sat_alone = sat_s[len(sat_s) // 2], sat_a[len(sat_a) // 2]
    srv.close()
    torch.cuda.empty_cache()
    px = float(sum(d["n"] * d["n"] for d in reqs))
    return {"requests": len(reqs), "pixels": int(px), "rate_per_s": 200,
            "span_s": served["span_s"],
            "gpix_s": whole_job_rate(world, px, served["span_s"], dev) / 1e9,
            "latency_ms": {"p50": served["p50_ms"], "p99": served["p99_ms"], "max": served["max_ms"]},
            "dispatches": dispatches,
            "per_frame_ask": {"p50_ms": alone["p50_ms"], "p99_ms": alone["p99_ms"],
                              "max_ms": alone["max_ms"], "gpix_s": alone["gpix_s"]},
            "saturated_600": {"served_gpix_s": sat_served["gpix_s"],
                              "per_frame_gpix_s": sat_alone["gpix_s"],
                              "served_p50_ms": sat_served["p50_ms"],
                              "served_p99_ms": sat_served["p99_ms"],
                              "per_frame_p50_ms": sat_alone["p50_ms"],
                              "per_frame_p99_ms": sat_alone["p99_ms"],
                              "passes": sat_passes, "reported": "median pass",
                              "served_gpix_s_all": [r["gpix_s"] for r in sat_s],
                              "per_frame_gpix_s_all": [r["gpix_s"] for r in sat_a]},
            "clocks": clk}


def run_serve(args):
    import torch

    from paper_2206_02255_gb300 import ask, build

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    ctx = ask.Context(local)
    res = measure_serve(ctx, dev, local, world, rank)
    if rank == 0:
        line = {
            "metric": METRIC, "value": res["gpix_s"], "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 * res["span_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serve_2000_poisson200_side256-4096_dwell512-4096",
                       "requests": res["requests"], "rate_per_s": 200, "budget_gb": 40, "slots": 2,
                       "pixels": res["pixels"]},
            "method": "ask continuous batching",
            "e2e": {"value": res["gpix_s"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 4 * res["pixels"],
                    "note": "latency includes the D2H copy"},
            "clocks": res.pop("clocks"),
        }
        line.update(res)
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# Deep zoom: one double-precision map per step
# ---------------------------------------------------------------------------
# FP64-pipe operations per update in ask_fp64.cu: 3 DFMA + 1 DADD (the |z|^2
# test is amortised over a block of updates)
FP64_OPS_PER_ITER = 4
# Nominal FP64 rate of the GB300 table (1.25 TFLOP/s with an FMA as 2 flops):
# 625 G FP64-pipe lane operations per second.  No measured FP64 peak exists.
FP64_PEAK_GOPS = 1.25e3 / 2
# FP32 instructions per float-float update (ArithFF::update: two squares of
# 7, three sums of 11, one product of 7, a doubling of 2)
FF_OPS_PER_ITER = 56
# FP32 pipe: 152 SMs x 128 lanes x 2070 MHz (operations per second, in G)
FP32_PEAK_GOPS = 152 * 128 * 2.07


def run_deep(args):
    import torch

    from paper_2206_02255_gb300 import ask, build, inputs

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    ctx = ask.Context(local)
    stream = torch.cuda.current_stream(dev)
    spot = "seahorse_2^-30"
    win, M = inputs.deep_window(spot)
    n = args.n or 8192
    M = args.max_dwell or M
    out = torch.empty((n, n), dtype=torch.int32, device=dev)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        barrier(world)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(world, e0.elapsed_time(e1) / steps, dev)

    # untimed tune: one warp per region at every level, so g runs higher
    # than in single precision
    def tune(flags):
        cands = [(args.g, args.r, args.B)] if args.no_tune else \
            [(g, r, B) for g in (32, 64, 128, 256) for r in (2, 4) for B in (8, 16, 32)]
        best = None
        for g, r, B in cands:
            p = ask.make_params(g, r, B, flags=flags)
            ms = timed(lambda: ctx.render64("ask", win, n, M, p, out=out), 1, 1)
            if best is None or ms < best[0]:
                best = (ms, g, r, B)
        return best[1:]

    g, r, B = tune(0)
    p = ask.make_params(g, r, B)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_ask = timed(lambda: ctx.render64("ask", win, n, M, p, out=out), args.steps,
                   max(3, args.warmup))
    clk = clocks.stop()
    ask_map = out.clone()
    ex_out = torch.empty_like(out)
    ms_ex = timed(lambda: ctx.render64("exhaustive", win, n, M, None, out=ex_out),
                  max(2, args.steps // 4), 1)
    ex_iters = int(ex_out.to(torch.int64).sum().item())      # exhaustive-equivalent work
    mism = int((ask_map != ex_out).sum().item())
    _, cst = ctx.render64("ask", win, n, M, ask.make_params(g, r, B, flags=ask.FLAG_COUNT),
                          out=out, stats=True)
    # per-kernel device times (CUDA events around each launch), mean of 3 renders
    runs = [ctx.render64("ask", win, n, M, p, out=out, stats=True)[1] for _ in range(3)]
    leaf_ms = sum(st["ms_leaf"] for st in runs) / len(runs)
    level_ms = [sum(st["ms_per_level"][i] for st in runs) / len(runs) for i in range(runs[0]["levels"])]

    # the same map in float-float arithmetic on the FP32 pipe
    FF = ask.FLAG_FLOAT_FLOAT
    gf, rf, Bf = tune(FF)
    pff = ask.make_params(gf, rf, Bf, flags=FF)
    ms_ff = timed(lambda: ctx.render64("ask", win, n, M, pff, out=out), args.steps, max(3, args.warmup))
    ff_diff = int((out != ask_map).sum().item())
    ms_ex_ff = timed(lambda: ctx.render64("exhaustive", win, n, M, ask.make_params(1, 2, 1, flags=FF),
                                          out=ex_out), max(2, args.steps // 4), 1)
    _, cff = ctx.render64("ask", win, n, M, ask.make_params(gf, rf, Bf, flags=FF | ask.FLAG_COUNT),
                          out=out, stats=True)
    runs_ff = [ctx.render64("ask", win, n, M, pff, out=out, stats=True)[1] for _ in range(3)]
    leaf_ff_ms = sum(st["ms_leaf"] for st in runs_ff) / len(runs_ff)

    # end to end: render into device memory, map copied to pinned host memory
    host = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
    k_e2e = max(2, args.steps // 2)
    ctx.render64("ask", win, n, M, p, out=out)
    host.copy_(out, non_blocking=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        ctx.render64("ask", win, n, M, p, out=out)
        host.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(world, (time.perf_counter() - t0) / k_e2e, dev)

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        # the same window at n = 1024, rendered again until about 10 s have passed
        n_cpu, g_cpu, reps = 1024, max(1, g * 1024 // n), 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and reps < 200:
            oracle.render_ms(win, n_cpu, M, g_cpu, r, B, fp64=True)
            reps += 1
        dt = time.perf_counter() - t0
        cpu = {"value": reps * n_cpu * n_cpu / dt / 1e9, "unit": UNIT,
               "cores": oracle.default_threads(), "kind": "oracle",
               "sample": "%d double-precision Mariani-Silver maps of the same window at n=%d "
                         "(g=%d r=%d B=%d), %.1f s" % (reps, n_cpu, g_cpu, r, B, dt)}

    if rank == 0:
        gp = lambda ms: world * n * n / (ms / 1e3) / 1e9
        leaf_gops = cst["leaf_iterations"] * FP64_OPS_PER_ITER / (leaf_ms / 1e3) / 1e9
        ex_gops = ex_iters * FP64_OPS_PER_ITER / (ms_ex / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": gp(ms_ask), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_ask,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "mandelbrot_fp64_%s_n%d_d%d" % (spot, n, M), "window": list(win),
                       "zoom": 2.0 / (win[1] - win[0]), "n": n, "max_dwell": M,
                       "g": g, "r": r, "B": B, "method": "ask_render64",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "%.0f MB map > 129 MB L2" % (4 * n * n / 1e6)},
            "exhaustive64": {"ms": ms_ex, "gpix_s": gp(ms_ex),
                             "fp64_gops": ex_gops, "frac_of_nominal_fp64": ex_gops / FP64_PEAK_GOPS},
            "speedup_vs_exhaustive": ms_ex / ms_ask,
            "dwell_iter_s": {"executed": cst["iterations"] / (ms_ask / 1e3),
                             "exhaustive_equivalent": ex_iters / (ms_ask / 1e3)},
            "mismatch_vs_exhaustive_pixels": mism,
            "levels": cst["levels"], "leaves": cst["leaves"],
            "ms_per_level": level_ms, "ms_leaf": leaf_ms,
            "roofline": {"bound": "alu", "kernel": "leaf64_kernel", "achieved": leaf_gops,
                         "peak": FP64_PEAK_GOPS, "unit": "G FP64-pipe ops/s",
                         "frac": leaf_gops / FP64_PEAK_GOPS, "traffic": None,
                         "of": "nominal (no measured FP64 peak on this GPU)",
                         "peak_source": "nominal 1.25 TFLOP/s FP64 (FMA = 2 flops); no measured "
                                        "FP64 peak",
                         "work": "leaf pixels' dwells x %d FP64 ops / mean leaf-kernel time" %
                                 FP64_OPS_PER_ITER},
            "float_float": {
                "flag": "ASK_FLAG_FLOAT_FLOAT", "g": gf, "r": rf, "B": Bf,
                "ms": ms_ff, "gpix_s": gp(ms_ff), "speedup_vs_binary64": ms_ask / ms_ff,
                "exhaustive_ms": ms_ex_ff, "speedup_vs_exhaustive": ms_ex_ff / ms_ff,
                "pixels_differing_from_binary64": ff_diff,
                "ms_leaf": leaf_ff_ms,
                "leaf_roofline": {"bound": "alu", "achieved": cff["leaf_iterations"] * FF_OPS_PER_ITER /
                                  (leaf_ff_ms / 1e3) / 1e9,
                                  "peak": FP32_PEAK_GOPS, "unit": "G FP32-pipe ops/s",
                                  "frac": cff["leaf_iterations"] * FF_OPS_PER_ITER /
                                  (leaf_ff_ms / 1e3) / 1e9 / FP32_PEAK_GOPS,
                                  "work": "leaf pixels' dwells x %d FP32 ops / mean leaf-kernel time"
                                          % FF_OPS_PER_ITER}},
            "cpu_baseline": cpu,
            "e2e": {"value": gp(t_e2e * 1e3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 4 * n * n, "ms_per_step": 1e3 * t_e2e},
            "gpu_launches": (2 + cst["levels"]) * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "deep":
        run_deep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
