"""Benchmark: fused vector-bytecode execution on one B300 (or N replicas).

Default workload: Black-Scholes call+put over 16,777,216 options in float64
(a second run in float32 is reported beside it). One step = one submitted
batch of the whole program (about 65 elementwise bytecodes) through the C
ABI, fused into one kernel and replayed as a CUDA graph, with the inputs
already resident in device memory. ``value`` is the compulsory HBM traffic
of the batch (inputs read once + outputs written once) per second; the plain
path (one launch per bytecode) is timed on the same GPU beside it.
``--impl reference`` times the oracle (the CPU reference interpreter) on a
bounded sample of the same workload instead.

Other workloads: ``--workload jacobi|shallow_water|stencil|knn|montecarlo|serving``.
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

METRIC = "fused bytecode-batch HBM GB/s (% of peak) vs per-bytecode path; p50/p99 latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6400.0


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ reference arm

def cpu_reference(args, rank, world):
    """The oracle, as it stands, on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    from workloads import blackscholes
    dtype = "float64"
    n_sample = args.ref_sample
    prog = blackscholes(n_sample, dtype)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.run(prog)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(prog)
        times.append(time.perf_counter() - t0)
    per_step = statistics.median(times)
    value = prog.compulsory_bytes() / per_step / 1e9
    cores = 1  # NumPy ufuncs run on one thread
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(1 << 24, dtype),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_sample} options per step (of 16,777,216), float64"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(sec: float, dist=None) -> float:
    """The slowest rank's per-step time (every rank takes part)."""
    if not dist:
        return sec
    import torch
    t = torch.tensor([sec], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def aggregate_value(units_per_rank: float, sec_max: float, world: int) -> float:
    """Whole-job throughput of weak scaling: every rank processes its own
    units_per_rank per step, the job's step takes the slowest rank's time."""
    return world * units_per_rank / sec_max


def workload_config(n, dtype):
    return {"workload": f"Black-Scholes call+put, {n} options, {dtype}", "options": n,
            "bytes_per_option": 7 * (8 if dtype == "float64" else 4),
            "l2": "inputs larger than L2 (no flush needed)",
            "path": "fused (one kernel per batch), cached launch replayed with programmatic dependent launch, "
                    "autotuned launch shape"}


# ------------------------------------------------------------------ GPU arm

def time_steps(fn, steps, warmup, torch, dist=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return ev0.elapsed_time(ev1) / 1e3 / steps


def kernel_hash(ex, L):
    import hashlib
    js = json.loads(ex.plan(L, 0, source=True))
    srcs = [i["run"]["source"] for i in js["items"] if "run" in i]
    return hashlib.sha1("".join(srcs).encode()).hexdigest()[:16]


def measured_counters(name, khash):
    """ncu counters recorded for this kernel (profiles/traffic.json), or None
    when the kernel has changed since they were taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)[name]
        return t if t.get("kernel_hash") == khash else None
    except Exception:
        return None


def measure_fp64_peak(V, torch, local, stream):
    """The FP64 pipe's rate, measured on this GPU by the library's throughput
    kernel (8 independent chains per thread, 8 blocks of 256 threads per SM):
    fused multiply-add, add and multiply, each the median of 5 launches of
    about 30 ms after one warm-up launch, with the SM clocks sampled
    meanwhile. ``peak`` is the fastest of the three medians (one FP64
    instruction per lane either way)."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    scratch = torch.empty(2048 * sms, dtype=torch.float64, device=f"cuda:{local}")
    ck = Clocks(local)
    ck.start()
    res = {}
    for op in ("dfma", "dadd", "dmul"):
        V.vbe_measure_fp64_rate(op, 512, scratch.data_ptr(), stream)
        vals = [V.vbe_measure_fp64_rate(op, 8192, scratch.data_ptr(), stream) for _ in range(5)]
        res[op] = statistics.median(vals) / 1e9
    clocks = ck.stop()
    peak = max(res.values())
    mhz = clocks.get("sm_mhz") or 2032.0
    return {"peak": peak, "unit": "G FP64-inst/s", "dfma": res["dfma"], "dadd": res["dadd"], "dmul": res["dmul"],
            "sms": sms, "per_sm_per_clk": peak * 1e9 / (sms * mhz * 1e6), "clocks": clocks,
            "how": "library throughput kernel (vbe_measure_fp64_rate): 8 chains/thread, 8x256 threads/SM, "
                   "median of 5 launches of 8192 rounds, CUDA events"}


FP64_PIPE_OPS = {"ADD", "SUBTRACT", "MULTIPLY", "MAXIMUM", "MINIMUM", "LESS", "LESS_EQUAL", "GREATER",
                 "GREATER_EQUAL", "EQUAL", "NOT_EQUAL"}


def fp64_bytecode_ops(program, lo=0, hi=None):
    """Float64 operations of the bytecodes in ``program.instrs[lo:hi]`` that
    must run on the FP64 pipe: element counts of the float64 add, subtract,
    multiply, min/max and compare bytecodes and of float64 sums, products by
    a constant +-2^k excluded (the library does those exactly on the integer
    pipes, as it does divide, sqrt, exp and log). This is the scheme's own
    ALU work, before any recomputation a kernel form adds."""
    from workloads.program import Const, View
    n = 0
    for ins in program.instrs[lo:hi]:
        views = [x for x in ins.ins if isinstance(x, View)]
        if ins.op == "ADD_REDUCE" and views and program.bases[views[0].base].dtype == "float64":
            n += views[0].size
            continue
        if ins.op not in FP64_PIPE_OPS or not views or program.bases[views[0].base].dtype != "float64":
            continue
        if ins.op == "MULTIPLY" and any(isinstance(x, Const) and x.value != 0 and
                                        float(abs(x.value)) == 2.0 ** int(np.round(np.log2(abs(x.value))))
                                        for x in ins.ins):
            continue
        n += ins.out.size
    return n


def roofline_f64(achieved_gbs, hbm, src, counters, n, sec, fp64, clk_mhz):
    hbm_part = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                "peak_source": src}
    if not counters or "fp64_inst_per_unit" not in counters:
        hbm_part["traffic"] = counters["dram_bytes_per_launch"] if counters else None
        return hbm_part
    peak = fp64["peak"]
    ach = counters["fp64_inst_per_unit"] * n / sec / 1e9
    out = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP64-inst/s", "frac": ach / peak,
           "peak_source": "measured in this run (vbe_measure_fp64_rate; see fp64_peak)",
           "work": f"{counters['fp64_inst_per_unit']:.1f} FP64 instructions per option (ncu, this kernel)",
           "traffic": counters["dram_bytes_per_launch"], "hbm": hbm_part}
    if "inst_per_unit" in counters:
        # all instructions against the issue rate (4 schedulers x 32 lanes per SM)
        ipeak = fp64["sms"] * 128 * clk_mhz * 1e6 / 1e12
        iach = counters["inst_per_unit"] * n / sec / 1e12
        out["issue"] = {"achieved": iach, "peak": ipeak, "unit": "T thread-inst/s", "frac": iach / ipeak,
                        "work": f"{counters['inst_per_unit']:.0f} instructions per option",
                        "peak_source": f"derived: {fp64['sms']} SMs x 128 lanes/clk x {clk_mhz:.0f} MHz"}
    return out


def gpu_blackscholes(args, rank, world, local):
    import torch
    from paper_1210_7774_b300 import build
    build.build()
    from paper_1210_7774_b300 import vbe as V
    from paper_1210_7774_b300.runner import Executor
    from workloads import blackscholes, bs_inputs

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    # a dedicated stream: the library launches on it and the CUDA events
    # that time the steps are recorded on it
    ts = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(ts)
    stream = ts.cuda_stream
    assert stream != 0
    n = args.options
    cache = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
    flags_fused = V.VBE_FUSE | V.VBE_GRAPHS | V.VBE_AUTOTUNE | V.VBE_PACK
    res = {"_fp64": measure_fp64_peak(V, torch, local, stream), "_ctx": (V, torch, local, stream)}
    for dtype in args.dtypes.split(","):
        inp = bs_inputs(n, dtype, seed=1210_7774 + 2 + rank)
        prog = blackscholes(n, dtype, inputs=inp)
        cbytes = prog.compulsory_bytes()
        out = {}
        for name, flags in (("fused", flags_fused), ("plain", 0)):
            if name not in args.paths.split(","):
                continue
            ex = Executor(flags, device=local, stream=stream, cache_dir=cache)
            L = ex.load(prog)
            st0 = ex.stats()
            steps = args.steps if name == "fused" else max(3, args.steps // 4)
            sec = time_steps(lambda: ex.submit(L, 0), steps, max(3, args.warmup), torch, dist)
            st1 = ex.stats()
            out[name] = {"sec": sec, "GB/s": cbytes / sec / 1e9,
                         "launches_per_step": (st1["kernel_launches"] - st0["kernel_launches"]) / (steps + max(3, args.warmup))}
            if name == "fused":
                out["kernel_hash"] = kernel_hash(ex, L)
                # end to end: pinned host inputs -> device, batch, results -> pinned host
                host_in = {bid: torch.from_numpy(b.init).pin_memory() for bid, b in prog.bases.items()
                           if b.init is not None}
                host_out = {bid: torch.empty(prog.bases[bid].nelem, dtype=getattr(torch, dtype)).pin_memory()
                            for bid in prog.outputs}
                h2d = sum(t.numel() * t.element_size() for t in host_in.values())
                d2h = sum(t.numel() * t.element_size() for t in host_out.values())

                def e2e_step():
                    for bid, t in host_in.items():
                        V.vbe_base_upload(ex.ctx, L.base[bid], t.data_ptr(), t.numel() * t.element_size())
                    ex.submit(L, 0)
                    for bid, t in host_out.items():
                        V.vbe_sync(ex.ctx, L.base[bid], t.data_ptr(), t.numel() * t.element_size())
                e2e_steps = max(2, args.steps // 4)
                for _ in range(2):
                    e2e_step()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(e2e_steps):
                    e2e_step()
                torch.cuda.synchronize()
                e2e_sec = (time.perf_counter() - t0) / e2e_steps
                out["e2e_serial"] = {"value": cbytes / e2e_sec / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                                     "d2h_bytes_per_step": d2h,
                                     "how": "one context: upload the inputs, submit, sync the outputs, in turn"}
                ex.close()
                if dtype == "float64":
                    out["e2e"] = e2e_pipelined(V, Executor, prog, dtype, flags_fused, local, cache, args, torch,
                                               workers=args.e2e_workers)
            if ex.ctx:
                ex.close()
        out["cbytes"] = cbytes
        res[dtype] = out
    return res, dist


def e2e_pipelined(V, Executor, prog, dtype, flags, local, cache, args, torch, workers=4):
    """End to end through the C ABI with the copies overlapped: the options
    are split over ``workers`` contexts (each with its own stream), each
    driven by a host thread that uploads its share of the inputs from pinned
    memory (vbe_base_upload), submits the batch and reads its results back
    (vbe_sync). The calls block their own thread only, so while one share's
    inputs go to the device another's results come back and a third computes:
    both directions of the host link are busy at once. The threads start
    together and run their steps without waiting for one another (so they
    drift apart and their copies interleave); a step is every share's
    upload, batch and read-back, and its time is the wall clock until the
    last thread has finished all its steps, divided by the steps."""
    import threading

    from workloads import blackscholes
    n = prog.meta["n"]
    cuts = np.linspace(0, n, workers + 1).astype(np.int64)
    ins = {k: prog.bases[i].init for k, i in prog.meta["input_ids"].items()}
    shares = []
    for w in range(workers):
        lo, hi = int(cuts[w]), int(cuts[w + 1])
        p = blackscholes(hi - lo, dtype, inputs={k: v[lo:hi] for k, v in ins.items()})
        ex = Executor(flags, device=local, cache_dir=cache)
        L = ex.load(p)
        host_in = {bid: torch.from_numpy(b.init).pin_memory() for bid, b in p.bases.items() if b.init is not None}
        host_out = {bid: torch.empty(p.bases[bid].nelem, dtype=getattr(torch, dtype)).pin_memory()
                    for bid in p.outputs}
        shares.append((ex, L, host_in, host_out))
    h2d = sum(t.numel() * t.element_size() for sh in shares for t in sh[2].values())
    d2h = sum(t.numel() * t.element_size() for sh in shares for t in sh[3].values())
    cbytes = prog.compulsory_bytes()

    def one(sh):
        ex, L, host_in, host_out = sh
        for bid, t in host_in.items():
            V.vbe_base_upload(ex.ctx, L.base[bid], t.data_ptr(), t.numel() * t.element_size())
        ex.submit(L, 0)
        for bid, t in host_out.items():
            V.vbe_sync(ex.ctx, L.base[bid], t.data_ptr(), t.numel() * t.element_size())

    def run_steps(k):
        barrier = threading.Barrier(workers)

        def worker(sh):
            torch.cuda.set_device(local)
            barrier.wait()  # the shares start together, then run their steps freely
            for _ in range(k):
                one(sh)
        th = [threading.Thread(target=worker, args=(sh,)) for sh in shares]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        return time.perf_counter() - t0

    run_steps(2)  # warm-up (tuning, first launches)
    steps = max(5, args.steps // 2)
    sec = run_steps(steps) / steps
    for sh in shares:
        sh[0].close()
    link = link_rates(torch, h2d, d2h)
    value = cbytes / sec / 1e9
    return {"value": value, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "workers": workers, "steps": steps, "link": link,
            "frac_of_link": value / link["same_bytes_gbs"],
            "how": f"{workers} contexts, one host thread each, over equal shares of the options: pinned inputs "
                   "uploaded, batch submitted, results synced back, each thread in turn; the threads overlap"}


def link_rates(torch, h2d, d2h, reps=5):
    """The host link's rates for the end-to-end step's copies, measured with
    plain copies between page-locked host memory and the device: each
    direction alone, both directions at once with equal sizes, and the
    step's own bytes (h2d to the device, d2h back, started together on two
    streams). The last is the bound of any end-to-end step that moves these
    bytes: ``same_bytes_gbs`` = (h2d + d2h) / its time (best of ``reps``)."""
    dev = torch.cuda.current_device()
    hin = torch.empty(h2d, dtype=torch.uint8).pin_memory()
    hout = torch.empty(d2h, dtype=torch.uint8).pin_memory()
    din = torch.empty(h2d, dtype=torch.uint8, device=dev)
    dout = torch.empty(d2h, dtype=torch.uint8, device=dev)
    s_up, s_down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(up, down):
        best = None
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if up is not None:
                with torch.cuda.stream(s_up):
                    up[0].copy_(up[1], non_blocking=True)
            if down is not None:
                with torch.cuda.stream(s_down):
                    down[0].copy_(down[1], non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best
    m = min(h2d, d2h)
    r = {"h2d_gbs": h2d / timed((din, hin), None) / 1e9,
         "d2h_gbs": d2h / timed(None, (hout, dout)) / 1e9,
         "both_equal_gbs": 2 * m / timed((din[:m], hin[:m]), (hout[:m], dout[:m])) / 1e9,
         "same_bytes_gbs": (h2d + d2h) / timed((din, hin), (hout, dout)) / 1e9,
         "how": "plain copies between page-locked host memory and the device, best of %d: each direction "
                "alone, both at once with equal sizes, and the step's own bytes both ways at once" % reps}
    del hin, hout, din, dout
    return r


# ------------------------------------------------- per-configuration keys

def _oracle_seconds(program, reps=1):
    import oracle
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.run(program)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best


def _oracle_job(args):
    """One oracle run in a worker process (a spawn pool): the program is
    rebuilt there from its generator and arguments."""
    kind, params = args
    sys.path.insert(0, ROOT)
    import oracle
    if kind == "mc":
        from workloads import montecarlo_pi
        p = montecarlo_pi(sizes=np.array(params["sizes"]), keys=params["keys"])
    else:
        from workloads.serving import request_program
        p = request_program(kind, params)
    t0 = time.perf_counter()
    oracle.run(p)
    return time.perf_counter() - t0


def _pool_rate(jobs, units):
    """Wall-clock rate of the oracle over all host cores: ``jobs`` run by a
    spawn process pool with one worker per usable core."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_job, jobs[:cores]))  # workers started and warm
        t0 = time.perf_counter()
        list(pool.map(_oracle_job, jobs))
        wall = time.perf_counter() - t0
    return units / wall, cores, wall


def _mcore_seconds(program, reps=2):
    """Best wall time of the mcore engine (the paper's multi-core blocked
    Vector Engine, restated in C++) on every usable core, after one
    untimed run."""
    import mcore
    prep = mcore.Prepared(program)
    prep.run()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        prep.run()
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best, mcore.cores()


def config_subkeys(args, V, torch, local, stream, hbm, fp64):
    """One sub-key per configuration beside the headline: Jacobi 256^2,
    shallow water 4096^2 float64 (50 steps), Monte-Carlo pi (256 instances)
    and the serving loop, each fused against the per-bytecode path on this
    GPU with the oracle timed beside it (``cpu_baseline``)."""
    from paper_1210_7774_b300.runner import Executor
    from workloads import jacobi, mc_sizes, montecarlo_pi, shallow_water
    cache = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
    F = V.VBE_FUSE | V.VBE_AUTOTUNE | V.VBE_PACK
    G = V.VBE_GRAPHS

    def timed(program, flags, reps, warmup=3):
        with Executor(flags, device=local, stream=stream, cache_dir=cache) as ex:
            L = ex.load(program)
            nb = len(L.batches)
            st0 = ex.stats()

            def step():
                for k in range(nb):
                    ex.submit(L, k)
            sec = time_steps(step, reps, warmup, torch)
            st1 = ex.stats()
        per = reps + warmup
        return sec, {k: (st1[k] - st0[k]) / per for k in ("kernel_launches", "graph_launches", "list_replays",
                                                             "packed_launches", "sweep_group_launches")}

    out = {}
    # --- Jacobi 256^2 float64, 10 iterations (launch-bound: the grid is L2-resident)
    p = jacobi(256, 10)
    cb = 256 * 256 * 8 + 254 * 254 * 8
    jr = {}
    for name, flags in (("fused_graphs", F | G), ("plain_graphs", G), ("plain", 0)):
        sec, st = timed(p, flags, 100, warmup=20)
        jr[name] = {"us_per_iteration": sec / 10 * 1e6, "GB/s": cb * 10 / sec / 1e9,
                    "launches_per_iteration": st["kernel_launches"] / 10}
    # the whole 10-iteration program as one batch (the paper's Bridge hands
    # over everything recorded up to a flush): one graph of ten kernels
    p1 = jacobi(256, 10, one_batch=True)
    sec, st = timed(p1, F | G, 100, warmup=20)
    jr["fused_graphs_one_batch"] = {"us_per_iteration": sec / 10 * 1e6, "GB/s": cb * 10 / sec / 1e9,
                                    "launches_per_iteration": st["kernel_launches"] / 10,
                                    "note": "one submit per 10 iterations"}
    osec = _oracle_seconds(p, 3)
    jr.update(speedup_vs_plain=jr["plain"]["us_per_iteration"] / jr["fused_graphs"]["us_per_iteration"],
              speedup_vs_plain_graphs=jr["plain_graphs"]["us_per_iteration"] / jr["fused_graphs"]["us_per_iteration"],
              note="256x256 float64, 10 iterations of 9 bytecodes; the 0.5 MB grid stays in L2, so launch latency "
                   "bounds it, not HBM",
              cpu_baseline={"value": osec / 10 * 1e6, "unit": "us/iteration", "cores": 1, "kind": "oracle",
                            "sample": "the whole configuration (10 iterations), best of 3"})
    msec, mcores = _mcore_seconds(p)
    jr["cpu_mcore"] = {"value": msec / 10 * 1e6, "unit": "us/iteration", "cores": mcores, "kind": "mcore",
                       "sample": "the whole configuration (10 iterations), best of 2"}
    out["jacobi_256_f64_10it"] = jr
    # --- shallow water 4096^2 float64, 50 steps
    N, steps = 4096, 50
    p = shallow_water(N, steps)
    cb = 6 * 8 * N * N
    lo, hi = p.meta["batches"][1]
    ops = fp64_bytecode_ops(p, lo, hi)
    sw = {}
    for name, flags in (("fused_graphs", F | G), ("plain_graphs", G)):
        sec, st = timed(p, flags, 2 if name == "fused_graphs" else 1, warmup=1)
        ms = sec / steps * 1e3
        sw[name] = {"ms_per_step": ms, "GB/s": cb / (ms / 1e3) / 1e9, "hbm_fraction": cb / (ms / 1e3) / 1e9 / hbm,
                    "launches_per_step": st["kernel_launches"] / steps}
    ms = sw["fused_graphs"]["ms_per_step"]
    floor_ms = ops / (fp64["peak"] * 1e9) * 1e3
    sw["speedup_vs_plain"] = sw["plain_graphs"]["ms_per_step"] / ms
    sw["roofline"] = {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e9, "peak": fp64["peak"],
                      "unit": "G FP64-inst/s", "frac": floor_ms / ms,
                      "work": f"{ops / (N * N):.2f} float64 add/subtract/multiply operations per cell per step "
                              "(the bytecodes' own, products by 2^k excluded)",
                      "floor_ms_per_step": floor_ms,
                      "hbm": {"achieved": cb / (ms / 1e3) / 1e9, "peak": hbm, "frac": cb / (ms / 1e3) / 1e9 / hbm,
                              "bytes_per_cell": 48}}
    ps = shallow_water(1024, 1)
    osec = _oracle_seconds(ps)
    sw["cpu_baseline"] = {"value": 6 * 8 * 1024 * 1024 / osec / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                          "ms_per_step_at_4096": osec * (N * N) / (1024 * 1024) * 1e3,
                          "sample": f"one step of 1024x1024 ({osec:.1f} s), scaled by cells"}
    ps = shallow_water(2048, 2)
    msec, mcores = _mcore_seconds(ps)
    sw["cpu_mcore"] = {"value": 6 * 8 * 2048 * 2048 * 2 / msec / 1e9, "unit": "GB/s", "cores": mcores,
                       "kind": "mcore", "ms_per_step_at_4096": msec / 2 * (N * N) / (2048 * 2048) * 1e3,
                       "sample": f"two steps of 2048x2048 ({msec:.2f} s), scaled by cells"}
    # the same program in float32, where the memory roofline is within reach
    # (fused path only: its plain path is timed by --workload shallow_water)
    p32 = shallow_water(N, steps, "float32")
    sec, st = timed(p32, F | G, 2, warmup=1)
    ms32 = sec / steps * 1e3
    cb32 = 6 * 4 * N * N
    sw["float32"] = {"ms_per_step": ms32, "GB/s": cb32 / (ms32 / 1e3) / 1e9,
                     "roofline": {"bound": "hbm", "achieved": cb32 / (ms32 / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": cb32 / (ms32 / 1e3) / 1e9 / hbm, "bytes_per_cell": 24},
                     "launches_per_step": st["kernel_launches"] / steps,
                     # graph replays are not counted: whether the form was issued (or captured) at all
                     "row_sweep_form": st["sweep_group_launches"] > 0}
    out["shallow_water_4096_f64_50st"] = sw
    # --- Monte-Carlo pi, 256 instances in one packed launch
    sizes = mc_sizes(256)
    p = montecarlo_pi(sizes=sizes)
    samples = int(sizes.sum())
    mc = {}
    for name, flags in (("packed", F), ("unpacked", V.VBE_FUSE | V.VBE_AUTOTUNE), ("plain", 0)):
        sec, st = timed(p, flags, 3 if name != "plain" else 1, warmup=2 if name != "plain" else 1)
        mc[name] = {"ms_per_step": sec * 1e3, "samples_per_s": samples / sec,
                    "launches_per_step": st["kernel_launches"], "packed_launches_per_step": st["packed_launches"]}
    ops = fp64_bytecode_ops(p)
    mc["speedup_vs_plain"] = mc["plain"]["ms_per_step"] / mc["packed"]["ms_per_step"]
    mc["roofline"] = {"bound": "alu", "achieved": ops / (mc["packed"]["ms_per_step"] / 1e3) / 1e9,
                      "peak": fp64["peak"], "unit": "G FP64-inst/s",
                      "frac": ops / (mc["packed"]["ms_per_step"] / 1e3) / 1e9 / fp64["peak"],
                      "work": f"{ops / samples:.1f} float64 operations per sample (2 multiplies, add, compare)"}
    order = np.argsort(sizes)
    pick = order[:192]  # a bounded sample: the 192 smallest instances
    sub = montecarlo_pi(sizes=sizes[pick], keys=pick)
    osec = _oracle_seconds(sub)
    ns = int(sizes[pick].sum())
    jobs = [("mc", {"sizes": [int(sizes[k])], "keys": [int(k)]}) for k in pick]
    prate, cores, wall = _pool_rate(jobs, ns)
    mc["cpu_baseline"] = {"value": ns / osec, "unit": "samples/s", "cores": 1, "kind": "oracle",
                          "sample": f"the 192 smallest instances ({ns} samples, {osec:.1f} s)",
                          "all_cores": {"value": prate, "cores": cores,
                                        "sample": f"the same instances, one per task, spawn process pool ({wall:.1f} s)"}}
    msec, mcores = _mcore_seconds(sub)
    mc["cpu_mcore"] = {"value": ns / msec, "unit": "samples/s", "cores": mcores, "kind": "mcore",
                       "sample": f"the 192 smallest instances ({ns} samples, {msec:.2f} s)"}
    mc["samples"] = samples
    out["montecarlo_pi_256"] = mc
    # --- serving loop
    sv = serving_bench(args, V, local)
    from workloads.serving import request_mix
    mix = request_mix(64, seed=1210_7774 + 55)
    jobs = [(k, prm) for k, prm in mix]
    t0 = time.perf_counter()
    for j in jobs[:8]:
        _oracle_job(j)
    one = time.perf_counter() - t0
    prate, cores, wall = _pool_rate(jobs, len(jobs))
    sv["cpu_baseline"] = {"value": 8 / one, "unit": "requests/s", "cores": 1, "kind": "oracle",
                          "sample": f"8 requests of the same mix (another seed), {one:.1f} s",
                          "all_cores": {"value": prate, "cores": cores,
                                        "sample": f"64 requests of that mix, spawn process pool ({wall:.1f} s)"}}
    import mcore
    from workloads.serving import request_program
    progs = [request_program(k, prm) for k, prm in jobs[:8]]
    for q in progs[:2]:
        mcore.run(q)
    t0 = time.perf_counter()
    for q in progs:
        mcore.run(q)
    msec = time.perf_counter() - t0
    sv["cpu_mcore"] = {"value": len(progs) / msec, "unit": "requests/s", "cores": mcore.cores(), "kind": "mcore",
                       "sample": f"the same 8 requests, one after another, each on every core ({msec:.1f} s)"}
    out["serving_64_clients"] = sv
    return out


# ------------------------------------------------------ the other workloads

def other_workload(args, local):
    """Jacobi, shallow water, Monte-Carlo pi and the serving loop: one JSON
    line each with fused / plain timings (these are reported beside the
    headline, not as it)."""
    import torch
    from paper_1210_7774_b300 import build
    build.build()
    from paper_1210_7774_b300 import vbe as V
    from paper_1210_7774_b300.runner import Executor

    torch.cuda.set_device(local)
    ts = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(ts)
    stream = ts.cuda_stream
    cache = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
    hbm, _ = peaks()
    F = V.VBE_FUSE | V.VBE_AUTOTUNE | V.VBE_PACK
    modes = {"fused_graphs": F | V.VBE_GRAPHS, "fused": F, "plain": 0, "plain_graphs": V.VBE_GRAPHS}
    out = {"workload": args.workload}

    def group_forms(st):
        # tile-fused group launches by form (tuning trials included); VBE_TILE
        # in the environment fixes the form
        return {"tensor_copy": st["tma_group_launches"], "row_sweep": st["sweep_group_launches"],
                "forced": os.environ.get("VBE_TILE") or None}

    def timed_batches(program, flags, reps, warmup=2):
        ex = Executor(flags, device=local, stream=stream, cache_dir=cache)
        L = ex.load(program)
        nb = len(L.batches)

        def step():
            for k in range(nb):
                ex.submit(L, k)
        sec = time_steps(step, reps, warmup, torch)
        st = ex.stats()
        ex.close()
        return sec, st

    if args.workload == "jacobi":
        from workloads import jacobi
        only_paper = args.paths == "paper_size"  # profiling: the 7168^2 part alone
        p = jacobi(256, 10)
        cbytes = 256 * 256 * 8 + 254 * 254 * 8  # read the grid, write the interior, per iteration
        for name, flags in ({} if only_paper else modes).items():
            # host-bound at this size: enough warm-up for the host path to settle
            sec, st = timed_batches(p, flags, 100, warmup=20)
            out[name] = {"us_per_iteration": sec / 10 * 1e6, "GB/s": cbytes * 10 / sec / 1e9}
        out["note"] = "256x256 float64, 10 iterations; the grid (0.5 MB) is L2-resident, so this is launch-bound"
        # the paper's size: 7168^2 float64, 4 iterations, HBM-bound
        n = 7168
        p = jacobi(n, 4)
        cbytes = n * n * 8 + (n - 2) * (n - 2) * 8
        big = {}
        modes["fused_graphs_untiled"] = F | V.VBE_GRAPHS | V.VBE_NO_TILE_FUSION
        for name in ("fused_graphs", "fused_graphs_untiled", "plain_graphs"):
            sec, st = timed_batches(p, modes[name], 3)
            big[name] = {"ms_per_iteration": sec / 4 * 1e3, "GB/s": cbytes * 4 / sec / 1e9,
                         "hbm_fraction": cbytes * 4 / sec / 1e9 / hbm}
        big["note"] = "7168x7168 float64, 4 iterations; bytes = grid read + interior written once per iteration"
        out["paper_size"] = big
    elif args.workload == "shallow_water":
        from workloads import shallow_water
        for dtype in [d for d in ("float64", "float32") if d in args.dtypes.split(",")]:
            p = shallow_water(4096, 50, dtype)
            isz = 8 if dtype == "float64" else 4
            cbytes = 6 * isz * 4096 * 4096 * 50  # H, U, V read once and written once per step
            res = {}
            modes["fused_graphs_untiled"] = F | V.VBE_GRAPHS | V.VBE_NO_TILE_FUSION
            names = [m for m in ("fused_graphs", "fused_graphs_untiled", "plain_graphs")
                     if args.paths == "fused,plain" or m in args.paths.split(",")]
            for name in names:
                sec, st = timed_batches(p, modes[name], 2)
                res[name] = {"ms_per_step": sec / 50 * 1e3, "GB/s": cbytes / sec / 1e9,
                             "hbm_fraction": cbytes / sec / 1e9 / hbm, "group_forms": group_forms(st)}
            if "plain_graphs" in res and "fused_graphs" in res:
                res["speedup_vs_plain"] = res["plain_graphs"]["ms_per_step"] / res["fused_graphs"]["ms_per_step"]
            out[dtype] = res
    elif args.workload == "stencil":
        from workloads import gray_scott
        R, C, steps = 10240, 1024, 10
        for dtype in [d for d in ("float64", "float32") if d in args.dtypes.split(",")]:
            p = gray_scott(R, C, steps, dtype)
            isz = 8 if dtype == "float64" else 4
            cbytes = (2 * R * C + 2 * (R - 2) * (C - 2)) * isz * steps  # U, V read once, interiors written once
            res = {}
            modes["fused_graphs_untiled"] = F | V.VBE_GRAPHS | V.VBE_NO_TILE_FUSION
            for name in ("fused_graphs", "fused_graphs_untiled", "plain_graphs"):
                sec, st = timed_batches(p, modes[name], 3)
                res[name] = {"ms_per_step": sec / steps * 1e3, "GB/s": cbytes / sec / 1e9,
                             "hbm_fraction": cbytes / sec / 1e9 / hbm, "group_forms": group_forms(st)}
            res["speedup_vs_plain"] = res["plain_graphs"]["ms_per_step"] / res["fused_graphs"]["ms_per_step"]
            out[dtype] = res
        out["note"] = "Gray-Scott reaction-diffusion, 10240x1024, 10 steps (the paper's synthetic-stencil size)"
    elif args.workload == "knn":
        from workloads import knn
        N, M, D, k = 10_000, 1_000, 16, 4
        for dtype in [d for d in ("float64", "float32") if d in args.dtypes.split(",")]:
            p = knn(N, M, D, k, dtype)
            res = {}
            for name in ("fused_graphs", "plain_graphs"):
                sec, st = timed_batches(p, modes[name], 5)
                res[name] = {"ms_per_job": sec * 1e3, "queries_per_s": M / sec,
                             "distance_terms_per_s": M * N * D / sec}
            res["speedup_vs_plain"] = res["plain_graphs"]["ms_per_job"] / res["fused_graphs"]["ms_per_job"]
            out[dtype] = res
        out["note"] = ("naive kNN, 10,000 points x 1,000 queries (16-D, k = 4): broadcast differences, "
                       "axis sums, then k rounds of MIN/ARGMIN reductions and masking")
    elif args.workload == "montecarlo":
        from workloads import mc_sizes, montecarlo_pi
        p = montecarlo_pi(sizes=mc_sizes(256))
        samples = p.meta["samples"]
        for name, flags in (("packed", F), ("unpacked", V.VBE_FUSE | V.VBE_AUTOTUNE), ("plain", 0)):
            sec, st = timed_batches(p, flags, 3 if name != "plain" else 1)
            out[name] = {"ms_per_step": sec * 1e3, "samples_per_s": samples / sec}
        out["samples"] = samples
    elif args.workload == "serving":
        out.update(serving_bench(args, V, local))
    print(json.dumps(out), flush=True)


def serving_bench(args, V, local):
    """64 clients, Poisson arrivals at 0.7 of the measured capacity, the
    request mix of the serving workload; p50/p99 latency and throughput,
    fused versus plain."""
    import threading

    import torch

    from paper_1210_7774_b300.runner import Request
    from workloads.program import NP_DTYPE
    from workloads.serving import poisson_arrivals, request_mix, request_program

    n_req = args.requests
    mix = request_mix(n_req)
    cache = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
    res = {}
    nclients = 64
    # each client's results land in a page-locked arena of its own (it has
    # one request in flight at a time): the server copies them there straight
    # from the device
    progs_all = [request_program(*m) for m in mix]
    need = [0] * nclients
    for i, p in enumerate(progs_all):
        nb = sum((p.bases[b].nelem * np.dtype(NP_DTYPE[p.bases[b].dtype]).itemsize + 63) // 64 * 64
                 for b in p.outputs)
        need[i % nclients] = max(need[i % nclients], nb)
    extra_mix = request_mix(256 + 3072, seed=1210_7774 + 99)
    for i, m in enumerate(extra_mix):
        p = request_program(*m)
        nb = sum((p.bases[b].nelem * np.dtype(NP_DTYPE[p.bases[b].dtype]).itemsize + 63) // 64 * 64
                 for b in p.outputs)
        need[i % nclients] = max(need[i % nclients], nb)
    arenas = [torch.empty(max(64, nb), dtype=torch.uint8).pin_memory().numpy() for nb in need]
    # the 64 clients are Python threads: after a submit returns, a client
    # needs the interpreter lock again before it can wait, and at the
    # default 5 ms switch interval that hand-over alone reached 20 ms at p99
    # (measured: results ready in host memory at p99 within 3 ms of issue,
    # clients back 19-24 ms later). The interval is shortened for the runs,
    # and the latency reported is the server's: from submit until the
    # request's results are in the client's host memory (the stream callback
    # after the result copies); what the Python clients saw is reported too.
    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    for name, flags in (("fused", V.VBE_FUSE | V.VBE_PACK), ("plain", 0)):
        ctx = V.vbe_init(local, flags, 0, None, cache)
        srv = V.vbe_server_create(ctx, args.serve_slots, 60 << 30, flags, workers=args.serve_workers)
        # every request is built and packed (views, bytecodes, result buffers
        # not yet touched) before the clock starts, so the Python load
        # generator stays off the measured path; the clients only submit,
        # wait and drop the request (its result memory) when it is done
        reqs = [Request(p) for p in progs_all]
        # capacity: after a pass over 256 requests of the same mix (kernel
        # compilation), a closed loop of the 64 clients over 3072 further
        # requests that have not been seen (another seed), so per-size work is
        # paid as it is in the timed run: each client submits its next
        # request as soon as its previous one is back
        extra = [Request(request_program(*m)) for m in extra_mix]
        for batch in (extra[:256], extra[256:]):
            def closed(c, batch=batch):
                for i in range(c, len(batch), 64):
                    batch[i].bind_results(arenas[c])
                    V.vbe_server_wait(srv, V.vbe_server_submit(srv, batch[i].req), -1)
            th = [threading.Thread(target=closed, args=(c,)) for c in range(64)]
            t0 = time.perf_counter()
            for t in th:
                t.start()
            for t in th:
                t.join()
            cap = len(batch) / (time.perf_counter() - t0)
        del extra
        rate = 0.7 * cap if name == "fused" else res["fused"]["arrival_rate"]
        arrivals = poisson_arrivals(n_req, rate)
        lat = [None] * n_req  # submit -> results in the client's host memory
        lat_client = [None] * n_req  # submit -> the client's wait returned
        parts = [None] * n_req  # (queued, planning, device and copies, waking the client) per request, ms
        start = time.perf_counter() + 0.2

        def client(c):
            for i in range(c, n_req, nclients):
                delay = start + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                reqs[i].bind_results(arenas[c])
                rid = V.vbe_server_submit(srv, reqs[i].req)
                r = V.vbe_server_wait(srv, rid, -1)
                reqs[i] = None
                lat[i] = (r.t_ready_ns - r.t_arrive_ns) / 1e6
                lat_client[i] = (r.t_done_ns - r.t_arrive_ns) / 1e6
                parts[i] = ((r.t_admit_ns - r.t_arrive_ns) / 1e6, (r.t_issued_ns - r.t_admit_ns) / 1e6,
                            (r.t_ready_ns - r.t_issued_ns) / 1e6, (r.t_done_ns - r.t_ready_ns) / 1e6)

        th = [threading.Thread(target=client, args=(c,)) for c in range(nclients)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        wall = time.perf_counter() - start
        V.vbe_server_destroy(srv)
        V.vbe_finalize(ctx)
        lat = np.array(lat)
        lc = np.array(lat_client)
        pa = np.array(parts)
        res[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "p99_over_p50": float(np.percentile(lat, 99) / np.percentile(lat, 50)),
                     "latency": "submit to results in the client's host memory (server side)",
                     "client_p50_ms": float(np.percentile(lc, 50)), "client_p99_ms": float(np.percentile(lc, 99)),
                     "throughput_req_s": n_req / wall, "capacity_req_s": cap, "arrival_rate": rate,
                     "breakdown_ms": {k: {"p50": float(np.percentile(pa[:, q], 50)),
                                          "p99": float(np.percentile(pa[:, q], 99))}
                                      for q, k in enumerate(("queued", "host_planning", "device_and_copies", "wake_client"))}}
        # the same per request kind (Jacobi solves, Black-Scholes pricings)
        by_kind = {}
        for kind in ("jacobi", "blackscholes"):
            sel = np.array([m[0] == kind for m in mix])
            if sel.any():
                by_kind[kind] = {"requests": int(sel.sum()),
                                 "latency_ms": {"p50": float(np.percentile(lat[sel], 50)),
                                                "p99": float(np.percentile(lat[sel], 99))},
                                 **{k: {"p50": float(np.percentile(pa[sel, q], 50)),
                                        "p99": float(np.percentile(pa[sel, q], 99))}
                                    for q, k in enumerate(("queued", "host_planning", "device_and_copies", "wake_client"))}}
        res[name]["by_kind"] = by_kind
    sys.setswitchinterval(switch)
    res["requests"] = n_req
    res["server"] = {"slots": args.serve_slots, "workers": args.serve_workers, "mem_cap_bytes": 60 << 30, "clients": 64,
                     "rate": "0.7 x the fused capacity, for both paths",
                     "results": "each client's results in a page-locked arena of its own (one request in flight "
                                "per client), filled by the server straight from the device"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vbe", choices=["vbe", "reference"])
    ap.add_argument("--workload", default="blackscholes")
    ap.add_argument("--options", type=int, default=1 << 24)
    ap.add_argument("--ref-sample", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the per-configuration sub-keys (Jacobi, shallow water, MC, serving)")
    ap.add_argument("--dtypes", default="float64,float32", help="profiling: restrict the dtypes run")
    ap.add_argument("--requests", type=int, default=10000, help="serving: number of requests")
    ap.add_argument("--serve-workers", type=int, default=8, help="serving: scheduler threads of the server")
    ap.add_argument("--serve-slots", type=int, default=16, help="serving: slots (streams) over all workers")
    ap.add_argument("--e2e-workers", type=int, default=4,
                    help="end-to-end: contexts (and host threads) the options are split over")
    ap.add_argument("--paths", default="fused,plain", help="profiling: restrict the paths run (jacobi: paper_size runs the 7168^2 part alone)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        cpu_reference(args, rank, world)
        return
    if args.workload != "blackscholes":
        other_workload(args, local)
        return
    clocks = Clocks(local)
    clocks.start()
    res, dist = gpu_blackscholes(args, rank, world, local)
    ck = clocks.stop()
    fp64 = res.pop("_fp64")
    V, torch, _, stream = res.pop("_ctx")
    if args.dtypes != "float64,float32" or args.paths != "fused,plain":
        if rank == 0:  # a restricted profiling run prints only its timings
            print(json.dumps({k: {p: v[p]["sec"] for p in ("fused", "plain") if p in v} for k, v in res.items()}))
        return
    # max over ranks of the per-step time
    sec = max_over_ranks(res["float64"]["fused"]["sec"], dist)
    if rank != 0:
        return
    hbm, src = peaks()
    f64 = res["float64"]
    value = aggregate_value(f64["cbytes"], sec, world) / 1e9
    achieved = f64["cbytes"] / sec / 1e9
    cpu = cpu_mcore = None
    if not args.no_cpu_baseline:
        import oracle
        from workloads import blackscholes
        prog = blackscholes(args.ref_sample, "float64")
        t0 = time.perf_counter()
        oracle.run(prog)
        dt = time.perf_counter() - t0
        cpu = {"value": prog.compulsory_bytes() / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.ref_sample} options of the same workload, float64, one pass ({dt:.1f} s)"}
        pm = blackscholes(4 * args.ref_sample, "float64")
        msec, mcores = _mcore_seconds(pm)
        cpu_mcore = {"value": pm.compulsory_bytes() / msec / 1e9, "unit": "GB/s", "cores": mcores, "kind": "mcore",
                     "sample": f"{4 * args.ref_sample} options of the same workload, float64, best of 2 "
                               f"({msec:.2f} s)"}
    f32 = res["float32"]
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args.options, "float64"),
        "hbm_fraction": achieved / hbm,
        "plain": {"value": f64["plain"]["GB/s"], "ms_per_step": f64["plain"]["sec"] * 1e3,
                  "launches_per_step": f64["plain"]["launches_per_step"]},
        "speedup_vs_plain": f64["plain"]["sec"] / sec,
        "float32": {"value": f32["fused"]["GB/s"], "hbm_fraction": f32["fused"]["GB/s"] / hbm,
                    "ms_per_step": f32["fused"]["sec"] * 1e3, "plain_value": f32["plain"]["GB/s"],
                    "speedup_vs_plain": f32["plain"]["sec"] / f32["fused"]["sec"],
                    "roofline": {"bound": "hbm", "achieved": f32["fused"]["GB/s"], "peak": hbm, "unit": "GB/s",
                                 "frac": f32["fused"]["GB/s"] / hbm, "peak_source": src,
                                 "traffic": (measured_counters("blackscholes_f32", f32["kernel_hash"]) or {}).get(
                                     "dram_bytes_per_launch"),
                                 "kernel_hash": f32["kernel_hash"]}},
        "roofline": dict(roofline_f64(achieved, hbm, src, measured_counters("blackscholes_f64", f64["kernel_hash"]),
                                      args.options, sec, fp64, ck.get("sm_mhz") or 2032.0),
                         kernel_hash=f64["kernel_hash"]),
        "fp64_peak": fp64,
        "e2e": f64["e2e"],
        "e2e_serial": f64["e2e_serial"],
        "gpu_launches": int(round(f64["fused"]["launches_per_step"] * args.steps)),
        "clocks": ck,
        "cpu_baseline": cpu,
        "cpu_mcore": cpu_mcore,
    }
    if not args.no_configs and world == 1:
        ck2 = Clocks(local)
        ck2.start()
        line["configs"] = config_subkeys(args, V, torch, local, stream, hbm, fp64)
        line["configs"]["clocks"] = ck2.stop()
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
