"""Benchmark: gate-level re-simulation throughput on one GB300.

One step = one full re-simulation of the benchmark workload (every gate of
every level over every cycle, SAIF included): the 200k-gate, depth-60,
10,000-cycle netlist of the "mid" recipe (4-input cells, geometric fanout,
COND delays on XOR2/MUX2, 20% narrow pulses), synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is gate x cycle evaluations per second over
the timed steps (CUDA events on the library's stream, inputs resident in HBM),
``e2e`` the same metric through the C interface from pinned host buffers
(stimulus upload, simulation, SAIF read-back every step), ``roofline`` the propagation
kernel's algorithmic HBM bandwidth against the measured copy peak, and
``cpu_baseline`` the CPU oracle on a bounded sample of the same workload.
``--impl reference`` times the CPU oracle as the reference arm.
With ``--gpus N`` under torchrun every rank runs an independent replica
(the path does not shard across GPUs); ``value`` sums all ranks' work over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "mid"
SEED = 1
METRIC = "gate*cycle evals/s"
UNIT = "gate-cycles/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(tile_threads, items_per_thread):
    """DRAM bytes per level (the level's propagation launches: the pair
    kernel's and propagate_kernel's) from the committed ncu summary, or None
    once the kernel source or the launch shape differs from the one the
    counters were taken on."""
    import hashlib
    try:
        fields = {}
        with open(os.path.join(ROOT, "profiles", "propagate_kernel_traffic.txt")) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        with open(os.path.join(ROOT, "paper_2203_06117_gb300", "csrc", "kernels.cuh"), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        if fields.get("kernels_cuh_sha256") != digest:
            return None
        return int(fields[f"traffic_bytes_per_level_{tile_threads}x{items_per_thread}"])
    except (OSError, KeyError, ValueError):
        return None


# ----------------------------------------------------------- CPU oracle leg

_WORKER = {}


def _oracle_init(name, seed):
    sys.path.insert(0, ROOT)
    import gen
    import oracle
    wl = gen.make_workload(name, seed=seed)
    _WORKER["wl"] = wl
    _WORKER["sim"] = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)


def _oracle_windows(windows):
    sim, wl = _WORKER["sim"], _WORKER["wl"]
    t = time.perf_counter()
    for w in windows:
        sim.window(w)
    return time.perf_counter() - t, len(windows) * wl.netlist.num_gates


class OraclePool:
    """The event-driven oracle, as it stands, timed on a bounded sample of
    windows of the benchmark workload: one spawned process per host core,
    each simulating its own windows (windows are independent).  Workers
    build the workload once, outside the timed region."""

    CYCLES = {"tiny": 1000, "mid": 10_000, "large": 20_000}

    def __init__(self, name=WORKLOAD, seed=SEED, cores=None):
        self.name, self.cores = name, cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(name, seed))
        dt, _ = self.pool.apply(_oracle_windows, ([0, 1],))
        self.per_window = max(dt / 2, 1e-6)
        self.offset = 0

    def measure(self, seconds):
        C = self.CYCLES[self.name]
        per_core = max(1, int(seconds / self.per_window))
        step = max(1, C // (per_core * self.cores))
        jobs = [[(self.offset + (k * self.cores + c) * step) % C for k in range(per_core)]
                for c in range(self.cores)]
        self.offset += 1
        res = self.pool.map(_oracle_windows, jobs, chunksize=1)
        wall = max(r[0] for r in res)
        work = sum(r[1] for r in res)
        sample = (f"{per_core * self.cores} of {C} windows of the {self.name} workload "
                  f"(every {step}th), {self.cores} processes x {per_core} windows, "
                  f"slowest process {wall:.1f} s")
        return work / wall, self.cores, sample

    def close(self):
        self.pool.terminate()


def cpu_oracle(seconds: float = 12.0):
    p = OraclePool()
    try:
        return p.measure(seconds)
    finally:
        p.close()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- main

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def dist_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands, on host cores."""
    if rank != 0:
        return
    per_step = []
    pool = OraclePool(cores=args.ref_cores or None)
    # whole run bounded to about ref_seconds of oracle work
    budget = args.ref_seconds / (args.warmup + args.steps)
    try:
        for s in range(args.warmup + args.steps):
            v, cores, sample = pool.measure(budget)
            if s >= args.warmup:
                per_step.append(v)
    finally:
        pool.close()
    value = statistics.mean(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


_PINNED = []


def _pinned(a):
    """A copy of a numpy array in page-locked host memory (kept alive for
    the process)."""
    import torch
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype, pin_memory=True)
    out = t.numpy()
    out[...] = a
    _PINNED.append(t)
    return out


def format_bytes_per_step(netlist, tc, num_windows):
    """Algorithmic bytes of one step by the per-(gate, window) figure of the
    paper's waveform format: each fanin waveform read once (a start value,
    an end marker and its edges, 4 bytes each), the output written once
    likewise, plus an 8-byte offset:
        4 * sum_pins (2 + e_pin) + 4 * (2 + e_out) + 8
    summed exactly over every item from the step's toggle counts."""
    I, G = netlist.num_inputs, netlist.num_gates
    P = int(netlist.fanin_ptr[-1])
    fanout = np.bincount(netlist.fanin_net.astype(np.int64), minlength=I + G)
    tc = np.asarray(tc, np.int64)
    edges_read = int((tc * fanout).sum())
    edges_written = int(tc[I:].sum())
    return 8 * num_windows * (P + G) + 8 * num_windows * G + 4 * edges_read + 4 * edges_written


def _config(args):
    return {"workload": "mid: 200k gates, depth 60, 512 inputs, 10,000 cycles of 1,000 ps, "
                        "fanin 1-4, geometric fanout mean 2.5, toggle p=0.3, 5% pulses (20% narrow), "
                        "COND on XOR2/MUX2, delays 2-120 ps, seed 1",
            "gates": 200_000, "cycles": 10_000, "window_cycles": 1,
            "parallelism": f"replicas x{args.gpus}", "l2": "inputs larger than L2 (waveform store ~20 GB)"}


def _saif_equal(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def run_batched_mode(args):
    """64 jobs over 8 netlists: engine (continuous batching) vs the plain
    single-job loop on the same GPU, bit-exact SAIF between the two."""
    import gen
    import paper_2203_06117_gb300 as gs
    from paper_2203_06117_gb300 import serve
    gs.build()
    nets, specs = gen.batched_workload(seed=SEED, scale=args.scale)
    work = sum(nets[s["netlist"]].netlist.num_gates * s["stim"].num_cycles for s in specs)
    reqs = [serve.Request.from_spec(s) for s in specs]
    opts = dict(tile_items=args.tile or 256, items_per_thread=args.ipt or 4)
    tuning = None
    if args.tile or args.ipt or args.step_items:
        eopts = dict(opts, step_items=args.step_items)
    else:  # the engine autotuner on a sample of the stream (outside the timed runs)
        eopts, timings = serve.autotune_engine(nets, reqs)
        tuning = {"chosen": eopts, "candidates_ms": [[round(t, 1), o] for t, o in timings]}
    serve.run_batched(nets, reqs, keep_results=False, **eopts)         # warm-up
    t_b = []
    for _ in range(args.steps):
        dt, st = serve.run_batched(nets, reqs, **eopts)
        t_b.append(dt)
    batched = [r.result for r in reqs]
    serve.run_plain_loop(nets, reqs, keep_results=False, **opts)       # warm-up
    t_p = [serve.run_plain_loop(nets, reqs, **opts) for _ in range(args.steps)]
    exact = all(_saif_equal(a, r.result) for a, r in zip(batched, reqs))
    tb, tp = statistics.median(t_b), statistics.median(t_p)
    line = {"metric": "batched gate*cycle evals/s", "value": work / tb, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": tb * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "64 jobs over 8 netlists of 10k-500k gates (mid recipe), cycles "
                                   "log-normal median 2,000 in [100, 20,000], toggle p in [0.05, 0.5]",
                       "jobs": len(reqs), "gate_cycles": int(work),
                       "gates": [n.netlist.num_gates for n in nets]},
            "plain_loop": {"value": work / tp, "ms": tp * 1e3},
            "speedup_vs_plain": tp / tb, "saif_bit_exact_vs_plain": exact, "engine": st,
            "engine_options": eopts, "autotune": tuning,
            "repeats_ms": {"engine": [round(t * 1e3, 1) for t in t_b], "plain": [round(t * 1e3, 1) for t in t_p]}}
    print(json.dumps(line), flush=True)


def run_served_mode(args):
    """Poisson stream at 200 req/s over 4 resident netlists: continuous
    batching vs serving one request at a time with the plain path."""
    import gen
    import paper_2203_06117_gb300 as gs
    from paper_2203_06117_gb300 import serve
    gs.build()
    nets, specs = gen.served_workload(seed=SEED, rate=args.rate, seconds=args.seconds, scale=args.scale)
    work = sum(nets[s["netlist"]].netlist.num_gates * s["stim"].num_cycles for s in specs)
    # warm-up on a short prefix of the stream
    warm = [serve.Request.from_spec(s) for s in specs[:8]]
    opts = dict(tile_items=args.tile or 256, items_per_thread=args.ipt or 4)
    eopts = dict(opts, step_items=args.step_items)
    serve.run_served(nets, warm, keep_results=False, **eopts)
    reqs = [serve.Request.from_spec(s) for s in specs]
    mk, st = serve.run_served(nets, reqs, **eopts)
    served = [r.result for r in reqs]
    lat = serve.latency_summary(reqs)
    reqs_p = [serve.Request.from_spec(s) for s in specs]
    serve.run_served_plain(nets, warm, keep_results=False, **opts)
    mk_p = serve.run_served_plain(nets, reqs_p, **opts)
    lat_p = serve.latency_summary(reqs_p)
    exact = all(_saif_equal(a, r.result) for a, r in zip(served, reqs_p))
    line = {"metric": "served gate*cycle evals/s", "value": work / mk, "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": mk * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"Poisson {args.rate:g} req/s for {args.seconds:g} s over 4 resident "
                                   "netlists (50k/200k/500k/1M gates, tiny recipe), 100-5,000 cycles "
                                   "log-uniform, 30% with a 1% delay edit",
                       "requests": len(reqs), "gate_cycles": int(work)},
            "latency_ms": lat, "plain_serial": {"value": work / mk_p, "latency_ms": lat_p},
            "saif_bit_exact_vs_plain": exact, "engine": st}
    print(json.dumps(line), flush=True)


def run_ingest_mode(args):
    """Stimulus ingest: the benchmark workload's 512 inputs x 10,000 cycles
    as raw (input, absolute ps) toggles in shuffled order, restructured per
    (input, cycle) on the GPU (gatspi_set_stimulus_events, host arrays in,
    device stimulus out, copies included), against the per-cycle upload
    (gatspi_set_stimulus, host validation) and the oracle's numpy
    restructuring on the host."""
    import gen
    import paper_2203_06117_gb300 as gs
    from oracle import stimulus as ostim
    gs.build()
    wl = gen.make_workload(WORKLOAD, seed=SEED, num_cycles=args.cycles or None)
    st = wl.stim
    inp, t = ostim.cycles_to_events(st)
    perm = np.random.Generator(np.random.PCG64(SEED)).permutation(inp.size)
    inp, t = np.ascontiguousarray(inp[perm]), np.ascontiguousarray(t[perm])
    I = wl.netlist.num_inputs

    def timed(fn, k):
        out = []
        for _ in range(k):
            a = time.perf_counter()
            fn()
            out.append(time.perf_counter() - a)
        return statistics.median(out)

    with gs.Simulator(wl.netlist, wl.delays, st) as sim:
        ev = lambda: gs.gatspi_set_stimulus_events(sim.ctx, st.num_cycles, st.cycle_ps, st.init, inp, t)
        cyc = lambda: gs.gatspi_set_stimulus(sim.ctx, st.num_cycles, st.cycle_ps, st.init, st.edge_ptr,
                                             st.edge_time)
        for _ in range(args.warmup):
            ev()
            cyc()
        t_ev = timed(ev, args.steps)
        t_cyc = timed(cyc, args.steps)
    t_host = timed(lambda: ostim.events_to_cycles(I, st.num_cycles, st.cycle_ps, inp, t), 3)
    n = int(inp.size)
    line = {"metric": "stimulus toggles restructured/s", "value": n / t_ev, "unit": "toggles/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ev * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"the mid workload's stimulus: {I} inputs x {st.num_cycles} cycles of "
                                   f"{st.cycle_ps} ps, {n} toggles in shuffled order",
                       "bytes_in": int(inp.nbytes + t.nbytes)},
            "per_cycle_upload_ms": t_cyc * 1e3, "host_numpy_restructure_ms": t_host * 1e3}
    print(json.dumps(line), flush=True)


def _levels(netlist):
    """Logic level of every gate (caller numbering)."""
    I = netlist.num_inputs
    lvl = np.zeros(netlist.num_nets, np.int64)
    for g in range(netlist.num_gates):
        a, b = netlist.fanin_ptr[g], netlist.fanin_ptr[g + 1]
        lvl[I + g] = 1 + lvl[netlist.fanin_net[a:b]].max()
    return lvl[I:]


def run_resim_mode(args):
    """Delay edits on the benchmark workload (Section 4's loop: simulate,
    re-time a cell, simulate again): gatspi_resimulate_edit, which runs
    only the fanout cone of the re-timed gate, against a full simulation
    with the same edit, for one gate at each of several depths."""
    import gen
    import paper_2203_06117_gb300 as gs
    gs.build()
    wl = gen.make_workload(WORKLOAD, seed=SEED, num_cycles=args.cycles or None)
    lvl = _levels(wl.netlist)
    D = int(lvl.max())
    rng = np.random.Generator(np.random.PCG64(SEED))
    opts = dict(window_cycles=1, tile_items=args.tile or 256, items_per_thread=args.ipt or 4)
    G, C = wl.netlist.num_gates, wl.stim.num_cycles
    rows = []
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(**opts)
        for frac in (0.1, 0.5, 0.9, 1.0):
            L = max(1, min(D, int(round(frac * D))))
            g = int(rng.choice(np.nonzero(lvl == L)[0]))
            cone, full, modes = [], [], []
            for k in range(args.warmup + args.steps):
                a = time.perf_counter()
                info = sim.resimulate_edit([g], [25 + (k % 2)])   # a new edit every time
                dt = time.perf_counter() - a
                modes.append(info["mode"])
                if k >= args.warmup and info["mode"] == 1:     # cone runs only (not a fallback)
                    cone.append(dt)
            gs.gatspi_set_edit(sim.ctx, [g], [30])
            for k in range(args.warmup + args.steps):
                a = time.perf_counter()
                sim.simulate(**opts)
                dt = time.perf_counter() - a
                if k >= args.warmup:
                    full.append(dt)
            gs.gatspi_set_edit(sim.ctx, [], [])
            sim.simulate(**opts)                                   # resident again, no edit
            rows.append({"level": L, "cone_gates": info["cone_gates"], "cone_items": info["items"],
                         "modes": modes, "cone_ms": statistics.median(cone) * 1e3 if cone else None,
                         "full_ms": statistics.median(full) * 1e3})
    best = max(r["full_ms"] / r["cone_ms"] for r in rows if r["cone_ms"])
    line = {"metric": "re-simulation after a one-gate delay edit, speedup over a full run", "value": best,
            "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": min(r["cone_ms"] for r in rows if r["cone_ms"]), "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"mid: {G} gates, depth {D}, {C} cycles; one gate re-timed by +25/26 ps "
                                   "at each of four depths; host wall time of each call"},
            "edits": rows}
    print(json.dumps(line), flush=True)


def run_pulse_mode(args):
    """Throughput of the pulse-limit kernels (PATHPULSEPERCENT other than
    100) on the benchmark workload, next to Algorithm 1 as printed."""
    import gen
    import paper_2203_06117_gb300 as gs
    gs.build()
    wl = gen.make_workload(WORKLOAD, seed=SEED, num_cycles=args.cycles or None)
    G, C = wl.netlist.num_gates, wl.stim.num_cycles
    rows = []
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        for pulse in (None, (50, 100), (0, 0)):
            opts = dict(window_cycles=1, tile_items=256, items_per_thread=4, time_kernels=1, pulse=pulse)
            for _ in range(args.warmup):
                sim.simulate(**opts)
            ms = []
            for _ in range(args.steps):
                sim.simulate(**opts)
                ms.append(sim.stats()["prop_ms"])
            st = sim.stats()
            tc = sim.saif()[2]
            # edges: the waveforms' edges (SAIF toggle counts); arena: entries
            # the waveforms take, which with pulse limits include the unused
            # rest of each tile's upper-bound claim
            rows.append({"limits": "100/100" if pulse is None else f"{pulse[0]}/{pulse[1]}",
                         "prop_ms": statistics.median(ms), "edges": int(tc.sum()), "arena": int(st["edges"]),
                         "gate_cycles_per_s": G * C / (statistics.median(ms) / 1e3)})
    line = {"metric": "gate*cycle evals/s with transport delay (pulse limits 0/0)",
            "value": rows[-1]["gate_cycles_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rows[-1]["prop_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"mid: {G} gates x {C} cycles, 256 x 4 launch shape"}, "limits": rows}
    print(json.dumps(line), flush=True)


def run_features_mode(args):
    """The kernel-time cost of two features of Algorithm 1 on the benchmark
    workload, as the paper measures it (Section 5, Table "features"): the
    full kernel against the kernel without the interconnect inertial filter,
    and against that without full SDF either (one averaged delay per arc
    and output edge).  Same launch shape, same stimulus; the steps of the
    three kernels are interleaved so that clock drift hits them alike."""
    import gen
    import paper_2203_06117_gb300 as gs
    gs.build()
    wl = gen.make_workload(WORKLOAD, seed=SEED, num_cycles=args.cycles or None)
    G, C = wl.netlist.num_gates, wl.stim.num_cycles
    variants = [("full features", 0), ("no interconnect filter", gs.NO_INTERCONNECT_FILTER),
                ("no interconnect filter + partial SDF", gs.NO_INTERCONNECT_FILTER | gs.PARTIAL_SDF)]
    ms = {name: [] for name, _ in variants}
    edges = {}
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        for k in range(args.warmup + args.steps):
            for name, mask in variants:
                sim.simulate(window_cycles=1, tile_items=256, items_per_thread=4, time_kernels=1, features=mask)
                if k >= args.warmup:
                    ms[name].append(sim.stats()["prop_ms"])
                edges[name] = int(sim.stats()["edges"])
    full = statistics.median(ms["full features"])
    rows = [{"kernel": name, "prop_ms": statistics.median(ms[name]), "edges": edges[name],
             "gate_cycles_per_s": G * C / (statistics.median(ms[name]) / 1e3),
             "overhead_of_full_kernel": full / statistics.median(ms[name]) - 1.0} for name, _ in variants]
    line = {"metric": "kernel-time overhead of interconnect filtering and full SDF (fraction of the reduced kernel)",
            "value": rows[-1]["overhead_of_full_kernel"], "unit": "fraction", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": full, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"mid: {G} gates x {C} cycles, 256 x 4 launch shape"}, "kernels": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=0, help="threads per block (0 with --ipt 0: autotuned)")
    ap.add_argument("--ipt", type=int, default=0, help="consecutive windows per thread (0: autotuned)")
    ap.add_argument("--cycles", type=int, default=0,
                    help="cycles of the benchmark workload (0 = the full 10,000); smaller values "
                         "only for profiler captures")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="total oracle seconds of the reference arm (split over its steps)")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="host processes of the reference arm (0: every core)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="mid", choices=["mid", "batched", "served", "ingest", "resim", "pulse", "features"],
                    help="mid = the headline single-job benchmark; batched / served = the "
                         "multi-job engine against the plain per-job path")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink batched/served workloads")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--step-items", type=int, default=0,
                    help="engine: (gate, window) items per step to admit up to (0: the engine's default)")
    ap.add_argument("--seconds", type=float, default=1.0)
    args = ap.parse_args()
    if args.workload == "batched":
        return run_batched_mode(args)
    if args.workload == "served":
        return run_served_mode(args)
    if args.workload == "ingest":
        return run_ingest_mode(args)
    if args.workload == "resim":
        return run_resim_mode(args)
    if args.workload == "pulse":
        return run_pulse_mode(args)
    if args.workload == "features":
        return run_features_mode(args)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    # the oracle's spawn pool starts before any GPU work in this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample = cpu_oracle(seconds=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    import gen
    import paper_2203_06117_gb300 as gs
    gs.build()
    device = local
    import torch
    torch.cuda.set_device(device)  # pinned staging below belongs to this rank's GPU
    wl = gen.make_workload(WORKLOAD, seed=SEED, num_cycles=args.cycles or None)
    G, C = wl.netlist.num_gates, wl.stim.num_cycles
    units = G * C
    sim = gs.Simulator(wl.netlist, wl.delays, wl.stim, device=device)
    opts = dict(window_cycles=1, tile_items=args.tile, items_per_thread=args.ipt, time_kernels=1)
    for _ in range(args.warmup):
        sim.simulate(**opts)
    dist_barrier(world)
    dev_ms, prop_ms, algo, launches, prop_launches = [], [], [], 0, 0
    with ClockSampler(device) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.simulate(**opts)
            st = sim.stats()
            dev_ms.append(st["device_ms"])
            prop_ms.append(st["prop_ms"])
            algo.append(st["algo_bytes"])
            launches += st["kernel_launches"]
            prop_launches += st["prop_launches"]
        host_s = time.perf_counter() - t0
    dist_barrier(world)
    total_s = dist_max(sum(dev_ms) / 1e3, world)
    value = units * args.steps * world / total_s
    ms_per_step = total_s * 1e3 / args.steps
    peak, peak_kind = _peaks()
    # the layout's own bytes (2-byte records, 8-byte tile runs): the stricter figure
    layout_achieved = (sum(algo) / (sum(prop_ms) / 1e3)) / 1e9
    edges = st["edges"]

    # end to end through the C interface from pinned host buffers
    e2e_times = []
    stim = wl.stim
    # the step's inputs sit in pinned host memory (staged once, before timing)
    p_init, p_ptr, p_time = (_pinned(a) for a in (stim.init, stim.edge_ptr, stim.edge_time))
    h2d = p_init.nbytes + p_ptr.nbytes + p_time.nbytes
    d2h = 2 * 8 * wl.netlist.num_nets
    for k in range(args.e2e_steps + 1):
        t = time.perf_counter()
        gs.gatspi_set_stimulus(sim.ctx, stim.num_cycles, stim.cycle_ps, p_init, p_ptr, p_time)
        gs.gatspi_simulate(sim.ctx, window_cycles=1, tile_items=args.tile, items_per_thread=args.ipt)
        saif = sim.saif()
        if k:
            e2e_times.append(time.perf_counter() - t)
    e2e_s = dist_max(statistics.median(e2e_times), world)
    sim.close()
    # the per-unit figure of the waveform format (Holst arrays with start
    # value and end marker) times the step's (gate, cycle) units
    format_step = format_bytes_per_step(wl.netlist, saif[2], C)
    achieved = format_step / (statistics.mean(prop_ms) / 1e3) / 1e9

    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(_config(args), cycles=C),
        "e2e": {"value": units * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": _traffic(st["tile_threads"], st["items_per_thread"])
                     if WORKLOAD == "mid" and not args.cycles else None,
                     "peak_kind": peak_kind,
                     "kernel": "propagate_kernel + propagate_pair_kernel (one level)",
                     "traffic_per": "level",
                     "algo_bytes_per_step": int(format_step),
                     "bytes_per_unit": "4*sum_pins(2+e_pin) + 4*(2+e_out) + 8 per (gate, cycle)",
                     "layout_bytes_per_step": int(algo[-1]),
                     "layout_achieved": layout_achieved, "layout_frac": layout_achieved / peak,
                     "prop_ms_per_step": statistics.mean(prop_ms),
                     "launches_per_step": prop_launches // args.steps},
        "cpu_baseline": cpu,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "gpu_launches": int(launches),
        "detail": {"edges_per_step": int(edges), "host_s": host_s, "clock_samples": clocks["samples"],
                   "saif_tc_total": int(saif[2].sum()), "tile_threads": st["tile_threads"],
                   "items_per_thread": st["items_per_thread"]},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
