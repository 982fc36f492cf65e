"""Batched and served re-simulation on top of the multi-job engine.

* ``run_batched``: submit every job at once and drain the engine (one
  propagation launch per step covers the next level of every admitted job
  part), against ``run_plain_loop``: the single-job path, one job after the
  other.
* ``run_served``: an open-loop request stream (arrival times given) served
  by continuous batching: requests are submitted when they arrive, admitted
  by the engine as device memory frees up, and stepped together with the
  requests already in flight; latency = completion - arrival.  Against
  ``run_served_plain``: the same stream served one request at a time with
  the single-job path (first come, first served).

The paper runs one design and testbench at a time (Section 3) and re-runs
the simulator inside a glitch-optimization loop after netlist edits
(Section 4); the delay edits here are that loop's re-timing step.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Engine, JOB_DONE, JOB_FAILED, Simulator, gatspi_set_edit, gatspi_set_stimulus, \
    gatspi_simulate


@dataclass
class Request:
    arrival: float             # seconds after the start of the stream
    netlist: int               # index into the resident netlists
    stim: object               # gen.Stimulus
    window_cycles: int = 1
    edit_gate: np.ndarray | None = None
    edit_delta: np.ndarray | None = None
    result: tuple | None = None
    digest: np.ndarray | None = None  # per-net waveform digests, when asked for
    done: float = field(default=float("nan"))

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @classmethod
    def from_spec(cls, spec: dict) -> "Request":
        """From a request description (keys arrival, netlist, stim and
        optionally window_cycles, edit_gate, edit_delta)."""
        return cls(spec.get("arrival", 0.0), spec["netlist"], spec["stim"], spec.get("window_cycles", 1),
                   spec.get("edit_gate"), spec.get("edit_delta"))


def _work(netlists, reqs):
    return sum(netlists[r.netlist].netlist.num_gates * r.stim.num_cycles for r in reqs)


def run_batched(netlists, reqs, keep_results=True, **engine_opts):
    """All jobs available at t=0, engine drained.  Each submission (which
    copies the job's stimulus to the device) is followed by one engine step,
    so the device works on the jobs already admitted while later ones are
    still being uploaded.  Returns (seconds, stats)."""
    with Engine(**engine_opts) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in netlists]
        t0 = time.perf_counter()
        jobs = []
        for r in reqs:
            jobs.append(eng.submit(ids[r.netlist], r.stim, r.window_cycles, r.edit_gate, r.edit_delta))
            eng.step()
        eng.drain()
        for r, j in zip(reqs, jobs):
            state, saif = eng.poll(j, ids[r.netlist] if keep_results else None)
            if state != JOB_DONE:
                raise RuntimeError(f"job {j} ended in state {state}")
            r.result = saif
            if engine_opts.get("digest"):
                r.digest = eng.digest(j, ids[r.netlist])
            r.done = time.perf_counter() - t0
        dt = time.perf_counter() - t0
        return dt, eng.stats()


# launch shapes (threads x windows per thread) and admission sizes (step
# items) the engine autotuner times; the kernel has one merge strategy
TUNE_SHAPES = ((256, 4), (128, 8), (256, 2))
TUNE_STEPS = (1 << 23, 1 << 24, 1 << 25, 1 << 26)
_TUNED = {}


def _mix_key(netlists):
    return tuple((w.netlist.num_inputs, w.netlist.num_gates, int(w.netlist.fanin_ptr[-1])) for w in netlists)


def autotune_engine(netlists, reqs, sample=16, shapes=TUNE_SHAPES, steps=TUNE_STEPS, cache=_TUNED):
    """Engine options for a netlist mix: every (launch shape, step items)
    pair is timed on a sample of the stream's jobs (every k-th job, so that
    sizes and activities stay representative; one warm-up run each), and the
    fastest is kept.  The choice is cached per netlist mix (inputs, gates
    and pins of each netlist), so later streams over the same mix reuse it.
    Returns (options, timings in ms per candidate)."""
    key = _mix_key(netlists)
    if key in cache:
        return dict(cache[key][0]), cache[key][1]
    k = max(1, len(reqs) // sample)
    pick = [Request(0.0, r.netlist, r.stim, r.window_cycles, r.edit_gate, r.edit_delta) for r in reqs[::k]]
    timings = []
    for nt, ipt in shapes:
        for si in steps:
            opts = dict(tile_items=nt, items_per_thread=ipt, step_items=si)
            run_batched(netlists, pick, keep_results=False, **opts)
            dt, _ = run_batched(netlists, pick, keep_results=False, **opts)
            timings.append((dt * 1e3, opts))
    best = min(timings, key=lambda x: x[0])[1]
    cache[key] = (best, timings)
    return dict(best), timings


def run_plain_loop(netlists, reqs, keep_results=True, tile_items=256, items_per_thread=4):
    """The single-job path, one job after the other (netlists resident), with
    the engine's default launch shape (no per-netlist autotuning inside the
    timed loop)."""
    sims = [Simulator(w.netlist, w.delays, _dummy_stim(w)) for w in netlists]
    try:
        t0 = time.perf_counter()
        for r in reqs:
            ctx = sims[r.netlist].ctx
            gatspi_set_edit(ctx, r.edit_gate, r.edit_delta)
            gatspi_set_stimulus(ctx, r.stim.num_cycles, r.stim.cycle_ps, r.stim.init, r.stim.edge_ptr,
                                r.stim.edge_time)
            gatspi_simulate(ctx, window_cycles=r.window_cycles, tile_items=tile_items,
                            items_per_thread=items_per_thread)
            saif = sims[r.netlist].saif()
            r.result = saif if keep_results else None
            r.done = time.perf_counter() - t0
        return time.perf_counter() - t0
    finally:
        for s in sims:
            s.close()


class _NoStimulus:
    """An edge-free one-cycle stimulus to open a context before requests."""

    def __init__(self, num_inputs):
        self.num_cycles, self.cycle_ps = 1, 1000
        self.init = np.zeros(num_inputs, np.uint8)
        self.edge_ptr = np.zeros(num_inputs + 1, np.int64)
        self.edge_time = np.zeros(0, np.int32)


def _dummy_stim(wl):
    return _NoStimulus(wl.netlist.num_inputs)


def run_served(netlists, reqs, keep_results=True, **engine_opts):
    """Open-loop stream with continuous batching.  Returns (makespan, stats).
    With ``digest=1`` among the engine options each request also gets its
    per-net waveform digests (read before the request is released)."""
    reqs = sorted(reqs, key=lambda r: r.arrival)
    want_digest = bool(engine_opts.get("digest"))
    with Engine(**engine_opts) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in netlists]
        inflight = {}
        i = 0
        t0 = time.perf_counter()
        while i < len(reqs) or inflight:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                r = reqs[i]
                inflight[eng.submit(ids[r.netlist], r.stim, r.window_cycles, r.edit_gate,
                                    r.edit_delta)] = r
                i += 1
            if inflight:
                eng.step()
            elif i < len(reqs):
                time.sleep(max(0.0, min(reqs[i].arrival - now, 0.0005)))
                continue
            for j in list(inflight):
                r = inflight[j]
                state, saif = eng.poll(j, ids[r.netlist] if keep_results else None)
                if state == JOB_DONE:
                    r.done = time.perf_counter() - t0
                    r.result = saif
                    if want_digest:
                        r.digest = eng.digest(j, ids[r.netlist])
                    eng.release(j)
                    del inflight[j]
                elif state == JOB_FAILED:
                    raise RuntimeError(f"request failed: job {j}")
        makespan = time.perf_counter() - t0
        return makespan, eng.stats()


def run_served_plain(netlists, reqs, keep_results=True, tile_items=256, items_per_thread=4):
    """The same stream, one request at a time on the single-job path, with
    the engine's default launch shape."""
    reqs = sorted(reqs, key=lambda r: r.arrival)
    sims = [Simulator(w.netlist, w.delays, _dummy_stim(w)) for w in netlists]
    try:
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if r.arrival > now:
                time.sleep(r.arrival - now)
            ctx = sims[r.netlist].ctx
            gatspi_set_edit(ctx, r.edit_gate, r.edit_delta)
            gatspi_set_stimulus(ctx, r.stim.num_cycles, r.stim.cycle_ps, r.stim.init, r.stim.edge_ptr,
                                r.stim.edge_time)
            gatspi_simulate(ctx, window_cycles=r.window_cycles, tile_items=tile_items,
                            items_per_thread=items_per_thread)
            saif = sims[r.netlist].saif()
            r.result = saif if keep_results else None
            r.done = time.perf_counter() - t0
        return time.perf_counter() - t0
    finally:
        for s in sims:
            s.close()


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "n": int(lat.size)}
