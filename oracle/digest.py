"""ORACLE -- test infrastructure: per-net waveform digests.

A check of bit-exactness at scale, where comparing every waveform one by
one would not fit in memory: each net's waveforms over all windows reduce
to one 64-bit number.  For net n and window w (global index) with start
value v and edge times t_1..t_c:

    h = mix(v + 1)
    h = mix(h + 0x9E3779B97F4A7C15 + t_k)        for k = 1..c
    digest[n] = sum over windows of mix(h ^ mix(w + 1))   (mod 2^64)

``mix`` is the output function of SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  The sum
does not depend on the order of the windows.  This module computes it from
the event-driven oracle's waveforms with numpy (arithmetic mod 2^64) and
shares no code with the GPU library, which computes the same definition in
its own kernel.
"""
from __future__ import annotations

import numpy as np

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, elementwise on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def window_terms(init: np.ndarray, ptr: np.ndarray, times: np.ndarray, w: int) -> np.ndarray:
    """Per-net digest terms of one window's waveforms (init[N], ptr[N+1],
    times as returned by the oracle's ``EventSim.window``)."""
    init = np.asarray(init, dtype=np.uint64)
    ptr = np.asarray(ptr, dtype=np.int64)
    t = np.asarray(times, dtype=np.int64).astype(np.uint32).astype(np.uint64)
    cnt = np.diff(ptr)
    with np.errstate(over="ignore"):
        h = mix(init + np.uint64(1))
        for k in range(int(cnt.max()) if cnt.size else 0):
            sel = np.nonzero(cnt > k)[0]
            h[sel] = mix(h[sel] + _GAMMA + t[ptr[sel] + k])
        return mix(h ^ mix(np.array([w + 1], dtype=np.uint64)))


def digest(sim, windows) -> np.ndarray:
    """Sum (mod 2^64) of the digest terms over the given windows of an
    oracle ``EventSim``."""
    acc = np.zeros(sim.N, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for w in windows:
            init, ptr, times = sim.window(int(w))
            acc += window_terms(init, ptr, times, int(w))
    return acc


def workload_digest(recipe: str, seed: int, num_cycles: int | None, windows) -> np.ndarray:
    """Digest over the given windows of a generator recipe's workload (one
    cycle per window), simulated by the event-driven oracle.  Self-contained
    so that it can run in a spawned worker process."""
    import gen
    from . import EventSim
    wl = gen.make_workload(recipe, seed=seed, num_cycles=num_cycles)
    return digest(EventSim(wl.netlist, wl.delays, wl.stim, W=1), windows)


def workload_digest_parallel(recipe: str, seed: int, num_cycles: int, procs: int) -> np.ndarray:
    """All windows of a recipe's workload, split over ``procs`` spawned
    processes (strided windows); the per-process sums add mod 2^64."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    parts = [list(range(k, num_cycles, procs)) for k in range(procs)]
    with ctx.Pool(procs) as pool:
        res = pool.starmap(workload_digest, [(recipe, seed, num_cycles, p) for p in parts])
    acc = np.zeros_like(res[0])
    with np.errstate(over="ignore"):
        for r in res:
            acc += r
    return acc
