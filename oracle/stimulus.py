"""ORACLE -- test infrastructure only (tests, smoke check, CPU baseline).

Restructuring of a raw input stimulus into the layout the re-simulator
takes.  A waveform dump gives each input's changes as (input, absolute
time) toggles; cycle-parallel re-simulation needs them grouped per (input,
cycle), in time order, with times relative to the cycle start (Section 3:
the input waveforms are re-structured to match the cycle-parallelism
schema; Section 4 counts this step in the application time).

Plain numpy: a lexicographic sort by (input, time) and a histogram of
(input, cycle) buckets.  Parity status: pinned by round trips with the
generator's per-cycle stimuli and by brute-force grouping on small cases
(tests/test_stimulus_io.py).
"""
from __future__ import annotations

import numpy as np


def events_to_cycles(num_inputs: int, num_cycles: int, cycle_ps: int, ev_input, ev_time):
    """(input, absolute ps) toggles in any order -> (edge_ptr int64[I*C+1],
    edge_time int32[]) with the toggles of input i in cycle c at
    edge_time[edge_ptr[i*C + c] : edge_ptr[i*C + c + 1]], strictly
    increasing, relative to the cycle start.  Raises ValueError on an input
    id out of range, a time outside [0, C*L) or two toggles of one input at
    the same time."""
    I, C, L = int(num_inputs), int(num_cycles), int(cycle_ps)
    inp = np.asarray(ev_input, np.int64)
    t = np.asarray(ev_time, np.int64)
    if inp.shape != t.shape:
        raise ValueError("event arrays differ in length")
    if inp.size and (inp.min() < 0 or inp.max() >= I):
        raise ValueError("event input id out of range")
    if t.size and (t.min() < 0 or t.max() >= C * L):
        raise ValueError("event time outside the stimulus")
    order = np.lexsort((t, inp))            # by input, then by time
    inp, t = inp[order], t[order]
    if np.any((inp[1:] == inp[:-1]) & (t[1:] == t[:-1])):
        raise ValueError("an input toggles twice at the same time")
    cyc = t // L
    counts = np.bincount(inp * C + cyc, minlength=I * C)
    edge_ptr = np.zeros(I * C + 1, np.int64)
    np.cumsum(counts, out=edge_ptr[1:])
    return edge_ptr, (t - cyc * L).astype(np.int32)


def cycles_to_events(stim):
    """The inverse: a per-cycle stimulus as (input int32[], absolute ps
    int64[]) toggles, input-major, in time order."""
    I = stim.init.shape[0]
    C, L = stim.num_cycles, stim.cycle_ps
    counts = np.diff(stim.edge_ptr)
    bucket = np.repeat(np.arange(I * C, dtype=np.int64), counts)
    inp = (bucket // C).astype(np.int32)
    t = (bucket % C) * L + stim.edge_time.astype(np.int64)
    return inp, t
