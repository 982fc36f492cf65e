"""Repeated simulations replay the batch from a CUDA graph.

The first simulation of a batch runs eagerly, the second captures the
batch's launches into a graph and later ones replay it while nothing the
graph bakes in has changed.  Every run must give the oracle's results, and
a new stimulus or delay edit must not replay a stale graph.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _ref(wl):
    o = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    return o.saif(), odig.digest(o, range(wl.stim.num_cycles))


def test_replayed_runs_match_the_oracle_and_follow_new_inputs():
    a = gen.make_workload("tiny", seed=11, num_cycles=150)
    b = gen.make_workload("tiny", seed=11, num_cycles=150)
    b_stim = gen.make_workload("tiny", seed=12, num_cycles=150).stim  # same netlist, other stimulus
    (a_saif, a_dig) = _ref(a)
    ob = oracle.EventSim(b.netlist, b.delays, b_stim, W=1)
    b_saif, b_dig = ob.saif(), odig.digest(ob, range(150))
    with gs.Simulator(a.netlist, a.delays, a.stim) as sim:
        for run in range(4):                      # eager, capture, replay, replay
            sim.simulate(window_cycles=1, tile_items=256, items_per_thread=4, digest=1, time_kernels=run % 2)
            got = sim.saif()
            assert all(np.array_equal(x, y) for x, y in zip(got, a_saif)), f"run {run}: SAIF"
            assert np.array_equal(sim.digest(), a_dig), f"run {run}: waveforms"
        # a new stimulus: the cached graph must not be replayed
        gs.gatspi_set_stimulus(sim.ctx, b_stim.num_cycles, b_stim.cycle_ps, b_stim.init, b_stim.edge_ptr,
                               b_stim.edge_time)
        for run in range(3):
            sim.simulate(window_cycles=1, tile_items=256, items_per_thread=4, digest=1)
            assert all(np.array_equal(x, y) for x, y in zip(sim.saif(), b_saif)), f"new stimulus run {run}"
            assert np.array_equal(sim.digest(), b_dig), f"new stimulus run {run}: waveforms"


def test_replay_after_a_delay_edit():
    wl = gen.make_workload("tiny", seed=13, num_cycles=120)
    nl = wl.netlist
    gates = np.arange(0, nl.num_gates, 37, dtype=np.int32)
    deltas = ((gates % 5) * 7 - 10).astype(np.int32)
    gd = wl.delays.gate_delay.copy().reshape(-1, 2, 2, 8)
    for g, dlt in zip(gates, deltas):     # the oracle gets the edit folded into the delay table
        a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
        ncol = 1 << (b - a - 1)
        gd[a:b, :, :, :ncol] = np.maximum(1, gd[a:b, :, :, :ncol] + int(dlt))
    edited = gen.Delays(gd.reshape(-1), wl.delays.wire_delay)
    ref = oracle.EventSim(nl, edited, wl.stim, W=1).saif()
    with gs.Simulator(nl, wl.delays, wl.stim) as sim:
        for run in range(3):
            sim.simulate(window_cycles=1, tile_items=256, items_per_thread=4)
        gs.gatspi_set_edit(sim.ctx, gates, deltas)
        for run in range(3):
            sim.simulate(window_cycles=1, tile_items=256, items_per_thread=4)
            assert all(np.array_equal(x, y) for x, y in zip(sim.saif(), ref)), f"edited run {run}"
