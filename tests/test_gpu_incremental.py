"""Re-simulation after a delay edit (gatspi_resimulate_edit): the glitch-
optimization loop of Section 4 -- simulate, re-time some cells, simulate
again -- running only the fanout cone of the re-timed gates.

Every result is compared bit-exactly with the CPU oracle on the edited
delays and with a full GPU simulation of the same edit: SAIF on every net,
the per-net digest of every waveform, and the resident waveforms of sampled
windows.  Edits follow one another (each replaces the last, so a gate left
out of the next edit reverts), and the paths that fall back to a full run
(several batches, too little free arena) are checked the same way.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs
from helpers import assert_saif_equal, assert_window_equal, edited_delays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _ext_gates_at_levels(wl, levels, rng):
    """Caller-numbered gates drawn from the given logic levels."""
    nl = wl.netlist
    lvl = np.zeros(nl.num_nets, np.int64)
    for g in range(nl.num_gates):
        a, b = nl.fanin_ptr[g], nl.fanin_ptr[g + 1]
        lvl[nl.num_inputs + g] = 1 + lvl[nl.fanin_net[a:b]].max()
    out = []
    for L in levels:
        cand = np.nonzero(lvl[nl.num_inputs:] == L)[0]
        out.append(int(rng.choice(cand)))
    return out


def _check_against_full_and_oracle(sim, wl, gates, deltas, windows, pulse=(100, 100), full_opts=None):
    dl = edited_delays(wl.netlist, wl.delays, gates, deltas) if gates else wl.delays
    ref = oracle.EventSim(wl.netlist, dl, wl.stim, W=1, pulse_gate=pulse[0], pulse_wire=pulse[1])
    assert_saif_equal(sim, ref)
    for w in windows:
        assert_window_equal(sim, ref, w, f"edit {list(zip(gates, deltas))}")
    got = sim.digest()
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as full:
        if gates:
            gs.gatspi_set_edit(full.ctx, gates, deltas)
        full.simulate(window_cycles=1, digest=1, pulse=None if pulse == (100, 100) else pulse,
                      **(full_opts or {}))
        assert np.array_equal(got, full.digest())
        assert all(np.array_equal(a, b) for a, b in zip(sim.saif(), full.saif()))
    return ref


def test_cone_edits_in_a_row_tiny():
    wl = gen.make_workload("tiny", seed=41, num_cycles=300)
    rng = np.random.Generator(np.random.PCG64(41))
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1, tile_items=256, items_per_thread=4)
        G = wl.netlist.num_gates
        steps = [
            (_ext_gates_at_levels(wl, [12], rng), [37]),             # one deep gate: a small cone
            (_ext_gates_at_levels(wl, [3, 15], rng), [-20, 45]),     # the first gate reverts
            (_ext_gates_at_levels(wl, [1], rng), [50]),              # a shallow gate: a wide cone
            ([], []),                                                # clear the edit: all revert
        ]
        for gates, deltas in steps:
            info = sim.resimulate_edit(gates, deltas)
            assert info["mode"] == 1, info
            assert 0 < info["cone_gates"] <= G
            ref = _check_against_full_and_oracle(sim, wl, gates, deltas, windows=range(0, 300, 11))
            # the digest also matches the oracle's own waveforms
            assert np.array_equal(sim.digest(), odig.digest(ref, range(300)))
        info = sim.resimulate_edit([], [])                         # the same (empty) edit again
        assert info["mode"] == 0


def test_deep_edit_runs_a_small_cone_mid_recipe():
    wl = gen.make_workload("mid", seed=42, num_gates=20_000, depth=40, num_inputs=256, num_cycles=256)
    rng = np.random.Generator(np.random.PCG64(42))
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1)
        gates = _ext_gates_at_levels(wl, [36, 38, 39], rng)
        info = sim.resimulate_edit(gates, [-30, 25, 40])
        assert info["mode"] == 1 and info["first_level"] >= 36
        assert info["cone_gates"] < wl.netlist.num_gates // 10
        assert sim.stats()["items"] == info["items"]
        _check_against_full_and_oracle(sim, wl, gates, [-30, 25, 40], windows=range(0, 256, 17))
        gates2 = _ext_gates_at_levels(wl, [5, 20], rng)
        info = sim.resimulate_edit(gates2, [15, -15])
        assert info["mode"] == 1 and info["first_level"] <= 20
        _check_against_full_and_oracle(sim, wl, gates2, [15, -15], windows=range(3, 256, 29))


def test_pulse_limits_carry_over():
    wl = gen.make_workload("tiny", seed=43, num_cycles=128)
    rng = np.random.Generator(np.random.PCG64(43))
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1, pulse=(0, 40))
        gates = _ext_gates_at_levels(wl, [8, 10], rng)
        info = sim.resimulate_edit(gates, [30, -10])
        assert info["mode"] == 1
        _check_against_full_and_oracle(sim, wl, gates, [30, -10], windows=range(0, 128, 9), pulse=(0, 40))


def test_falls_back_to_a_full_run_with_several_batches():
    wl = gen.make_workload("tiny", seed=44, num_cycles=300)
    rng = np.random.Generator(np.random.PCG64(44))
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1, batch_windows=100, tile_items=256, items_per_thread=4)
        gates = _ext_gates_at_levels(wl, [10], rng)
        info = sim.resimulate_edit(gates, [33])
        assert info["mode"] == 2
        st = sim.stats()
        assert st["batches"] == 3
        last = range(200, 300, 7)                                  # the resident (last) batch
        _check_against_full_and_oracle(sim, wl, gates, [33], windows=last,
                                       full_opts=dict(batch_windows=100, tile_items=256, items_per_thread=4))


def test_falls_back_to_a_full_run_without_free_arena():
    wl = gen.make_workload("tiny", seed=45, num_cycles=200)
    rng = np.random.Generator(np.random.PCG64(45))
    # an arena just large enough for the batch: the cone's new runs do not fit
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as probe:
        probe.simulate(window_cycles=1, tile_items=256, items_per_thread=4)
        edges = probe.stats()["edges"]
    N = wl.netlist.num_nets
    fixed = N * 2 * 8 + N * 200 * 2 + 64 * 1024
    with gs.Simulator(wl.netlist, wl.delays, wl.stim, arena_bytes=fixed + 4 * (edges + edges * 3 // 10)) as sim:
        sim.simulate(window_cycles=1, digest=1, tile_items=256, items_per_thread=4)
        if sim.stats()["batches"] != 1:
            pytest.skip("the arena estimate split the batch")
        gates = _ext_gates_at_levels(wl, [1, 2], rng)
        info = sim.resimulate_edit(gates, [40, 40])
        assert info["mode"] == 2
        _check_against_full_and_oracle(sim, wl, gates, [40, 40], windows=range(0, 200, 13))


def test_falls_back_to_a_full_run_after_a_new_stimulus():
    wl = gen.make_workload("tiny", seed=47, num_cycles=150)
    wl2 = gen.make_workload("tiny", seed=48, num_cycles=150)
    rng = np.random.Generator(np.random.PCG64(47))
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1)
        st = wl2.stim                                   # same netlist, another stimulus
        gs.gatspi_set_stimulus(sim.ctx, st.num_cycles, st.cycle_ps, st.init, st.edge_ptr, st.edge_time)
        gates = _ext_gates_at_levels(wl, [9], rng)
        info = sim.resimulate_edit(gates, [21])
        assert info["mode"] == 2
        wl_new = gen.Workload(wl.name, wl.netlist, wl.delays, st, 0, {})
        _check_against_full_and_oracle(sim, wl_new, gates, [21], windows=range(0, 150, 10))
        info = sim.resimulate_edit(gates, [21])         # the same edit again: nothing to do
        assert info["mode"] == 0


def test_resimulate_needs_a_simulation_and_valid_edits():
    wl = gen.make_workload("tiny", seed=46, num_cycles=70)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        with pytest.raises(gs.GatspiError) as e:
            sim.resimulate_edit([1], [5])
        assert e.value.code == gs.ESTATE
        sim.simulate(window_cycles=1)
        with pytest.raises(gs.GatspiError) as e:
            sim.resimulate_edit([wl.netlist.num_gates], [5])
        assert e.value.code == gs.EINVAL
