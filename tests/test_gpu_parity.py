"""Parity of the CUDA path with the CPU oracle, through the C interface.

Integer event work: every comparison is bit-exact (waveform start values,
edge times, SAIF T0/T1/TC).  Sizes run from single gates to the full
benchmark configurations; at full size the oracle recomputes sampled
windows one by one and the rest is checked through properties that hold at
any size.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2203_06117_gb300 as gs
from cases import case_workload, load_hand_traced
from helpers import assert_saif_equal, assert_window_equal

pytestmark = pytest.mark.gpu

CASES = load_hand_traced()


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_traced(case):
    wl = case_workload(case)
    pulse = (case["pulse"]["gate"], case["pulse"]["wire"]) if "pulse" in case else None
    f = case.get("features", {})
    features = (0 if f.get("interconnect_filter", True) else gs.NO_INTERCONNECT_FILTER) | \
               (0 if f.get("full_sdf", True) else gs.PARTIAL_SDF)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=case["W"], pulse=pulse, features=features)
        for e in case["expect"]:
            init, ptr, times = sim.window(e["window"])
            n = e["net"]
            assert int(init[n]) == e["init"]
            assert times[ptr[n]:ptr[n + 1]].tolist() == e["times"]
        t0, t1, tc = sim.saif()
        for s in case["saif"]:
            n = s["net"]
            assert (int(t0[n]), int(t1[n]), int(tc[n])) == (s["T0"], s["T1"], s["TC"])


@pytest.mark.parametrize("block", range(4))
def test_random_small_circuits(block):
    for s in range(block * 60, block * 60 + 60):
        wl = gen.random_small(10_000 + s, max_cycles=5)
        W = 1 + s % 3
        ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W)
        with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
            sim.simulate(window_cycles=W, tile_items=(128, 256, 512)[s % 3])
            for w in range(ref.num_windows):
                assert_window_equal(sim, ref, w, f"case {s}")
            assert_saif_equal(sim, ref)


def test_tiny_config_full():
    """2,000 gates x 1,000 cycles: every window of every net."""
    wl = gen.make_workload("tiny", seed=1)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1)
        st = sim.stats()
        assert st["batches"] == 1 and st["windows"] == 1000
        for w in range(1000):
            assert_window_equal(sim, ref, w)
        assert_saif_equal(sim, ref)
        assert st["edges"] == int(sim.saif()[2].sum())


@pytest.mark.parametrize("W,batch", [(4, 0), (1, 96), (3, 7)])
def test_windows_and_batches(W, batch):
    """Multi-cycle windows, a ragged last window, several device batches."""
    wl = gen.make_workload("tiny", seed=2, num_cycles=301)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=W, batch_windows=batch)
        assert_saif_equal(sim, ref)
        st = sim.stats()
        last0 = (st["batches"] - 1) * st["batch_windows"]
        for w in range(last0, ref.num_windows):
            assert_window_equal(sim, ref, w)


def test_mid_recipe_reduced_full():
    """The mid recipe (4-input cells, COND on XOR2/MUX2, narrow pulses) at
    20k gates x 300 cycles: every window."""
    wl = gen.make_workload("mid", seed=3, num_gates=20_000, depth=40, num_inputs=256, num_cycles=300)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate()
        for w in range(300):
            assert_window_equal(sim, ref, w)
        assert_saif_equal(sim, ref)


def test_large_recipe_reduced_full():
    """The large recipe (Zipf fanout, 10% COND, high activity) reduced."""
    wl = gen.make_workload("large", seed=4, num_gates=30_000, depth=60, num_inputs=400, num_cycles=120)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(batch_windows=50)
        assert_saif_equal(sim, ref)
        for w in range(100, 120):
            assert_window_equal(sim, ref, w)


def test_gates_out_of_level_order():
    """Gates given in an order that is topological but not sorted by level:
    the library levelizes and reports results in the caller's numbering."""
    wl = gen.make_workload("tiny", seed=6, num_cycles=40)
    nl = wl.netlist
    I, G = nl.num_inputs, nl.num_gates
    # interleave levels: a valid topological order that is not level-sorted
    rng = np.random.Generator(np.random.PCG64(0))
    order = list(range(G))
    for _ in range(4 * G):
        a = int(rng.integers(0, G - 1))
        g1, g2 = order[a], order[a + 1]
        f2 = nl.fanin_net[nl.fanin_ptr[g2]:nl.fanin_ptr[g2 + 1]]
        if (I + g1) not in f2:
            order[a], order[a + 1] = g2, g1
    new_id = {g: k for k, g in enumerate(order)}
    remap = lambda n: n if n < I else I + new_id[n - I]
    fp, fn, lut, gd, wd = [0], [], [], [], []
    for g in order:
        a, b = nl.fanin_ptr[g], nl.fanin_ptr[g + 1]
        fn += [remap(int(x)) for x in nl.fanin_net[a:b]]
        fp.append(len(fn))
        lut.append(nl.lut[g])
        gd.append(wl.delays.gate_delay[32 * a:32 * b])
        wd.append(wl.delays.wire_delay[2 * a:2 * b])
    nl2 = gen.Netlist(I, np.asarray(fp, np.int32), np.asarray(fn, np.int32), np.diff(fp).astype(np.uint8),
                      np.asarray(lut, np.uint16))
    dl2 = gen.Delays(np.concatenate(gd), np.concatenate(wd))
    ref = oracle.EventSim(nl2, dl2, wl.stim, W=1)
    with gs.Simulator(nl2, dl2, wl.stim) as sim:
        sim.simulate()
        assert_saif_equal(sim, ref)
        for w in (0, 17, 39):
            assert_window_equal(sim, ref, w)


def test_degenerate_inputs():
    # no gates at all
    nl = gen.Netlist(3, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                     np.zeros(0, np.uint16))
    dl = gen.Delays(np.zeros(0, np.int32), np.zeros(0, np.int32))
    st = gen.Stimulus(2, 100, np.array([0, 1, 0], np.uint8), np.array([0, 2, 2, 3, 3, 3, 3], np.int64),
                      np.array([5, 50, 7], np.int32))
    ref = oracle.EventSim(nl, dl, st, W=1)
    with gs.Simulator(nl, dl, st) as sim:
        sim.simulate()
        assert_saif_equal(sim, ref)
        assert_window_equal(sim, ref, 0)
    # no stimulus edges at all: nothing moves, every net keeps its settled value
    wl = gen.make_workload("tiny", seed=1, num_cycles=5)
    st0 = gen.Stimulus(5, 1000, wl.stim.init, np.zeros(64 * 5 + 1, np.int64), np.zeros(0, np.int32))
    ref = oracle.EventSim(wl.netlist, wl.delays, st0, W=1)
    with gs.Simulator(wl.netlist, wl.delays, st0) as sim:
        sim.simulate()
        assert_saif_equal(sim, ref)
        assert sim.stats()["edges"] == 0


def test_small_arena_retries_then_matches():
    """An arena too small for all windows: the library shrinks the batch
    and still produces the oracle's SAIF; an arena too small for one window
    is reported as ECAPACITY."""
    wl = gen.make_workload("tiny", seed=8, num_cycles=200)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim, arena_bytes=1 << 20) as sim:
        sim.simulate()
        assert sim.stats()["batches"] > 1
        assert_saif_equal(sim, ref)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim, arena_bytes=12 << 10) as sim:
        with pytest.raises(gs.GatspiError) as e:
            sim.simulate()
        assert e.value.code == gs.ECAPACITY


def test_invalid_arguments_are_rejected():
    wl = gen.make_workload("tiny", seed=1, num_cycles=3)
    nl = wl.netlist
    ctx = gs.gatspi_create(0)
    try:
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_simulate(ctx)
        assert e.value.code == gs.ESTATE
        bad = nl.fanin_net.copy()
        bad[-1] = nl.num_nets - 1          # a gate reading its own output
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_load_netlist(ctx, nl.num_inputs, nl.fanin_ptr, bad, nl.lut)
        assert e.value.code == gs.EINVAL
        gs.gatspi_load_netlist(ctx, nl.num_inputs, nl.fanin_ptr, nl.fanin_net, nl.lut)
        gd = wl.delays.gate_delay.copy()
        gd[0] = 0                          # delays must be >= 1 ps
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_load_delays(ctx, gd, wl.delays.wire_delay)
        assert e.value.code == gs.EINVAL
        gs.gatspi_load_delays(ctx, wl.delays.gate_delay, wl.delays.wire_delay)
        st = wl.stim
        et = st.edge_time.copy()
        et[0] = st.cycle_ps                # outside the cycle
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_set_stimulus(ctx, st.num_cycles, st.cycle_ps, st.init, st.edge_ptr, et)
        assert e.value.code == gs.EINVAL
        gs.gatspi_set_stimulus(ctx, st.num_cycles, st.cycle_ps, st.init, st.edge_ptr, st.edge_time)
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_simulate(ctx, tile_items=100)
        assert e.value.code == gs.EINVAL
        gs.gatspi_simulate(ctx)
        with pytest.raises(gs.GatspiError) as e:
            gs.gatspi_read_window(ctx, 5, nl.num_nets)
        assert e.value.code == gs.ESTATE
    finally:
        gs.gatspi_destroy(ctx)


def _sampled_windows(wl, sim, windows, W=1):
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W)
    for w in windows:
        assert_window_equal(sim, ref, w)


def _saif_properties(wl, sim):
    t0, t1, tc = sim.saif()
    total = wl.stim.num_cycles * wl.stim.cycle_ps
    assert np.all(t0 + t1 == total)
    assert np.all(t0 >= 0) and np.all(t1 >= 0) and np.all(tc >= 0)
    assert int(tc.sum()) == sim.stats()["edges"]
    # inputs: TC and T1 straight from the stimulus
    I, C = wl.netlist.num_inputs, wl.stim.num_cycles
    ptr = wl.stim.edge_ptr
    assert np.array_equal(tc[:I], ptr[np.arange(1, I + 1) * C] - ptr[np.arange(I) * C])


def test_mid_config_full_size():
    """200k gates x 10,000 cycles in the benchmark's launch configuration:
    sampled windows against the oracle, SAIF through invariants."""
    wl = gen.make_workload("mid", seed=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, time_kernels=1)
        assert sim.stats()["batches"] == 1
        _saif_properties(wl, sim)
        _sampled_windows(wl, sim, [0, 1, 4999, 9998, 9999])


def test_large_config_full_size():
    """2M gates x 20,000 cycles in 2,000-cycle device batches: the last
    batch's sampled windows against the oracle, SAIF through invariants."""
    wl = gen.make_workload("large", seed=1)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, batch_windows=2000)
        st = sim.stats()
        assert st["batches"] == 10
        _saif_properties(wl, sim)
        _sampled_windows(wl, sim, [18000, 19999])


def test_delay_edit_on_plain_path():
    """A request-scoped delay edit (every delay of 1% of gates shifted by
    +-10..50 ps, clamped at 1 ps) equals the oracle on the edited table;
    clearing it restores the unedited result."""
    wl = gen.make_workload("mid", seed=9, num_gates=5000, depth=30, num_inputs=80, num_cycles=60)
    nl = wl.netlist
    rng = np.random.Generator(np.random.PCG64(2))
    gates = rng.choice(nl.num_gates, size=50, replace=False)
    deltas = rng.choice([-1, 1], size=50) * rng.integers(10, 51, size=50)
    gd = wl.delays.gate_delay.copy().reshape(-1, 2, 2, 8)
    for g, d in zip(gates, deltas):
        a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
        ncol = 1 << (b - a - 1)
        gd[a:b, :, :, :ncol] = np.maximum(1, gd[a:b, :, :, :ncol] + int(d))
    edited = gen.Delays(gd.reshape(-1), wl.delays.wire_delay)
    with gs.Simulator(nl, wl.delays, wl.stim) as sim:
        gs.gatspi_set_edit(sim.ctx, gates, deltas)
        sim.simulate()
        assert_saif_equal(sim, oracle.EventSim(nl, edited, wl.stim, W=1))
        assert_window_equal(sim, oracle.EventSim(nl, edited, wl.stim, W=1), 59)
        gs.gatspi_set_edit(sim.ctx)
        sim.simulate()
        assert_saif_equal(sim, oracle.EventSim(nl, wl.delays, wl.stim, W=1))
