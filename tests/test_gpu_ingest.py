"""Stimulus ingest on the GPU (gatspi_set_stimulus_events): raw (input,
absolute ps) toggles in any order, restructured per (input, cycle) by the
library's kernels, must give the very stimulus the per-cycle interface
takes.  Checked through simulation results, bit-exact: the digest of every
waveform of every net (input nets included, so the restructured stimulus
itself is compared window by window) and SAIF, against the per-cycle path
and the CPU oracle; and end to end from a VCD file to a SAIF file.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
from oracle import stimulus as ostim
import paper_2203_06117_gb300 as gs
from helpers import parse_saif, write_vcd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _shuffled_events(stim, seed):
    inp, t = ostim.cycles_to_events(stim)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(inp.size)
    return inp[perm], t[perm]


def _digest_saif(sim):
    sim.simulate(window_cycles=1, digest=1, tile_items=256, items_per_thread=4)
    return sim.digest(), sim.saif()


@pytest.mark.parametrize("name,kw", [("tiny", dict()),
                                     ("mid", dict(num_cycles=400, num_gates=20_000, depth=40,
                                                  num_inputs=256))])
def test_events_give_the_per_cycle_stimulus(name, kw):
    wl = gen.make_workload(name, seed=51, **kw)
    st = wl.stim
    inp, t = _shuffled_events(st, 51)
    with gs.Simulator(wl.netlist, wl.delays, st) as sim:
        d_cycles, s_cycles = _digest_saif(sim)
        gs.gatspi_set_stimulus_events(sim.ctx, st.num_cycles, st.cycle_ps, st.init, inp, t)
        d_events, s_events = _digest_saif(sim)
    assert np.array_equal(d_events, d_cycles)
    assert all(np.array_equal(a, b) for a, b in zip(s_events, s_cycles))
    ref = oracle.EventSim(wl.netlist, wl.delays, st, W=1)
    assert all(np.array_equal(a, b) for a, b in zip(s_events, ref.saif()))
    if name == "tiny":
        assert np.array_equal(d_events, odig.digest(ref, range(st.num_cycles)))


def test_benchmark_stimulus_every_window():
    """The 200k-gate workload's whole stimulus (512 inputs x 10,000 cycles)."""
    wl = gen.make_workload("mid", seed=1)
    st = wl.stim
    inp, t = _shuffled_events(st, 52)
    with gs.Simulator(wl.netlist, wl.delays, st) as sim:
        d_cycles, s_cycles = _digest_saif(sim)
        gs.gatspi_set_stimulus_events(sim.ctx, st.num_cycles, st.cycle_ps, st.init, inp, t)
        d_events, s_events = _digest_saif(sim)
    assert np.array_equal(d_events, d_cycles)
    assert all(np.array_equal(a, b) for a, b in zip(s_events, s_cycles))


def test_no_events_and_bad_events():
    wl = gen.make_workload("tiny", seed=53, num_cycles=30)
    st = wl.stim
    I = wl.netlist.num_inputs
    empty = gen.Stimulus(st.num_cycles, st.cycle_ps, st.init, np.zeros(I * st.num_cycles + 1, np.int64),
                         np.zeros(0, np.int32))
    with gs.Simulator(wl.netlist, wl.delays, empty) as sim:
        d0, s0 = _digest_saif(sim)
        gs.gatspi_set_stimulus_events(sim.ctx, st.num_cycles, st.cycle_ps, st.init, np.zeros(0, np.int32),
                                      np.zeros(0, np.int64))
        d1, s1 = _digest_saif(sim)
        assert np.array_equal(d0, d1) and all(np.array_equal(a, b) for a, b in zip(s0, s1))
        inp, t = ostim.cycles_to_events(st)
        C, L = st.num_cycles, st.cycle_ps
        for bi, bt in [(np.r_[inp, I], np.r_[t, 5]), (np.r_[inp, 0], np.r_[t, C * L]),
                       (np.r_[inp, -1], np.r_[t, 0]), (np.r_[inp, inp[0]], np.r_[t, t[0]])]:
            with pytest.raises(gs.GatspiError) as e:
                gs.gatspi_set_stimulus_events(sim.ctx, C, L, st.init, bi, bt)
            assert e.value.code == gs.EINVAL
        with pytest.raises(gs.GatspiError) as e:       # nothing valid is loaded after a failure
            sim.simulate(window_cycles=1)
        assert e.value.code == gs.ESTATE
        gs.gatspi_set_stimulus_events(sim.ctx, C, L, st.init, inp, t)
        d2, _ = _digest_saif(sim)
        ref = oracle.EventSim(wl.netlist, wl.delays, st, W=1)
        assert np.array_equal(d2, odig.digest(ref, range(C)))


def test_vcd_file_to_saif_file(tmp_path):
    wl = gen.make_workload("tiny", seed=54, num_cycles=120)
    st = wl.stim
    I, N = wl.netlist.num_inputs, wl.netlist.num_nets
    in_names = [f"pi{k}" for k in range(I)]
    vcd = os.path.join(tmp_path, "tb.vcd")
    write_vcd(vcd, st, in_names, scope=("tb", "dut"))
    init, ei, et = gs.gatspi_vcd_read(vcd, [f"tb.dut.{n}" for n in in_names])
    with gs.Simulator(wl.netlist, wl.delays, st) as sim:
        gs.gatspi_set_stimulus_events(sim.ctx, st.num_cycles, st.cycle_ps, init, ei, et)
        sim.simulate(window_cycles=1)
        t0, t1, tc = sim.saif()
    net_names = in_names + [f"g{g}" for g in range(N - I)]
    out = os.path.join(tmp_path, "act.saif")
    gs.gatspi_saif_write(out, "dut", st.num_cycles * st.cycle_ps, net_names, t0, t1, tc)
    head, nets = parse_saif(out)
    r0, r1, rc = oracle.EventSim(wl.netlist, wl.delays, st, W=1).saif()
    assert int(head["DURATION"]) == st.num_cycles * st.cycle_ps
    for n, nm in enumerate(net_names):
        assert nets[nm] == (int(r0[n]), int(r1[n]), 0, int(rc[n]), 0), nm


def test_per_cycle_stimulus_is_checked_on_the_device():
    """gatspi_set_stimulus checks its arrays' contents with a kernel: each
    kind of fault is rejected and named with its input and cycle, and a
    valid stimulus loaded afterwards simulates correctly."""
    wl = gen.make_workload("tiny", seed=55, num_cycles=20)
    st = wl.stim
    C, L = st.num_cycles, st.cycle_ps
    counts = np.diff(st.edge_ptr)
    k = int(np.nonzero(counts >= 2)[0][0])        # the first slot with two edges
    a = int(st.edge_ptr[k])
    where = f"input {k // C} cycle {k % C}"
    with gs.Simulator(wl.netlist, wl.delays, st) as sim:
        et = st.edge_time.copy()
        et[a + 1] = et[a]                          # not strictly increasing
        et2 = st.edge_time.copy()
        et2[a] = -1                                # before the cycle
        et3 = st.edge_time.copy()
        et3[a + 1] = L                             # after the cycle
        ep = st.edge_ptr.copy()
        ep[k + 1] = ep[k] - 1 if ep[k] > 0 else ep[k + 2] + 1   # edge_ptr goes back
        for p, t, msg in [(st.edge_ptr, et, where), (st.edge_ptr, et2, where), (st.edge_ptr, et3, where),
                          (ep, st.edge_time, "")]:
            with pytest.raises(gs.GatspiError) as e:
                gs.gatspi_set_stimulus(sim.ctx, C, L, st.init, p, t)
            assert e.value.code == gs.EINVAL and msg in str(e.value), str(e.value)
        gs.gatspi_set_stimulus(sim.ctx, C, L, st.init, st.edge_ptr, st.edge_time)
        sim.simulate(window_cycles=1)
        ref = oracle.EventSim(wl.netlist, wl.delays, st, W=1)
        assert all(np.array_equal(x, y) for x, y in zip(sim.saif(), ref.saif()))
