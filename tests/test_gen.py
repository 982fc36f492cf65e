"""The seeded input generator: determinism, shapes and the recipe rules."""
import numpy as np
import pytest

import gen


def _levels(nl):
    lv = np.zeros(nl.num_nets, np.int32)
    for g in range(nl.num_gates):
        a, b = nl.fanin_ptr[g], nl.fanin_ptr[g + 1]
        lv[nl.num_inputs + g] = 1 + lv[nl.fanin_net[a:b]].max()
    return lv


@pytest.mark.parametrize("name", ["tiny", "mid", "large"])
def test_deterministic_and_seed_sensitive(name):
    kw = dict(num_cycles=5) if name == "tiny" else dict(num_cycles=3, num_gates=3000, depth=30,
                                                         num_inputs=64)
    a = gen.make_workload(name, seed=4, **kw)
    b = gen.make_workload(name, seed=4, **kw)
    c = gen.make_workload(name, seed=5, **kw)
    for x, y in [(a.netlist.fanin_net, b.netlist.fanin_net), (a.delays.gate_delay, b.delays.gate_delay),
                 (a.stim.edge_time, b.stim.edge_time), (a.stim.edge_ptr, b.stim.edge_ptr)]:
        assert np.array_equal(x, y)
    assert not np.array_equal(a.stim.edge_ptr, c.stim.edge_ptr)


def test_tiny_recipe_shape():
    wl = gen.make_workload("tiny", seed=1)
    nl = wl.netlist
    assert (nl.num_inputs, nl.num_gates, wl.stim.num_cycles, wl.stim.cycle_ps) == (64, 2000, 1000, 1000)
    lv = _levels(nl)
    # pin 1 always comes from the previous level: exact depth, G/D per level
    assert lv.max() == 20
    assert np.all(np.bincount(lv[64:])[1:] == 100)
    gates = np.repeat(np.arange(nl.num_gates), np.diff(nl.fanin_ptr))
    assert np.all(nl.fanin_net < nl.num_inputs + gates)
    # no net twice on one gate
    for g in range(nl.num_gates):
        f = nl.fanin_net[nl.fanin_ptr[g]:nl.fanin_ptr[g + 1]]
        assert len(set(f.tolist())) == f.size
    # delays within the recipe's ranges on used columns
    gd = wl.delays.gate_delay.reshape(-1, 2, 2, 8)
    n = np.repeat(np.diff(nl.fanin_ptr), np.diff(nl.fanin_ptr))
    for k in (1, 2, 3):
        used = gd[n == k][..., :1 << (k - 1)]
        assert used.min() >= 5 and used.max() <= 50
    assert wl.delays.wire_delay.min() >= 1 and wl.delays.wire_delay.max() <= 5


def test_stimulus_rules():
    wl = gen.make_workload("tiny", seed=2)
    st = wl.stim
    E = st.edge_time
    assert E.min() >= 0 and E.max() < 240
    seg = np.diff(st.edge_ptr)
    assert seg.max() <= 3
    # strictly increasing inside each (input, cycle)
    starts = st.edge_ptr[:-1][seg >= 2]
    for s, k in zip(starts.tolist(), seg[seg >= 2].tolist()):
        assert np.all(np.diff(E[s:s + k]) > 0)
    # toggle rate near p = 0.2 plus pulses
    assert 0.2 < seg.mean() < 0.35


def test_mid_conditional_arcs_only_on_xor_mux():
    wl = gen.make_workload("mid", seed=1, num_gates=4000, depth=40, num_cycles=2, num_inputs=64)
    nl = wl.netlist
    gd = wl.delays.gate_delay.reshape(-1, 2, 2, 8)
    cell = np.repeat(nl.cell, np.diff(nl.fanin_ptr))
    n = np.repeat(np.diff(nl.fanin_ptr), np.diff(nl.fanin_ptr))
    xor_mux = np.isin(cell, [gen.CELL_NAMES.index("XOR2"), gen.CELL_NAMES.index("MUX2")])
    # non-conditional arcs repeat one value per output edge
    for p in np.nonzero(~xor_mux)[0][:2000]:
        k = 1 << (n[p] - 1)
        for oe in range(2):
            assert len(set(gd[p, :, oe, :k].reshape(-1).tolist())) == 1
    assert xor_mux.sum() > 0
    assert nl.num_pins.max() == 4


def test_cell_truth_tables():
    assert gen.cell_lut("INV") == 0b01
    assert gen.cell_lut("NAND2") == 0b0111
    assert gen.cell_lut("XOR2") == 0b0110
    # MUX2 (A, B, S): S ? B : A
    for col in range(8):
        a, b, s = col & 1, (col >> 1) & 1, (col >> 2) & 1
        assert (gen.cell_lut("MUX2") >> col) & 1 == (b if s else a)
    for col in range(16):
        a1, a2, b1, b2 = [(col >> k) & 1 for k in range(4)]
        assert (gen.cell_lut("AOI22") >> col) & 1 == int(not ((a1 and a2) or (b1 and b2)))
        assert (gen.cell_lut("OAI22") >> col) & 1 == int(not ((a1 or a2) and (b1 or b2)))


def test_depth_interpolation():
    assert gen.interp_depth(2000) == 20
    assert gen.interp_depth(200_000) == 60
    assert gen.interp_depth(2_000_000) == 120
