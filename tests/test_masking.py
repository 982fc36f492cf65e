"""Logically masked windows (CPU).

The propagation kernel settles a (gate, window) without simulating it when
the gate's truth table is constant on every input combination that its
switching pins (the pins with edges in the window) can reach from their
start values, the other pins held.  Algorithm 1 then finds the output value
unchanged at every event, so the window keeps its start value and has no
edge, whatever the arrival times, delays, pulse limits or features.  These
tests check that property on the oracle (both formulations), and the
kernel's column-set construction against plain subset enumeration.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import algo1


def _reachable(col, sw, k):
    """Truth-table columns reachable from col by flipping any subset of the
    pins in sw (plain enumeration)."""
    pins = [i for i in range(k) if (sw >> i) & 1]
    out = set()
    for m in range(1 << len(pins)):
        c = col
        for b, i in enumerate(pins):
            if (m >> b) & 1:
                c ^= 1 << i
        out.add(c)
    return out


def _masked(lut, col, sw, k):
    cols = _reachable(col, sw, k)
    return len({(lut >> c) & 1 for c in cols}) == 1


def _kernel_cube(col, sw):
    """The kernel's construction: each switching pin i doubles the column set
    by its mirror image in bit i."""
    low = [0x5555, 0x3333, 0x0F0F, 0x00FF]
    cube = 1 << col
    for i in range(4):
        if (sw >> i) & 1:
            cube |= ((cube & low[i]) << (1 << i)) | ((cube >> (1 << i)) & low[i])
    return cube


def test_column_set_construction_matches_enumeration():
    for k in range(1, 5):
        for col in range(1 << k):
            for sw in range(1 << k):
                want = sum(1 << c for c in _reachable(col, sw, k))
                assert _kernel_cube(col, sw) == want, (k, col, sw)


def test_masking_test_matches_definition():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(4000):
        k = int(rng.integers(1, 5))
        lut = int(rng.integers(0, 1 << (1 << k)))
        col = int(rng.integers(0, 1 << k))
        sw = int(rng.integers(1, 1 << k))
        cube = _kernel_cube(col, sw)
        hit = lut & cube
        assert (hit == 0 or hit == cube) == _masked(lut, col, sw, k)


def _check_masked_windows(wl, W, **kw):
    """Every masked (gate, window) of the oracle's run has no output edge and
    the truth table's value at the start values.  Returns how many there were."""
    nl = wl.netlist
    I, G = nl.num_inputs, nl.num_gates
    sim = oracle.EventSim(nl, wl.delays, wl.stim, W=W, **kw)
    found = 0
    for w in range(sim.num_windows):
        init, ptr, _ = sim.window(w)
        cnt = np.diff(ptr)
        for g in range(G):
            a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
            nets = [int(x) for x in nl.fanin_net[a:b]]
            col = sum(int(init[n]) << i for i, n in enumerate(nets))
            sw = sum((1 << i) for i, n in enumerate(nets) if cnt[n] > 0)
            if sw and _masked(int(nl.lut[g]), col, sw, b - a):
                found += 1
                assert cnt[I + g] == 0, (g, w)
                assert int(init[I + g]) == (int(nl.lut[g]) >> col) & 1, (g, w)
    return found


@pytest.mark.parametrize("pulse", [(100, 100), (0, 0), (30, 60)], ids=["g100w100", "g0w0", "g30w60"])
def test_masked_windows_keep_their_start_value(pulse):
    found = 0
    for s in range(300):
        wl = gen.random_small(60_000 + s)
        found += _check_masked_windows(wl, 1 + s % 2, pulse_gate=pulse[0], pulse_wire=pulse[1])
    assert found > 100  # the property was exercised


@pytest.mark.parametrize("wire_filter,full_sdf", [(False, True), (True, False)])
def test_masked_windows_keep_their_start_value_reduced_features(wire_filter, full_sdf):
    found = 0
    for s in range(200):
        wl = gen.random_small(61_000 + s)
        found += _check_masked_windows(wl, 1, interconnect_filter=wire_filter, full_sdf=full_sdf)
    assert found > 50


def test_masked_windows_in_algorithm1():
    # the second formulation agrees window by window (it shares nothing with
    # the event-driven simulator)
    found = 0
    for s in range(150):
        wl = gen.random_small(62_000 + s)
        nl = wl.netlist
        I, G = nl.num_inputs, nl.num_gates
        for w in range(wl.stim.num_cycles):
            waves = algo1.simulate_window(nl, wl.delays, wl.stim, w, 1)
            for g in range(G):
                a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
                fan = [waves[int(x)] for x in nl.fanin_net[a:b]]
                col = sum(v << i for i, (v, _) in enumerate(fan))
                sw = sum(1 << i for i, (_, t) in enumerate(fan) if t)
                if sw and _masked(int(nl.lut[g]), col, sw, b - a):
                    found += 1
                    assert waves[I + g] == ((int(nl.lut[g]) >> col) & 1, [])
    assert found > 50
