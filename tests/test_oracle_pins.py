"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, not against the oracle itself.

* hand-traced single-gate cases (``golden/hand_traced.json``), each derived
  step by step from Algorithm 1;
* settled values: the last value of every net in a window equals the
  zero-delay truth-table evaluation of the inputs' final values (filters
  drop edges in pairs, so they never change a settled value);
* SAIF invariants: T0 + T1 = simulated time, TC parity = start/end change,
  strictly increasing times;
* closed forms: a BUF/INV chain with wide pulses shifts every edge by the
  sum of its delays; pulses narrower than every wire delay never pass;
* the event-driven simulator and the Algorithm 1 formulation agree on
  thousands of random tiny circuits;
* every planted mistake in the event simulator is caught by the pins above
  (not counting the cross-check);
* pulse limits other than 100 percent (PATHPULSEPERCENT, Section 3): the
  hand-traced cases that carry a 'pulse' entry, settled values and
  invariants at several limits, a transport-delay chain whose narrow pulses
  all pass shifted by the path delay (closed form), and the two
  formulations agreeing on random circuits at random limits.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import algo1
from cases import case_workload, load_hand_traced

CASES = load_hand_traced()


def _pulse(case):
    p = case.get("pulse", {})
    return p.get("gate", 100), p.get("wire", 100)


def _features(case):
    f = case.get("features", {})
    return f.get("interconnect_filter", True), f.get("full_sdf", True)


def _event_windows(wl, W, mutation="none", pulse=(100, 100), features=(True, True)):
    sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, mutation=mutation,
                          pulse_gate=pulse[0], pulse_wire=pulse[1], interconnect_filter=features[0],
                          full_sdf=features[1])
    out = []
    for w in range(sim.num_windows):
        out.append(oracle.windows_as_lists(*sim.window(w)))
    return sim, out


def _golden_failures(case, mutation="none"):
    wl = case_workload(case)
    sim, wins = _event_windows(wl, case["W"], mutation, _pulse(case), _features(case))
    fails = []
    for e in case["expect"]:
        got = wins[e["window"]][e["net"]]
        if got != (e["init"], e["times"]):
            fails.append(f"{case['name']}: net {e['net']} window {e['window']}: {got}")
    t0, t1, tc = sim.saif()
    for s in case["saif"]:
        n = s["net"]
        if (int(t0[n]), int(t1[n]), int(tc[n])) != (s["T0"], s["T1"], s["TC"]):
            fails.append(f"{case['name']}: SAIF net {n}: {(t0[n], t1[n], tc[n])}")
    return fails


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_traced_event_sim(case):
    assert _golden_failures(case) == []


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_traced_algo1(case):
    wl = case_workload(case)
    W = case["W"]
    nwin = (wl.stim.num_cycles + W - 1) // W
    pg, pw = _pulse(case)
    wire_filter, full_sdf = _features(case)
    if not wire_filter:
        pw = 0  # the interconnect test deleted: only crossing arrivals cancel
    wins = [algo1.simulate_window(wl.netlist, wl.delays, wl.stim, w, W, pg, pw, full_sdf) for w in range(nwin)]
    for e in case["expect"]:
        init, times = wins[e["window"]][e["net"]]
        assert (init, list(times)) == (e["init"], e["times"])
    for s in case["saif"]:
        n = s["net"]
        t1 = tc = total = 0
        for w in range(nwin):
            length = algo1.window_length(wl.stim, w, W)
            a, b = algo1.saif_of_waves([wins[w][n]], length)[0]
            t1, tc, total = t1 + a, tc + b, total + length
        assert (total - t1, t1, tc) == (s["T0"], s["T1"], s["TC"])


# ----------------------------------------------------------- settled values

def _final_input_values(stim, w, W):
    I, C = stim.init.shape[0], stim.num_cycles
    c1 = min((w + 1) * W, C)
    idx = np.arange(I, dtype=np.int64) * C
    return (stim.init.astype(np.int64) ^ ((stim.edge_ptr[idx + c1] - stim.edge_ptr[idx]) & 1)).astype(np.uint8)


def _zero_delay(netlist, inputs):
    """Brute-force truth-table evaluation of every net (net id order)."""
    vals = list(inputs.tolist())
    for g in range(netlist.num_gates):
        a, b = int(netlist.fanin_ptr[g]), int(netlist.fanin_ptr[g + 1])
        col = 0
        for k, q in enumerate(range(a, b)):
            col |= vals[int(netlist.fanin_net[q])] << k
        vals.append((int(netlist.lut[g]) >> col) & 1)
    return np.asarray(vals, np.uint8)


def _settled_failures(wl, W, mutation="none", windows=None, pulse=(100, 100)):
    sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, mutation=mutation,
                          pulse_gate=pulse[0], pulse_wire=pulse[1])
    fails = []
    for w in (windows if windows is not None else range(sim.num_windows)):
        init, ptr, times = sim.window(w)
        final = init ^ (np.diff(ptr) & 1).astype(np.uint8)
        ref_final = _zero_delay(wl.netlist, _final_input_values(wl.stim, w, W))
        c0 = w * W
        start_inputs = (wl.stim.init.astype(np.int64) ^ (
            (wl.stim.edge_ptr[np.arange(wl.netlist.num_inputs) * wl.stim.num_cycles + c0]
             - wl.stim.edge_ptr[np.arange(wl.netlist.num_inputs) * wl.stim.num_cycles]) & 1)).astype(np.uint8)
        ref_init = _zero_delay(wl.netlist, start_inputs)
        if not np.array_equal(final, ref_final):
            fails.append(f"window {w}: final values differ at {np.nonzero(final != ref_final)[0][:5]}")
        if not np.array_equal(init, ref_init):
            fails.append(f"window {w}: start values differ")
    return fails


SETTLED = [("tiny", dict(num_cycles=30)), ("mid", dict(num_cycles=4, num_gates=3000, depth=30,
                                                       num_inputs=64)),
           ("large", dict(num_cycles=3, num_gates=4000, depth=40, num_inputs=100))]


@pytest.mark.parametrize("name,kw", SETTLED, ids=[s[0] for s in SETTLED])
@pytest.mark.parametrize("W", [1, 3])
def test_settled_values(name, kw, W):
    wl = gen.make_workload(name, seed=7, **kw)
    assert _settled_failures(wl, W) == []


# ------------------------------------------------------------- invariants

def _invariant_failures(wl, W, mutation="none", pulse=(100, 100)):
    sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, mutation=mutation,
                          pulse_gate=pulse[0], pulse_wire=pulse[1])
    fails = []
    I = wl.netlist.num_inputs
    inits, finals = [], []
    for w in range(sim.num_windows):
        init, ptr, times = sim.window(w)
        t1, length = sim.window_t1()
        for n in range(init.shape[0]):
            ts = times[ptr[n]:ptr[n + 1]]
            if ts.size and (np.any(np.diff(ts) <= 0) or ts[0] < 0):
                fails.append(f"net {n} window {w}: times not strictly increasing / negative")
            if n >= I and ts.size and ts[0] < 1:
                fails.append(f"gate net {n} window {w}: edge before 1 ps")
        if np.any(t1 < 0) or np.any(t1 > length):
            fails.append(f"window {w}: T1 outside [0, {length}]")
        inits.append(init)
        finals.append(init ^ (np.diff(ptr) & 1).astype(np.uint8))
    t0, t1, tc = sim.saif()
    total = wl.stim.num_cycles * wl.stim.cycle_ps
    if not np.all(t0 + t1 == total):
        fails.append("T0 + T1 != simulated time")
    parity = np.zeros_like(tc)
    for a, b in zip(inits, finals):
        parity += (a ^ b).astype(np.int64)
    if not np.array_equal(tc & 1, parity & 1):
        fails.append("TC parity != number of windows whose value changed")
    return fails


@pytest.mark.parametrize("W", [1, 2])
def test_invariants(W):
    wl = gen.make_workload("tiny", seed=11, num_cycles=12)
    assert _invariant_failures(wl, W) == []


PULSES = [(0, 0), (0, 100), (100, 0), (50, 50), (30, 80)]


@pytest.mark.parametrize("pulse", PULSES, ids=[f"g{a}w{b}" for a, b in PULSES])
def test_settled_values_and_invariants_at_pulse_limits(pulse):
    # a cancel removes one output edge and a dropped wire pulse two input
    # edges, so the settled values never depend on the limits
    wl = gen.make_workload("tiny", seed=13, num_cycles=10)
    assert _settled_failures(wl, 1, pulse=pulse) == []
    assert _invariant_failures(wl, 2, pulse=pulse) == []
    wl = gen.make_workload("mid", seed=13, num_cycles=3, num_gates=2000, depth=25, num_inputs=48)
    assert _settled_failures(wl, 1, pulse=pulse) == []


# ------------------------------------------------------------- closed forms

def _chain(seed, depth):
    rng = np.random.Generator(np.random.PCG64(seed))
    inv = rng.integers(0, 2, depth)
    lut = np.where(inv == 1, gen.cell_lut("INV"), gen.cell_lut("BUF")).astype(np.uint16)
    wire = rng.integers(1, 21, (depth, 2)).astype(np.int32)      # [rise, fall]
    io = rng.integers(1, 51, (depth, 2)).astype(np.int32)        # [out-fall, out-rise]
    gd = np.zeros((depth, 2, 2, 8), np.int32)
    gd[:, :, 0, 0] = io[:, 0:1]
    gd[:, :, 1, 0] = io[:, 1:2]
    nl = gen.Netlist(1, np.arange(depth + 1, dtype=np.int32), np.arange(depth, dtype=np.int32),
                     np.ones(depth, np.uint8), lut, np.zeros(depth, np.uint8))
    return nl, gen.Delays(gd.reshape(-1), wire.reshape(-1)), inv, wire, io


@pytest.mark.parametrize("seed", range(6))
def test_chain_shift_closed_form(seed):
    depth = 3 + seed * 3
    nl, dl, inv, wire, io = _chain(seed, depth)
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    spacing = 100 * (depth + 1)
    k = 6
    L = spacing * (k + 2)
    init0 = int(rng.integers(0, 2))
    t_in = (np.arange(1, k + 1) * spacing + rng.integers(0, 20, k)).astype(np.int64)
    st = gen.Stimulus(1, L, np.asarray([init0], np.uint8), np.asarray([0, k], np.int64),
                      t_in.astype(np.int32))
    sim = oracle.EventSim(nl, dl, st, W=1)
    init, ptr, times = sim.window(0)
    # closed form: each edge keeps its identity; at stage j it arrives after
    # the wire delay of its direction and leaves after the gate delay of the
    # output direction
    v = init0
    cur = [(int(t), 1 - ((init0 + i) % 2)) for i, t in enumerate(t_in)]   # (time, rising?)
    for j in range(depth):
        v = v ^ int(inv[j])
        nxt = []
        for t, rising in cur:
            arr = t + int(wire[j, 0] if rising else wire[j, 1])
            out_rising = rising ^ int(inv[j])
            nxt.append((arr + int(io[j, 1] if out_rising else io[j, 0]), out_rising))
        cur = nxt
        net = 1 + j
        assert int(init[net]) == v
        assert times[ptr[net]:ptr[net + 1]].tolist() == [t for t, _ in cur]


@pytest.mark.parametrize("seed", range(4))
def test_transport_chain_passes_narrow_pulses_shifted(seed):
    # equal rise and fall delays at every stage keep every pulse's width, so
    # with both limits at 0 (transport) each input edge comes out shifted by
    # the sum of the path's delays, however narrow its pulse; at 100 percent
    # the same pulses (narrower than every delay) all vanish
    depth = 4 + 3 * seed
    rng = np.random.Generator(np.random.PCG64(500 + seed))
    inv = rng.integers(0, 2, depth)
    lut = np.where(inv == 1, gen.cell_lut("INV"), gen.cell_lut("BUF")).astype(np.uint16)
    w = rng.integers(10, 30, depth)
    g = rng.integers(10, 50, depth)
    wire = np.stack([w, w], 1).astype(np.int32)
    gd = np.zeros((depth, 2, 2, 8), np.int32)
    gd[:, :, :, 0] = g[:, None, None]
    nl = gen.Netlist(1, np.arange(depth + 1, dtype=np.int32), np.arange(depth, dtype=np.int32),
                     np.ones(depth, np.uint8), lut, np.zeros(depth, np.uint8))
    dl = gen.Delays(gd.reshape(-1), wire.reshape(-1))
    starts = np.arange(1, 6) * 150 + rng.integers(0, 20, 5)
    widths = rng.integers(1, 10, 5)
    t_in = np.sort(np.concatenate([starts, starts + widths])).astype(np.int32)
    init0 = int(rng.integers(0, 2))
    st = gen.Stimulus(1, 4000, np.asarray([init0], np.uint8), np.asarray([0, t_in.size], np.int64), t_in)
    init, ptr, times = oracle.EventSim(nl, dl, st, W=1, pulse_gate=0, pulse_wire=0).window(0)
    shift = np.cumsum(w + g)
    v = init0
    for j in range(depth):
        v ^= int(inv[j])
        net = 1 + j
        assert int(init[net]) == v
        assert times[ptr[net]:ptr[net + 1]].tolist() == (t_in + shift[j]).tolist()
    a1 = algo1.simulate_window(nl, dl, st, 0, 1, 0, 0)
    assert [list(t) for _, t in a1[1:]] == [times[ptr[n]:ptr[n + 1]].tolist() for n in range(1, depth + 1)]
    _, ptr100, _ = oracle.EventSim(nl, dl, st, W=1).window(0)
    assert np.all(np.diff(ptr100)[1:] == 0)


def test_narrow_pulses_never_pass():
    wl = gen.make_workload("tiny", seed=5, num_cycles=10)
    # every input pulse narrower than every wire delay (>= 3 here)
    dl = gen.Delays(wl.delays.gate_delay, np.maximum(wl.delays.wire_delay, 3))
    I, C = wl.netlist.num_inputs, 10
    ptr, times = [0], []
    for i in range(I):
        for c in range(C):
            s = 10 + (i * 7 + c * 13) % 150
            times += [s, s + 1 + (i + c) % 2]          # width 1 or 2
            ptr.append(len(times))
    st = gen.Stimulus(C, 1000, wl.stim.init, np.asarray(ptr, np.int64), np.asarray(times, np.int32))
    sim = oracle.EventSim(wl.netlist, dl, st, W=1)
    for w in range(C):
        init, p, _ = sim.window(w)
        assert np.all(np.diff(p)[I:] == 0)


# -------------------------------------------- the two formulations agree

@pytest.mark.parametrize("block", range(4))
def test_event_sim_matches_algorithm1_random(block):
    for s in range(block * 500, block * 500 + 500):
        wl = gen.random_small(s)
        W = 1 + s % 2
        sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W)
        for w in range(sim.num_windows):
            ev = oracle.windows_as_lists(*sim.window(w))
            a1 = [(i, list(t)) for i, t in algo1.simulate_window(wl.netlist, wl.delays, wl.stim, w, W)]
            assert ev == a1, f"random case {s} window {w}"


@pytest.mark.parametrize("block", range(2))
def test_event_sim_matches_algorithm1_random_pulse_limits(block):
    rng = np.random.Generator(np.random.PCG64(77 + block))
    for s in range(5000 + block * 400, 5000 + block * 400 + 400):
        wl = gen.random_small(s)
        W = 1 + s % 2
        pg, pw = (int(x) for x in rng.choice([0, 1, 25, 50, 99, 100], 2))
        sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, pulse_gate=pg, pulse_wire=pw)
        for w in range(sim.num_windows):
            ev = oracle.windows_as_lists(*sim.window(w))
            a1 = [(i, list(t)) for i, t in algo1.simulate_window(wl.netlist, wl.delays, wl.stim, w, W, pg, pw)]
            assert ev == a1, f"random case {s} window {w} limits {pg}/{pw}"


@pytest.mark.parametrize("wire_filter,full_sdf", [(False, True), (True, False), (False, False)])
def test_event_sim_matches_algorithm1_reduced_features(wire_filter, full_sdf):
    """The paper's reduced-feature variants (Section 5, Table "features"):
    no interconnect filter, averaged (partial-SDF) arc delays, and both."""
    for s in range(9000, 9300):
        wl = gen.random_small(s)
        W = 1 + s % 2
        sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, interconnect_filter=wire_filter,
                              full_sdf=full_sdf)
        for w in range(sim.num_windows):
            ev = oracle.windows_as_lists(*sim.window(w))
            a1 = [(i, list(t)) for i, t in algo1.simulate_window(
                wl.netlist, wl.delays, wl.stim, w, W, 100, 100 if wire_filter else 0, full_sdf)]
            assert ev == a1, f"random case {s} window {w}"
    # settled values and invariants hold in both variants too
    wl = gen.make_workload("tiny", seed=13, num_cycles=40)
    sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1, interconnect_filter=wire_filter,
                          full_sdf=full_sdf)
    t0, t1, tc = sim.saif()
    assert np.all(t0 + t1 == 40 * wl.stim.cycle_ps) and np.all(t0 >= 0) and np.all(t1 >= 0)
    for w in (0, 17, 39):
        init, ptr, times = sim.window(w)
        final = init ^ (np.diff(ptr) & 1).astype(np.uint8)
        assert np.array_equal(final, _zero_delay(wl.netlist, _final_input_values(wl.stim, w, 1)))
        for n in range(sim.N):
            assert np.all(np.diff(times[ptr[n]:ptr[n + 1]]) > 0)


def test_event_sim_matches_algorithm1_recipes():
    for name, kw in [("tiny", dict(num_cycles=6)),
                     ("mid", dict(num_cycles=3, num_gates=1500, depth=20, num_inputs=40))]:
        wl = gen.make_workload(name, seed=3, **kw)
        sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=2)
        for w in range(sim.num_windows):
            ev = oracle.windows_as_lists(*sim.window(w))
            a1 = [(i, list(t)) for i, t in algo1.simulate_window(wl.netlist, wl.delays, wl.stim, w, 2)]
            assert ev == a1


# ----------------------------------------------- planted-mistake coverage

@pytest.mark.parametrize("mutation", [m for m in oracle.MUTATIONS if m != "none"])
def test_planted_mistake_is_caught(mutation):
    fails = []
    for case in CASES:
        fails += _golden_failures(case, mutation)
    wl = gen.make_workload("tiny", seed=7, num_cycles=6)
    fails += _settled_failures(wl, 1, mutation)
    fails += _invariant_failures(wl, 1, mutation)
    assert fails, f"planted mistake '{mutation}' passes every pin"


# ---------------------------------------------------------------- digests
# The per-net waveform digest (oracle/digest.py) checks bit-exactness at
# scale.  Its mixing function is the SplitMix64 output function; the
# generator module implements the same published function independently in
# C (its counter-keyed draws), which pins the oracle's version.

from oracle import digest as odig  # noqa: E402

_G = 0x9E3779B97F4A7C15
_C2 = 0xD1B54A32D192ED03


@pytest.mark.parametrize("seed,stream,idx", [(1, 0, 0), (7, 3, 12345), (2**63 + 5, 17, 2**40 + 3)])
def test_digest_mix_matches_generator_splitmix(seed, stream, idx):
    m = 2**64 - 1
    a = int(odig.mix(np.array([(seed + _G * (stream + 1)) & m], np.uint64))[0])
    x = int(odig.mix(np.array([a ^ ((idx * _C2 + _G) & m)], np.uint64))[0])
    assert x == gen.draw(seed, stream, idx)


def test_digest_empty_waveform_closed_form():
    init = np.array([0, 1], np.uint8)
    ptr = np.array([0, 0, 0], np.int64)
    t = odig.window_terms(init, ptr, np.zeros(0, np.int32), 41)
    mw = odig.mix(np.array([42], np.uint64))[0]
    for n, v in enumerate((0, 1)):
        h = odig.mix(np.array([v + 1], np.uint64))[0]
        assert t[n] == odig.mix(np.array([h ^ mw], np.uint64))[0]


def test_digest_is_order_free_and_local():
    wl = gen.make_workload("tiny", seed=4, num_cycles=40)
    sim = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    fwd = odig.digest(sim, range(40))
    rev = odig.digest(sim, reversed(range(40)))
    assert np.array_equal(fwd, rev)
    # one changed edge time changes exactly one net's term
    init, ptr, times = sim.window(7)
    base = odig.window_terms(init, ptr, times, 7)
    n = int(np.nonzero(np.diff(ptr) > 0)[0][0])
    times2 = times.copy()
    times2[ptr[n]] += 1
    moved = odig.window_terms(init, ptr, times2, 7)
    assert np.count_nonzero(moved != base) == 1 and moved[n] != base[n]
    # the window index enters: the same waveforms at another index differ
    assert not np.array_equal(odig.window_terms(init, ptr, times, 8), base)


# ---------------------------------------------------------- time translation

@pytest.mark.parametrize("pulse", [(100, 100), (0, 0), (40, 70)], ids=["g100w100", "g0w0", "g40w70"])
def test_shifting_every_input_edge_shifts_every_waveform(pulse):
    # nothing in the method depends on absolute time: moving all of a
    # window's input edges later by d moves every net's edges later by d
    # (start values unchanged), in both formulations
    rng = np.random.Generator(np.random.PCG64(99))
    for s in range(120):
        wl = gen.random_small(40_000 + s, max_cycles=1)
        st = wl.stim
        d = int(rng.integers(1, 300))
        big = st.cycle_ps + d + 10
        shifted = gen.Stimulus(st.num_cycles, big, st.init, st.edge_ptr, (st.edge_time + d).astype(np.int32))
        base = gen.Stimulus(st.num_cycles, big, st.init, st.edge_ptr, st.edge_time)
        a = oracle.EventSim(wl.netlist, wl.delays, base, W=1, pulse_gate=pulse[0], pulse_wire=pulse[1])
        b = oracle.EventSim(wl.netlist, wl.delays, shifted, W=1, pulse_gate=pulse[0], pulse_wire=pulse[1])
        ia, pa, ta = a.window(0)
        ib, pb, tb = b.window(0)
        assert np.array_equal(ia, ib) and np.array_equal(pa, pb), f"case {s}"
        assert np.array_equal(ta.astype(np.int64) + d, tb), f"case {s}"
        a1 = algo1.simulate_window(wl.netlist, wl.delays, shifted, 0, 1, *pulse)
        assert [(i, list(t)) for i, t in a1] == oracle.windows_as_lists(ib, pb, tb)
