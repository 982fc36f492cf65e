"""Stimulus restructuring and file formats, on the CPU.

* The oracle's restructuring (oracle/stimulus.py) of raw (input, absolute
  time) toggles into per-(input, cycle) lists is pinned by round trips with
  the generator's stimuli (in shuffled order) and by brute-force grouping
  with plain dictionaries on small random cases.
* The library's VCD reader (host code, no GPU) reads dumps that a small
  writer here produces from generator stimuli -- several timescales, scopes,
  aliases, glitches inside one time step -- and must give back the same
  stimulus; malformed dumps are rejected.
* The library's SAIF writer's files parse back to the arrays written.
"""
import os

import numpy as np
import pytest

import gen
import paper_2203_06117_gb300 as gs
from oracle import stimulus as ostim
from helpers import parse_saif, write_vcd


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()


def _same_stim(a_ptr, a_time, stim):
    return np.array_equal(a_ptr, stim.edge_ptr) and np.array_equal(a_time, stim.edge_time)


# ------------------------------------------------------------ oracle pins

@pytest.mark.parametrize("name,kw", [("tiny", dict(num_cycles=50)),
                                     ("mid", dict(num_cycles=20, num_gates=3000, depth=20, num_inputs=64))])
def test_oracle_round_trip_shuffled(name, kw):
    wl = gen.make_workload(name, seed=3, **kw)
    st = wl.stim
    inp, t = ostim.cycles_to_events(st)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(inp.size)
    ptr, times = ostim.events_to_cycles(st.init.size, st.num_cycles, st.cycle_ps, inp[perm], t[perm])
    assert _same_stim(ptr, times, st)


def test_oracle_matches_brute_force_grouping():
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(200):
        I, C, L = int(rng.integers(1, 5)), int(rng.integers(1, 6)), int(rng.integers(1, 50))
        n = int(rng.integers(0, 30))
        pairs = set()
        while len(pairs) < min(n, I * C * L):
            pairs.add((int(rng.integers(0, I)), int(rng.integers(0, C * L))))
        pairs = list(pairs)
        rng.shuffle(pairs)
        inp = np.array([p[0] for p in pairs], np.int64)
        t = np.array([p[1] for p in pairs], np.int64)
        ptr, times = ostim.events_to_cycles(I, C, L, inp, t)
        groups = {}
        for i, tt in pairs:
            groups.setdefault((i, tt // L), []).append(tt % L)
        for i in range(I):
            for c in range(C):
                assert times[ptr[i * C + c]:ptr[i * C + c + 1]].tolist() == sorted(groups.get((i, c), []))


@pytest.mark.parametrize("inp,t", [([2], [0]), ([0], [-1]), ([0], [30]), ([0, 0], [5, 5])])
def test_oracle_rejects_bad_events(inp, t):
    with pytest.raises(ValueError):
        ostim.events_to_cycles(2, 3, 10, np.array(inp), np.array(t))


# -------------------------------------------------------------- VCD reader

def _check_vcd_round_trip(tmp_path, stim, **kw):
    names = [f"in{k}" for k in range(stim.init.size)]
    p = os.path.join(tmp_path, "s.vcd")
    write_vcd(p, stim, names, **kw)
    init, ei, et = gs.gatspi_vcd_read(p, names)
    assert np.array_equal(init, stim.init)
    ptr, times = ostim.events_to_cycles(stim.init.size, stim.num_cycles, stim.cycle_ps, ei, et)
    assert _same_stim(ptr, times, stim)
    assert np.all(np.diff(et) >= 0)            # file (time) order


@pytest.mark.parametrize("unit", ["1ps", "1 ps"])
def test_vcd_round_trip_generator_stimulus(tmp_path, unit):
    wl = gen.make_workload("tiny", seed=5, num_cycles=40)
    _check_vcd_round_trip(tmp_path, wl.stim, unit=unit, glitch_every=7)


def test_vcd_coarse_timescales(tmp_path):
    wl = gen.make_workload("tiny", seed=6, num_cycles=30)
    st = wl.stim
    for unit, ps in [("10ps", 10), ("1ns", 1000)]:
        # a stimulus whose times are multiples of the unit
        t = (st.edge_time // ps) * ps
        ptr, times = ostim.events_to_cycles(st.init.size, st.num_cycles, st.cycle_ps,
                                            *_dedup(st, t))
        s2 = gen.Stimulus(st.num_cycles, st.cycle_ps, st.init, ptr, times)
        _check_vcd_round_trip(tmp_path, s2, unit=unit)


def _dedup(st, t):
    """Events of a stimulus with times t (per cycle), dropping toggles that
    land on the same ps as another of the same input in pairs."""
    C, L = st.num_cycles, st.cycle_ps
    counts = np.diff(st.edge_ptr)
    bucket = np.repeat(np.arange(st.init.size * C, dtype=np.int64), counts)
    inp = bucket // C
    at = (bucket % C) * L + t
    keep = {}
    for i, x in zip(inp.tolist(), at.tolist()):
        keep[(i, x)] = keep.get((i, x), 0) ^ 1
    pairs = sorted(k for k, v in keep.items() if v)
    return np.array([p[0] for p in pairs], np.int64), np.array([p[1] for p in pairs], np.int64)


def test_vcd_scopes_and_hierarchical_names(tmp_path):
    wl = gen.make_workload("tiny", seed=8, num_cycles=10)
    st = wl.stim
    names = [f"in{k}" for k in range(st.init.size)]
    p = os.path.join(tmp_path, "h.vcd")
    write_vcd(p, st, names, scope=("top", "u_core"), alias="in0_alias")
    full = [f"top.u_core.{n}" for n in names]
    init, ei, et = gs.gatspi_vcd_read(p, full)
    ptr, times = ostim.events_to_cycles(st.init.size, st.num_cycles, st.cycle_ps, ei, et)
    assert _same_stim(ptr, times, st)
    # an alias of input 0 read as its own signal has input 0's waveform
    init2, ei2, et2 = gs.gatspi_vcd_read(p, ["in0_alias", "in1"])
    init0, ei0, et0 = gs.gatspi_vcd_read(p, ["in0", "in1"])
    assert np.array_equal(init2, init0) and np.array_equal(ei2, ei0) and np.array_equal(et2, et0)


BAD_VCDS = {
    "x value": "$timescale 1ps $end $var wire 1 ! a $end $enddefinitions $end #0 0! #5 x!",
    "first value late": "$timescale 1ps $end $var wire 1 ! a $end $enddefinitions $end #0 #5 1!",
    "unknown signal": "$timescale 1ps $end $var wire 1 ! b $end $enddefinitions $end #0 0!",
    "wide signal": "$timescale 1ps $end $var wire 2 ! a $end $enddefinitions $end #0 b00 !",
    "time goes back": "$timescale 1ps $end $var wire 1 ! a $end $enddefinitions $end #0 0! #9 1! #5 0!",
    "fs timescale": "$timescale 100fs $end $var wire 1 ! a $end $enddefinitions $end #0 0!",
    "no enddefinitions": "$timescale 1ps $end $var wire 1 ! a $end #0 0!",
    "time beyond int64": "$timescale 1ps $end $var wire 1 ! a $end $enddefinitions $end #0 0! "
                         "#99999999999999999999 1!",
    "time beyond int64 ps": "$timescale 1s $end $var wire 1 ! a $end $enddefinitions $end #0 0! "
                            "#100000000 1!",
}


@pytest.mark.parametrize("why", list(BAD_VCDS))
def test_vcd_rejects_malformed_dumps(tmp_path, why):
    p = os.path.join(tmp_path, "bad.vcd")
    with open(p, "w") as f:
        f.write(BAD_VCDS[why])
    with pytest.raises(gs.GatspiError) as e:
        gs.gatspi_vcd_read(p, ["a"])
    assert e.value.code == gs.EINVAL


def test_vcd_values_inside_one_step_count_by_their_last_value(tmp_path):
    p = os.path.join(tmp_path, "g.vcd")
    with open(p, "w") as f:
        f.write("$timescale 1ns $end $scope module t $end $var wire 1 ! a $end $var reg 1 \" b $end "
                "$upscope $end $enddefinitions $end #0 $dumpvars 1! 0\" $end "
                "#3 0! 1! 1\" #4 0! b0 \" #7 1! #7 0!\n")
    init, ei, et = gs.gatspi_vcd_read(p, ["a", "b"])
    # a: 1, glitch at 3 ns (no toggle), falls at 4 ns, glitch at 7 ns; b: 0, rises 3 ns, falls 4 ns
    assert init.tolist() == [1, 0]
    assert list(zip(ei.tolist(), et.tolist())) == [(1, 3000), (0, 4000), (1, 4000)]


# -------------------------------------------------------------- SAIF writer

def test_saif_file_round_trip(tmp_path):
    rng = np.random.Generator(np.random.PCG64(2))
    n = 50
    names = [f"n{k}" for k in range(n - 3)] + ["u1/a[3]", "weird name", "x(1)"]
    t1 = rng.integers(0, 10**9, n)
    total = 10**9
    tc = rng.integers(0, 10**6, n)
    p = os.path.join(tmp_path, "o.saif")
    gs.gatspi_saif_write(p, "top", total, names, total - t1, t1, tc)
    head, nets = parse_saif(p)
    assert head["DURATION"] == str(total) and head["TIMESCALE"] == "1 ps"
    assert len(nets) == n
    for k, nm in enumerate(names):
        assert nets[nm] == (total - int(t1[k]), int(t1[k]), 0, int(tc[k]), 0)
    text = open(p).read()
    assert r"u1\/a\[3\]" in text and r"weird\ name" in text and r"x\(1\)" in text


def test_vcd_dumpoff_blocks_are_not_changes(tmp_path):
    p = os.path.join(tmp_path, "off.vcd")
    with open(p, "w") as f:
        f.write("$timescale 1ps $end $var wire 1 ! a $end $var wire 1 # b $end $enddefinitions $end "
                "#0 $dumpvars 0! 1# $end #10 1! #20 $dumpoff x! x# $end #50 $dumpon 0! 1# $end "
                "#60 0#\n")
    init, ei, et = gs.gatspi_vcd_read(p, ["a", "b"])
    # a: 0, rises at 10, the dump is off 20-50, back on at 50 with a = 0:
    # a toggle at 50; b: 1 throughout the gap, falls at 60
    assert init.tolist() == [0, 1]
    assert list(zip(ei.tolist(), et.tolist())) == [(0, 10), (0, 50), (1, 60)]
