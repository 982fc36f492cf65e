"""Segments of a long stimulus (gatspi_opts.first_window / num_windows).

The paper runs a testbench too long for device memory as shorter segments
and combines their results (Section 4); windows are independent, so a run
can also resume at any window.  The SAIF figures and the digests of
consecutive segments must add up, bit for bit, to those of the whole run,
and each segment's resident waveforms must equal the oracle's.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2203_06117_gb300 as gs
from helpers import assert_window_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


@pytest.mark.parametrize("W,cuts,batch", [(1, [0, 250, 600, 1000], 0), (1, [0, 1, 999, 1000], 128),
                                          (3, [0, 100, 334], 40)])
def test_segments_add_up_to_the_whole_run(W, cuts, batch):
    wl = gen.make_workload("tiny", seed=61)
    nwin = (wl.stim.num_cycles + W - 1) // W
    assert cuts[-1] == nwin
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=W, digest=1)
        whole = sim.saif(), sim.digest()
        t0 = np.zeros_like(whole[0][0]); t1 = np.zeros_like(t0); tc = np.zeros_like(t0)
        dg = np.zeros_like(whole[1])
        for a, b in zip(cuts[:-1], cuts[1:]):
            sim.simulate(window_cycles=W, digest=1, first_window=a, num_windows=b - a, batch_windows=batch)
            st = sim.stats()
            assert st["windows"] == b - a
            s0, s1, sc = sim.saif()
            t0 += s0; t1 += s1; tc += sc
            with np.errstate(over="ignore"):
                dg += sim.digest()
            last0 = a + (st["batches"] - 1) * st["batch_windows"]
            for w in sorted({last0, b - 1, (last0 + b - 1) // 2}):
                assert_window_equal(sim, ref, w, f"segment [{a}, {b})")
    assert np.array_equal(t0, whole[0][0]) and np.array_equal(t1, whole[0][1]) and np.array_equal(tc, whole[0][2])
    assert np.array_equal(dg, whole[1])
    r0, r1, rc = ref.saif()
    assert np.array_equal(t1, r1) and np.array_equal(tc, rc) and np.array_equal(t0, r0)


def test_segment_bounds_are_checked():
    wl = gen.make_workload("tiny", seed=62, num_cycles=50)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        for bad in [dict(first_window=50), dict(first_window=-1), dict(num_windows=-2)]:
            with pytest.raises(gs.GatspiError) as e:
                sim.simulate(window_cycles=1, **bad)
            assert e.value.code == gs.EINVAL
        sim.simulate(window_cycles=1, first_window=40, num_windows=1000)   # clipped at the end
        assert sim.stats()["windows"] == 10
