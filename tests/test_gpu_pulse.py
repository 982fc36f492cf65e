"""Pulse limits (PATHPULSEPERCENT other than 100, Section 3) on the GPU,
bit-exact against the oracle at the same limits.

The kernels with pulse limits are separate instantiations; these tests run
them through the C interface on every tiling (gate-aligned tiles with 1, 2,
4 or 8 windows per lane, linear tiles for small batches), with high enough
activity that lanes overflow their staging and are simulated again into
global memory, and check that limits of 100 / 100 give the default path's
results.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2203_06117_gb300 as gs
from helpers import assert_saif_equal, assert_window_equal

pytestmark = pytest.mark.gpu

LIMITS = [(0, 0), (0, 100), (100, 0), (50, 50), (25, 75), (99, 1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


@pytest.mark.parametrize("pulse", LIMITS, ids=[f"g{a}w{b}" for a, b in LIMITS])
def test_tiny_every_window(pulse):
    wl = gen.make_workload("tiny", seed=21, num_cycles=200)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1, pulse_gate=pulse[0], pulse_wire=pulse[1])
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, pulse=pulse)
        for w in range(200):
            assert_window_equal(sim, ref, w, f"limits {pulse}")
        assert_saif_equal(sim, ref)


@pytest.mark.parametrize("shape", [(256, 1), (256, 2), (256, 4), (128, 8)],
                         ids=["256x1", "256x2", "256x4", "128x8"])
def test_launch_shapes_transport(shape):
    wl = gen.make_workload("mid", seed=22, num_gates=6000, depth=30, num_inputs=128, num_cycles=300)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1, pulse_gate=0, pulse_wire=0)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, pulse=(0, 0), tile_items=shape[0], items_per_thread=shape[1])
        for w in range(0, 300, 7):
            assert_window_equal(sim, ref, w, f"shape {shape}")
        assert_saif_equal(sim, ref)


@pytest.mark.parametrize("W,batch", [(1, 20), (3, 0), (2, 9)])
def test_linear_tiles_and_windows(W, batch):
    """Small batches (linear tiling), multi-cycle windows, ragged tails."""
    wl = gen.make_workload("tiny", seed=23, num_cycles=101)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, pulse_gate=30, pulse_wire=60)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=W, batch_windows=batch, pulse=(30, 60))
        assert_saif_equal(sim, ref)
        st = sim.stats()
        for w in range((st["batches"] - 1) * st["batch_windows"], ref.num_windows):
            assert_window_equal(sim, ref, w, f"W={W} batch={batch}")


def test_random_small_circuits_random_limits():
    rng = np.random.Generator(np.random.PCG64(31))
    for s in range(120):
        wl = gen.random_small(20_000 + s, max_cycles=5)
        W = 1 + s % 2
        pg, pw = (int(x) for x in rng.choice([0, 1, 40, 99, 100], 2))
        ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W, pulse_gate=pg, pulse_wire=pw)
        with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
            sim.simulate(window_cycles=W, pulse=(pg, pw))
            for w in range(ref.num_windows):
                assert_window_equal(sim, ref, w, f"case {s} limits {pg}/{pw}")
            assert_saif_equal(sim, ref)


def test_limits_of_100_equal_the_default_path():
    wl = gen.make_workload("mid", seed=24, num_gates=5000, depth=25, num_inputs=100, num_cycles=200)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1, tile_items=256, items_per_thread=4)
        d0, s0 = sim.digest(), sim.saif()
        sim.simulate(window_cycles=1, digest=1, tile_items=256, items_per_thread=4, pulse=(100, 100))
        d1, s1 = sim.digest(), sim.saif()
    assert np.array_equal(d0, d1)
    assert all(np.array_equal(a, b) for a, b in zip(s0, s1))


def test_transport_changes_results_and_rejects_bad_options():
    wl = gen.make_workload("tiny", seed=25, num_cycles=50)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1)
        tc100 = sim.saif()[2]
        sim.simulate(window_cycles=1, pulse=(0, 0))
        tc0 = sim.saif()[2]
        assert tc0.sum() > tc100.sum()          # transport keeps the glitches inertia removes
        for bad in [dict(pulse=(101, 0)), dict(pulse=(0, -1)),
                    dict(pulse=(0, 0), tile_items=512, items_per_thread=4)]:
            with pytest.raises(gs.GatspiError) as e:
                sim.simulate(window_cycles=1, **bad)
            assert e.value.code == gs.EINVAL
