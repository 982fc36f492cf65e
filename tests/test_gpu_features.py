"""The kernels without some of Algorithm 1's features -- the paper's cost
comparison (Section 5, Table "features": no interconnect inertial filter;
that plus partial SDF, i.e. one averaged delay per arc and output edge) --
against the oracle with the same features switched off, bit for bit: every
waveform (digests) and SAIF, on gate-aligned and linear tiles, with
multi-cycle windows, plus the option checks."""
import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs
from helpers import assert_window_equal

pytestmark = pytest.mark.gpu

MASKS = [gs.NO_INTERCONNECT_FILTER, gs.PARTIAL_SDF, gs.NO_INTERCONNECT_FILTER | gs.PARTIAL_SDF]


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _oracle(wl, mask, W=1):
    return oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=W,
                           interconnect_filter=not mask & gs.NO_INTERCONNECT_FILTER,
                           full_sdf=not mask & gs.PARTIAL_SDF)


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("recipe,cycles,W,ipt", [("tiny", 400, 1, 4), ("mid", 120, 1, 4), ("tiny", 90, 3, 1)])
def test_reduced_features_match_oracle(mask, recipe, cycles, W, ipt):
    kw = dict(num_gates=20_000, depth=40, num_inputs=200) if recipe == "mid" else {}
    wl = gen.make_workload(recipe, seed=7, num_cycles=cycles, **kw)
    ref = _oracle(wl, mask, W)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=W, features=mask, digest=1, tile_items=256, items_per_thread=ipt)
        got = sim.digest()
        want = odig.digest(ref, range(ref.num_windows))
        assert np.array_equal(got, want), f"{np.count_nonzero(got != want)} nets differ"
        for a, b in zip(sim.saif(), ref.saif()):
            assert np.array_equal(a, b)
        assert_window_equal(sim, ref, ref.num_windows - 1)


def test_linear_tiles_without_features():
    """Batches of fewer than 64 windows take the linear tiles."""
    wl = gen.make_workload("tiny", seed=8, num_cycles=50)
    mask = gs.NO_INTERCONNECT_FILTER | gs.PARTIAL_SDF
    ref = _oracle(wl, mask)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, features=mask, batch_windows=20, tile_items=256, items_per_thread=4)
        for a, b in zip(sim.saif(), ref.saif()):
            assert np.array_equal(a, b)
        assert_window_equal(sim, ref, 49)


def test_features_change_the_result_and_options_are_checked():
    wl = gen.make_workload("mid", seed=3, num_cycles=40, num_gates=5000, depth=20, num_inputs=64)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        tcs = []
        for mask in [0] + MASKS:
            sim.simulate(window_cycles=1, features=mask)
            tcs.append(sim.saif()[2].copy())
        # the narrow pulses the mid recipe plants reach the gates without the
        # interconnect filter (and may pass, or cancel other output edges there)
        assert not np.array_equal(tcs[1], tcs[0])
        assert not np.array_equal(tcs[2], tcs[0])       # averaged arcs move edges
        for bad in (dict(features=4), dict(features=1, pulse=(50, 100)),
                    dict(features=1, tile_items=128, items_per_thread=4)):
            with pytest.raises(gs.GatspiError) as e:
                sim.simulate(window_cycles=1, **bad)
            assert e.value.code == gs.EINVAL
