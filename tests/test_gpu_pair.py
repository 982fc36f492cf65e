"""The kernel for a level's gates of at most two pins (propagate_pair_kernel)
against the oracle, bit for bit: every waveform (digests) and SAIF.

A level's pair class gets a launch of its own only from 32,768 tiles, so the
netlist here is shallow and wide: 40,000 gates in 4 levels of 10,000, 640
windows (5 tiles per gate), which splits every level.  Both compiled launch
shapes of Algorithm 1 as printed, and the reduced-feature modes at 256 x 4,
which have their own pair kernels."""
import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs
from helpers import assert_window_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


@pytest.fixture(scope="module")
def wide():
    return gen.make_workload("tiny", seed=17, num_gates=40_000, depth=4, num_inputs=256, num_cycles=640)


@pytest.mark.parametrize("mask,nt", [(0, 256), (0, 128), (gs.NO_INTERCONNECT_FILTER, 256), (gs.PARTIAL_SDF, 256),
                                     (gs.NO_INTERCONNECT_FILTER | gs.PARTIAL_SDF, 256)])
def test_pair_kernel_matches_oracle(wide, mask, nt):
    wl = wide
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1,
                          interconnect_filter=not mask & gs.NO_INTERCONNECT_FILTER,
                          full_sdf=not mask & gs.PARTIAL_SDF)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, features=mask, digest=1, tile_items=nt, items_per_thread=4)
        st = sim.stats()
        levels = 4
        assert st["prop_launches"] > levels, "no level split into the pair kernel and the rest"
        got = sim.digest()
        want = odig.digest(ref, range(ref.num_windows))
        assert np.array_equal(got, want), f"{np.count_nonzero(got != want)} nets differ"
        for a, b in zip(sim.saif(), ref.saif()):
            assert np.array_equal(a, b)
        assert_window_equal(sim, ref, ref.num_windows - 1)
