"""Bit-exactness at scale through per-net waveform digests.

The library reduces every (net, window) waveform it produced to a per-net
64-bit digest (gatspi_digest); the oracle computes the same definition from
its own event-driven waveforms (oracle/digest.py).  Equal digests on every
net mean every waveform of every window matched, beyond the SAIF totals
and the sampled windows the other parity tests compare.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _gpu_digest(wl, **opts):
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1, digest=1, **opts)
        return sim.digest(), sim.saif()


def test_tiny_all_windows_gate_aligned_tiles():
    wl = gen.make_workload("tiny", seed=2)                    # 1,000 windows: gate-aligned tiles
    got, _ = _gpu_digest(wl, tile_items=256, items_per_thread=4)
    ref = odig.digest(oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1), range(wl.stim.num_cycles))
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} nets differ"


def test_large_cut_small_batches_linear_tiles():
    wl = gen.make_workload("large", seed=3, num_cycles=24)    # 2M gates; 5-window batches: linear tiles
    got, _ = _gpu_digest(wl, batch_windows=5, tile_items=256, items_per_thread=4)
    ref = odig.workload_digest_parallel("large", 3, 24, min(8, os.cpu_count() or 1))
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} nets differ"


def test_mid_config_every_window():
    """The 200k-gate, 10,000-cycle workload: every waveform of every net."""
    procs = max(1, min(16, os.cpu_count() or 1))
    ref = odig.workload_digest_parallel("mid", 1, 10000, procs)
    wl = gen.make_workload("mid", seed=1)
    got, _ = _gpu_digest(wl)
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} nets differ"


def test_digest_requires_a_digest_run():
    wl = gen.make_workload("tiny", seed=1, num_cycles=5)
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=1)
        with pytest.raises(gs.GatspiError) as e:
            sim.digest()
        assert e.value.code == gs.ESTATE
