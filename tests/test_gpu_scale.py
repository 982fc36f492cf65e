"""Bit-exact parity with the oracle at the stated sizes of the large,
batched and served workloads, and on tile runs long enough to take the
propagation kernel's chunked count scan.

* Large (2M gates, depth 120, Zipf fanout up to 64, 20,000 cycles): the
  first and the last 2,000-window device batch, simulated as segments with
  gate-aligned tiles at the benchmark's launch shape, against the oracle's
  per-net waveform digests and SAIF over the same windows (computed here, on
  one spawned process per host core).
* Batched (64 jobs over 8 netlists) and served (200 requests/s for 1 s over
  four resident netlists, continuous batching): every batched job and a
  sample of 27 served requests, 11 of them with a delay edit, against the
  oracle's folds of SAIF and digests kept in tests/golden/engine_streams.json
  (written by tests/golden/make_engine_golden.py from the oracle alone; the
  oracle needs about 4e10 gate-cycles for them, too long to rerun here).
"""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import digest as odig
import paper_2203_06117_gb300 as gs
from paper_2203_06117_gb300 import serve

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "engine_streams.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    oracle.build()


def _fold(v):
    """sum_n mix(v[n] ^ mix(n + 1)) mod 2^64 (as in make_engine_golden.py)."""
    v = np.asarray(v).astype(np.uint64)
    n = np.arange(v.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(odig.mix(v ^ odig.mix(n + np.uint64(1))), dtype=np.uint64))


def _procs(gb_each):
    """Worker processes for the oracle: one per core, fewer if the host's
    available memory would not hold gb_each GB per worker."""
    procs = max(1, min(16, os.cpu_count() or 1))
    try:
        with open("/proc/meminfo") as f:
            avail = dict(l.split(":", 1) for l in f)["MemAvailable"]
        gb = int(avail.strip().split()[0]) / 2 ** 20
        procs = max(1, min(procs, int(gb * 0.6 / gb_each)))
    except (OSError, KeyError, ValueError):
        procs = min(procs, 4)
    return procs


_W = {}


def _large_init():
    _W["wl"] = gen.make_workload("large", seed=1)
    _W["sim"] = oracle.EventSim(_W["wl"].netlist, _W["wl"].delays, _W["wl"].stim, W=1)


def _large_unit(windows):
    sim = _W["sim"]
    dig = np.zeros(sim.N, np.uint64)
    t1 = np.zeros(sim.N, np.int64)
    tc = np.zeros(sim.N, np.int64)
    with np.errstate(over="ignore"):
        for w in windows:
            init, ptr, times = sim.window(int(w))
            dig += odig.window_terms(init, ptr, times, int(w))
            t1 += sim.window_t1()[0]
            tc += np.diff(ptr)
    return dig, t1, tc


def test_large_config_first_and_last_device_batches():
    import multiprocessing as mp
    wl = gen.make_workload("large", seed=1)
    segs = [(0, 2000), (18000, 2000)]
    got = []
    with gs.Simulator(wl.netlist, wl.delays, wl.stim) as sim:
        for w0, nw in segs:
            sim.simulate(window_cycles=1, first_window=w0, num_windows=nw, batch_windows=nw, digest=1,
                         tile_items=256, items_per_thread=4)
            st = sim.stats()
            assert st["batches"] == 1 and st["windows"] == nw
            got.append((sim.digest(), sim.saif()))
    procs = _procs(4.0)
    with mp.get_context("spawn").Pool(procs, initializer=_large_init) as pool:
        for (w0, nw), (g_dig, (g0, g1, gc)) in zip(segs, got):
            parts = pool.map(_large_unit, [list(range(w0 + k, w0 + nw, procs)) for k in range(procs)])
            dig = np.zeros_like(parts[0][0])
            t1 = np.zeros_like(parts[0][1])
            tc = np.zeros_like(parts[0][2])
            with np.errstate(over="ignore"):
                for d, a, c in parts:
                    dig += d
                    t1 += a
                    tc += c
            bad = np.count_nonzero(g_dig != dig)
            assert bad == 0, f"windows {w0}..{w0 + nw - 1}: {bad} nets' waveforms differ"
            assert np.array_equal(g1, t1) and np.array_equal(gc, tc), f"windows {w0}..: SAIF differs"
            assert np.array_equal(g0, nw * wl.stim.cycle_ps - t1)


def _golden():
    if not os.path.exists(GOLDEN):
        pytest.fail("tests/golden/engine_streams.json is missing: run tests/golden/make_engine_golden.py")
    with open(GOLDEN) as f:
        return json.load(f)


def _check(what, ref, saif, digest):
    t0, t1, tc = saif
    assert int(t1.sum()) == ref["sum_t1"] and int(tc.sum()) == ref["sum_tc"], f"{what}: SAIF totals differ"
    assert f"{_fold(t1):016x}" == ref["fold_t1"], f"{what}: T1 differs"
    assert f"{_fold(tc):016x}" == ref["fold_tc"], f"{what}: TC differs"
    assert f"{_fold(digest):016x}" == ref["fold_digest"], f"{what}: waveforms differ"


def test_batched_stream_every_job():
    g = _golden()
    nets, jobs = gen.batched_workload(seed=g["seed"])
    reqs = [serve.Request.from_spec(j) for j in jobs]
    serve.run_batched(nets, reqs, digest=1)
    assert len(g["batched"]) == len(reqs) == 64
    for ref, r in zip(g["batched"], reqs):
        assert ref["cycles"] == r.stim.num_cycles
        _check(f"batched job {ref['job']}", ref, r.result, r.digest)


def test_served_stream_sampled_requests():
    g = _golden()
    nets, specs = gen.served_workload(seed=g["seed"], rate=g["served_rate"], seconds=g["served_seconds"])
    reqs = [serve.Request.from_spec(s) for s in specs]
    serve.run_served(nets, reqs, digest=1)
    edited = 0
    for ref in g["served"]:
        r = reqs[ref["job"]]
        assert ref["cycles"] == r.stim.num_cycles
        edited += r.edit_gate is not None
        _check(f"served request {ref['job']}", ref, r.result, r.digest)
    assert len(g["served"]) >= 20 and edited >= 5


def test_tile_runs_of_65536_edges_or_more():
    """Windows of 600 cycles with a toggle in every cycle: a 128-window tile
    of an input-fed pin carries more than 65,536 edges, so the kernel scans
    the run's counts chunk by chunk instead of in packed 16-bit fields."""
    base = gen.make_workload("tiny", seed=31, num_gates=300, depth=8, num_inputs=16, num_cycles=1)
    C, W = 128 * 600, 600
    st = gen.make_stimulus(16, C, 31, 1000, 200)
    per_run = np.diff(st.edge_ptr[::W]).reshape(16, 128).sum(axis=1)  # each input's one tile run
    assert per_run.max() >= 65536
    with gs.Simulator(base.netlist, base.delays, st) as sim:
        sim.simulate(window_cycles=W, digest=1, tile_items=256, items_per_thread=4)
        got_dig, got_saif = sim.digest(), sim.saif()
    ref = oracle.EventSim(base.netlist, base.delays, st, W=W)
    assert np.array_equal(got_dig, odig.digest(ref, range(ref.num_windows)))
    for a, b in zip(got_saif, ref.saif()):
        assert np.array_equal(a, b)
