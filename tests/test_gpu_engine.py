"""The multi-job engine (batched and served re-simulation) through the C
interface: every job's SAIF must equal the oracle's for the same netlist,
delays (with the job's delay edit applied) and stimulus, bit for bit, and
be the same whether the job runs alone or mixed with others."""
import numpy as np
import pytest

import gen
import oracle
import paper_2203_06117_gb300 as gs
from helpers import edited_delays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()


def oracle_saif(nl, dl, st, W=1):
    return oracle.EventSim(nl, dl, st, W=W).saif()


def assert_saif(got, ref, what=""):
    for name, a, b in zip(("T0", "T1", "TC"), got, ref):
        if not np.array_equal(a, b):
            n = int(np.nonzero(a != b)[0][0])
            raise AssertionError(f"{what} SAIF {name} of net {n}: engine {a[n]} oracle {b[n]}")


def small_netlists():
    out = []
    for k, (name, kw) in enumerate([("tiny", dict(num_gates=600, depth=8, num_inputs=24)),
                                    ("mid", dict(num_gates=1500, depth=25, num_inputs=40)),
                                    ("large", dict(num_gates=900, depth=30, num_inputs=30)),
                                    ("tiny", dict(num_gates=2000, depth=20, num_inputs=64))]):
        wl = gen.make_workload(name, seed=20 + k, num_cycles=1, **kw)
        out.append(wl)
    return out


def job_stimulus(wl, seed, cycles):
    r = wl.params
    return gen.make_stimulus(wl.netlist.num_inputs, cycles, seed, r["p"], r["q"])


def test_batched_jobs_match_oracle():
    nets = small_netlists()
    rng = np.random.Generator(np.random.PCG64(1))
    with gs.Engine(part_items=40_000) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in nets]
        jobs = []
        for k in range(24):
            n = int(rng.integers(0, len(nets)))
            cycles = int(rng.integers(1, 90))
            W = int(rng.integers(1, 4))
            st = job_stimulus(nets[n], 1000 + k, cycles)
            edit = None
            if k % 3 == 0:
                G = nets[n].netlist.num_gates
                gates = rng.choice(G, size=max(1, G // 100), replace=False)
                deltas = rng.choice([-1, 1], size=gates.size) * rng.integers(10, 51, size=gates.size)
                edit = (gates, deltas)
            jid = eng.submit(ids[n], st, W, *(edit or (None, None)))
            jobs.append((jid, n, st, W, edit))
        eng.drain()
        s = eng.stats()
        assert s["parts_done"] >= 24 and s["active"] == 0 and s["queued"] == 0
        for jid, n, st, W, edit in jobs:
            state, saif = eng.poll(jid, ids[n])
            assert state == gs.JOB_DONE
            dl = nets[n].delays if edit is None else edited_delays(nets[n].netlist, nets[n].delays, *edit)
            assert_saif(saif, oracle_saif(nets[n].netlist, dl, st, W), f"job {jid}")


def test_engine_digests_match_oracle():
    """Per-job waveform digests (every waveform of every window) equal the
    oracle's, for jobs split into several parts, with and without edits."""
    from oracle import digest as odig
    nets = small_netlists()
    rng = np.random.Generator(np.random.PCG64(4))
    with gs.Engine(part_items=25_000, digest=1) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in nets]
        jobs = []
        for k in range(10):
            n = k % len(nets)
            st = job_stimulus(nets[n], 4000 + k, int(rng.integers(20, 120)))
            W = 1 + k % 3
            edit = None
            if k % 2:
                G = nets[n].netlist.num_gates
                gates = rng.choice(G, size=max(1, G // 50), replace=False)
                edit = (gates, rng.choice([-1, 1], size=gates.size) * rng.integers(10, 51, size=gates.size))
            jobs.append((eng.submit(ids[n], st, W, *(edit or (None, None))), n, st, W, edit))
        eng.drain()
        assert eng.stats()["parts_done"] > 10            # several jobs span more than one part
        for jid, n, st, W, edit in jobs:
            dl = nets[n].delays if edit is None else edited_delays(nets[n].netlist, nets[n].delays, *edit)
            ref = oracle.EventSim(nets[n].netlist, dl, st, W=W)
            got = eng.digest(jid, ids[n])
            want = odig.digest(ref, range(ref.num_windows))
            assert np.array_equal(got, want), f"job {jid}: {np.count_nonzero(got != want)} nets differ"
    with gs.Engine() as eng:                             # no digests asked for
        nid = eng.add_netlist(nets[0].netlist, nets[0].delays)
        j = eng.submit(nid, job_stimulus(nets[0], 9, 10))
        eng.drain()
        with pytest.raises(gs.GatspiError) as e:
            eng.digest(j, nid)
        assert e.value.code == gs.ESTATE


def test_same_alone_and_in_the_mix():
    """A job's SAIF does not depend on what else runs with it, and equals the
    plain single-job path."""
    nets = small_netlists()
    target = (3, job_stimulus(nets[3], 77, 150))
    with gs.Engine() as eng:
        nid = eng.add_netlist(nets[3].netlist, nets[3].delays)
        j = eng.submit(nid, target[1])
        eng.drain()
        alone = eng.poll(j, nid)[1]
    with gs.Engine(part_items=30_000, max_active=7) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in nets]
        others = [eng.submit(ids[k % 4], job_stimulus(nets[k % 4], 500 + k, 40 + 7 * k)) for k in range(10)]
        j = eng.submit(ids[3], target[1])
        more = [eng.submit(ids[k % 4], job_stimulus(nets[k % 4], 600 + k, 30 + k)) for k in range(6)]
        eng.drain()
        mixed = eng.poll(j, ids[3])[1]
        assert all(eng.poll(x)[0] == gs.JOB_DONE for x in others + more)
    with gs.Simulator(nets[3].netlist, nets[3].delays, target[1]) as sim:
        plain = sim.simulate().saif()
    for a, b, c in zip(alone, mixed, plain):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_arrivals_between_steps():
    """Continuous batching: jobs submitted while others are mid-flight join
    at their level 0; all results still match the oracle."""
    nets = small_netlists()
    with gs.Engine(part_items=50_000) as eng:
        ids = [eng.add_netlist(w.netlist, w.delays) for w in nets]
        pending, done = [], {}
        k = 0
        for step in range(400):
            if step % 3 == 0 and k < 15:
                n = k % 4
                st = job_stimulus(nets[n], 3000 + k, 20 + 5 * k)
                pending.append((eng.submit(ids[n], st), n, st))
                k += 1
            a, q = eng.step()
            for jid, n, st in pending:
                if jid not in done:
                    state, saif = eng.poll(jid, ids[n])
                    if state == gs.JOB_DONE:
                        done[jid] = saif
            if k == 15 and a == 0 and q == 0:
                break
        eng.drain()
        for jid, n, st in pending:
            saif = done.get(jid) or eng.poll(jid, ids[n])[1]
            assert_saif(saif, oracle_saif(nets[n].netlist, nets[n].delays, st), f"job {jid}")
            eng.release(jid)


def test_memory_pressure_queues_and_splits():
    """A budget far below the total: parts wait for memory, oversized parts
    are split, undersized edge stores are retried, results unchanged."""
    nets = small_netlists()
    wl = nets[3]
    with gs.Engine(arena_bytes=6 << 20, part_items=400_000) as eng:
        nid = eng.add_netlist(wl.netlist, wl.delays)
        jobs = [(eng.submit(nid, job_stimulus(wl, 40 + k, 200)), job_stimulus(wl, 40 + k, 200))
                for k in range(4)]
        eng.drain()
        s = eng.stats()
        assert s["bytes_peak"] <= 6 << 20
        for jid, st in jobs:
            state, saif = eng.poll(jid, nid)
            assert state == gs.JOB_DONE
            assert_saif(saif, oracle_saif(wl.netlist, wl.delays, st))


def test_job_that_cannot_fit_fails_cleanly():
    wl = small_netlists()[3]
    with gs.Engine(arena_bytes=64 << 10) as eng:
        nid = eng.add_netlist(wl.netlist, wl.delays)
        jid = eng.submit(nid, job_stimulus(wl, 5, 10))
        with pytest.raises(gs.GatspiError) as e:
            eng.drain()
        assert e.value.code == gs.ECAPACITY
        assert eng.poll(jid)[0] == gs.JOB_FAILED


def test_engine_rejects_bad_submissions():
    wl = small_netlists()[0]
    with gs.Engine() as eng:
        nid = eng.add_netlist(wl.netlist, wl.delays)
        st = job_stimulus(wl, 1, 5)
        with pytest.raises(gs.GatspiError) as e:
            eng.submit(nid + 5, st)
        assert e.value.code == gs.EINVAL
        with pytest.raises(gs.GatspiError) as e:
            eng.submit(nid, st, 1, [wl.netlist.num_gates], [5])
        assert e.value.code == gs.EINVAL
        with pytest.raises(gs.GatspiError) as e:
            eng.poll(12345)
        assert e.value.code == gs.EINVAL
