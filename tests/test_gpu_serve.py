"""Batched and served front-ends (small versions of the 64-job and the
Poisson-stream workloads): every request's SAIF is the same when it runs
alone on the single-job path and when it runs in the mix."""
import numpy as np
import pytest

import gen
import paper_2203_06117_gb300 as gs
from paper_2203_06117_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_batched_equals_plain_loop():
    nets, specs = gen.batched_workload(seed=3, n_jobs=20, n_netlists=4, scale=0.02)
    reqs = [serve.Request.from_spec(s) for s in specs]
    dt, st = serve.run_batched(nets, reqs, part_items=200_000)
    batched = [r.result for r in reqs]
    serve.run_plain_loop(nets, reqs)
    for k, (a, r) in enumerate(zip(batched, reqs)):
        assert _same(a, r.result), f"job {k}"


def test_served_stream_equals_alone():
    nets, specs = gen.served_workload(seed=4, rate=2000.0, seconds=0.05, scale=0.01)
    reqs = [serve.Request.from_spec(s) for s in specs]
    assert len(reqs) > 20 and any(r.edit_gate is not None for r in reqs)
    makespan, st = serve.run_served(nets, reqs, part_items=300_000)
    mixed = [r.result for r in reqs]
    lat = serve.latency_summary(reqs)
    assert lat["p99_ms"] >= lat["p50_ms"] > 0
    serve.run_served_plain(nets, reqs)
    for k, (a, r) in enumerate(zip(mixed, reqs)):
        assert _same(a, r.result), f"request {k}"


def test_engine_autotuner_picks_a_timed_candidate_and_caches_it():
    """The engine autotuner times every (launch shape, step items) candidate
    on a sample of the stream, returns the fastest, and reuses its choice for
    the same netlist mix; jobs run with the chosen options give the same SAIF
    as the plain path."""
    nets, specs = gen.batched_workload(seed=5, n_jobs=12, n_netlists=3, scale=0.02)
    reqs = [serve.Request.from_spec(s) for s in specs]
    cache = {}
    shapes, steps = ((256, 4), (128, 8)), (1 << 20, 1 << 24)
    opts, timings = serve.autotune_engine(nets, reqs, sample=6, shapes=shapes, steps=steps, cache=cache)
    assert len(timings) == 4
    assert opts == min(timings, key=lambda x: x[0])[1]
    assert (opts["tile_items"], opts["items_per_thread"]) in shapes and opts["step_items"] in steps
    again, _ = serve.autotune_engine(nets, reqs, sample=6, shapes=shapes, steps=steps, cache=cache)
    assert again == opts and len(cache) == 1
    serve.run_batched(nets, reqs, **opts)
    batched = [r.result for r in reqs]
    serve.run_plain_loop(nets, reqs)
    for k, (a, r) in enumerate(zip(batched, reqs)):
        assert _same(a, r.result), f"job {k}"
