"""Expected results of the batched and served job streams, from the CPU oracle.

Writes tests/golden/engine_streams.json: for every job of the batched stream
(64 jobs over 8 netlists of the mid recipe, gen.batched_workload, seed 1) and
for a sample of the served stream (gen.served_workload, seed 1, 200 requests/s
for 1 s: every tenth request plus the first edited requests not among them),
three 64-bit folds over the job's nets -- of the SAIF T1, of the SAIF TC and
of the per-net waveform digests (oracle/digest.py) -- and the T1 and TC
totals.  A fold of a per-net vector v is  sum_n mix(v[n] ^ mix(n + 1))  mod
2^64, with mix the SplitMix64 output function, so it changes when any one
net's value changes.  Every value comes from the event-driven oracle
(oracle.EventSim) on the job's netlist, its delays with the job's delay edit
applied, and its stimulus, one cycle per window; nothing comes from the GPU
library.  The oracle is too slow to rerun inside the GPU tests (about 4e10
gate-cycles), so its results are kept here.

    python tests/golden/make_engine_golden.py [processes]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "engine_streams.json")
SEED = 1
SERVED_RATE, SERVED_SECONDS = 200.0, 1.0


def served_sample(reqs):
    """Every tenth request, plus the first six edited requests not among them."""
    pick = list(range(0, len(reqs), 10))
    extra = [k for k, r in enumerate(reqs) if "edit_gate" in r and k not in pick][:6]
    return sorted(pick + extra)


def fold(v):
    from oracle.digest import mix
    v = np.asarray(v).astype(np.uint64)
    n = np.arange(v.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(mix(v ^ mix(n + np.uint64(1))), dtype=np.uint64))


_W = {}


def _init():
    import gen
    _W["batched"] = gen.batched_workload(seed=SEED)
    _W["served"] = gen.served_workload(seed=SEED, rate=SERVED_RATE, seconds=SERVED_SECONDS)
    _W["sims"] = {}


def _sim(stream, k):
    import oracle
    from helpers import edited_delays
    key = (stream, k)
    if key not in _W["sims"]:
        nets, jobs = _W[stream]
        j = jobs[k]
        wl = nets[j["netlist"]]
        dl = wl.delays
        if j.get("edit_gate") is not None:
            dl = edited_delays(wl.netlist, wl.delays, j["edit_gate"], j["edit_delta"])
        _W["sims"].clear()  # one job's oracle at a time per worker
        _W["sims"][key] = oracle.EventSim(wl.netlist, dl, j["stim"], W=1)
    return _W["sims"][key]


def _unit(stream, k, windows):
    from oracle import digest as odig
    sim = _sim(stream, k)
    dig = np.zeros(sim.N, np.uint64)
    t1 = np.zeros(sim.N, np.int64)
    tc = np.zeros(sim.N, np.int64)
    with np.errstate(over="ignore"):
        for w in windows:
            init, ptr, times = sim.window(int(w))
            dig += odig.window_terms(init, ptr, times, int(w))
            t1 += sim.window_t1()[0]
            tc += np.diff(ptr)
    return stream, k, dig, t1, tc


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    import gen
    import oracle
    gen.build()
    oracle.build()
    b_nets, b_jobs = gen.batched_workload(seed=SEED)
    s_nets, s_reqs = gen.served_workload(seed=SEED, rate=SERVED_RATE, seconds=SERVED_SECONDS)
    sample = served_sample(s_reqs)
    todo = [("batched", k, b_nets[j["netlist"]].netlist.num_gates, j["stim"].num_cycles)
            for k, j in enumerate(b_jobs)]
    todo += [("served", k, s_nets[s_reqs[k]["netlist"]].netlist.num_gates, s_reqs[k]["stim"].num_cycles)
             for k in sample]
    units = []
    for stream, k, G, C in todo:  # large jobs split into window chunks
        chunks = max(1, min(procs * 2, int(G * C // 400_000_000)))
        units += [(stream, k, list(range(c, C, chunks))) for c in range(chunks)]
    units.sort(key=lambda u: -len(u[2]) * (b_nets if u[0] == "batched" else s_nets)[
        (b_jobs if u[0] == "batched" else s_reqs)[u[1]]["netlist"]].netlist.num_gates)
    acc = {}
    t = time.time()
    with mp.get_context("spawn").Pool(procs, initializer=_init) as pool:
        for stream, k, dig, t1, tc in pool.imap_unordered(_unit_star, units):
            a = acc.setdefault((stream, k), [np.zeros_like(dig), np.zeros_like(t1), np.zeros_like(tc)])
            with np.errstate(over="ignore"):
                a[0] += dig
            a[1] += t1
            a[2] += tc
    out = {"what": __doc__.split("\n\n")[0], "seed": SEED, "served_rate": SERVED_RATE,
           "served_seconds": SERVED_SECONDS, "served_sample": sample, "batched": [], "served": []}
    for stream, k, G, C in todo:
        dig, t1, tc = acc[(stream, k)]
        out[stream].append({"job": k, "gates": int(G), "cycles": int(C),
                            "fold_t1": f"{fold(t1):016x}", "fold_tc": f"{fold(tc):016x}",
                            "fold_digest": f"{fold(dig):016x}", "sum_t1": int(t1.sum()),
                            "sum_tc": int(tc.sum())})
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}: {len(out['batched'])} batched, {len(out['served'])} served jobs in {time.time() - t:.0f} s")


def _unit_star(u):
    return _unit(*u)


if __name__ == "__main__":
    main()
