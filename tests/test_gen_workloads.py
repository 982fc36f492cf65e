"""The multi-job workloads match the recipes the design notes state
(batched: 64 jobs over 8 mid-recipe netlists of 10k-500k gates, cycles in
[100, 20,000], toggle probability in [0.05, 0.5]; served: 4 resident
netlists of 50k/200k/500k/1M gates, Poisson arrivals at 200/s, windows of
100-5,000 cycles, 30% of requests re-timing 1% of gates by +-[10, 50] ps),
and are reproducible from their seed."""
import numpy as np

import gen


def _toggle_rate(st):
    return st.edge_time.size / (st.init.size * st.num_cycles)


def test_batched_workload_recipe():
    nets, specs = gen.batched_workload(seed=1)
    assert len(nets) == 8 and len(specs) == 64
    for wl in nets:
        G = wl.netlist.num_gates
        assert 10_000 <= G <= 500_000
        assert wl.netlist.num_inputs == max(16, G // 400)
        assert wl.depth == min(gen.interp_depth(G), G)
    cycles = np.array([s["stim"].num_cycles for s in specs])
    assert cycles.min() >= 100 and cycles.max() <= 20_000
    assert 1000 <= np.median(cycles) <= 4000                      # log-normal around 2,000
    rates = np.array([_toggle_rate(s["stim"]) for s in specs])
    # toggle probability 0.05-0.5 plus 5% two-edge pulses (some cancel)
    assert rates.min() > 0.03 and rates.max() < 0.65
    assert all(0 <= s["netlist"] < 8 for s in specs)
    nets2, specs2 = gen.batched_workload(seed=1)
    assert all(np.array_equal(a["stim"].edge_time, b["stim"].edge_time) for a, b in zip(specs, specs2))


def test_served_workload_recipe():
    nets, reqs = gen.served_workload(seed=1, rate=200.0, seconds=1.0)
    assert [wl.netlist.num_gates for wl in nets] == [50_000, 200_000, 500_000, 1_000_000]
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] <= 1.0
    assert 150 <= len(reqs) <= 250                                 # Poisson, mean 200
    cycles = np.array([r["stim"].num_cycles for r in reqs])
    assert cycles.min() >= 100 and cycles.max() <= 5000
    edited = [r for r in reqs if "edit_gate" in r]
    assert 0.2 <= len(edited) / len(reqs) <= 0.4                  # 30% of requests
    for r in edited:
        G = nets[r["netlist"]].netlist.num_gates
        assert r["edit_gate"].size == max(1, G // 100)
        assert np.unique(r["edit_gate"]).size == r["edit_gate"].size
        d = np.abs(r["edit_delta"])
        assert d.min() >= 10 and d.max() <= 50
    rates = np.array([_toggle_rate(r["stim"]) for r in reqs])
    assert np.all(np.abs(rates - 0.3) < 0.1)                       # toggle 0.2 plus 5% pulses
