"""Host-side logic of bench.py. The roofline's algorithmic bytes: the per-(gate, cycle)
figure of the waveform format (every fanin waveform read once and the
output written once, each as a start value, an end marker and its edges, 4
bytes apiece, plus an 8-byte offset), summed in closed form from toggle
counts and fanouts, must equal the per-item sum taken item by item."""
import numpy as np

import bench
import gen
import oracle


def test_format_bytes_match_a_per_item_sum():
    wl = gen.make_workload("tiny", seed=1, num_cycles=4)
    ref = oracle.EventSim(wl.netlist, wl.delays, wl.stim, W=1)
    _, _, tc = ref.saif()
    nl, I = wl.netlist, wl.netlist.num_inputs
    brute = 0
    for w in range(4):
        _, ptr, _ = ref.window(w)
        e = np.diff(ptr)
        for g in range(nl.num_gates):
            pins = nl.fanin_net[nl.fanin_ptr[g]:nl.fanin_ptr[g + 1]]
            brute += sum(4 * (2 + int(e[n])) for n in pins) + 4 * (2 + int(e[I + g])) + 8
    assert bench.format_bytes_per_step(nl, tc, 4) == brute


def test_clock_samples_summary():
    """bench.py's record of clocks during the timed region: the median SM
    clock, the maximum, and every throttle reason seen active."""
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
               "2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line",
               "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["1500, 2070, 1000, 0x48, Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["sm_mhz"] is None


def test_traffic_record_is_read_per_shape_and_only_for_its_kernel_source(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from the committed ncu record only while
    the kernel source hashes to the recorded value, for the launch shapes it
    lists; otherwise it is null."""
    import hashlib
    import os
    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "paper_2203_06117_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "kernels.cuh").write_bytes(b"kernel source")
    digest = hashlib.sha256(b"kernel source").hexdigest()
    rec = root / "profiles" / "propagate_kernel_traffic.txt"
    rec.write_text(f"# comment: a line\nkernels_cuh_sha256: {digest}\ntraffic_bytes_per_level_128x4: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic(128, 4) == 1234
    assert bench._traffic(256, 4) is None
    rec.write_text("kernels_cuh_sha256: 00\ntraffic_bytes_per_level_128x4: 1234\n")
    assert bench._traffic(128, 4) is None
    os.remove(rec)
    assert bench._traffic(128, 4) is None
