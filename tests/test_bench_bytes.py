"""The roofline's algorithmic bytes in bench.py: the per-(gate, cycle)
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
