"""Helpers shared by the tests: hand-traced golden cases -> input arrays."""
import json
import os

import numpy as np

import gen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_hand_traced():
    with open(os.path.join(GOLDEN, "hand_traced.json")) as f:
        return json.load(f)["cases"]


def case_workload(case) -> gen.Workload:
    """Build netlist, delays and stimulus arrays from a golden case."""
    I = len(case["inputs"])
    fp, fn, npins, lut, gd, wd = [0], [], [], [], [], []
    for g in case["gates"]:
        n = len(g["pins"])
        npins.append(n)
        lut.append(gen.cell_lut(g["cell"]))
        for pin in g["pins"]:
            fn.append(pin["net"])
            tab = np.zeros((2, 2, 8), np.int32)
            ncol = 1 << (n - 1)
            if "iopath" in pin:
                for oe in range(2):
                    tab[:, oe, :ncol] = pin["iopath"][oe]
            else:
                for row in range(4):
                    tab[row // 2, row % 2, :ncol] = pin["cond"][row]
            gd.append(tab.reshape(-1))
            wd += list(pin["wire"])
        fp.append(len(fn))
    nl = gen.Netlist(I, np.asarray(fp, np.int32), np.asarray(fn, np.int32),
                     np.asarray(npins, np.uint8), np.asarray(lut, np.uint16),
                     np.zeros(len(npins), np.uint8))
    dl = gen.Delays(np.concatenate(gd).astype(np.int32), np.asarray(wd, np.int32))
    C = len(case["inputs"][0]["cycles"])
    ptr, times = [0], []
    for inp in case["inputs"]:
        assert len(inp["cycles"]) == C
        for cyc in inp["cycles"]:
            times += cyc
            ptr.append(len(times))
    st = gen.Stimulus(C, case["cycle_ps"], np.asarray([x["init"] for x in case["inputs"]], np.uint8),
                      np.asarray(ptr, np.int64), np.asarray(times, np.int32))
    return gen.Workload(case["name"], nl, dl, st, 0, {})
