"""Helpers shared by several test modules: bit-exact comparisons of the
library's results with the oracle's, delay edits applied to a delay table,
and a small VCD writer and SAIF parser for the file-format tests."""
import re

import numpy as np

import gen
from oracle import stimulus as ostim


def assert_window_equal(sim, ref, w, what=""):
    gi, gp, gt = sim.window(w)
    oi, op, ot = ref.window(w)
    if not np.array_equal(gi, oi):
        n = int(np.nonzero(gi != oi)[0][0])
        raise AssertionError(f"{what} window {w}: start value of net {n}: gpu {gi[n]} oracle {oi[n]}")
    if not (np.array_equal(gp, op) and np.array_equal(gt, ot)):
        cg, co = np.diff(gp), np.diff(op)
        bad = np.nonzero(cg != co)[0]
        n = int(bad[0]) if bad.size else -1
        if n < 0:
            for m in range(gi.shape[0]):
                if not np.array_equal(gt[gp[m]:gp[m + 1]], ot[op[m]:op[m + 1]]):
                    n = m
                    break
        raise AssertionError(f"{what} window {w}: net {n}: gpu {gt[gp[n]:gp[n + 1]].tolist()} "
                             f"oracle {ot[op[n]:op[n + 1]].tolist()}")

def assert_saif_equal(sim, ref):
    g = sim.saif()
    o = ref.saif()
    for name, a, b in zip(("T0", "T1", "TC"), g, o):
        if not np.array_equal(a, b):
            n = int(np.nonzero(a != b)[0][0])
            raise AssertionError(f"SAIF {name} of net {n}: gpu {a[n]} oracle {b[n]}")

def edited_delays(nl, dl, gates, deltas):
    """The delay table with a job's edit applied: every gate delay of an
    edited gate shifted by its delta, clamped at 1 ps."""
    gd = dl.gate_delay.copy().reshape(-1, 2, 2, 8)
    for g, d in zip(gates, deltas):
        a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
        ncol = 1 << (b - a - 1)
        blk = gd[a:b, :, :, :ncol]
        gd[a:b, :, :, :ncol] = np.maximum(1, blk + int(d))
    return gen.Delays(gd.reshape(-1), dl.wire_delay)

def _codes(k):
    """VCD identifier codes: printable characters 33..126, several per code."""
    out = []
    for n in range(k):
        s, n = "", n + 1
        while n:
            n, r = divmod(n - 1, 94)
            s = chr(33 + r) + s
        out.append(s)
    return out

def write_vcd(path, stim, names, unit="1ps", scope=("top",), glitch_every=0, alias=None):
    """A VCD dump of a per-cycle stimulus (absolute times divided by the
    unit's picoseconds, which must divide them)."""
    ps = {"1ps": 1, "10ps": 10, "100ps": 100, "1ns": 1000, "1 ps": 1}[unit]
    I = stim.init.size
    codes = _codes(I)
    inp, t = gs_events = ostim.cycles_to_events(stim)
    assert np.all(t % ps == 0)
    order = np.lexsort((inp, t))
    lines = ["$date today $end", "$version writer in the tests $end", f"$timescale {unit} $end"]
    for s in scope:
        lines.append(f"$scope module {s} $end")
    for k in range(I):
        lines.append(f"$var wire 1 {codes[k]} {names[k]} $end")
    if alias is not None:                      # a second name sharing input 0's code
        lines.append(f"$var wire 1 {codes[0]} {alias} $end")
    lines.append("$var wire 4 " + "%%" + " bus [3:0] $end")
    for _ in scope:
        lines.append("$upscope $end")
    lines += ["$enddefinitions $end", "#0", "$dumpvars"]
    lines += [f"{int(stim.init[k])}{codes[k]}" for k in range(I)] + ["b0000 %%", "$end"]
    val = stim.init.astype(np.int64).copy()
    cur = None
    for j, e in enumerate(order):
        tt, k = int(t[e]) // ps, int(inp[e])
        if tt != cur:
            lines.append(f"#{tt}")
            cur = tt
            if glitch_every and j % glitch_every == 0:
                # a zero-width glitch on another input: two changes in one step
                o = (k + 1) % I
                lines += [f"{1 - val[o]}{codes[o]}", f"{val[o]}{codes[o]}"]
        val[k] ^= 1
        lines.append(f"{val[k]}{codes[k]}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")

def parse_saif(path):
    text = open(path).read()
    head = dict(re.findall(r"\((DURATION|DESIGN|TIMESCALE) ([^)]*)\)", text))
    nets = {}
    for name, t0, t1, tx, tc, ig in re.findall(
            r"\(((?:\\.|[A-Za-z0-9_])+)\s*\(T0 (\d+)\) \(T1 (\d+)\) \(TX (\d+)\)\s*\(TC (\d+)\) \(IG (\d+)\)",
            text):
        nets[re.sub(r"\\(.)", r"\1", name)] = (int(t0), int(t1), int(tx), int(tc), int(ig))
    return head, nets
