"""ORACLE -- test infrastructure only (tests, smoke check, CPU baseline).

Second, independent CPU formulation of GATSPI re-simulation (Zhang et al.,
DAC'22, Section 3 and Algorithm 1): gates are evaluated one at a time in
topological (net id) order for each window, each from the complete
waveforms of its fanin nets.  It shares nothing with the event-driven
simulator in ``event_sim.c``, which keeps one global event queue per window
instead.  One gate in one window takes three steps:

1. Arrivals per pin.  A fanin edge reaches the gate after the pin's
   interconnect delay for its direction (rising or falling).  Interconnect
   inertial filter: a pulse -- an edge and the pin's next edge -- narrower
   than the delay of its first edge is rejected as a pair, and the scan goes
   on after the pair, so a run of narrow pulses is rejected pulse by pulse;
   a pin's last edge has no partner and always arrives.
2. Events.  The distinct arrival times of all pins, in time order.  Every
   pin with an arrival at a time switches at that time (multiple
   simultaneous input switching), then the truth table gives the new output
   value.  The delay of an output change comes from the highest-index pin
   that switched: its table row is 2 * (its new value) + (new output value),
   its column the other pins' values after the switch (the COND condition).
3. Output.  The kept output edges form a stack.  An output change at time t
   with delay d proposes an edge at t + d; gate inertial filter: if that is
   closer than d to the last kept edge, the last kept edge is removed
   instead (so the output keeps its value), else the new edge is kept.

Readings where Algorithm 1 is silent or literally inconsistent (also taken
by the event-driven simulator):
  * the interconnect test repeats until the next edge survives (the listing
    takes one skip per step of its loop);
  * a pin's last edge is never tested (the listing would read past its end
    marker);
  * with several pins switching at once, the highest-index pin picks the
    delay arc, with the post-switch column.

Pulse limits (PATHPULSEPERCENT; Section 3: Algorithm 1 assumes 100, other
values edit its output test).  With ``pulse_gate`` = pct the gate test is
100 (t_o - E) < pct d for the last kept edge E; with ``pulse_wire`` = pct
the interconnect test is 100 (width) < pct delay.  Below 100 a pulse can be
shorter than the difference of its two edges' delays, so both tests also
reject a pulse that would come out with zero or negative width.  0 is
transport delay; an interconnect limit of 0 is also the paper's variant
without interconnect filtering (Section 5, Table "features").
``full_sdf=False`` is the paper's partial-SDF variant (same table): every
arc keeps only its average delay per output edge over all COND columns and
both input edges, rounded to the nearest ps (halves up).

Pure Python: use it on small cases only.
"""
from __future__ import annotations


def _side(col: int, i: int) -> int:
    """The other pins' bits of col: pin i's bit removed."""
    return (col & ((1 << i) - 1)) | ((col >> (i + 1)) << i)


def pin_arrivals(start: int, times, rise: int, fall: int, pct: int = 100) -> list:
    """Arrival times at the gate of one fanin pin's edges (window-relative,
    strictly increasing), after the interconnect inertial filter.  Edge k
    rises when start and k have equal parity."""
    delay = [rise if ((start ^ k) & 1) == 0 else fall for k in range(len(times))]
    out, k = [], 0
    while k < len(times):
        if k + 1 < len(times):
            narrow = 100 * (times[k + 1] - times[k]) < pct * delay[k]
            crossing = times[k + 1] + delay[k + 1] <= times[k] + delay[k]
            if narrow or crossing:
                k += 2                      # the pulse is rejected as a pair
                continue
        out.append(times[k] + delay[k])
        k += 1
    return out


def averaged_table(table: list, n: int) -> list:
    """Partial SDF: a pin's 32-entry table [inEdge][outEdge][side] with every
    entry replaced by the arc's mean for its output edge over both input
    edges and the gate's 2^(n-1) COND columns (nearest ps, halves up)."""
    ncol = 1 << (n - 1)
    out = [0] * 32
    for oe in range(2):
        vals = [table[(2 * ie + oe) * 8 + c] for ie in range(2) for c in range(ncol)]
        avg = (sum(vals) + len(vals) // 2) // len(vals)
        for ie in range(2):
            for c in range(8):
                out[(2 * ie + oe) * 8 + c] = avg
    return out


def gate_window(fanins, n: int, truth: int, wire: list, tables: list, pulse_gate: int = 100,
                pulse_wire: int = 100) -> tuple:
    """One gate in one window.

    fanins -- per pin (0-based; pin 0 is the least significant truth-table
              bit) the driving net's waveform (start value, edge times);
    truth  -- truth table as an int, bit c = output for input combination c;
    wire   -- per pin (rise, fall) interconnect delay;
    tables -- per pin a 32-entry gate delay table [inEdge][outEdge][side].
    Returns the output waveform (start value, edge times).
    """
    arrivals = [pin_arrivals(s, t, wire[i][0], wire[i][1], pulse_wire) for i, (s, t) in enumerate(fanins)]
    col = sum(s << i for i, (s, _) in enumerate(fanins))
    y0 = (truth >> col) & 1
    kept = []
    for t in sorted({a for arr in arrivals for a in arr}):
        switching = [i for i in range(n) if t in arrivals[i]]
        for i in switching:
            col ^= 1 << i
        y = (truth >> col) & 1
        if y == y0 ^ (len(kept) & 1):      # the output value does not change
            continue
        i = switching[-1]
        d = tables[i][(2 * ((col >> i) & 1) + y) * 8 + _side(col, i)]
        to = t + d
        if kept and (100 * (to - kept[-1]) < pulse_gate * d or to <= kept[-1]):
            kept.pop()
        else:
            kept.append(to)
    return y0, kept


def simulate_window(netlist, delays, stim, w: int, W: int = 1, pulse_gate: int = 100,
                    pulse_wire: int = 100, full_sdf: bool = True):
    """All nets of window w (cycles [w W, (w+1) W) clipped to the stimulus):
    a list of (start value, edge times) per net id.  Inputs start from their
    value after the cycles before the window; their edges are placed on the
    window's own time axis.  Gates start from the zero-delay values of their
    fanins' start values (step 3 begins from the truth table there)."""
    I, G = netlist.num_inputs, netlist.num_gates
    C, L = stim.num_cycles, stim.cycle_ps
    c0, c1 = w * W, min((w + 1) * W, C)
    waves = []
    for i in range(I):
        before = int(stim.edge_ptr[i * C + c0] - stim.edge_ptr[i * C])
        times = []
        for c in range(c0, c1):
            a, b = int(stim.edge_ptr[i * C + c]), int(stim.edge_ptr[i * C + c + 1])
            times += [(c - c0) * L + int(t) for t in stim.edge_time[a:b]]
        waves.append((int(stim.init[i]) ^ (before & 1), times))
    for g in range(G):
        a, b = int(netlist.fanin_ptr[g]), int(netlist.fanin_ptr[g + 1])
        n = b - a
        fanins = [waves[int(netlist.fanin_net[q])] for q in range(a, b)]
        wire = [(int(delays.wire_delay[2 * q]), int(delays.wire_delay[2 * q + 1])) for q in range(a, b)]
        tables = [[int(v) for v in delays.gate_delay[32 * q:32 * q + 32]] for q in range(a, b)]
        if not full_sdf:
            tables = [averaged_table(tb, n) for tb in tables]
        waves.append(gate_window(fanins, n, int(netlist.lut[g]), wire, tables, pulse_gate, pulse_wire))
    return waves


def window_length(stim, w: int, W: int = 1) -> int:
    c0 = w * W
    return (min(c0 + W, stim.num_cycles) - c0) * stim.cycle_ps


def saif_of_waves(waves, length: int):
    """Per net (T1, TC) of one window: time at 1 within [0, length), edges."""
    out = []
    for init, times in waves:
        v, prev, t1 = init, 0, 0
        for t in times:
            t = min(int(t), length)
            if v:
                t1 += t - prev
            prev, v = t, v ^ 1
        if v:
            t1 += length - prev
        out.append((t1, len(times)))
    return out
