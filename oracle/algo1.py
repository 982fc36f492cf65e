"""ORACLE -- test infrastructure only (tests, smoke check, CPU baseline).

Second, independent CPU formulation of GATSPI re-simulation (Zhang et al.,
DAC'22): the per-gate, per-cycle procedure of Algorithm 1, applied gate by
gate in topological (net id) order for each window.  It is written in the
paper's notation -- the waveform array ``allW`` in the array format the paper
takes from Holst et al. (Section 3, Fig. "Waveform"), pin pointers ``p_i``,
output pointer ``p_o``, ``colInd``, ``y``, ``t_i``, ``netDelay``,
``gateDelay``, ``EOW`` -- so that it can be read against Algorithm 1, and it
shares nothing with the event-driven simulator in ``event_sim.c``.

Array format (Section 3; the figure itself is not reproduced in the text, the
format is implied by Algorithm 1): a waveform is a list of int timestamps;
the entry at index k opens an interval whose logic value is k % 2; a signal
that starts at 1 is written ``[-1, 0, ...]`` so that index 1 (odd) opens the
first interval; the list ends with EOW = INT_MAX.

Readings where Algorithm 1 is silent or literally inconsistent:
  * the interconnect pulse test is repeated until the next edge survives
    (the literal "p_i += 2; continue" takes one skip per outer step and can
    process another pin's later edge first);
  * a pin whose next entry is EOW offers no candidate and is not tested
    (the literal test would read past EOW);
  * with several pins switching at t_i, the last pin in loop order (the
    highest index) sets gateDelay, read in row 2*(new pin value) + (new y)
    and in the column of the other pins' values after the switch.

PATHPULSEPERCENT (Section 3: Algorithm 1 assumes 100, and other values edit
the output test).  ``pulse_gate`` = pct turns the output test into
100 (t_o - allW[p_o]) < pct gateDelay; ``pulse_wire`` = pct turns the
interconnect test into 100 (allW[p_i+2] - allW[p_i+1]) < pct netDelay.
Below 100 a pulse can be shorter than the delay difference of its two
edges, so both tests also drop a pulse whose width after the delays is
zero or negative (at 100 that case is already covered).  0 is transport
delay.

Pure Python: use it on small cases only.
"""
from __future__ import annotations

EOW = 2**31 - 1


def to_array(init: int, times) -> list:
    """(initial value, edge times) -> array format with EOW."""
    return ([-1, 0] if init else [0]) + [int(t) for t in times] + [EOW]


def from_array(w: list) -> tuple:
    """array format -> (initial value, edge times)."""
    if w[0] == -1:
        return 1, w[2:-1]
    return 0, w[1:-1]


def _without_bit(col: int, i: int) -> int:
    return (col & ((1 << i) - 1)) | ((col >> (i + 1)) << i)


def resimulate_gate(allW_in: list, n: int, Y: int, delta: list, d: list,
                    pulse_gate: int = 100, pulse_wire: int = 100) -> list:
    """Algorithm 1 for one gate and one window.

    allW_in  -- per pin i (0-based; the paper's pin i+1) the input waveform
                in array format;
    Y        -- truth table as an int, bit colInd = output value;
    delta    -- per pin (rise, fall) interconnect delay;
    d        -- per pin a flat 32-entry gate delay table indexed
                [inEdge][outEdge][side] (row = 2*inEdge + outEdge, 8 columns).
    Returns the output waveform in array format.
    """
    p = [0] * n
    # initial value: skip the -1 marker of signals that start at 1
    for i in range(n):
        if allW_in[i][p[i]] == -1:
            p[i] += 1
    colInd = 0
    for i in range(n):
        colInd |= (p[i] % 2) << i
    y = (Y >> colInd) & 1
    out = [0] if y == 0 else [-1, 0]
    p_o = len(out) - 1
    gateDelay = None
    t_i = None
    while t_i != EOW:
        # next event: earliest delayed arrival over the pins, after dropping
        # pulses narrower than the interconnect delay of their first edge
        t_i = EOW
        for i in range(n):
            W = allW_in[i]
            netDelay = delta[i][1] if p[i] % 2 else delta[i][0]
            while W[p[i] + 1] != EOW and W[p[i] + 2] != EOW:
                # the pulse (p_i+1, p_i+2): its second edge has the other
                # direction, so the other delay
                nextDelay = delta[i][0] if p[i] % 2 else delta[i][1]
                narrow = 100 * (W[p[i] + 2] - W[p[i] + 1]) < pulse_wire * netDelay
                crossed = W[p[i] + 2] + nextDelay <= W[p[i] + 1] + netDelay
                if not (narrow or crossed):
                    break
                p[i] += 2
            if W[p[i] + 1] != EOW:
                t_i = min(t_i, W[p[i] + 1] + netDelay)
        if t_i != EOW:
            # every pin arriving at t_i switches (MSI), then y is re-evaluated
            for i in range(n):
                W = allW_in[i]
                netDelay = delta[i][1] if p[i] % 2 else delta[i][0]
                if W[p[i] + 1] != EOW and W[p[i] + 1] + netDelay == t_i:
                    p[i] += 1
                    colInd = (colInd & ~(1 << i)) | ((p[i] % 2) << i)
                    y = (Y >> colInd) & 1
                    gateDelay = d[i][(2 * (p[i] % 2) + y) * 8 + _without_bit(colInd, i)]
            if y != p_o % 2:
                t_o = t_i + gateDelay
                if 100 * (t_o - out[p_o]) < pulse_gate * gateDelay or t_o <= out[p_o]:
                    p_o -= 1                       # cancel the last kept edge
                else:
                    p_o += 1
                    if p_o == len(out):
                        out.append(t_o)
                    else:
                        out[p_o] = t_o
    return out[:p_o + 1] + [EOW]


def simulate_window(netlist, delays, stim, w: int, W: int = 1, pulse_gate: int = 100,
                    pulse_wire: int = 100):
    """All nets of window w: returns a list of (init, times) per net id.

    Inputs of window w start from their value after the cycles before the
    window; their edges are placed on the window's own time axis.
    """
    I = netlist.num_inputs
    G = netlist.num_gates
    C, L = stim.num_cycles, stim.cycle_ps
    c0, c1 = w * W, min((w + 1) * W, C)
    waves = []
    for i in range(I):
        before = int(stim.edge_ptr[i * C + c0] - stim.edge_ptr[i * C])
        init = int(stim.init[i]) ^ (before & 1)
        times = []
        for c in range(c0, c1):
            a, b = int(stim.edge_ptr[i * C + c]), int(stim.edge_ptr[i * C + c + 1])
            times += [(c - c0) * L + int(t) for t in stim.edge_time[a:b]]
        waves.append(to_array(init, times))
    for g in range(G):
        a, b = int(netlist.fanin_ptr[g]), int(netlist.fanin_ptr[g + 1])
        n = b - a
        ins = [waves[int(netlist.fanin_net[q])] for q in range(a, b)]
        delta = [(int(delays.wire_delay[2 * q]), int(delays.wire_delay[2 * q + 1])) for q in range(a, b)]
        d = [[int(v) for v in delays.gate_delay[32 * q:32 * q + 32]] for q in range(a, b)]
        waves.append(resimulate_gate(ins, n, int(netlist.lut[g]), delta, d, pulse_gate, pulse_wire))
    return [from_array(x) for x in waves]


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
