"""The allocation-free level propagation entry point.

Callers that cannot allocate device memory themselves at run time (memory
owned by a framework or a pool, no implicit device synchronization allowed,
everything reserved up front) pass their own buffers to
gatspi_propagate_level_noalloc.  This test plays such a caller: it lays out
the waveform store the way the header describes, fills level 0 from the
stimulus on the host (record metas plus tile runs or record starts),
runs every level through the new entry point -- twice
in a row, since calls share the library's fixed scratch -- and checks each
run against gatspi_simulate bit for bit (SAIF of every gate net and the
waveforms of sampled windows).  The cases cover both record layouts (tile
runs with 64 or more windows, record starts with fewer), a segment that
starts past window 0, and windows of several cycles with a ragged last one.
Kept in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

import gen
import paper_2203_06117_gb300 as gs

pytestmark = pytest.mark.gpu


def _levels(nl):
    lv = np.zeros(nl.num_nets, np.int32)
    for g in range(nl.num_gates):
        a, b = nl.fanin_ptr[g], nl.fanin_ptr[g + 1]
        lv[nl.num_inputs + g] = 1 + lv[nl.fanin_net[a:b]].max()
    return lv


TW = 128  # windows per gate-aligned tile of the allocation-free entry point


def _level0(wl, NW, fw, W):
    """Input records of batch windows 0..NW-1 (global windows fw..fw+NW-1 of
    W cycles each, the last one clipped to the stimulus): meta (start value
    in bit 15, edge count below), edge times shifted onto each window's own
    time axis (input-major, window order), and where each record's edges
    start: tile runs (first edge, edges) of 128-window tiles with 64 or more
    windows, else one start per record."""
    st, I = wl.stim, wl.netlist.num_inputs
    C, L = st.num_cycles, st.cycle_ps
    T = -(-NW // TW)
    meta = np.zeros(I * NW, np.uint16)
    rstart = np.zeros(I * NW, np.int32)
    tinfo = np.zeros((I * T, 2), np.int32)
    times = []
    for i in range(I):
        for w in range(NW):
            c0 = (fw + w) * W
            c1 = min(c0 + W, C)
            a, b = int(st.edge_ptr[i * C + c0]), int(st.edge_ptr[i * C + c1])
            v0 = int(st.init[i]) ^ ((a - int(st.edge_ptr[i * C])) & 1)
            meta[i * NW + w] = (v0 << 15) | (b - a)
            rstart[i * NW + w] = len(times)
            if w % TW == 0:
                tinfo[i * T + w // TW, 0] = len(times)
            tinfo[i * T + w // TW, 1] += b - a
            for c in range(c0, c1):
                e0, e1 = int(st.edge_ptr[i * C + c]), int(st.edge_ptr[i * C + c + 1])
                times += (st.edge_time[e0:e1].astype(np.int64) + (c - c0) * L).tolist()
    return meta, rstart, tinfo, np.asarray(times, np.int32)


# (tiny workload seed, cycles, window cycles, first window, windows per call)
CASES = [
    (5, 300, 1, 0, 300),     # gate-aligned tiles (tile runs), the whole stimulus
    (6, 200, 1, 37, 40),     # fewer than 64 windows: linear tiles (record starts), a later segment
    (7, 1001, 3, 200, 134),  # three-cycle windows, the last one ragged, a partial second tile
    (8, 120, 2, 5, 20),      # linear tiles with two-cycle windows
]


@pytest.mark.parametrize("seed,C,W,fw,NW", CASES)
def test_noalloc_levels_match_simulate_twice(seed, C, W, fw, NW):
    torch = pytest.importorskip("torch")
    gs.build()
    wl = gen.make_workload("tiny", seed=seed, num_cycles=C)
    nl = wl.netlist
    I, G, N, L = nl.num_inputs, nl.num_gates, nl.num_nets, wl.stim.cycle_ps
    lv = _levels(nl)
    D = int(lv.max())
    assert np.all(np.diff(lv[I:]) >= 0)            # the generator's gates come in level order
    gate_begin = [0] * (D + 2)
    for l in range(1, D + 2):
        gate_begin[l] = int(np.searchsorted(lv[I:], l))
    sample = sorted({fw, fw + NW // 2, fw + NW - 1})

    with gs.Simulator(nl, wl.delays, wl.stim) as sim:
        sim.simulate(window_cycles=W, first_window=fw, num_windows=NW)
        ref_t0, ref_t1, ref_tc = sim.saif()
        ref_windows = {w: sim.window(w) for w in sample}
    seg_time = (min((fw + NW) * W, C) - fw * W) * L

    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    fanin_ptr = t(nl.fanin_ptr, torch.int32)
    fanin_net = t(nl.fanin_net, torch.int32)
    lut = t(nl.lut.astype(np.int16), torch.int16)
    gate_delay = t(wl.delays.gate_delay, torch.int32)
    wire_delay = t(wl.delays.wire_delay, torch.int32)
    net_level = t(lv, torch.int32)
    wide = NW >= 64                                 # gate-aligned tiles: tile runs, no record starts
    T = -(-NW // TW)
    meta0, rstart0, tinfo0, times0 = _level0(wl, NW, fw, W)
    capacity = 8 * N * NW * W + times0.size
    tinfo = torch.zeros((N * T, 2), dtype=torch.int32, device=dev)
    rstart = torch.zeros(N * NW, dtype=torch.int32, device=dev)
    rmeta = torch.zeros(N * NW, dtype=torch.int16, device=dev)
    times = torch.zeros(capacity, dtype=torch.int32, device=dev)
    lvl_base = torch.zeros(D + 2, dtype=torch.int64, device=dev)
    saif_t1 = torch.zeros(N, dtype=torch.int64, device=dev)
    saif_tc = torch.zeros(N, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    err = ctypes.create_string_buffer(256)

    for run in range(2):
        tinfo[:I * T] = t(tinfo0, torch.int32)
        rstart[:I * NW] = t(rstart0, torch.int32)
        rmeta[:I * NW] = t(meta0.view(np.int16), torch.int16)
        times[:times0.size] = t(times0, torch.int32)
        lvl_base.zero_()
        lvl_base[1] = int(times0.size)
        saif_t1.zero_()
        saif_tc.zero_()
        status.zero_()
        torch.cuda.synchronize()
        for level in range(1, D + 1):
            a = gs.gatspi_level_args(
                fanin_ptr.data_ptr(), fanin_net.data_ptr(), lut.data_ptr(), gate_delay.data_ptr(),
                wire_delay.data_ptr(), net_level.data_ptr(), None if wide else rstart.data_ptr(),
                tinfo.data_ptr() if wide else None, rmeta.data_ptr(),
                times.data_ptr(), lvl_base.data_ptr(), capacity, saif_t1.data_ptr(),
                saif_tc.data_ptr(), status.data_ptr(), I, level, gate_begin[level],
                gate_begin[level + 1], NW, fw, W, C, L, 256, ctypes.cast(err, ctypes.c_char_p))
            rc = gs.lib().gatspi_propagate_level_noalloc(ctypes.byref(a), None)
            assert rc == gs.OK, err.value.decode()
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"run {run}: status {int(status.item())}"

        t1 = saif_t1.cpu().numpy()
        tc = saif_tc.cpu().numpy()
        assert np.array_equal(t1[I:], ref_t1[I:]), f"run {run}: T1 differs"
        assert np.array_equal(tc[I:], ref_tc[I:]), f"run {run}: TC differs"
        assert np.array_equal(seg_time - t1[I:], ref_t0[I:])

        h_tinfo = tinfo.cpu().numpy()
        h_rstart = rstart.cpu().numpy()
        h_meta = rmeta.cpu().numpy().view(np.uint16)
        h_times, h_base = times.cpu().numpy(), lvl_base.cpu().numpy()
        for gw, (ri, rp, rt) in ref_windows.items():
            w = gw - fw                             # the window's index in the call's batch
            for n in range(I, N):
                r = n * NW + w
                if wide:                            # the window's tile: run start + earlier counts
                    t0 = w // TW * TW
                    s = int(h_tinfo[n * T + w // TW, 0]) + int((h_meta[n * NW + t0:r] & 0x7FFF).sum())
                else:
                    s = int(h_rstart[r])
                c = int(h_meta[r]) & 0x7FFF
                b0 = int(h_base[lv[n]])
                got = h_times[b0 + s:b0 + s + c].tolist()
                assert int(h_meta[r]) >> 15 == int(ri[n]), f"run {run} window {gw} net {n}: start value"
                assert got == rt[rp[n]:rp[n + 1]].tolist(), f"run {run} window {gw} net {n}: edges"


def test_noalloc_rejects_levels_beyond_its_limit():
    pytest.importorskip("torch")
    gs.build()
    err = ctypes.create_string_buffer(256)
    dummy = 16  # never dereferenced: the size check comes first
    # 4096 gates x 2^20 windows = 2^32 items, beyond GATSPI_NOALLOC_MAX_ITEMS
    a = gs.gatspi_level_args(*([dummy] * 11), 1 << 20, dummy, dummy, dummy, 4, 1, 0, 4096,
                             1 << 20, 0, 1, 1 << 20, 1000, 256,
                             ctypes.cast(err, ctypes.c_char_p))
    rc = gs.lib().gatspi_propagate_level_noalloc(ctypes.byref(a), None)
    assert rc == gs.ECAPACITY
    assert b"GATSPI_NOALLOC_MAX_ITEMS" in err.value
