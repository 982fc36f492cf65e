"""ORACLE -- test infrastructure.

Plain, slow CPU re-simulators of GATSPI (Zhang et al., DAC'22) used to check
the GPU library.  Only the tests, the smoke check (``__graft_entry__.smoke``)
and the CPU-baseline leg of ``bench.py`` may import this package; the
library itself never does, and nothing here is a fallback for it.

* ``event_sim.c`` -- event-driven simulator with one global time-ordered
  event queue per window (the primary oracle).
* ``algo1.py``    -- Algorithm 1 applied gate by gate in the paper's array
  format (second formulation, pure Python, small cases).

Every function cites the passage it follows in its own docstring or in the
source file's header.  Parity status: the event simulator and the Algorithm 1
formulation are pinned by hand-traced single-gate cases, zero-delay settled
values, SAIF invariants and closed forms for chains (see ``tests/``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import algo1  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
# test-only build of the same file with the planted-mistake switches compiled
# in (OSIM_PLANTED_MISTAKES); the oracle itself is built without them
_SO_PLANTED = os.path.join(_HERE, "_build", "liboracle_planted.so")
_libs = {}

MUTATIONS = {
    "none": 0, "wire_rise_fall_swapped": 1, "wire_cancel_on_equal": 2,
    "gate_cancel_on_equal": 3, "msi_lowest_pin": 4, "side_before_switch": 5,
    "row_transposed": 6, "t1_unclipped": 7, "window_init_from_cycle0": 8,
    "no_wire_filter": 9, "no_gate_filter": 10, "out_delay_from_old_y": 11,
    "gate_stack_depth_one": 12, "wire_crossing_kept": 13, "side_low_bits": 14,
}


def build(force: bool = False, planted: bool = False) -> str:
    """Compile event_sim.c with the host C compiler (``planted``: the
    test-only build with the planted-mistake switches)."""
    src = os.path.join(_HERE, "event_sim.c")
    so = _SO_PLANTED if planted else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(so), exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", *(
            ["-DOSIM_PLANTED_MISTAKES"] if planted else []), "-o", tmp, src])
        os.replace(tmp, so)
    return so


def _load(planted: bool = False):
    if planted not in _libs:
        lib = ctypes.CDLL(build(planted=planted))
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.osim_create.restype = vp
        lib.osim_create.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, i32, i32]
        lib.osim_destroy.restype = None
        lib.osim_destroy.argtypes = [vp]
        lib.osim_num_windows.restype = i32
        lib.osim_num_windows.argtypes = [vp]
        lib.osim_run_window.restype = i64
        lib.osim_run_window.argtypes = [vp, i32]
        lib.osim_get.restype = None
        lib.osim_get.argtypes = [vp, vp, vp, vp]
        lib.osim_t1.restype = i32
        lib.osim_t1.argtypes = [vp, vp]
        lib.osim_saif.restype = i64
        lib.osim_saif.argtypes = [vp, i32, i32, vp, vp]
        lib.osim_set_pulse.restype = i32
        lib.osim_set_pulse.argtypes = [vp, i32, i32]
        lib.osim_set_full_sdf.restype = i32
        lib.osim_set_full_sdf.argtypes = [vp, i32]
        _libs[planted] = lib
    return _libs[planted]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class EventSim:
    """Event-driven oracle over one netlist + delays + stimulus.

    ``W`` is the window length in cycles (each window starts from its
    settled values and runs on its own time axis).  ``pulse_gate`` and
    ``pulse_wire`` are the pulse limits (PATHPULSEPERCENT, 0..100) of the
    gate and interconnect inertial tests; 100 is Algorithm 1 as printed,
    0 transport delay (Section 3: other values edit the output test).

    The two features the paper switches off to measure their cost (Section
    5, Table "features"):
    ``interconnect_filter=False`` deletes Algorithm 1's interconnect test;
    arrivals of one pin that would cross or coincide still cancel as a pair,
    which keeps each pin's arrivals in time order as Algorithm 1 assumes (the
    same as an interconnect pulse limit of 0 percent).
    ``full_sdf=False`` replaces each arc's table by its average rise and
    fall delay over all COND columns and both input edges (osim_set_full_sdf).
    ``mutation`` selects a planted mistake of the test-only build.
    """

    def __init__(self, netlist, delays, stim, W: int = 1, mutation: str = "none",
                 pulse_gate: int = 100, pulse_wire: int = 100, interconnect_filter: bool = True,
                 full_sdf: bool = True):
        if not interconnect_filter:
            if pulse_wire != 100:
                raise ValueError("oracle: interconnect_filter=False sets the interconnect limit itself")
            pulse_wire = 0
        self._lib = _load(planted=mutation != "none")
        # keep contiguous copies alive for the lifetime of the C object
        self._arrs = [np.ascontiguousarray(a) for a in (
            netlist.fanin_ptr.astype(np.int32), netlist.fanin_net.astype(np.int32),
            netlist.lut.astype(np.uint16), delays.gate_delay.astype(np.int32),
            delays.wire_delay.astype(np.int32), stim.init.astype(np.uint8),
            stim.edge_ptr.astype(np.int64), stim.edge_time.astype(np.int32))]
        fp, fn, lut, gd, wd, init, ep, et = self._arrs
        self.N = netlist.num_nets
        self.I = netlist.num_inputs
        self.W = int(W)
        self._h = self._lib.osim_create(
            netlist.num_inputs, netlist.num_gates, _p(fp), _p(fn), _p(lut), _p(gd), _p(wd),
            stim.num_cycles, stim.cycle_ps, _p(init), _p(ep), _p(et), self.W,
            MUTATIONS[mutation])
        if not self._h:
            raise ValueError("oracle: invalid netlist or stimulus")
        if self._lib.osim_set_pulse(self._h, int(pulse_gate), int(pulse_wire)) != 0:
            raise ValueError("oracle: pulse limits must be 0..100 percent")
        if self._lib.osim_set_full_sdf(self._h, 1 if full_sdf else 0) != 0:
            raise MemoryError("oracle: averaged delay table")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.osim_destroy(h)
            self._h = None

    @property
    def num_windows(self) -> int:
        return int(self._lib.osim_num_windows(self._h))

    def window(self, w: int):
        """Waveforms of window w: (init uint8[N], ptr int64[N+1], times int32[])."""
        E = self._lib.osim_run_window(self._h, int(w))
        if E < 0:
            raise RuntimeError("oracle: window simulation failed")
        init = np.empty(self.N, np.uint8)
        ptr = np.empty(self.N + 1, np.int64)
        times = np.empty(max(E, 1), np.int32)
        self._lib.osim_get(self._h, _p(init), _p(ptr), _p(times))
        return init, ptr, times[:E]

    def window_t1(self):
        """T1 per net of the last simulated window and the window length."""
        t1 = np.empty(self.N, np.int64)
        length = self._lib.osim_t1(self._h, _p(t1))
        return t1, int(length)

    def saif(self, w0: int = 0, w1: int | None = None):
        """SAIF over windows [w0, w1): (T0, T1, TC) int64 per net."""
        if w1 is None:
            w1 = self.num_windows
        t1 = np.empty(self.N, np.int64)
        tc = np.empty(self.N, np.int64)
        total = self._lib.osim_saif(self._h, int(w0), int(w1), _p(t1), _p(tc))
        if total < 0:
            raise RuntimeError("oracle: SAIF failed")
        return total - t1, t1, tc


def windows_as_lists(init, ptr, times):
    """(init, ptr, times) arrays -> list of (init, [times]) per net."""
    return [(int(init[n]), times[ptr[n]:ptr[n + 1]].tolist()) for n in range(init.shape[0])]
