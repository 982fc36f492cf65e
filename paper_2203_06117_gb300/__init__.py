"""GB300-native gate-level re-simulator with GATSPI delay semantics.

A thin ctypes binding over the C interface in ``include/gatspi.h`` (the
shared library ``_build/libgatspi.so`` built from ``csrc/`` for sm_103a).
Functions keep the C names and only marshal arguments; every step of the
simulation runs in the library's CUDA kernels.  There is no CPU path: if the
library is missing, importing its functions raises.

    import paper_2203_06117_gb300 as gs
    ctx = gs.gatspi_create(0)
    gs.gatspi_load_netlist(ctx, I, fanin_ptr, fanin_net, lut)
    gs.gatspi_load_delays(ctx, gate_delay, wire_delay)
    gs.gatspi_set_stimulus(ctx, C, L, init, edge_ptr, edge_time)
    gs.gatspi_simulate(ctx, window_cycles=1)
    t0, t1, tc = gs.gatspi_saif(ctx)
    gs.gatspi_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "_build", "libgatspi.so")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = [os.path.join(_HERE, "csrc", f) for f in ("gatspi.cu", "engine.cu", "noalloc.cu", "fileio.cpp")]
DEPS = SOURCES + [os.path.join(_HERE, "csrc", f) for f in ("kernels.cuh", "digest.cuh", "ingest.cuh",
                                                           "host_common.h", "per_device.h")] + \
    [os.path.join(INCLUDE, "gatspi.h")]

NVCC_FLAGS = ["-Xcompiler", "-fPIC", "-std=c++17",
              "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo"]

OK, EINVAL, ENOMEM, ECAPACITY, ECUDA, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECAPACITY: "ECAPACITY", ECUDA: "ECUDA",
          ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE"}

#: every entry point declared in include/gatspi.h
EXPORTS = ["gatspi_create", "gatspi_destroy", "gatspi_last_error", "gatspi_load_netlist",
           "gatspi_load_delays", "gatspi_set_edit", "gatspi_set_stimulus", "gatspi_simulate", "gatspi_saif",
           "gatspi_read_window", "gatspi_get_stats", "gatspi_digest",
           "gatspi_engine_create", "gatspi_engine_destroy", "gatspi_engine_last_error",
           "gatspi_engine_add_netlist", "gatspi_engine_submit", "gatspi_engine_step",
           "gatspi_engine_drain", "gatspi_engine_poll", "gatspi_engine_release",
           "gatspi_engine_get_stats", "gatspi_engine_digest", "gatspi_propagate_level_noalloc", "gatspi_resimulate_edit",
           "gatspi_set_stimulus_events", "gatspi_vcd_read", "gatspi_saif_write"]

JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


class GatspiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False, nvcc: str = "nvcc") -> str:
    """Compile the CUDA library (sm_103a) into ``_build/libgatspi.so``: one
    nvcc process per translation unit, in parallel, then one link."""
    newest = max(os.path.getmtime(p) for p in DEPS)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        bdir = os.path.dirname(LIB_PATH)
        os.makedirs(bdir, exist_ok=True)
        tag = f".tmp{os.getpid()}"
        objs = [os.path.join(bdir, os.path.basename(src) + tag + ".o") for src in SOURCES]
        procs = [subprocess.Popen([nvcc, "-c", *NVCC_FLAGS, "-I" + INCLUDE, "-o", o, src])
                 for src, o in zip(SOURCES, objs)]
        codes = [p.wait() for p in procs]
        if any(codes):
            raise RuntimeError(f"nvcc failed: {codes}")
        tmp = LIB_PATH + tag
        subprocess.check_call([nvcc, "-shared", *NVCC_FLAGS, "-o", tmp, *objs])
        os.replace(tmp, LIB_PATH)
        for o in objs:
            os.remove(o)
    return LIB_PATH


class gatspi_opts(ctypes.Structure):
    _fields_ = [("window_cycles", ctypes.c_int32), ("batch_windows", ctypes.c_int32),
                ("tile_items", ctypes.c_int32), ("time_kernels", ctypes.c_int32),
                ("items_per_thread", ctypes.c_int32), ("digest", ctypes.c_int32),
                ("pulse_limits", ctypes.c_int32), ("gate_pulse_percent", ctypes.c_int32),
                ("wire_pulse_percent", ctypes.c_int32), ("first_window", ctypes.c_int32),
                ("num_windows", ctypes.c_int32), ("features", ctypes.c_int32)]


class gatspi_engine_opts(ctypes.Structure):
    _fields_ = [("tile_items", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("part_items", ctypes.c_int64), ("items_per_thread", ctypes.c_int32),
                ("digest", ctypes.c_int32), ("step_items", ctypes.c_int64)]


class gatspi_engine_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("parts_done", ctypes.c_int64), ("parts_retried", ctypes.c_int64),
                ("items", ctypes.c_int64), ("bytes_peak", ctypes.c_int64),
                ("active", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("host_ms", ctypes.c_double), ("wait_ms", ctypes.c_double), ("prop_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gatspi_level_args(ctypes.Structure):
    """Arguments of gatspi_propagate_level_noalloc (device pointers as ints)."""
    _fields_ = [(n, ctypes.c_void_p) for n in ("fanin_ptr", "fanin_net", "lut", "gate_delay",
                                                 "wire_delay", "net_level", "rstart", "tile_info", "rmeta", "times",
                                                 "lvl_base")] + \
               [("capacity", ctypes.c_int64)] + \
               [(n, ctypes.c_void_p) for n in ("saif_t1", "saif_tc", "status")] + \
               [(n, ctypes.c_int32) for n in ("num_inputs", "level", "gate_begin", "gate_end",
                                               "num_windows", "first_window", "window_cycles",
                                               "num_cycles", "cycle_ps", "err_len")] + \
               [("err", ctypes.c_char_p)]


class gatspi_resim_info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("cone_gates", ctypes.c_int32),
                ("first_level", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("items", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gatspi_stats(ctypes.Structure):
    _fields_ = [("prop_ms", ctypes.c_double), ("input_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64),
                ("prop_launches", ctypes.c_int64), ("items", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("algo_bytes", ctypes.c_int64),
                ("batches", ctypes.c_int32), ("windows", ctypes.c_int32),
                ("batch_windows", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("tile_threads", ctypes.c_int32), ("items_per_thread", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run build() (nvcc, sm_103a) first; "
                              "this package has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.gatspi_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, sz]
        L.gatspi_destroy.argtypes = [vp]
        L.gatspi_last_error.argtypes = [vp]
        L.gatspi_last_error.restype = ctypes.c_char_p
        L.gatspi_load_netlist.argtypes = [vp, i32, i32, vp, vp, vp]
        L.gatspi_load_delays.argtypes = [vp, vp, vp]
        L.gatspi_set_stimulus.argtypes = [vp, i32, i32, vp, vp, vp]
        L.gatspi_set_edit.argtypes = [vp, i32, vp, vp]
        L.gatspi_resimulate_edit.argtypes = [vp, i32, vp, vp, ctypes.POINTER(gatspi_resim_info)]
        L.gatspi_set_stimulus_events.argtypes = [vp, i32, i32, vp, i64, vp, vp]
        L.gatspi_vcd_read.argtypes = [ctypes.c_char_p, i32, vp, vp, vp, vp, i64,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_char_p, i32]
        L.gatspi_saif_write.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i64, i32, vp, vp, vp, vp,
                                        ctypes.c_char_p, i32]
        L.gatspi_simulate.argtypes = [vp, ctypes.POINTER(gatspi_opts)]
        L.gatspi_saif.argtypes = [vp, vp, vp, vp]
        L.gatspi_read_window.argtypes = [vp, i32, vp, vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.gatspi_get_stats.argtypes = [vp, ctypes.POINTER(gatspi_stats)]
        L.gatspi_engine_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, sz,
                                           ctypes.POINTER(gatspi_engine_opts)]
        L.gatspi_engine_destroy.argtypes = [vp]
        L.gatspi_engine_last_error.argtypes = [vp]
        L.gatspi_engine_last_error.restype = ctypes.c_char_p
        L.gatspi_engine_add_netlist.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp,
                                                ctypes.POINTER(ctypes.c_int32)]
        L.gatspi_engine_submit.argtypes = [vp, i32, i32, i32, vp, vp, vp, i32, i32, vp, vp,
                                           ctypes.POINTER(ctypes.c_int64)]
        L.gatspi_engine_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.gatspi_engine_drain.argtypes = [vp]
        L.gatspi_engine_poll.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int32), vp, vp, vp]
        L.gatspi_engine_release.argtypes = [vp, i64]
        L.gatspi_engine_digest.argtypes = [vp, i64, vp]
        L.gatspi_engine_get_stats.argtypes = [vp, ctypes.POINTER(gatspi_engine_stats)]
        L.gatspi_propagate_level_noalloc.argtypes = [ctypes.POINTER(gatspi_level_args), vp]
        for name in EXPORTS:
            if not name.endswith("last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, rc):
    if rc != OK:
        msg = lib().gatspi_last_error(ctx).decode() if ctx else ""
        raise GatspiError(rc, msg)


def _arr(a, dt):
    return np.ascontiguousarray(np.asarray(a), dtype=dt)


def gatspi_create(device: int = 0, arena_bytes: int = 0):
    h = ctypes.c_void_p()
    rc = lib().gatspi_create(ctypes.byref(h), int(device), int(arena_bytes))
    if rc != OK:
        raise GatspiError(rc, f"cannot create a context on device {device}")
    return h


def gatspi_destroy(ctx) -> None:
    lib().gatspi_destroy(ctx)


def gatspi_last_error(ctx) -> str:
    return lib().gatspi_last_error(ctx).decode()


def gatspi_load_netlist(ctx, num_inputs, fanin_ptr, fanin_net, lut) -> None:
    fp, fn, lt = _arr(fanin_ptr, np.int32), _arr(fanin_net, np.int32), _arr(lut, np.uint16)
    _check(ctx, lib().gatspi_load_netlist(ctx, int(num_inputs), int(fp.shape[0] - 1), _ptr(fp),
                                          _ptr(fn), _ptr(lt)))


def gatspi_load_delays(ctx, gate_delay, wire_delay) -> None:
    gd, wd = _arr(gate_delay, np.int32), _arr(wire_delay, np.int32)
    _check(ctx, lib().gatspi_load_delays(ctx, _ptr(gd), _ptr(wd)))


def gatspi_set_edit(ctx, edit_gate=None, edit_delta=None) -> None:
    n = 0 if edit_gate is None else len(edit_gate)
    eg = None if n == 0 else _arr(edit_gate, np.int32)
    ed = None if n == 0 else _arr(edit_delta, np.int32)
    _check(ctx, lib().gatspi_set_edit(ctx, n, _ptr(eg), _ptr(ed)))


def gatspi_resimulate_edit(ctx, edit_gate=None, edit_delta=None) -> dict:
    """Set a delay edit and bring the last simulation up to date (only the
    fanout cone of the changed gates runs when the result is resident).
    Returns the call's gatspi_resim_info as a dict (mode 0: nothing changed,
    1: cone only, 2: everything again)."""
    n = 0 if edit_gate is None else len(edit_gate)
    eg = None if n == 0 else _arr(edit_gate, np.int32)
    ed = None if n == 0 else _arr(edit_delta, np.int32)
    info = gatspi_resim_info()
    _check(ctx, lib().gatspi_resimulate_edit(ctx, n, _ptr(eg), _ptr(ed), ctypes.byref(info)))
    return info.as_dict()


def gatspi_set_stimulus_events(ctx, num_cycles, cycle_ps, init, ev_input, ev_time) -> None:
    """Stimulus from raw (input, absolute ps) toggles in any order,
    restructured per (input, cycle) on the GPU."""
    iv, ei, et = _arr(init, np.uint8), _arr(ev_input, np.int32), _arr(ev_time, np.int64)
    _check(ctx, lib().gatspi_set_stimulus_events(ctx, int(num_cycles), int(cycle_ps), _ptr(iv),
                                                 int(ei.shape[0]), _ptr(ei), _ptr(et)))


def _names(names):
    arr = (ctypes.c_char_p * len(names))(*[n.encode() for n in names])
    return arr, ctypes.cast(arr, ctypes.c_void_p)


def gatspi_vcd_read(path, names):
    """(init uint8[k], ev_input int32[], ev_time int64[]) of the named 1-bit
    signals of a VCD file (host only)."""
    keep, pn = _names(list(names))
    init = np.zeros(len(names), np.uint8)
    total = ctypes.c_int64(0)
    err = ctypes.create_string_buffer(512)
    cap = 0
    while True:
        ei = np.empty(max(cap, 1), np.int32)
        et = np.empty(max(cap, 1), np.int64)
        rc = lib().gatspi_vcd_read(os.fsencode(path), len(names), pn, _ptr(init), _ptr(ei), _ptr(et), cap,
                                   ctypes.byref(total), err, len(err))
        if rc == ECAPACITY and total.value > cap:
            cap = total.value
            continue
        if rc != OK:
            raise GatspiError(rc, err.value.decode())
        return init, ei[:total.value], et[:total.value]


def gatspi_saif_write(path, design, duration_ps, names, t0, t1, tc) -> None:
    """Write a SAIF file for the given nets (host only)."""
    keep, pn = _names(list(names))
    a, b, c = _arr(t0, np.int64), _arr(t1, np.int64), _arr(tc, np.int64)
    err = ctypes.create_string_buffer(512)
    rc = lib().gatspi_saif_write(os.fsencode(path), design.encode(), int(duration_ps), len(names), pn,
                                 _ptr(a), _ptr(b), _ptr(c), err, len(err))
    if rc != OK:
        raise GatspiError(rc, err.value.decode())


def gatspi_set_stimulus(ctx, num_cycles, cycle_ps, init, edge_ptr, edge_time) -> None:
    iv, ep, et = _arr(init, np.uint8), _arr(edge_ptr, np.int64), _arr(edge_time, np.int32)
    _check(ctx, lib().gatspi_set_stimulus(ctx, int(num_cycles), int(cycle_ps), _ptr(iv), _ptr(ep),
                                          _ptr(et)))


#: features masks of gatspi_opts (the paper's variants without them)
NO_INTERCONNECT_FILTER, PARTIAL_SDF = 1, 2


def gatspi_simulate(ctx, window_cycles=0, batch_windows=0, tile_items=0, time_kernels=0,
                    items_per_thread=0, digest=0, pulse=None, first_window=0, num_windows=0,
                    features=0) -> None:
    """``pulse``: None for Algorithm 1 as printed, else (gate percent, wire
    percent), the PATHPULSEPERCENT limits of the two inertial tests.
    ``first_window`` / ``num_windows``: a segment of the windows (0 = to the
    end); segments' SAIF and digests add up to the whole run's.
    ``features``: a mask of NO_INTERCONNECT_FILTER and PARTIAL_SDF."""
    pg, pw = pulse if pulse is not None else (100, 100)
    o = gatspi_opts(int(window_cycles), int(batch_windows), int(tile_items), int(time_kernels),
                    int(items_per_thread), int(digest), 1 if pulse is not None else 0, int(pg), int(pw),
                    int(first_window), int(num_windows), int(features))
    _check(ctx, lib().gatspi_simulate(ctx, ctypes.byref(o)))


def gatspi_digest(ctx, num_nets: int):
    """Per-net uint64 waveform digest of the last simulation run with digest=1."""
    out = np.empty(num_nets, np.uint64)
    _check(ctx, lib().gatspi_digest(ctx, _ptr(out)))
    return out


def gatspi_saif(ctx, num_nets: int):
    """(T0, T1, TC) int64 per net."""
    t0, t1, tc = (np.empty(num_nets, np.int64) for _ in range(3))
    _check(ctx, lib().gatspi_saif(ctx, _ptr(t0), _ptr(t1), _ptr(tc)))
    return t0, t1, tc


def gatspi_read_window(ctx, window: int, num_nets: int):
    """All nets of one window: (init uint8[N], ptr int64[N+1], times int32[])."""
    init = np.empty(num_nets, np.uint8)
    ptr = np.empty(num_nets + 1, np.int64)
    total = ctypes.c_int64(0)
    _check(ctx, lib().gatspi_read_window(ctx, int(window), _ptr(init), _ptr(ptr), None, 0,
                                         ctypes.byref(total)))
    times = np.empty(max(total.value, 1), np.int32)
    _check(ctx, lib().gatspi_read_window(ctx, int(window), _ptr(init), _ptr(ptr), _ptr(times),
                                         int(times.shape[0]), ctypes.byref(total)))
    return init, ptr, times[:total.value]


def gatspi_get_stats(ctx) -> dict:
    s = gatspi_stats()
    _check(ctx, lib().gatspi_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


class Simulator:
    """One context with a netlist, its delays and a stimulus loaded."""

    def __init__(self, netlist, delays, stim, device: int = 0, arena_bytes: int = 0):
        self.ctx = gatspi_create(device, arena_bytes)
        self.N = netlist.num_nets
        try:
            gatspi_load_netlist(self.ctx, netlist.num_inputs, netlist.fanin_ptr, netlist.fanin_net,
                                netlist.lut)
            gatspi_load_delays(self.ctx, delays.gate_delay, delays.wire_delay)
            gatspi_set_stimulus(self.ctx, stim.num_cycles, stim.cycle_ps, stim.init, stim.edge_ptr,
                                stim.edge_time)
        except Exception:
            self.close()
            raise

    def simulate(self, **opts):
        gatspi_simulate(self.ctx, **opts)
        return self

    def saif(self):
        return gatspi_saif(self.ctx, self.N)

    def window(self, w: int):
        return gatspi_read_window(self.ctx, w, self.N)

    def resimulate_edit(self, edit_gate=None, edit_delta=None) -> dict:
        return gatspi_resimulate_edit(self.ctx, edit_gate, edit_delta)

    def digest(self):
        return gatspi_digest(self.ctx, self.N)

    def stats(self) -> dict:
        return gatspi_get_stats(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            gatspi_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        self.close()


# ------------------------------------------------------------------ engine

def _echeck(eng, rc):
    if rc != OK:
        raise GatspiError(rc, lib().gatspi_engine_last_error(eng).decode() if eng else "")


def gatspi_engine_create(device=0, arena_bytes=0, tile_items=0, max_active=0, part_items=0,
                         items_per_thread=0, step_items=0, digest=0):
    h = ctypes.c_void_p()
    o = gatspi_engine_opts(int(tile_items), int(max_active), int(part_items), int(items_per_thread),
                           int(digest), int(step_items))
    rc = lib().gatspi_engine_create(ctypes.byref(h), int(device), int(arena_bytes), ctypes.byref(o))
    if rc != OK:
        raise GatspiError(rc, f"cannot create an engine on device {device}")
    return h


def gatspi_engine_destroy(eng) -> None:
    lib().gatspi_engine_destroy(eng)


def gatspi_engine_last_error(eng) -> str:
    return lib().gatspi_engine_last_error(eng).decode()


def gatspi_engine_add_netlist(eng, netlist, delays) -> int:
    fp, fn = _arr(netlist.fanin_ptr, np.int32), _arr(netlist.fanin_net, np.int32)
    lt = _arr(netlist.lut, np.uint16)
    gd, wd = _arr(delays.gate_delay, np.int32), _arr(delays.wire_delay, np.int32)
    nid = ctypes.c_int32(-1)
    _echeck(eng, lib().gatspi_engine_add_netlist(eng, int(netlist.num_inputs), int(fp.shape[0] - 1),
                                                 _ptr(fp), _ptr(fn), _ptr(lt), _ptr(gd), _ptr(wd),
                                                 ctypes.byref(nid)))
    return nid.value


def gatspi_engine_submit(eng, netlist_id, stim, window_cycles=0, edit_gate=None, edit_delta=None) -> int:
    iv, ep, et = _arr(stim.init, np.uint8), _arr(stim.edge_ptr, np.int64), _arr(stim.edge_time, np.int32)
    n = 0 if edit_gate is None else len(edit_gate)
    eg = None if n == 0 else _arr(edit_gate, np.int32)
    ed = None if n == 0 else _arr(edit_delta, np.int32)
    jid = ctypes.c_int64(-1)
    _echeck(eng, lib().gatspi_engine_submit(eng, int(netlist_id), int(stim.num_cycles), int(stim.cycle_ps),
                                            _ptr(iv), _ptr(ep), _ptr(et), int(window_cycles), n,
                                            _ptr(eg), _ptr(ed), ctypes.byref(jid)))
    return jid.value


def gatspi_engine_step(eng):
    """One engine step; returns (active parts, queued parts)."""
    a, q = ctypes.c_int32(0), ctypes.c_int32(0)
    _echeck(eng, lib().gatspi_engine_step(eng, ctypes.byref(a), ctypes.byref(q)))
    return a.value, q.value


def gatspi_engine_drain(eng) -> None:
    _echeck(eng, lib().gatspi_engine_drain(eng))


def gatspi_engine_poll(eng, job_id, num_nets=None):
    """(state, saif) where saif is (T0, T1, TC) once the job is done and
    num_nets is given, else None."""
    st = ctypes.c_int32(-1)
    if num_nets is None:
        _echeck(eng, lib().gatspi_engine_poll(eng, int(job_id), ctypes.byref(st), None, None, None))
        return st.value, None
    t0, t1, tc = (np.empty(num_nets, np.int64) for _ in range(3))
    _echeck(eng, lib().gatspi_engine_poll(eng, int(job_id), ctypes.byref(st), _ptr(t0), _ptr(t1), _ptr(tc)))
    return st.value, ((t0, t1, tc) if st.value == JOB_DONE else None)


def gatspi_engine_digest(eng, job_id, num_nets) -> np.ndarray:
    """Per-net waveform digests (uint64 [num_nets]) of a finished job."""
    out = np.empty(num_nets, np.uint64)
    _echeck(eng, lib().gatspi_engine_digest(eng, int(job_id), _ptr(out)))
    return out


def gatspi_engine_release(eng, job_id) -> None:
    _echeck(eng, lib().gatspi_engine_release(eng, int(job_id)))


def gatspi_engine_get_stats(eng) -> dict:
    s = gatspi_engine_stats()
    _echeck(eng, lib().gatspi_engine_get_stats(eng, ctypes.byref(s)))
    return s.as_dict()


class Engine:
    """Multi-job engine: resident netlists, queued jobs, continuous batching."""

    def __init__(self, device=0, arena_bytes=0, **opts):
        self.h = gatspi_engine_create(device, arena_bytes, **opts)
        self.nets = {}

    def add_netlist(self, netlist, delays) -> int:
        nid = gatspi_engine_add_netlist(self.h, netlist, delays)
        self.nets[nid] = netlist.num_nets
        return nid

    def submit(self, netlist_id, stim, window_cycles=0, edit_gate=None, edit_delta=None) -> int:
        return gatspi_engine_submit(self.h, netlist_id, stim, window_cycles, edit_gate, edit_delta)

    def step(self):
        return gatspi_engine_step(self.h)

    def drain(self):
        gatspi_engine_drain(self.h)

    def poll(self, job_id, netlist_id=None):
        return gatspi_engine_poll(self.h, job_id, None if netlist_id is None else self.nets[netlist_id])

    def digest(self, job_id, netlist_id):
        return gatspi_engine_digest(self.h, job_id, self.nets[netlist_id])

    def release(self, job_id):
        gatspi_engine_release(self.h, job_id)

    def stats(self) -> dict:
        return gatspi_engine_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            gatspi_engine_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        self.close()
