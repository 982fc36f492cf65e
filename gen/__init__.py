"""Seeded synthetic inputs for gate-level re-simulation.

This module only produces inputs (netlists, delay tables, stimulus).  It
holds none of the simulation arithmetic and is the one piece shared by the
CPU oracle and the GPU path.  The heavy lifting is in ``gen.c`` (compiled on
first use, or by ``build()``), which draws every random number from a
counter-based SplitMix64 key, so the same seed gives the same bytes on x86-64
and AArch64.

The workload recipes follow the benchmark shapes of the GATSPI paper
(Section 4, Table "benchmarks"): gate counts 1k to 2M, thousands of cycles,
activity from low to above 1.  The paper's designs and testbenches are not
public; these synthetic inputs stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libgatspi_gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to this file."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32, i64, u64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.gen_netlist.restype = i64
        lib.gen_netlist.argtypes = [i32, i32, i32, u64, i32, i32, vp, vp, vp, vp, vp]
        lib.gen_delays.restype = None
        lib.gen_delays.argtypes = [i32, vp, vp, u64, i32, i32, i32, i32, i32, i32, vp, vp]
        lib.gen_stimulus_count.restype = i64
        lib.gen_stimulus_count.argtypes = [i32, i32, u64, i32, i32, i32, vp, vp, vp]
        lib.gen_stimulus_fill.restype = None
        lib.gen_stimulus_fill.argtypes = [i32, i32, u64, i32, i32, i32, vp, vp, vp]
        lib.gen_cell_lut.restype = ctypes.c_int
        lib.gen_cell_lut.argtypes = [ctypes.c_int]
        lib.gen_cell_pins.restype = ctypes.c_int
        lib.gen_cell_pins.argtypes = [ctypes.c_int]
        lib.gen_cell_count.restype = ctypes.c_int
        lib.gen_draw.restype = u64
        lib.gen_draw.argtypes = [u64, u64, u64]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


CELL_NAMES = ["INV", "BUF", "NAND2", "NOR2", "AND2", "OR2", "XOR2", "XNOR2",
              "AOI21", "OAI21", "MUX2", "NAND3", "NAND4", "NOR3", "NOR4",
              "AND3", "AND4", "OR3", "OR4", "AOI22", "OAI22"]


def cell_lut(name: str) -> int:
    """Truth table of a named cell (bit k = output for column index k)."""
    return _load().gen_cell_lut(CELL_NAMES.index(name))


def cell_pins(name: str) -> int:
    return _load().gen_cell_pins(CELL_NAMES.index(name))


@dataclass
class Netlist:
    num_inputs: int
    fanin_ptr: np.ndarray   # int32 [G+1]
    fanin_net: np.ndarray   # int32 [P]
    num_pins: np.ndarray    # uint8 [G]
    lut: np.ndarray         # uint16 [G]
    cell: np.ndarray = None  # uint8 [G] (cell index into CELL_NAMES), informational

    @property
    def num_gates(self) -> int:
        return int(self.num_pins.shape[0])

    @property
    def num_nets(self) -> int:
        return self.num_inputs + self.num_gates


@dataclass
class Delays:
    gate_delay: np.ndarray  # int32 [P*32]: [pin][inEdge][outEdge][side 8]
    wire_delay: np.ndarray  # int32 [P*2]: [pin][rise, fall]


@dataclass
class Stimulus:
    num_cycles: int
    cycle_ps: int
    init: np.ndarray        # uint8 [I]
    edge_ptr: np.ndarray    # int64 [I*C+1], index i*C+c
    edge_time: np.ndarray   # int32 [E], relative to the cycle start


@dataclass
class Workload:
    name: str
    netlist: Netlist
    delays: Delays
    stim: Stimulus
    depth: int
    params: dict = field(default_factory=dict)

    @property
    def gate_cycles(self) -> int:
        return self.netlist.num_gates * self.stim.num_cycles


def make_netlist(num_inputs, num_gates, depth, seed, cell_set=0, fanout_model=0) -> Netlist:
    """Levelized random netlist.  cell_set 0 = {INV, BUF, NAND2, NOR2, AND2,
    OR2, XOR2, XNOR2, AOI21, OAI21, MUX2}; 1 adds 3/4-input NAND/NOR/AND/OR
    and AOI22/OAI22.  fanout_model 0 = uniform fanin choice, 1 = geometric
    fanout quota (mean 2.5), 2 = Zipf(1.2) quota capped at 64."""
    lib = _load()
    G = int(num_gates)
    fp = np.zeros(G + 1, np.int32)
    fn = np.zeros(max(4 * G, 1), np.int32)
    npins = np.zeros(G, np.uint8)
    lut = np.zeros(G, np.uint16)
    cell = np.zeros(G, np.uint8)
    P = lib.gen_netlist(int(num_inputs), G, int(depth), int(seed) & (2**64 - 1),
                        int(cell_set), int(fanout_model), _p(fp), _p(fn), _p(npins),
                        _p(lut), _p(cell))
    if P < 0:
        raise ValueError("gen_netlist: bad arguments")
    return Netlist(int(num_inputs), fp, fn[:P].copy(), npins, lut, cell)


def make_delays(nl: Netlist, seed, dlo, dhi, wlo, whi, cond_mode=0, cond_permille=0) -> Delays:
    """IOPATH delays uniform in [dlo, dhi]; cond_mode 1 makes XOR2/MUX2 arcs
    conditional, cond_mode 2 makes cond_permille/1000 of arcs conditional.
    Wire delays uniform in [wlo, whi]."""
    lib = _load()
    P = int(nl.fanin_net.shape[0])
    gd = np.zeros(P * 32, np.int32)
    wd = np.zeros(P * 2, np.int32)
    lib.gen_delays(nl.num_gates, _p(nl.fanin_ptr), _p(nl.cell), int(seed) & (2**64 - 1),
                   int(dlo), int(dhi), int(wlo), int(whi), int(cond_mode),
                   int(cond_permille), _p(gd), _p(wd))
    return Delays(gd, wd)


def first_fanout_min_delay(nl: Netlist, d: Delays) -> np.ndarray:
    """Per input: the smallest IOPATH delay of the first gate it drives (0 if
    it drives nothing).  Used to size the deliberately narrow pulses."""
    I = nl.num_inputs
    out = np.zeros(I, np.int32)
    pins = np.nonzero(nl.fanin_net < I)[0]
    if pins.size == 0:
        return out
    nets, first = np.unique(nl.fanin_net[pins], return_index=True)
    pin = pins[first]
    gate = np.searchsorted(nl.fanin_ptr, pin, side="right") - 1
    gd = d.gate_delay.reshape(-1, 32)
    for net, g in zip(nets.tolist(), gate.tolist()):
        a, b = int(nl.fanin_ptr[g]), int(nl.fanin_ptr[g + 1])
        vals = gd[a:b]
        out[net] = int(vals[vals > 0].min())
    return out


def make_stimulus(num_inputs, num_cycles, seed, p_permille, q_permille,
                  narrow_permille=0, dmin=None, cycle_ps=1000) -> Stimulus:
    """Per (input, cycle): toggle with probability p at a uniform time in
    [0, 200) ps, plus a two-edge pulse with probability q (start uniform in
    [0, 200), width uniform in [1, 40], or narrower than dmin for
    narrow_permille/1000 of pulses).  Coincident edges cancel in pairs."""
    lib = _load()
    I, C = int(num_inputs), int(num_cycles)
    init = np.zeros(I, np.uint8)
    ptr = np.zeros(I * C + 1, np.int64)
    dm = None if dmin is None else np.ascontiguousarray(dmin, np.int32)
    E = lib.gen_stimulus_count(I, C, int(seed) & (2**64 - 1), int(p_permille), int(q_permille),
                               int(narrow_permille), _p(dm), _p(init), _p(ptr))
    times = np.zeros(max(E, 1), np.int32)
    lib.gen_stimulus_fill(I, C, int(seed) & (2**64 - 1), int(p_permille), int(q_permille),
                          int(narrow_permille), _p(dm), _p(ptr), _p(times))
    return Stimulus(C, int(cycle_ps), init, ptr, times[:E].copy())


def draw(seed, stream, idx) -> int:
    return int(_load().gen_draw(int(seed) & (2**64 - 1), int(stream), int(idx)))


# --------------------------------------------------------------- recipes

#: name -> (I, G, depth, cycles, cell_set, fanout_model, delay lo/hi,
#:          wire lo/hi, cond_mode, cond_permille, p, q, narrow) in permille
RECIPES = {
    # 2,000 gates, depth 20, 64 inputs, 1,000 cycles of 1,000 ps, p = 0.2,
    # 5% pulses of width 1-40 ps, delays 5-50 ps.
    "tiny": dict(I=64, G=2000, D=20, C=1000, cell_set=0, fanout=0, dlo=5, dhi=50,
                 wlo=1, whi=5, cond=0, cond_pm=0, p=200, q=50, narrow=0),
    # 200k gates, depth 60, fanin 1-4, geometric fanout (mean 2.5), 512
    # inputs, 10,000 cycles, p = 0.3, 20% of pulses narrower than the driven
    # gate's delay, XOR2/MUX2 conditional delays, delays 2-120 ps.
    "mid": dict(I=512, G=200_000, D=60, C=10_000, cell_set=1, fanout=1, dlo=2, dhi=120,
                wlo=1, whi=12, cond=1, cond_pm=0, p=300, q=50, narrow=200),
    # 2M gates, depth 120, Zipf(1.2) fanout capped at 64, 5,000 inputs,
    # 20,000 cycles, p = 0.5, 10% pulses, delays 1-200 ps with 10%
    # conditional arcs.
    "large": dict(I=5000, G=2_000_000, D=120, C=20_000, cell_set=1, fanout=2, dlo=1, dhi=200,
                  wlo=1, whi=20, cond=2, cond_pm=100, p=500, q=100, narrow=0),
}


def make_workload(name: str, seed: int = 1, num_cycles: int | None = None,
                  num_gates: int | None = None, depth: int | None = None,
                  num_inputs: int | None = None, **over) -> Workload:
    """Build one of the named recipes (optionally resized for tests)."""
    r = dict(RECIPES[name])
    r.update(over)
    I = int(num_inputs or r["I"])
    G = int(num_gates or r["G"])
    D = int(depth or r["D"])
    C = int(num_cycles or r["C"])
    nl = make_netlist(I, G, D, seed * 1000 + 1, r["cell_set"], r["fanout"])
    d = make_delays(nl, seed * 1000 + 2, r["dlo"], r["dhi"], r["wlo"], r["whi"],
                    r["cond"], r["cond_pm"])
    dmin = first_fanout_min_delay(nl, d) if r["narrow"] else None
    st = make_stimulus(I, C, seed * 1000 + 3, r["p"], r["q"], r["narrow"], dmin)
    return Workload(name, nl, d, st, D, dict(r, I=I, G=G, D=D, C=C, seed=seed))


def interp_depth(gates: int) -> int:
    """Depth for a gate count by log-linear interpolation through (2k, 20),
    (200k, 60), (2M, 120)."""
    pts = [(2e3, 20.0), (2e5, 60.0), (2e6, 120.0)]
    x = np.log10(max(gates, 1))
    xs = [np.log10(a) for a, _ in pts]
    ys = [b for _, b in pts]
    return int(round(float(np.interp(x, xs, ys, left=ys[0], right=ys[-1]))))


def random_small(seed: int, max_inputs: int = 4, max_gates: int = 12, max_cycles: int = 3,
                 dmax: int = 20, dense: bool = True, cycle_ps: int = 300) -> Workload:
    """A tiny random case for exhaustive cross-checks: up to ``max_inputs``
    inputs and ``max_gates`` gates, delays uniform in [1, dmax], conditional
    arcs on a random subset, and a dense stimulus (up to six edges per input
    and cycle, packed into the first fifth of the cycle) so that both
    inertial filters and simultaneous switching are exercised often."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    I = int(rng.integers(1, max_inputs + 1))
    G = int(rng.integers(1, max_gates + 1))
    D = int(rng.integers(1, G + 1))
    cs = int(rng.integers(0, 2))
    fm = int(rng.integers(0, 3))
    nl = make_netlist(I, G, D, int(rng.integers(1, 2**62)), cs, fm)
    cond = int(rng.integers(0, 3))
    d = make_delays(nl, int(rng.integers(1, 2**62)), 1, dmax, 1, dmax, cond, 300)
    C = int(rng.integers(1, max_cycles + 1))
    init = rng.integers(0, 2, I).astype(np.uint8)
    ptr = [0]
    times = []
    span = max(cycle_ps // 5, 8)
    for i in range(I):
        for c in range(C):
            k = int(rng.integers(0, 7)) if dense else int(rng.integers(0, 3))
            ts = np.unique(rng.integers(0, span, k)) if k else np.zeros(0, np.int64)
            times += ts.tolist()
            ptr.append(len(times))
    st = Stimulus(C, int(cycle_ps), init, np.asarray(ptr, np.int64), np.asarray(times, np.int32))
    return Workload(f"random_small_{seed}", nl, d, st, D, dict(seed=seed))


# ------------------------------------------------ job streams (batched / served)


def batched_workload(seed: int = 1, n_jobs: int = 64, n_netlists: int = 8, scale: float = 1.0):
    """64 jobs over 8 netlists of 10k-500k gates (log-uniform, mid recipe,
    depth by log-linear interpolation through (2k, 20), (200k, 60),
    (2M, 120)); cycles log-normal (median 2,000, sigma 1) clipped to
    [100, 20,000]; toggle probability uniform in [0.05, 0.5].  ``scale``
    shrinks gates and cycles for tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nets = []
    for k in range(n_netlists):
        G = int(10 ** rng.uniform(np.log10(10_000), np.log10(500_000)) * scale)
        G = max(G, 200)
        D = min(interp_depth(G), G)
        I = max(16, G // 400)
        nets.append(make_workload("mid", seed=seed * 100 + k, num_gates=G, depth=D, num_inputs=I,
                                      num_cycles=1))
    reqs = []
    for j in range(n_jobs):
        n = int(rng.integers(0, n_netlists))
        C = int(np.clip(np.exp(rng.normal(np.log(2000), 1.0)), 100, 20_000) * scale)
        C = max(C, 2)
        p = int(rng.uniform(50, 500))
        st = make_stimulus(nets[n].netlist.num_inputs, C, seed * 10_000 + j, p, 50, 200,
                               first_fanout_min_delay(nets[n].netlist, nets[n].delays))
        reqs.append(dict(arrival=0.0, netlist=n, stim=st))
    return nets, reqs


def served_workload(seed: int = 1, rate: float = 200.0, seconds: float = 2.0, scale: float = 1.0,
                    sizes=(50_000, 200_000, 500_000, 1_000_000)):
    """Four resident netlists (50k, 200k, 500k, 1M gates; the tiny recipe's
    cells and delays; depth interpolated), Poisson arrivals at ``rate``/s,
    window cycles log-uniform in [100, 5,000], 30% of requests with a delay
    edit re-timing 1% of gates by +-[10, 50] ps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nets = []
    for k, G0 in enumerate(sizes):
        G = max(200, int(G0 * scale))
        D = min(interp_depth(G), G)
        I = max(16, G // 400)
        nets.append(make_workload("tiny", seed=seed * 100 + k, num_gates=G, depth=D, num_inputs=I,
                                      num_cycles=1))
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        n = int(rng.integers(0, len(nets)))
        C = max(2, int(10 ** rng.uniform(2, np.log10(5000)) * scale))
        st = make_stimulus(nets[n].netlist.num_inputs, C, seed * 100_000 + len(reqs), 200, 50)
        r = dict(arrival=t, netlist=n, stim=st)
        if rng.uniform() < 0.3:
            G = nets[n].netlist.num_gates
            r["edit_gate"] = rng.choice(G, size=max(1, G // 100), replace=False).astype(np.int32)
            r["edit_delta"] = (rng.choice([-1, 1], size=r["edit_gate"].size) *
                               rng.integers(10, 51, size=r["edit_gate"].size)).astype(np.int32)
        reqs.append(r)
    return nets, reqs
