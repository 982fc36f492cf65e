// Device code of the re-simulator: input restructuring, the per-level
// propagation kernel, and waveform read-back.
//
// Propagation (GATSPI, Section 3 and Algorithm 1): each thread takes a few
// consecutive (gate, window) items of a logic level.  For each it merges
// the fanin pins' delayed, inertially filtered edges, evaluates the truth
// table, picks the switching pin's (COND) delay, applies the gate inertial
// filter and emits the output edges.
//
// Output allocation.  The paper simulates every item twice: a counting
// pass, then a storing pass at the scanned offsets.  Here one pass suffices.
// A warp stages its items' edges in shared memory, sums its edge count with
// shuffles, and takes its output range with one atomic add on the level's
// counter, so no tile waits for another.  The same add counts the tile as
// done (the counter packs tiles done above the edges allocated), so the
// level's last tile sees the final edge total and publishes it, which
// places the next level.
//
// Waveform store (one batch of NW windows):
//   rmeta[n*NW + w]   uint16  bit 15: value of net n at the start of window
//                             w; bits 0-14: its edge count in the window
//   times[lvl_base[level(n)] + ...]  int32 window-relative edge times
// and where each record's edges start, in one of two forms:
//   gate-aligned tiling (NW >= 16*IPT): tiles are one gate x TW = 32*IPT
//     windows, and the edges of a tile are one run in window order;
//     tinfo[n*T + t] = {first edge relative to lvl_base[level(n)], edges}
//     for tile t of net n (T = ceil(NW / TW)), and a window's first edge is
//     its tile's plus the counts of the tile's earlier windows;
//   linear tiling (fewer windows): rstart[n*NW + w] int32, the first edge of
//     each record relative to lvl_base[level(n)].
// A net's records are contiguous, so a warp's record loads for one pin
// cover one contiguous range.
#pragma once

#include <cstdint>

#include "per_device.h"

namespace gatspi_dev {
namespace {  // every translation unit gets its own copy of the kernels

constexpr int32_t kInf = 0x7fffffff;
constexpr int32_t kMaxCount = 0x7fff;  // edges per (net, window) record

// Level counter: tiles done in the top 27 bits, edges allocated in the low
// 37.  A level has fewer than 2^27 tiles (fewer than 2^31 items, at least 16
// per tile on average) and fewer than 2^37 edges (512 GB of times).
constexpr int kTileShift = 37;
constexpr unsigned long long kEdgeMask = (1ull << kTileShift) - 1ull;

// status bits (device -> host)
constexpr int kStCapacity = 1;  // arena too small for this batch
constexpr int kStTimeout = 2;   // reserved: a bounded device-side wait ran out
constexpr int kStCorrupt = 4;   // a record failed its bounds check
constexpr int kStOffset = 8;    // a level's edges exceed int32, or a record > kMaxCount

// One simulation job as the kernels see it: a netlist with its delays, one
// batch of windows of its stimulus, and where its waveforms and SAIF go.
struct JobView {
  // netlist (internal order: gates sorted by level)
  const int32_t* __restrict__ fanin_ptr;
  const int32_t* __restrict__ fanin_net;
  const uint16_t* __restrict__ lut;
  const int32_t* __restrict__ gate_delay;  // [P][2][2][8]
  const int32_t* __restrict__ wire_delay;  // [P][2]
  const int32_t* __restrict__ net_level;   // [N]
  const int32_t* __restrict__ gate_delta;  // [G] delay edit per gate, or null
  const int4* __restrict__ gdesc;          // [G][2] gate descriptors, or null (then the CSR arrays)
  // waveform store
  int32_t* rstart;  // linear tiling: [N*NW] record starts
  int2* tinfo;      // gate-aligned tiling: [N*T] tile runs
  int32_t T;        // tiles per net with gate-aligned tiling, 0 with linear
  uint16_t* rmeta;
  int32_t* times;
  long long* lvl_base;  // [D+2]
  long long capacity;   // elements of times
  // SAIF accumulators (per internal net)
  unsigned long long* saif_t1;
  unsigned long long* saif_tc;
  int32_t* status;
  int32_t I;
  int32_t NW;  // windows in the batch
  // window w of the batch is global window w0 + w; it spans cycles
  // [g*W, min(g*W + W, C)) of L ps each
  int32_t w0, W, C, L;
  // pulse limits of the gate and interconnect inertial tests, percent of
  // the delay (read only by the kernels compiled with pulse limits; the
  // others apply Algorithm 1 as printed, i.e. 100 / 100)
  int32_t pulse_g, pulse_w;
};

// One level of one job inside a launch.
struct SegView {
  unsigned long long* counters;  // [1]: packed level counter, zero before use
  int32_t level;
  int32_t gate_begin;  // first internal gate of the level
  int32_t n_items;     // gates of the level * NW
  int32_t n_tiles;
  // Re-simulation of a fanout cone (gate-aligned tiling only), null
  // otherwise: the tiles cover the listed gates (internal ids) instead of
  // all the level's gates, and their edges go to an append region past
  // everything stored, so that the other gates' waveforms stay in place.
  // The launch's edges start at *append_in; its last tile writes where the
  // next launch's start to *append_out (consecutive launches swap the two
  // words) and leaves lvl_base alone.  Tile runs stay relative to
  // lvl_base[level].
  const int32_t* gate_list;
  const long long* append_in;
  long long* append_out;
};

struct PropParams {
  JobView job;
  SegView seg;
  int32_t* tile_counter;  // zero before the launch
  int32_t n_tiles;        // tiles of this launch: seg.n_tiles, or the part of
                          // the level's gates it covers (seg.n_tiles counts the
                          // whole level, whose last tile publishes its end)
};

struct MultiSeg {
  JobView job;
  SegView seg;
  int32_t tile_begin;  // first launch-wide tile of this segment
};

// Segments of one multi-job launch.  The table travels in the kernel's
// parameter space (read through the constant cache), so finding a tile's
// job costs no global-memory round trip.
constexpr int kMaxSegs = 32;
struct MultiParams {
  int32_t n_segs;
  int32_t n_tiles;        // tiles of all segments
  int32_t* tile_counter;  // zero before the launch
  MultiSeg segs[kMaxSegs];  // sorted by tile_begin
};
static_assert(sizeof(MultiParams) < 32000, "kernel parameters are limited to 32 KB");

__device__ __forceinline__ int32_t window_len(int32_t wg, int32_t W, int32_t C, int32_t L) {
  const int32_t c0 = wg * W;
  const int32_t c1 = min(c0 + W, C);
  return (c1 - c0) * L;
}

// Features of Algorithm 1 a kernel can be compiled without, as the paper
// does to measure their cost (Section 5, Table "features"):
//   kNoWireFilter -- the interconnect inertial test deleted: every edge
//     arrives after its delay, except that two consecutive edges of a pin
//     whose arrivals would cross or coincide cancel as a pair (Algorithm 1
//     assumes each pin's arrivals in time order);
//   kAvgSdf -- partial SDF: each arc keeps one delay per output edge, the
//     mean over its COND columns and input edges, which the host stores in
//     every entry of the arc's table; the kernel reads the entry of row
//     outEdge, column 0, without the input-edge and COND index.
constexpr int kNoWireFilter = 1, kAvgSdf = 2;

// One fanin pin of one (gate, window) item.
struct Pin {
  const int32_t* t;  // edge times of the driving net in this window
  int32_t n;         // number of edges
  int32_t j;         // next edge not yet examined
  int32_t a;         // delayed time of the next surviving edge, or kInf
  int32_t dr, df;    // interconnect delay for a rising / falling edge
  uint32_t v0;       // value of the driving net at the window start
};

// Find the pin's next surviving edge: edge j has direction given by the
// parity of j and the start value; the pulse (j, j+1) is dropped when it is
// narrower than the delay of edge j (Algorithm 1, interconnect inertial
// test), repeatedly, until an edge survives or the list ends.
// The edge times may sit in shared memory (staged) or in global memory, so
// they are read with generic loads (a global-only load of a shared address
// faults).
template <int F = 0>
__device__ __forceinline__ void pin_advance(Pin& q) {
  int32_t j = q.j, a = kInf;
  while (j < q.n) {
    const int32_t t = q.t[j];
    const bool rise = ((q.v0 ^ (uint32_t)j) & 1u) == 0u;
    const int32_t d = rise ? q.dr : q.df;
    bool drop;
    if constexpr (F & kNoWireFilter) drop = j + 1 < q.n && q.t[j + 1] + (rise ? q.df : q.dr) <= t + d;
    else drop = j + 1 < q.n && q.t[j + 1] - t < d;
    if (drop) {
      j += 2;
      continue;
    }
    a = t + d;
    ++j;
    break;
  }
  q.j = j;
  q.a = a;
}

// Algorithm 1 for one gate and one window (`gd`: the gate's delay tables, 32
// entries per pin, in global or shared memory; `edit` shifts every gate delay of
// the gate, clamped at 1 ps; 0 without a delay edit).  The output keeps at
// most one edge that may still be cancelled (the last kept one, `pend`): a
// cancel needs the last kept edge to lie after the current time, and once an
// edge has been cancelled the kept edge before it is already in the past, so
// no deeper history is needed.  Edges are handed to `sink` as they become
// final; T1 (time at 1 inside [0, len)) is integrated on the way.
template <int K, int F = 0, class Sink>
__device__ __forceinline__ void run_gate(Pin (&pin)[K], uint32_t lut,
                                         const int32_t* __restrict__ gd, int32_t edit,
                                         int32_t len, Sink& sink, int32_t& count, int32_t& t1,
                                         uint32_t& y0) {
  uint32_t col = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) col |= (pin[i].v0 & 1u) << i;
  uint32_t y = (lut >> col) & 1u;
  y0 = y;
#pragma unroll
  for (int i = 0; i < K; ++i) pin_advance<F>(pin[i]);
  bool pend_on = false;
  int32_t pend = 0, nflush = 0, prev = 0, acc = 0;
  uint32_t cv = y;
  auto flush = [&](int32_t te) {
    sink.put(nflush++, te);
    const int32_t c = min(te, len);
    if (cv) acc += c - prev;
    prev = c;
    cv ^= 1u;
  };
  for (;;) {
    int32_t t = pin[0].a;
#pragma unroll
    for (int i = 1; i < K; ++i) t = min(t, pin[i].a);
    if (t == kInf) break;
    int istar = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (pin[i].a == t) {  // every pin arriving now switches (MSI)
        col ^= 1u << i;
        istar = i;
        pin_advance<F>(pin[i]);
      }
    }
    const uint32_t yn = (lut >> col) & 1u;
    if (yn != y) {
      if (pend_on && pend > t) {
        pend_on = false;  // gate inertial filter: cancel the last kept edge
      } else {
        if (pend_on) flush(pend);
        int32_t dg;
        if constexpr (F & kAvgSdf) {
          dg = gd[istar * 32 + (int)(yn * 8u)];
        } else {
          const uint32_t side = (col & ((1u << istar) - 1u)) | ((col >> (istar + 1)) << istar);
          const uint32_t ie = (col >> istar) & 1u;
          dg = gd[istar * 32 + (int)(ie * 16u + yn * 8u + side)];
        }
        pend = t + max(1, dg + edit);
        pend_on = true;
      }
      y = yn;
    }
  }
  if (pend_on) flush(pend);
  if (cv) acc += len - prev;
  count = nflush;
  t1 = acc;
}

// Interconnect test with a pulse limit of pw percent (Section 3 allows
// PATHPULSEPERCENT values other than 100): the pulse (j, j+1) is dropped
// when 100 (t_{j+1} - t_j) < pw delta(e_j), or when its two delayed edges
// would not stay in order (a width of zero or less after the delays, which
// the 100 percent test already covers); repeated until an edge survives.
__device__ __forceinline__ void pin_advance_pp(Pin& q, int32_t pw) {
  int32_t j = q.j, a = kInf;
  while (j < q.n) {
    const int32_t t = q.t[j];
    const bool rise = ((q.v0 ^ (uint32_t)j) & 1u) == 0u;
    const int32_t d = rise ? q.dr : q.df;
    if (j + 1 < q.n) {
      const int32_t t2 = q.t[j + 1];
      const int32_t d2 = rise ? q.df : q.dr;
      if (100ll * (t2 - t) < (long long)pw * d || t2 + d2 <= t + d) {
        j += 2;
        continue;
      }
    }
    a = t + d;
    ++j;
    break;
  }
  q.j = j;
  q.a = a;
}

// Algorithm 1 with pulse limits: pg percent for the gate test (cancel the
// last kept output edge E when 100 (t_o - E) < pg gateDelay, or t_o <= E)
// and pw percent for the interconnect test.  Below 100 percent a cancel
// can expose a kept edge that is itself still cancellable, so the kept
// edges form a stack (the paper's p_o moving back): the top lives in a
// register, the ones below it in the sink, which reads them back.  T1 is
// kept as y0 * len plus one signed term per kept edge (a rising edge at t
// adds len - min(t, len), a falling one subtracts it), so a cancel takes
// its edge's term back out.
template <int K, class Sink>
__device__ __forceinline__ void run_gate_pp(Pin (&pin)[K], uint32_t lut, const int32_t* __restrict__ gd,
                                            int32_t edit, int32_t len, int32_t pg, int32_t pw, Sink& sink,
                                            int32_t& count, int32_t& t1, uint32_t& y0) {
  uint32_t col = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) col |= (pin[i].v0 & 1u) << i;
  uint32_t y = (lut >> col) & 1u;
  y0 = y;
#pragma unroll
  for (int i = 0; i < K; ++i) pin_advance_pp(pin[i], pw);
  int32_t n = 0;  // kept edges below the top (in the sink)
  bool top_on = false;
  int32_t top = 0;
  long long acc = y ? (long long)len : 0ll;
  auto term = [&](int32_t k, int32_t te) -> long long {  // signed T1 term of kept edge k
    const long long r = (long long)len - min(te, len);
    return ((y0 ^ (uint32_t)k) & 1u) ? -r : r;
  };
  for (;;) {
    int32_t t = pin[0].a;
#pragma unroll
    for (int i = 1; i < K; ++i) t = min(t, pin[i].a);
    if (t == kInf) break;
    int istar = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (pin[i].a == t) {  // every pin arriving now switches (MSI)
        col ^= 1u << i;
        istar = i;
        pin_advance_pp(pin[i], pw);
      }
    }
    const uint32_t yn = (lut >> col) & 1u;
    if (yn != y) {
      const uint32_t side = (col & ((1u << istar) - 1u)) | ((col >> (istar + 1)) << istar);
      const uint32_t ie = (col >> istar) & 1u;
      const int32_t d = max(1, gd[istar * 32 + (int)(ie * 16u + yn * 8u + side)] + edit);
      const int32_t to = t + d;
      if (top_on && (100ll * (to - top) < (long long)pg * d || to <= top)) {
        acc -= term(n, top);  // cancel the last kept edge
        if (n > 0) {
          --n;
          top = sink.get(n);
        } else {
          top_on = false;
        }
      } else {
        if (top_on) sink.put(n++, top);
        top = to;
        top_on = true;
        acc += term(n, to);
      }
      y = yn;
    }
  }
  if (top_on) sink.put(n++, top);
  count = n;
  t1 = (int32_t)acc;
}

// Appends a lane's output edges to its column of its warp's staging buffer
// (element k of lane l's column at [k * 32 + l]); edges past the cap are
// dropped and the lane simulates again straight to global memory once its
// offsets are known.
template <int CAP>
struct WarpSink {
  int32_t* col;
  int32_t pos;  // edges already staged by this lane's earlier windows
  __device__ __forceinline__ void put(int k, int32_t t) {
    if (pos + k < CAP) col[(pos + k) * 32] = t;
  }
};

struct GlobalSink {
  int32_t* dst;
  long long limit;
  __device__ __forceinline__ void put(int k, int32_t t) {
    if (k < limit) dst[k] = t;
  }
  __device__ __forceinline__ int32_t get(int k) const { return k < limit ? dst[k] : 0; }
};

// Record of (net, window): start (relative to its level's base), count and
// start value; the bounds check keeps reads inside the arena even after an
// earlier error.
__device__ __forceinline__ void load_record(const JobView& J, long long rec, long long base,
                                            int32_t& s, int32_t& n, uint32_t& v0) {
  s = __ldg(J.rstart + rec);
  const uint32_t m = __ldg(J.rmeta + rec);
  n = (int32_t)(m & (uint32_t)kMaxCount);
  v0 = m >> 15;
  if (s < 0 || base + s + n > J.capacity) {
    s = 0;
    n = 0;
    atomicOr(J.status, kStCorrupt);
  }
}

// Everything about a gate that does not depend on the window: fetched once
// and reused for all of a lane's consecutive windows of that gate.
template <int K>
struct GateCtx {
  const int32_t* gd;  // gate delay table of pin 1 (pins follow, 32 entries each)
  uint32_t lut;
  int32_t edit;
  long long rec[K];   // record index of (driving net, window 0): net * NW
  long long base[K];  // times index of the driving net's level
  int32_t dr[K], df[K];
};

template <int K>
__device__ __forceinline__ void load_gate(const JobView& J, int32_t g, GateCtx<K>& c) {
  const int32_t p0 = __ldg(J.fanin_ptr + g);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int32_t pp = p0 + i;
    const int32_t net = __ldg(J.fanin_net + pp);
    c.rec[i] = (long long)net * J.NW;
    c.base[i] = __ldg(J.lvl_base + __ldg(J.net_level + net));
    c.dr[i] = __ldg(J.wire_delay + 2 * pp);
    c.df[i] = __ldg(J.wire_delay + 2 * pp + 1);
  }
  c.lut = __ldg(J.lut + g);
  c.edit = J.gate_delta ? __ldg(J.gate_delta + g) : 0;
  c.gd = J.gate_delay + (long long)p0 * 32;
}

// Windows w .. w+run-1 of gate g for one lane: counts go to cnt[0..run),
// edges to the lane's staging column, start values to bits m0.. of y0s.
template <int K, int CAP, int F>
__device__ __forceinline__ void simulate_run_k(const JobView& J, int32_t g, int32_t w, int32_t run,
                                               int32_t* cnt, int32_t* col, int32_t& total,
                                               uint32_t& y0s, int m0, long long& t1_acc) {
  GateCtx<K> c;
  load_gate<K>(J, g, c);
  for (int32_t j = 0; j < run; ++j) {
    Pin pin[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      int32_t s, n;
      uint32_t v0;
      load_record(J, c.rec[i] + w + j, c.base[i], s, n, v0);
      pin[i] = Pin{J.times + c.base[i] + s, n, 0, kInf, c.dr[i], c.df[i], v0};
    }
    WarpSink<CAP> sink{col, total};
    int32_t n = 0, t1 = 0;
    uint32_t y0 = 0;
    run_gate<K, F>(pin, c.lut, c.gd, c.edit, window_len(J.w0 + w + j, J.W, J.C, J.L), sink, n, t1, y0);
    cnt[j] = n;
    total += n;
    y0s |= y0 << (m0 + j);
    t1_acc += t1;
  }
}

template <int CAP, int F>
__device__ __forceinline__ void simulate_run(const JobView& J, int32_t g, int32_t w, int32_t run,
                                             int32_t* cnt, int32_t* col, int32_t& total, uint32_t& y0s,
                                             int m0, long long& t1_acc) {
  switch (__ldg(J.fanin_ptr + g + 1) - __ldg(J.fanin_ptr + g)) {
    case 1: simulate_run_k<1, CAP, F>(J, g, w, run, cnt, col, total, y0s, m0, t1_acc); break;
    case 2: simulate_run_k<2, CAP, F>(J, g, w, run, cnt, col, total, y0s, m0, t1_acc); break;
    case 3: simulate_run_k<3, CAP, F>(J, g, w, run, cnt, col, total, y0s, m0, t1_acc); break;
    default: simulate_run_k<4, CAP, F>(J, g, w, run, cnt, col, total, y0s, m0, t1_acc); break;
  }
}

// One window of one gate straight to global memory (lanes whose edges did
// not fit their staging column).
template <int K, int F>
__device__ __forceinline__ int32_t simulate_global_k(const JobView& J, int32_t g, int32_t w, int32_t* dst,
                                                     long long limit) {
  GateCtx<K> c;
  load_gate<K>(J, g, c);
  Pin pin[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    int32_t s, n;
    uint32_t v0;
    load_record(J, c.rec[i] + w, c.base[i], s, n, v0);
    pin[i] = Pin{J.times + c.base[i] + s, n, 0, kInf, c.dr[i], c.df[i], v0};
  }
  GlobalSink sink{dst, limit};
  int32_t n = 0, t1 = 0;
  uint32_t y0 = 0;
  run_gate<K, F>(pin, c.lut, c.gd, c.edit, window_len(J.w0 + w, J.W, J.C, J.L), sink, n, t1, y0);
  return n;
}

template <int F>
__device__ __forceinline__ int32_t simulate_global(const JobView& J, int32_t g, int32_t w, int32_t* dst,
                                                   long long limit) {
  switch (__ldg(J.fanin_ptr + g + 1) - __ldg(J.fanin_ptr + g)) {
    case 1: return simulate_global_k<1, F>(J, g, w, dst, limit);
    case 2: return simulate_global_k<2, F>(J, g, w, dst, limit);
    case 3: return simulate_global_k<3, F>(J, g, w, dst, limit);
    default: return simulate_global_k<4, F>(J, g, w, dst, limit);
  }
}

// Per-warp shared memory.  The linear tiling uses the output staging (each
// lane's column, the compacted tile, per-item edge counts).  The
// gate-aligned tiling stages, per fanin pin, the windows' metas, their edge
// starts inside the pin's tile run, the run itself (pins share one pool),
// and the gate's delay tables; and keeps per window its output meta, plus
// the list of windows that have fanin edges.
template <int IPT, int KMAX = 4>
struct WarpSmem {
  static constexpr int TW = 32 * IPT;    // windows (items) per tile
  static constexpr int POOL = 4 * TW;    // fanin edge times staged per tile
  static constexpr int CAP = 8;          // output edges staged per lane (per round)
  static constexpr int OCAP = (2 * TW > CAP * 32) ? 2 * TW : CAP * 32;  // compacted output edges
  int32_t sstart[KMAX][TW];
  int32_t spool[POOL];
  int32_t scr[CAP * 32];
  int32_t cmp[OCAP];
  int32_t cnt[TW];     // linear: per-item edge counts; gate-aligned: per-window output offsets
  int32_t sgd[KMAX][32];  // gate-aligned: the gate's delay tables
  uint16_t smeta[KMAX][TW];
  uint16_t omet[TW];
  uint8_t list[TW];
};

// Takes a tile's output range: one atomic add on the level counter both
// reserves `aggregate` edges and counts the tile done.  The tile that brings
// the done count to the level's tile count sees the final edge total and
// publishes it as the next level's base (later kernels see it after this
// launch ends).  Returns the range's start relative to the level base (same
// value in every lane).
__device__ __forceinline__ long long claim_range(const JobView& J, const SegView& S, int lane, long long aggregate,
                                                 long long base) {
  unsigned long long old = 0;
  if (lane == 0) old = atomicAdd(S.counters, (1ull << kTileShift) + (unsigned long long)aggregate);
  old = __shfl_sync(0xffffffffu, old, 0);
  const long long start = (long long)(old & kEdgeMask);
  if (lane == 0 && (long long)(old >> kTileShift) == (long long)S.n_tiles - 1) {
    const long long tot = start + aggregate;
    if (tot > 0x7fffffffll) atomicOr(J.status, kStOffset);
    J.lvl_base[S.level + 1] = base + tot;
    if (base + tot > J.capacity) atomicOr(J.status, kStCapacity);
  }
  return start;
}

// Everything after a linear tile's simulation: sum the lanes' edge counts
// with shuffles, take the tile's output range, write the records (start,
// count and start value of each item), store the edges (compacted through
// shared memory, or, when a lane's staging column overflowed, by `resim`
// straight to their final place), and add the SAIF of the lane's last gate.
template <int IPT, class Resim>
__device__ __forceinline__ void finish_tile(const JobView& J, const SegView& S, int lane, WarpSmem<IPT>& sm,
                                            int32_t n_mine, const int32_t* cnt, int32_t total, uint32_t y0s,
                                            long long rec_first, int32_t cur_gl, long long acc_t1,
                                            long long acc_tc, Resim&& resim) {
  constexpr int CAP = WarpSmem<IPT>::CAP;
  const bool any_over = __any_sync(0xffffffffu, total > CAP);
  int32_t incl = total;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const long long excl_l = incl - total;
  const long long aggregate = __shfl_sync(0xffffffffu, incl, 31);
  const long long base = __ldg(J.lvl_base + S.level);
  const long long start = claim_range(J, S, lane, aggregate, base);

  {
    long long o = start + excl_l;
    for (int m = 0; m < n_mine; ++m) {
      const int32_t c = cnt[m];
      J.rstart[rec_first + m] = (int32_t)o;
      J.rmeta[rec_first + m] = (uint16_t)(min(c, kMaxCount) | (int32_t)(((y0s >> m) & 1u) << 15));
      if (c > kMaxCount) atomicOr(J.status, kStOffset);
      o += c;
    }
    if (n_mine > 0 && o > 0x7fffffffll) atomicOr(J.status, kStOffset);
  }

  int32_t* dst = J.times + base + start;
  const long long room = J.capacity - base - start;  // elements left in the arena
  if (!any_over) {
    for (int k = 0; k < total; ++k) sm.cmp[excl_l + k] = sm.scr[k * 32 + lane];
    __syncwarp();
    const long long n = aggregate < room ? aggregate : (room > 0 ? room : 0);
    for (long long j = lane; j < n; j += 32) dst[j] = sm.cmp[j];
  } else if (n_mine > 0) {
    if (total <= CAP) {
      for (int k = 0; k < total; ++k)
        if (excl_l + k < room) dst[excl_l + k] = sm.scr[k * 32 + lane];
    } else {
      resim(dst, excl_l, room);
    }
  }
  __syncwarp();

  // SAIF: the lane's last gate; one atomic per warp when the warp agrees
  // (every lane takes part in every shuffle)
  const int32_t g_lane0 = __shfl_sync(0xffffffffu, cur_gl, 0);
  const bool uniform = __all_sync(0xffffffffu, cur_gl < 0 || cur_gl == g_lane0);
  if (uniform) {
    long long a = acc_t1, c = acc_tc;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, d);
      c += __shfl_xor_sync(0xffffffffu, c, d);
    }
    if (lane == 0 && g_lane0 >= 0) {
      const long long n = (long long)J.I + S.gate_begin + g_lane0;
      if (a) atomicAdd(J.saif_t1 + n, (unsigned long long)a);
      if (c) atomicAdd(J.saif_tc + n, (unsigned long long)c);
    }
  } else if (cur_gl >= 0) {
    const long long n = (long long)J.I + S.gate_begin + cur_gl;
    if (acc_t1) atomicAdd(J.saif_t1 + n, (unsigned long long)acc_t1);
    if (acc_tc) atomicAdd(J.saif_tc + n, (unsigned long long)acc_tc);
  }
}

// Linear tiling: 32 lanes x IPT consecutive items of the level in
// gate-major order (a tile may span gates); each lane fetches its gate's
// metadata once and reads its fanin records and edges from global memory.
template <int IPT, int F>
__device__ __forceinline__ void linear_tile(const JobView& J, const SegView& S, int32_t tile, WarpSmem<IPT>& sm) {
  constexpr int CAP = WarpSmem<IPT>::CAP;
  const int lane = threadIdx.x & 31;
  const int32_t r0 = tile * (32 * IPT) + lane * IPT;  // this lane's first item
  const int32_t n_mine = max(0, min(IPT, S.n_items - r0));
  int32_t* cnt = sm.cnt + lane * IPT;
  int32_t total = 0;
  uint32_t y0s = 0;
  int32_t cur_gl = -1;  // SAIF partial sums for the lane's current gate
  long long acc_t1 = 0, acc_tc = 0;
  if (n_mine > 0) {
    int32_t gl = r0 / J.NW, w = r0 - gl * J.NW, m = 0;
    while (m < n_mine) {
      const int32_t run = min(n_mine - m, J.NW - w);
      if (cur_gl >= 0) {  // the lane's windows cross into the next gate (small NW)
        const long long n = (long long)J.I + S.gate_begin + cur_gl;
        if (acc_t1) atomicAdd(J.saif_t1 + n, (unsigned long long)acc_t1);
        if (acc_tc) atomicAdd(J.saif_tc + n, (unsigned long long)acc_tc);
      }
      cur_gl = gl;
      acc_t1 = 0;
      const int32_t before = total;
      simulate_run<CAP, F>(J, S.gate_begin + gl, w, run, cnt + m, sm.scr + lane, total, y0s, m, acc_t1);
      acc_tc = total - before;
      m += run;
      ++gl;
      w = 0;
    }
  }
  // a level's records are linear in its item index
  const long long rec_first = ((long long)J.I + S.gate_begin) * J.NW + r0;
  finish_tile<IPT>(J, S, lane, sm, n_mine, cnt, total, y0s, rec_first, cur_gl, acc_t1, acc_tc,
                   [&](int32_t* dst, long long o, long long room) {
                     int32_t gl = r0 / J.NW, w = r0 - gl * J.NW;
                     for (int m = 0; m < n_mine; ++m) {
                       o += simulate_global<F>(J, S.gate_begin + gl, w, dst + o, room - o);
                       if (++w == J.NW) {
                         w = 0;
                         ++gl;
                       }
                     }
                   });
}

// Exclusive prefix sums, in window order, of one pin's per-window edge
// counts (bits 0-14 of m[k] for window k*32 + lane), written to out[] for
// the n windows.  While the pin's run has fewer than 65536 edges, four
// chunks of 32 windows share one 64-bit shuffle scan, 16 bits per chunk
// (no field can carry into the next); longer runs scan chunk by chunk.
template <int IPT>
__device__ __forceinline__ void run_starts(const uint32_t (&m)[IPT], int lane, int32_t n, int32_t run_edges,
                                           int32_t* out) {
  if (run_edges < 65536) {
    constexpr int NV = (IPT + 3) / 4;
    unsigned long long v[NV], incl[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      v[q] = 0;
#pragma unroll
      for (int k = 4 * q; k < IPT && k < 4 * q + 4; ++k)
        v[q] |= (unsigned long long)(m[k] & (uint32_t)kMaxCount) << (16 * (k - 4 * q));
      incl[q] = v[q];
    }
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl[q], dd);
        if (lane >= dd) incl[q] += u;
      }
    }
    int32_t carry = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const unsigned long long tot = __shfl_sync(0xffffffffu, incl[q], 31);
      const unsigned long long ex = incl[q] - v[q];
#pragma unroll
      for (int k = 4 * q; k < IPT && k < 4 * q + 4; ++k) {
        const int sh = 16 * (k - 4 * q);
        if (k * 32 + lane < n) out[k * 32 + lane] = carry + (int32_t)((ex >> sh) & 0xffffull);
        carry += (int32_t)((tot >> sh) & 0xffffull);
      }
    }
  } else {
    int32_t carry = 0;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int32_t c = (int32_t)(m[k] & (uint32_t)kMaxCount);
      int32_t incl = c;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += u;
      }
      if (k * 32 + lane < n) out[k * 32 + lane] = carry + incl - c;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// 4-byte asynchronous global-to-shared copy (cp.async, cached in L1), and
// the wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(int32_t* smem, const int32_t* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A gate's fanin nets and their levels, first pin, truth table and pin
// count: one 32-byte descriptor, or the CSR arrays when there is none.
struct GateDesc {
  int32_t net[4];
  int32_t lvl[4];
  int32_t p0, k;
  uint32_t lut;
};

__device__ __forceinline__ void load_desc(const JobView& J, int32_t g, GateDesc& d) {
  if (J.gdesc) {
    const int4 a = __ldg(J.gdesc + 2 * (long long)g);
    const int4 b = __ldg(J.gdesc + 2 * (long long)g + 1);
    d.net[0] = a.x; d.net[1] = a.y; d.net[2] = a.z; d.net[3] = a.w;
    d.p0 = b.x;
    d.lut = (uint32_t)b.y & 0xffffu;
    d.k = (int32_t)((uint32_t)b.y >> 16);
    d.lvl[0] = (int32_t)((uint32_t)b.z & 0xffffu); d.lvl[1] = (int32_t)((uint32_t)b.z >> 16);
    d.lvl[2] = (int32_t)((uint32_t)b.w & 0xffffu); d.lvl[3] = (int32_t)((uint32_t)b.w >> 16);
  } else {
    d.p0 = __ldg(J.fanin_ptr + g);
    d.k = __ldg(J.fanin_ptr + g + 1) - d.p0;
    d.lut = __ldg(J.lut + g);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      d.net[i] = __ldg(J.fanin_net + d.p0 + (i < d.k ? i : 0));
      d.lvl[i] = __ldg(J.net_level + d.net[i]);
    }
  }
}

// Simulation with pulse limits.  Below 100 percent a cancel can expose a
// kept output edge that is itself still cancellable, so the kept edges are
// a stack that must be read back, however deep it grows; staging columns of
// a fixed size cannot hold it.  So each window is simulated straight into
// global memory, into a slot sized by an upper bound of its output: every
// kept output edge follows an arrival of at least one pin, so a window has
// at most as many output edges as its pins have edges.

// The gate-aligned tile's steps after the quiet windows are settled and the
// others listed (steps 3 and 4 of wide_tile_k): the bounds are scanned in
// window order and the tile claims their sum; every listed window is
// simulated into its slot; then the windows' edges are moved down, in
// window order, into one run (a slot never starts before its run position,
// so in-order moves never overwrite edges not yet moved), leaving the
// unused rest of the claim empty.
template <int K, int IPT, class PinsOf>
__device__ __forceinline__ void wide_tail_pp(const JobView& J, const SegView& S, int32_t g, int32_t tg,
                                             int32_t wb, int32_t n, int32_t n_act, int lane, uint32_t lut,
                                             const int32_t* gd, int32_t edit, long long acc_t1,
                                             WarpSmem<IPT>& sm, PinsOf&& pins_of) {
  // slot of each listed window: exclusive scan of the bounds (in sm.cnt)
  int32_t U = 0;
  for (int32_t r0 = 0; r0 < n_act; r0 += 32) {
    const int32_t q = r0 + lane;
    int32_t ub = 0, wl = 0;
    if (q < n_act) {
      wl = sm.list[q];
#pragma unroll
      for (int i = 0; i < K; ++i) ub += sm.smeta[i][wl] & kMaxCount;
    }
    int32_t incl = ub;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += v;
    }
    if (q < n_act) sm.cnt[wl] = U + incl - ub;
    U += __shfl_sync(0xffffffffu, incl, 31);
  }
  // claim the bound (the level's range, or the append region)
  const long long lbase = __ldg(J.lvl_base + S.level);
  const long long obase = S.append_in ? __ldg(S.append_in) : lbase;
  unsigned long long old = 0;
  if (lane == 0) old = atomicAdd(S.counters, (1ull << kTileShift) + (unsigned long long)U);
  old = __shfl_sync(0xffffffffu, old, 0);
  const long long start = (long long)(old & kEdgeMask);
  if (lane == 0 && (long long)(old >> kTileShift) == (long long)S.n_tiles - 1) {
    const long long tot = start + U;
    if (tot > 0x7fffffffll) atomicOr(J.status, kStOffset);
    if (S.append_in) *S.append_out = obase + tot;
    else J.lvl_base[S.level + 1] = lbase + tot;
    if (obase + tot > J.capacity) atomicOr(J.status, kStCapacity);
  }
  int32_t* dst = J.times + obase + start;
  const long long room = J.capacity - obase - start;  // elements left in the arena
  __syncwarp();
  for (int32_t q = lane; q < n_act; q += 32) {
    const int32_t wl = sm.list[q];
    const int32_t at = sm.cnt[wl];
    Pin pin[K];
    pins_of(wl, pin);
    GlobalSink sink{dst + at, room - at};
    int32_t c = 0, t1 = 0;
    uint32_t y0 = 0;
    run_gate_pp<K>(pin, lut, gd, edit, window_len(J.w0 + wb + wl, J.W, J.C, J.L), J.pulse_g, J.pulse_w, sink,
                   c, t1, y0);
    acc_t1 += t1;
    sm.omet[wl] = (uint16_t)(min(c, kMaxCount) | (int32_t)(y0 << 15));
    if (c > kMaxCount) atomicOr(J.status, kStOffset);
  }
  __syncwarp();  // every lane's edges and metas are visible to the warp
  // move each window's edges from its slot to its place in the run
  int32_t out_n = 0;
  for (int32_t q = 0; q < n_act; ++q) {
    const int32_t wl = sm.list[q];
    const int32_t c = sm.omet[wl] & kMaxCount;
    const int32_t from = sm.cnt[wl];
    for (int32_t j0 = 0; j0 < c; j0 += 32) {
      const int32_t j = j0 + lane;
      int32_t v = 0;
      const bool ok = j < c && from + j < room && out_n + j < room;
      if (ok) v = dst[from + j];
      __syncwarp();
      if (ok) dst[out_n + j] = v;
      __syncwarp();
    }
    out_n += c;
  }
  {
    uint16_t* om = J.rmeta + ((long long)J.I + g) * J.NW + wb;
#pragma unroll
    for (int k = 0; k < IPT; ++k)
      if (k * 32 + lane < n) om[k * 32 + lane] = sm.omet[k * 32 + lane];
  }
  const long long rel = obase - lbase + start;
  if (lane == 0) {
    if (rel + out_n > 0x7fffffffll) atomicOr(J.status, kStOffset);
    J.tinfo[((long long)J.I + g) * J.T + tg] = make_int2((int32_t)rel, out_n);
  }
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) acc_t1 += __shfl_xor_sync(0xffffffffu, acc_t1, dd);
  if (lane == 0) {
    const long long net = (long long)J.I + g;
    if (acc_t1) atomicAdd(J.saif_t1 + net, (unsigned long long)acc_t1);
    if (out_n) atomicAdd(J.saif_tc + net, (unsigned long long)out_n);
  }
}

// One item (gate g, window w) with pulse limits, straight into dst.
template <int K>
__device__ __forceinline__ int32_t simulate_item_pp(const JobView& J, int32_t g, int32_t w, int32_t* dst,
                                                    long long limit, int32_t& t1, uint32_t& y0) {
  GateCtx<K> c;
  load_gate<K>(J, g, c);
  Pin pin[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    int32_t s, n;
    uint32_t v0;
    load_record(J, c.rec[i] + w, c.base[i], s, n, v0);
    pin[i] = Pin{J.times + c.base[i] + s, n, 0, kInf, c.dr[i], c.df[i], v0};
  }
  GlobalSink sink{dst, limit};
  int32_t n = 0;
  run_gate_pp<K>(pin, c.lut, c.gd, c.edit, window_len(J.w0 + w, J.W, J.C, J.L), J.pulse_g, J.pulse_w, sink, n,
                 t1, y0);
  return n;
}

// Linear tiling with pulse limits: every item gets a slot sized by its
// bound, in item order; records point at their slots (records carry their
// own starts here, so the slots need no compaction).
template <int IPT>
__device__ __forceinline__ void linear_tile_pp(const JobView& J, const SegView& S, int32_t tile) {
  const int lane = threadIdx.x & 31;
  const int32_t r0 = tile * (32 * IPT) + lane * IPT;  // this lane's first item
  const int32_t n_mine = max(0, min(IPT, S.n_items - r0));
  int32_t ub[IPT];
  int32_t mine = 0;
#pragma unroll
  for (int m = 0; m < IPT; ++m) {
    ub[m] = 0;
    if (m < n_mine) {
      const int32_t r = r0 + m, gl = r / J.NW, w = r - gl * J.NW, g = S.gate_begin + gl;
      const int32_t p0 = __ldg(J.fanin_ptr + g), p1 = __ldg(J.fanin_ptr + g + 1);
      for (int32_t p = p0; p < p1; ++p)
        ub[m] += __ldg(J.rmeta + (long long)__ldg(J.fanin_net + p) * J.NW + w) & kMaxCount;
      mine += ub[m];
    }
  }
  int32_t incl = mine;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl += v;
  }
  const long long aggregate = __shfl_sync(0xffffffffu, incl, 31);
  const long long base = __ldg(J.lvl_base + S.level);
  const long long start = claim_range(J, S, lane, aggregate, base);
  int32_t* dst = J.times + base + start;
  const long long room = J.capacity - base - start;
  long long o = incl - mine;
  int32_t cur_gl = -1;
  long long acc_t1 = 0, acc_tc = 0;
  const long long rec_first = ((long long)J.I + S.gate_begin) * J.NW + r0;
  for (int m = 0; m < n_mine; ++m) {
    const int32_t r = r0 + m, gl = r / J.NW, w = r - gl * J.NW, g = S.gate_begin + gl;
    if (gl != cur_gl) {
      if (cur_gl >= 0) {
        const long long net = (long long)J.I + S.gate_begin + cur_gl;
        if (acc_t1) atomicAdd(J.saif_t1 + net, (unsigned long long)acc_t1);
        if (acc_tc) atomicAdd(J.saif_tc + net, (unsigned long long)acc_tc);
      }
      cur_gl = gl;
      acc_t1 = acc_tc = 0;
    }
    int32_t c = 0, t1 = 0;
    uint32_t y0 = 0;
    const long long lim = room - o < (long long)ub[m] ? room - o : (long long)ub[m];
    switch (__ldg(J.fanin_ptr + g + 1) - __ldg(J.fanin_ptr + g)) {
      case 1: c = simulate_item_pp<1>(J, g, w, dst + o, lim, t1, y0); break;
      case 2: c = simulate_item_pp<2>(J, g, w, dst + o, lim, t1, y0); break;
      case 3: c = simulate_item_pp<3>(J, g, w, dst + o, lim, t1, y0); break;
      default: c = simulate_item_pp<4>(J, g, w, dst + o, lim, t1, y0); break;
    }
    if (start + o + c > 0x7fffffffll || c > kMaxCount) atomicOr(J.status, kStOffset);
    J.rstart[rec_first + m] = (int32_t)(start + o);
    J.rmeta[rec_first + m] = (uint16_t)(min(c, kMaxCount) | (int32_t)(y0 << 15));
    acc_t1 += t1;
    acc_tc += c;
    o += ub[m];
  }
  if (cur_gl >= 0) {
    const long long net = (long long)J.I + S.gate_begin + cur_gl;
    if (acc_t1) atomicAdd(J.saif_t1 + net, (unsigned long long)acc_t1);
    if (acc_tc) atomicAdd(J.saif_tc + net, (unsigned long long)acc_tc);
  }
}

// Gate-aligned tiling, up to K pins (pins from d.k on are absent: no edges,
// value 0): tile tg of gate g, windows wb .. wb+n-1 (n <= TW).
//  1. Everything that depends on the gate descriptor only is loaded at once:
//     each pin's level base, tile run, wire and gate delays, and the n metas
//     (kept in registers).  Then the pins' runs are staged into the pool
//     (in pin order while they fit), and each pin's per-window edge starts
//     inside its run are found by a warp scan of its counts.
//  2. Every window whose pins carry no edge is settled on the spot: its
//     output is the truth table at the pins' start values, with no edge.
//     The others are listed, in window order.
//  3. The listed windows are simulated (Algorithm 1) in rounds of 32, one
//     per lane, so lanes stay busy however sparse the activity; each round's
//     edges are compacted, in window order, into the tile's output buffer.
//  4. One atomic add claims the tile's run.  The output metas are stored
//     while it is in flight, then the run (coalesced) and the tile's entry.
//     If some lane's edges did not fit the staging, the listed windows are
//     simulated again straight into their final place instead.
// Kernel modes: Algorithm 1 as printed over all of a level's gates (the
// benchmark kernel, which carries no code of the other modes), pulse limits
// (with or without a gate list), and a gate list at 100 percent.
// Modes 4 + F are Algorithm 1 as printed without the features F (above).
constexpr int kModePlain = 0, kModePulse = 1, kModeCone = 2;
constexpr int kModeNoWireFilter = 4 + kNoWireFilter, kModeAvgSdf = 4 + kAvgSdf,
              kModeNoWireAvgSdf = 4 + kNoWireFilter + kAvgSdf;
__host__ __device__ constexpr int features_of(int mode) { return mode >= 4 ? mode - 4 : 0; }
// modes whose launches may cover a gate list and write to an append region
__host__ __device__ constexpr bool lists_of(int mode) { return mode == kModePulse || mode == kModeCone; }

template <int K, int IPT, int MODE, int KMAX = 4>
__device__ __forceinline__ void wide_tile_k(const JobView& J, const SegView& S, const GateDesc& d, int32_t g,
                                            int32_t tg, int32_t n, WarpSmem<IPT, KMAX>& sm) {
  static_assert(K <= KMAX, "the tile body stages at most KMAX pins");
  constexpr int CAP = WarpSmem<IPT, KMAX>::CAP;
  constexpr int POOL = WarpSmem<IPT, KMAX>::POOL;
  constexpr int OCAP = WarpSmem<IPT, KMAX>::OCAP;
  constexpr int TW = WarpSmem<IPT, KMAX>::TW;
  const int lane = threadIdx.x & 31;
  const int32_t wb = tg * TW;
  const int32_t p0 = d.p0;
  const int kp = d.k;  // pins kp..K-1 are absent: no edges, value 0

  // 1. loads that depend on the descriptor only, all in flight together
  long long base[K];
  int2 run[K];
  int32_t dr[K], df[K], gdv[K];
  uint32_t mv[K][IPT];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    base[i] = 0;
    run[i] = make_int2(0, 0);
    dr[i] = df[i] = gdv[i] = 0;
#pragma unroll
    for (int k = 0; k < IPT; ++k) mv[i][k] = 0u;
    if (i < kp) {
      const int32_t pp = p0 + i;
      base[i] = __ldg(J.lvl_base + d.lvl[i]);
      run[i] = __ldg(J.tinfo + (long long)d.net[i] * J.T + tg);
      dr[i] = __ldg(J.wire_delay + 2 * pp);
      df[i] = __ldg(J.wire_delay + 2 * pp + 1);
      gdv[i] = __ldg(J.gate_delay + (long long)pp * 32 + lane);
      const uint16_t* mp = J.rmeta + (long long)d.net[i] * J.NW + wb;
#pragma unroll
      for (int k = 0; k < IPT; ++k)
        if (k * 32 + lane < n) mv[i][k] = __ldg(mp + k * 32 + lane);
    }
  }
  const int32_t edit = J.gate_delta ? __ldg(J.gate_delta + g) : 0;

  // pins' runs into the pool; src[i] + s is where edge s of pin i's run is
  const int32_t* src[K];
  int32_t lim[K];  // edges in the pin's run (0 if it failed its bounds check)
  {
    int32_t used = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int32_t lo = run[i].x, c = run[i].y;
      const bool ok = lo >= 0 && c >= 0 && base[i] + lo + c <= J.capacity;
      if (!ok && lane == 0) atomicOr(J.status, kStCorrupt);
      lim[i] = ok ? c : 0;
      if (ok && used + c <= POOL) {
        // asynchronous copies: the pins' runs are all in flight while the
        // warp scans counts and settles quiet windows
        const int32_t* gsrc = J.times + base[i] + lo;
        for (int j = lane; j < c; j += 32) cp_async4(&sm.spool[used + j], gsrc + j);
        src[i] = &sm.spool[used];
        used += c;
      } else {
        src[i] = J.times + (ok ? base[i] + lo : 0);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    sm.sgd[i][lane] = gdv[i];
#pragma unroll
    for (int k = 0; k < IPT; ++k)
      if (k * 32 + lane < n) sm.smeta[i][k * 32 + lane] = (uint16_t)mv[i][k];
    // edge starts inside the run: exclusive scan of the counts in window order
    if (lim[i] > 0) run_starts<IPT>(mv[i], lane, n, lim[i], sm.sstart[i]);
  }

  // 2. settle the windows whose output cannot change, list the others
  // (window order: k-major, lane-minor).  A window's output cannot change
  // when no pin has an edge, and also when the truth table is constant on
  // every input combination its switching pins can reach from their start
  // values (the other pins fixed): then every event of Algorithm 1 finds
  // the output value unchanged, so the window keeps its start value and has
  // no edge, whatever the arrival times and delays.
  const uint32_t lut = d.lut;
  const uint32_t lt_mask = (1u << lane) - 1u;
  long long acc_t1 = 0;
  int32_t n_act = 0;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int32_t j = k * 32 + lane;
    const bool valid = j < n;
    uint32_t col = 0, sw = 0;  // start values; pins with edges
#pragma unroll
    for (int i = 0; i < K; ++i) {
      col |= (mv[i][k] >> 15) << i;
      sw |= ((mv[i][k] & (uint32_t)kMaxCount) != 0u ? 1u : 0u) << i;
    }
    // the reachable combinations as a set of truth-table columns: each
    // switching pin i doubles the set by its mirror image in bit i
    uint32_t cube = 1u << col;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      constexpr uint32_t kLow[4] = {0x5555u, 0x3333u, 0x0f0fu, 0x00ffu};  // columns with bit i clear
      if ((sw >> i) & 1u) cube |= ((cube & kLow[i]) << (1 << i)) | ((cube >> (1 << i)) & kLow[i]);
    }
    const uint32_t hit = lut & cube;
    const bool act = valid && sw != 0u && hit != 0u && hit != cube;
    const uint32_t amask = __ballot_sync(0xffffffffu, act);
    if (act) {
      sm.list[n_act + __popc(amask & lt_mask)] = (uint8_t)j;
    } else if (valid) {
      const uint32_t y = (lut >> col) & 1u;
      sm.omet[j] = (uint16_t)(y << 15);
      if (y) acc_t1 += window_len(J.w0 + wb + j, J.W, J.C, J.L);
    }
    n_act += __popc(amask);
  }
  cp_async_wait_all();  // the staged runs; the barrier then publishes every
  __syncwarp();         // lane's copies, list entries and metas

  const int32_t* gd = &sm.sgd[0][0];
  auto pins_of = [&](int32_t wl, Pin (&pin)[K]) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const uint32_t meta = sm.smeta[i][wl];
      int32_t c = (int32_t)(meta & (uint32_t)kMaxCount);
      int32_t s = c ? sm.sstart[i][wl] : 0;
      if (s < 0 || s + c > lim[i]) {  // never read outside the pin's run
        atomicOr(J.status, kStCorrupt);
        s = 0;
        c = 0;
      }
      pin[i].t = src[i] + s;
      pin[i].n = c;
      pin[i].j = 0;
      pin[i].a = kInf;
      pin[i].dr = dr[i];
      pin[i].df = df[i];
      pin[i].v0 = meta >> 15;
    }
  };

  if constexpr (MODE == kModePulse) {
    wide_tail_pp<K, IPT>(J, S, g, tg, wb, n, n_act, lane, lut, gd, edit, acc_t1, sm, pins_of);
    return;
  }

  // 3. listed windows, 32 per round, compacted in window order into cmp
  int32_t out_n = 0;    // the tile's edges so far
  bool spill = false;   // some round did not fit the staging (warp-uniform)
  for (int32_t r0 = 0; r0 < n_act; r0 += 32) {
    const int32_t q = r0 + lane;
    int32_t c = 0;
    if (q < n_act) {
      const int32_t wl = sm.list[q];
      Pin pin[K];
      pins_of(wl, pin);
      WarpSink<CAP> sink{sm.scr + lane, 0};
      int32_t t1 = 0;
      uint32_t y0 = 0;
      run_gate<K, features_of(MODE)>(pin, lut, gd, edit, window_len(J.w0 + wb + wl, J.W, J.C, J.L), sink, c, t1, y0);
      acc_t1 += t1;
      sm.omet[wl] = (uint16_t)(min(c, kMaxCount) | (int32_t)(y0 << 15));
      if (c > kMaxCount) atomicOr(J.status, kStOffset);
    }
    int32_t incl = c;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += v;
    }
    const int32_t round_n = __shfl_sync(0xffffffffu, incl, 31);
    const bool over = __any_sync(0xffffffffu, c > CAP);  // every lane votes
    spill = spill || over || out_n + round_n > OCAP;
    if (!spill) {
      const int32_t at = out_n + incl - c;
      for (int e = 0; e < c; ++e) sm.cmp[at + e] = sm.scr[e * 32 + lane];
    }
    out_n += round_n;
  }
  __syncwarp();

  // 4. claim the run; store the metas while the claim is in flight
  const long long lbase = __ldg(J.lvl_base + S.level);
  // where the launch's runs go: the level's range, or the append region
  long long obase = lbase;
  if constexpr (lists_of(MODE)) obase = S.append_in ? __ldg(S.append_in) : lbase;
  unsigned long long old = 0;
  if (lane == 0) old = atomicAdd(S.counters, (1ull << kTileShift) + (unsigned long long)out_n);
  {
    uint16_t* om = J.rmeta + ((long long)J.I + g) * J.NW + wb;
#pragma unroll
    for (int k = 0; k < IPT; ++k)
      if (k * 32 + lane < n) om[k * 32 + lane] = sm.omet[k * 32 + lane];
  }
  old = __shfl_sync(0xffffffffu, old, 0);
  const long long start = (long long)(old & kEdgeMask);
  const long long rel = obase - lbase + start;  // the run's start relative to the level base
  if (lane == 0) {
    if ((long long)(old >> kTileShift) == (long long)S.n_tiles - 1) {
      const long long tot = start + out_n;
      if (tot > 0x7fffffffll) atomicOr(J.status, kStOffset);
      if (lists_of(MODE) && S.append_in) *S.append_out = obase + tot;
      else J.lvl_base[S.level + 1] = lbase + tot;
      if (obase + tot > J.capacity) atomicOr(J.status, kStCapacity);
    }
    if (rel + out_n > 0x7fffffffll) atomicOr(J.status, kStOffset);
    J.tinfo[((long long)J.I + g) * J.T + tg] = make_int2((int32_t)rel, out_n);
  }
  int32_t* dst = J.times + obase + start;
  const long long room = J.capacity - obase - start;  // elements left in the arena
  if (!spill) {
    const long long m = out_n < room ? out_n : (room > 0 ? room : 0);
    for (long long e = lane; e < m; e += 32) dst[e] = sm.cmp[e];
  } else {
    // output offsets of the windows inside the run (consecutive windows per lane)
    const int32_t w_first = lane * IPT;
    int32_t mine = 0;
#pragma unroll
    for (int k = 0; k < IPT; ++k)
      if (w_first + k < n) mine += sm.omet[w_first + k] & kMaxCount;
    int32_t incl = mine;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += v;
    }
    int32_t o = incl - mine;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (w_first + k < n) {
        sm.cnt[w_first + k] = o;
        o += sm.omet[w_first + k] & kMaxCount;
      }
    }
    __syncwarp();
    for (int32_t q = lane; q < n_act; q += 32) {
      const int32_t wl = sm.list[q];
      const int32_t at = sm.cnt[wl];
      Pin pin[K];
      pins_of(wl, pin);
      GlobalSink sink{dst + at, room - at};
      int32_t c = 0, t1 = 0;
      uint32_t y0 = 0;
      run_gate<K, features_of(MODE)>(pin, lut, gd, edit, window_len(J.w0 + wb + wl, J.W, J.C, J.L), sink, c, t1, y0);
    }
  }

  // SAIF of the gate: one atomic per tile
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) acc_t1 += __shfl_xor_sync(0xffffffffu, acc_t1, dd);
  if (lane == 0) {
    const long long net = (long long)J.I + g;
    if (acc_t1) atomicAdd(J.saif_t1 + net, (unsigned long long)acc_t1);
    if (out_n) atomicAdd(J.saif_tc + net, (unsigned long long)out_n);
  }
}

template <int IPT, int MODE>
__device__ __forceinline__ void wide_tile(const JobView& J, const SegView& S, int32_t tile, WarpSmem<IPT>& sm) {
  constexpr int TW = 32 * IPT;
  const int32_t gl = tile / J.T;
  const int32_t tg = tile - gl * J.T;
  const int32_t n = min(TW, J.NW - tg * TW);
  int32_t g = S.gate_begin + gl;
  if constexpr (lists_of(MODE)) {
    if (S.gate_list) g = __ldg(S.gate_list + gl);
  }
  GateDesc d;
  load_desc(J, g, d);
  // two compiled bodies, not four: 1- and 3-pin gates run with an absent
  // pin (measured 3% faster than four bodies: the hot code then fits the
  // instruction cache better)
  if (d.k <= 2) wide_tile_k<2, IPT, MODE>(J, S, d, g, tg, n, sm);
  else wide_tile_k<4, IPT, MODE>(J, S, d, g, tg, n, sm);
}

// Gate lists (fanout cones) exist for gate-aligned tiles only.
template <int IPT, int MODE>
__device__ __forceinline__ void propagate_warp(const JobView& J, const SegView& S, int32_t tile, WarpSmem<IPT>& sm) {
  if (J.T > 0) wide_tile<IPT, MODE>(J, S, tile, sm);
  else if constexpr (MODE == kModePulse) linear_tile_pp<IPT>(J, S, tile);
  else linear_tile<IPT, features_of(MODE)>(J, S, tile, sm);
}

// Blocks per SM the launch bounds ask for: as many as the per-warp shared
// memory lets reside (227 KB per SM), capped at 1024 threads (64 registers
// per thread).  Where shared memory is the tighter limit, the threads get the
// registers that limit frees.
template <int NT, int IPT>
__host__ __device__ constexpr int smem_blocks() {
  return (int)((227u * 1024u) / (sizeof(WarpSmem<IPT>) * (NT / 32) + 2048u));
}
template <int NT, int IPT>
__host__ __device__ constexpr int min_blocks() {
  return smem_blocks<NT, IPT>() < 1 ? 1 : (smem_blocks<NT, IPT>() < 1024 / NT ? smem_blocks<NT, IPT>() : 1024 / NT);
}

// One level of one job; each warp takes one tile (one atomic per block hands
// out NT/32 consecutive tiles).  MODE: kModePlain, or one of the modes with
// pulse limits or gate lists (separate instantiations, so the kernel for
// Algorithm 1 as printed carries none of their code).
template <int NT, int IPT, int MODE = kModePlain>
__global__ void __launch_bounds__(NT, (min_blocks<NT, IPT>())) propagate_kernel(const __grid_constant__ PropParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<IPT>* sm = reinterpret_cast<WarpSmem<IPT>*>(smem_raw);
  __shared__ int32_t s_first;
  if (threadIdx.x == 0) s_first = atomicAdd(p.tile_counter, NT / 32);
  __syncthreads();
  const int32_t t = s_first + (int32_t)(threadIdx.x >> 5);
  if (t >= p.n_tiles) return;
  propagate_warp<IPT, MODE>(p.job, p.seg, t, sm[threadIdx.x >> 5]);
}

// Shared memory of the kernel for gates of at most two pins: two pins
// staged per tile.
template <int IPT>
using PairSmem = WarpSmem<IPT, 2>;
template <int NT, int IPT>
__host__ __device__ constexpr int pair_blocks() {
  return (int)((227u * 1024u) / (sizeof(PairSmem<IPT>) * (NT / 32) + 2048u)) < 1024 / NT
             ? (int)((227u * 1024u) / (sizeof(PairSmem<IPT>) * (NT / 32) + 2048u))
             : 1024 / NT;
}

// Algorithm 1 as printed (or without the features of MODE 4 + F) over
// gate-aligned tiles of a level's gates of at most two pins (the level's
// first gates).  The body is the 2-pin one of propagate_kernel; with two
// pins' staging per warp, four blocks of 256 threads fit an SM instead of
// three, and the registers fit the 64 that four blocks leave.
template <int NT, int IPT, int MODE = kModePlain>
__global__ void __launch_bounds__(NT, (pair_blocks<NT, IPT>())) propagate_pair_kernel(const __grid_constant__ PropParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PairSmem<IPT>* sm = reinterpret_cast<PairSmem<IPT>*>(smem_raw);
  __shared__ int32_t s_first;
  if (threadIdx.x == 0) s_first = atomicAdd(p.tile_counter, NT / 32);
  __syncthreads();
  const int32_t t = s_first + (int32_t)(threadIdx.x >> 5);
  if (t >= p.n_tiles) return;
  const JobView& J = p.job;
  constexpr int TW = 32 * IPT;
  const int32_t gl = t / J.T;
  const int32_t tg = t - gl * J.T;
  const int32_t n = min(TW, J.NW - tg * TW);
  const int32_t g = p.seg.gate_begin + gl;
  GateDesc d;
  load_desc(J, g, d);
  static_assert(!lists_of(MODE), "the pair kernel covers a level's gates, without a gate list");
  wide_tile_k<2, IPT, MODE, 2>(J, p.seg, d, g, tg, n, sm[threadIdx.x >> 5]);
}

// The pair kernel over several jobs' segments (the gates of at most two pins
// of each (part, level) segment; propagate_multi_kernel runs the rest of
// each level, into the same level counters).
template <int NT, int IPT>
__global__ void __launch_bounds__(NT, (pair_blocks<NT, IPT>()))
    propagate_pair_multi_kernel(const __grid_constant__ MultiParams m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PairSmem<IPT>* sm = reinterpret_cast<PairSmem<IPT>*>(smem_raw);
  __shared__ int32_t s_first;
  if (threadIdx.x == 0) s_first = atomicAdd(m.tile_counter, NT / 32);
  __syncthreads();
  const int32_t t = s_first + (int32_t)(threadIdx.x >> 5);
  if (t >= m.n_tiles) return;
  int32_t lo = 0, hi = m.n_segs - 1;
  while (lo < hi) {  // last segment with tile_begin <= t
    const int32_t mid = (lo + hi + 1) >> 1;
    if (m.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  const MultiSeg& sg = m.segs[lo];
  const JobView& J = sg.job;
  constexpr int TW = 32 * IPT;
  const int32_t tile = t - sg.tile_begin;
  const int32_t gl = tile / J.T;
  const int32_t tg = tile - gl * J.T;
  const int32_t n = min(TW, J.NW - tg * TW);
  const int32_t g = sg.seg.gate_begin + gl;
  GateDesc d;
  load_desc(J, g, d);
  wide_tile_k<2, IPT, kModePlain, 2>(J, sg.seg, d, g, tg, n, sm[threadIdx.x >> 5]);
}

// Several jobs (each at its own level) in one launch: tiles are handed out
// as above and mapped to (job, level) segments, each segment with its own
// counters and tiling.
template <int NT, int IPT>
__global__ void __launch_bounds__(NT, (min_blocks<NT, IPT>())) propagate_multi_kernel(const __grid_constant__ MultiParams m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<IPT>* sm = reinterpret_cast<WarpSmem<IPT>*>(smem_raw);
  __shared__ int32_t s_first;
  if (threadIdx.x == 0) s_first = atomicAdd(m.tile_counter, NT / 32);
  __syncthreads();
  const int32_t t = s_first + (int32_t)(threadIdx.x >> 5);
  if (t >= m.n_tiles) return;
  int32_t lo = 0, hi = m.n_segs - 1;
  while (lo < hi) {  // last segment with tile_begin <= t
    const int32_t mid = (lo + hi + 1) >> 1;
    if (m.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  const MultiSeg& sg = m.segs[lo];
  propagate_warp<IPT, kModePlain>(sg.job, sg.seg, t - sg.tile_begin, sm[threadIdx.x >> 5]);
}

// Items per tile (one warp's tile) for a variant.
inline int tile_items_of(int ipt) { return 32 * ipt; }

// Windows per batch from which a level uses gate-aligned tiles with staged
// fanins (below, tiles would be mostly empty).
inline bool wide_tiling(int32_t nw, int ipt) { return nw >= 16 * ipt; }

// Tiles of one level of `gates` gates and nw windows.
inline long long level_tiles(long long gates, int32_t nw, int ipt) {
  const long long tw = tile_items_of(ipt);
  return wide_tiling(nw, ipt) ? gates * ((nw + tw - 1) / tw) : (gates * nw + tw - 1) / tw;
}

template <int NT, int IPT>
inline size_t dyn_smem() { return sizeof(WarpSmem<IPT>) * (NT / 32); }

// Opts a kernel in to more than 48 KB of dynamic shared memory on the
// current device.  The attribute belongs to the kernel on one device, so it
// is set once per (kernel, device); `once` is the kernel's flag set.  On a
// failure the error is returned (and stays the runtime's last error) and
// the flag stays clear, so a later launch tries again.
template <class Kern>
inline cudaError_t smem_opt_in(Kern kern, size_t bytes, gatspi_host::PerDeviceOnce& once) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  once.run(dev, [&] {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e == cudaSuccess ? 0 : 1;
  });
  return e;
}

// Host-side launchers of the two propagation kernels for one compiled
// (threads, items per thread) variant.  `err` holds the failure to opt in
// to the variant's shared memory, if any (the kernel is then not launched).
struct SingleLaunch {
  const PropParams* p;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  template <int NT, int IPT>
  void go() {
    static gatspi_host::PerDeviceOnce once;
    if ((err = smem_opt_in(propagate_kernel<NT, IPT>, dyn_smem<NT, IPT>(), once)) != cudaSuccess) return;
    const unsigned grid = (unsigned)((p->n_tiles + NT / 32 - 1) / (NT / 32));
    propagate_kernel<NT, IPT><<<grid, NT, dyn_smem<NT, IPT>(), s>>>(*p);
  }
};

// The kernels of the other modes, compiled for a few launch shapes only.
template <int MODE>
struct SingleLaunchMode {
  const PropParams* p;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  template <int NT, int IPT>
  void go() {
    static gatspi_host::PerDeviceOnce once;
    if ((err = smem_opt_in(propagate_kernel<NT, IPT, MODE>, dyn_smem<NT, IPT>(), once)) != cudaSuccess) return;
    const unsigned grid = (unsigned)((p->n_tiles + NT / 32 - 1) / (NT / 32));
    propagate_kernel<NT, IPT, MODE><<<grid, NT, dyn_smem<NT, IPT>(), s>>>(*p);
  }
};

// The kernel for gates of at most two pins: Algorithm 1 as printed at
// 256 x 4 and 128 x 4, the reduced-feature modes at 256 x 4 (the other
// launch shapes run those gates in propagate_kernel).
inline bool pair_variant_compiled(int nt, int ipt, int features) {
  return ipt == 4 && (nt == 256 || (nt == 128 && features == 0));
}

// Fewest tiles of a level's gates of at most two pins for which they get a
// launch of their own (about seven waves of the pair kernel on 152 SMs):
// smaller parts stay in the level's one launch.
constexpr int64_t kPairMinTiles = 32768;

struct PairLaunch {
  const PropParams* p;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  template <int NT, int MODE>
  void go() {
    constexpr int IPT = 4;
    static gatspi_host::PerDeviceOnce once;
    const size_t bytes = sizeof(PairSmem<IPT>) * (NT / 32);
    if ((err = smem_opt_in(propagate_pair_kernel<NT, IPT, MODE>, bytes, once)) != cudaSuccess) return;
    const unsigned grid = (unsigned)((p->n_tiles + NT / 32 - 1) / (NT / 32));
    propagate_pair_kernel<NT, IPT, MODE><<<grid, NT, bytes, s>>>(*p);
  }
};

struct MultiPairLaunch {
  const MultiParams* m;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  template <int NT>
  void go() {
    constexpr int IPT = 4;
    static gatspi_host::PerDeviceOnce once;
    const size_t bytes = sizeof(PairSmem<IPT>) * (NT / 32);
    if ((err = smem_opt_in(propagate_pair_multi_kernel<NT, IPT>, bytes, once)) != cudaSuccess) return;
    const unsigned grid = (unsigned)((m->n_tiles + NT / 32 - 1) / (NT / 32));
    propagate_pair_multi_kernel<NT, IPT><<<grid, NT, bytes, s>>>(*m);
  }
};

// Pulse limits: 256 x {1, 2, 4} and 128 x 8.
inline bool pulse_variant_compiled(int nt, int ipt) {
  return (nt == 256 && (ipt == 1 || ipt == 2 || ipt == 4)) || (nt == 128 && ipt == 8);
}

inline bool launch_variant_pp(int nt, int ipt, SingleLaunchMode<kModePulse>& launch) {
  switch (nt * 16 + ipt) {
    case 256 * 16 + 1: launch.template go<256, 1>(); return true;
    case 256 * 16 + 2: launch.template go<256, 2>(); return true;
    case 256 * 16 + 4: launch.template go<256, 4>(); return true;
    case 128 * 16 + 8: launch.template go<128, 8>(); return true;
    default: return false;
  }
}

// Kernels without some features (the paper's cost comparison): 256 x 4 and
// 256 x 1.
template <int MODE>
inline bool launch_variant_features(int ipt, SingleLaunchMode<MODE>& launch) {
  switch (ipt) {
    case 1: launch.template go<256, 1>(); return true;
    case 4: launch.template go<256, 4>(); return true;
    default: return false;
  }
}

// Gate lists at 100 percent: 256 threads, any windows per thread (a cone
// must keep the tile width of the runs it updates).
inline bool launch_variant_cone(int ipt, SingleLaunchMode<kModeCone>& launch) {
  switch (ipt) {
    case 1: launch.template go<256, 1>(); return true;
    case 2: launch.template go<256, 2>(); return true;
    case 4: launch.template go<256, 4>(); return true;
    case 8: launch.template go<256, 8>(); return true;
    default: return false;
  }
}

struct MultiLaunch {
  const MultiParams* m;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  template <int NT, int IPT>
  void go() {
    static gatspi_host::PerDeviceOnce once;
    if ((err = smem_opt_in(propagate_multi_kernel<NT, IPT>, dyn_smem<NT, IPT>(), once)) != cudaSuccess) return;
    const unsigned grid = (unsigned)((m->n_tiles + NT / 32 - 1) / (NT / 32));
    propagate_multi_kernel<NT, IPT><<<grid, NT, dyn_smem<NT, IPT>(), s>>>(*m);
  }
};

// Launch one of the compiled (threads, items per thread) variants.
template <class Launch>
inline bool launch_variant(int nt, int ipt, Launch&& launch) {
  switch (nt * 16 + ipt) {
    case 128 * 16 + 1: launch.template go<128, 1>(); return true;
    case 128 * 16 + 2: launch.template go<128, 2>(); return true;
    case 128 * 16 + 4: launch.template go<128, 4>(); return true;
    case 128 * 16 + 8: launch.template go<128, 8>(); return true;
    case 256 * 16 + 1: launch.template go<256, 1>(); return true;
    case 256 * 16 + 2: launch.template go<256, 2>(); return true;
    case 256 * 16 + 4: launch.template go<256, 4>(); return true;
    case 256 * 16 + 8: launch.template go<256, 8>(); return true;
    case 512 * 16 + 1: launch.template go<512, 1>(); return true;
    case 512 * 16 + 2: launch.template go<512, 2>(); return true;
    case 512 * 16 + 4: launch.template go<512, 4>(); return true;
    default: return false;
  }
}

// Level 0: the inputs' records for the batch, read straight from the
// stimulus (edges of window w = edges of its cycles, shifted onto the
// window's time axis; start value = initial value toggled by every earlier
// edge).  Inputs' edges are laid out input-major, so record (i, w) starts at
// in_prefix[i] + (edges of input i in the batch before window w).
struct InputParams {
  const int64_t* __restrict__ edge_ptr;   // [I*C+1]
  const int32_t* __restrict__ edge_time;
  const uint8_t* __restrict__ init_in;    // [I]
  const long long* __restrict__ in_prefix;  // [I] edges of inputs < i in this batch
  int32_t* rstart;  // linear tiling
  int2* tinfo;      // gate-aligned tiling
  int32_t T, TW;    // tiles per net and windows per tile (gate-aligned), or 0
  uint16_t* rmeta;
  int32_t* times;
  unsigned long long* saif_t1;
  unsigned long long* saif_tc;
  long long total;  // level-0 edges of the batch
  long long* lvl_base;
  int32_t* status;
  int32_t I, NW, w0, W, C, L;
  int32_t n_items;
};

__global__ void inputs_kernel(const InputParams q) {
  const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = r < q.n_items;
  int32_t i = 0, cnt = 0;
  long long t1 = 0;
  if (valid) {
    i = r / q.NW;
    const int32_t w = r - i * q.NW;
    const int32_t wg = q.w0 + w;
    const int32_t c0 = wg * q.W, c1 = min(c0 + q.W, q.C);
    const int64_t* ep = q.edge_ptr + (long long)i * q.C;
    const long long a = ep[c0];
    const long long b = ep[c1];
    const long long o = q.in_prefix[i] + (a - ep[q.w0 * q.W]);
    uint32_t v = (q.init_in[i] ^ (uint32_t)((a - ep[0]) & 1)) & 1u;
    cnt = (int32_t)(b - a);
    if (q.T > 0) {
      if (w % q.TW == 0) {  // the tile's run: its windows' edges, in order
        const int32_t ct = min((q.w0 + min(w + q.TW, q.NW)) * q.W, q.C);
        q.tinfo[(long long)i * q.T + w / q.TW] = make_int2((int32_t)o, (int32_t)(ep[ct] - a));
      }
    } else {
      q.rstart[(long long)i * q.NW + w] = (int32_t)o;
    }
    q.rmeta[(long long)i * q.NW + w] = (uint16_t)(min(cnt, kMaxCount) | (int32_t)(v << 15));
    if (cnt > kMaxCount) atomicOr(q.status, kStOffset);
    const int32_t len = (c1 - c0) * q.L;
    int32_t prev = 0;
    long long k = o;
    for (int32_t c = c0; c < c1; ++c) {
      const int32_t shift = (c - c0) * q.L;
      for (long long e = ep[c]; e < ep[c + 1]; ++e) {
        const int32_t t = __ldg(q.edge_time + e) + shift;
        q.times[k++] = t;
        const int32_t cl = min(t, len);
        if (v) t1 += cl - prev;
        prev = cl;
        v ^= 1u;
      }
    }
    if (v) t1 += len - prev;
  }
  if (r == 0) {
    q.lvl_base[0] = 0;
    q.lvl_base[1] = q.total;
  }
  // every lane takes part in every shuffle
  const int32_t i0 = __shfl_sync(0xffffffffu, i, 0);
  const int lane0_valid = __shfl_sync(0xffffffffu, valid ? 1 : 0, 0);
  const bool uniform = __all_sync(0xffffffffu, !valid || i == i0);
  if (uniform) {
    long long c = cnt;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      t1 += __shfl_xor_sync(0xffffffffu, t1, d);
      c += __shfl_xor_sync(0xffffffffu, c, d);
    }
    if (lane == 0 && lane0_valid) {
      if (t1) atomicAdd(q.saif_t1 + i0, (unsigned long long)t1);
      if (c) atomicAdd(q.saif_tc + i0, (unsigned long long)c);
    }
  } else if (valid) {
    if (t1) atomicAdd(q.saif_t1 + i, (unsigned long long)t1);
    if (cnt) atomicAdd(q.saif_tc + i, (unsigned long long)cnt);
  }
}

// Read-back of one window: counts and start values per internal net, then
// the edges gathered to caller-ordered offsets.
__global__ void window_counts_kernel(int32_t N, int32_t NW, int32_t w, const uint16_t* rmeta, int32_t* cnt,
                                     uint8_t* init_out) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t m = rmeta[(long long)n * NW + w];
  cnt[n] = (int32_t)(m & (uint32_t)kMaxCount);
  init_out[n] = (uint8_t)(m >> 15);
}

__global__ void window_gather_kernel(int32_t N, int32_t NW, int32_t w, const int32_t* net_level,
                                     const int32_t* rstart, const int2* tinfo, int32_t T, int32_t TW,
                                     const uint16_t* rmeta, const long long* lvl_base, const int32_t* times,
                                     const long long* dst_ptr, int32_t* out) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const long long rec = (long long)n * NW + w;
  const int32_t c = (int32_t)(rmeta[rec] & (uint32_t)kMaxCount);
  long long s;
  if (T > 0) {  // the tile's run start plus the counts of its earlier windows
    const int32_t t = w / TW;
    s = tinfo[(long long)n * T + t].x;
    for (int32_t v = t * TW; v < w; ++v) s += rmeta[(long long)n * NW + v] & (uint32_t)kMaxCount;
  } else {
    s = rstart[rec];
  }
  const int32_t* src = times + lvl_base[net_level[n]] + s;
  const long long d = dst_ptr[n];
  for (int32_t k = 0; k < c; ++k) out[d + k] = src[k];
}

// Clear the SAIF of the listed gates' nets before their cone is simulated
// again (the new waveforms' SAIF is added by the propagation launches).
__global__ void clear_saif_kernel(int32_t n, const int32_t* __restrict__ gates, int32_t I,
                                  unsigned long long* t1, unsigned long long* tc) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long net = (long long)I + gates[k];
  t1[net] = 0;
  tc[net] = 0;
}

// Add a finished part's SAIF into its job's accumulators.
__global__ void saif_add_kernel(int32_t N, const unsigned long long* t1, const unsigned long long* tc,
                                unsigned long long* dst_t1, unsigned long long* dst_tc) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  if (t1[n]) atomicAdd(dst_t1 + n, t1[n]);
  if (tc[n]) atomicAdd(dst_tc + n, tc[n]);
}

}  // namespace
}  // namespace gatspi_dev
