// Device code of the re-simulator: input restructuring, the per-level
// propagation kernel, and waveform read-back.
//
// Propagation (GATSPI, Section 3 and Algorithm 1): one thread per (gate,
// window) item of a logic level.  Each thread merges its fanin pins'
// delayed, inertially filtered edges, evaluates the truth table, picks the
// switching pin's (COND) delay, applies the gate inertial filter and emits
// the output edges.  The paper simulates every item twice (a counting pass,
// then a storing pass at the scanned offsets); here one pass suffices:
// edges are staged in shared memory while the block's edge counts are
// scanned, and the block's global offset comes from a decoupled look-back
// scan across blocks (Merrill and Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", NVIDIA TR 2016).  Fanin waveforms are therefore
// read from HBM once per pin instead of twice.
//
// Waveform store (one batch of NW windows):
//   init[n*NW + w]            uint8   value of net n at the start of window w
//   off[n*NW + w + level(n)]  int32   first edge of (n, w), relative to the
//                                     level's base; every level keeps one
//                                     extra slot at its end, so the edges of
//                                     (n, w) end at the next slot
//   times[lvl_base[level(n)] + off ...]  int32 edge times, window-relative
// Items of a level are ordered gate-major, window-minor, so the windows of a
// net are contiguous and a warp's reads of one pin cover one contiguous
// range.
#pragma once

#include <cstdint>

namespace gatspi_dev {
namespace {  // every translation unit gets its own copy of the kernels

constexpr int32_t kInf = 0x7fffffff;
// output edges per thread staged in shared memory (two NT x cap int32
// buffers per block stay under the 48 KB static limit)
template <int NT>
__host__ __device__ constexpr int staging_cap() { return NT >= 512 ? 8 : 16; }

// status bits (device -> host)
constexpr int kStCapacity = 1;  // arena too small for this batch
constexpr int kStTimeout = 2;   // look-back wait ran out
constexpr int kStCorrupt = 4;   // a record failed its bounds check
constexpr int kStOffset = 8;    // a level's edges exceed the int32 offset range

// look-back state word: 2 flag bits over a 62-bit value
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr long long kSpinLimit = 1ll << 20;  // bounded wait (well under a second)

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
  // waveform store
  uint8_t* init;
  int32_t* off;
  int32_t* times;
  long long* lvl_base;
  long long capacity;  // elements of times
  // SAIF accumulators (per internal net)
  unsigned long long* saif_t1;
  unsigned long long* saif_tc;
  int32_t* status;
  int32_t I;
  int32_t NW;  // windows in the batch
  // window w of the batch is global window w0 + w; it spans cycles
  // [g*W, min(g*W + W, C)) of L ps each
  int32_t w0, W, C, L;
};

// One level of one job inside a launch.
struct SegView {
  unsigned long long* tile_state;  // [n_tiles] look-back words, zero before use
  int32_t level;
  int32_t gate_begin;  // first internal gate of the level
  int32_t net_end;     // one past the level's last net
  int32_t n_items;     // gates of the level * NW
  int32_t n_tiles;
};

struct PropParams {
  JobView job;
  SegView seg;
  int32_t* tile_counter;  // zero before the launch
};

struct MultiSeg {
  SegView seg;
  int32_t job;         // index into the job table
  int32_t tile_begin;  // first launch-wide tile of this segment
};

struct MultiParams {
  const JobView* jobs;
  const MultiSeg* segs;  // sorted by tile_begin
  int32_t n_segs;
  int32_t* tile_counter;  // zero before the launch
};

__device__ __forceinline__ int32_t window_len(int32_t wg, int32_t W, int32_t C, int32_t L) {
  const int32_t c0 = wg * W;
  const int32_t c1 = min(c0 + W, C);
  return (c1 - c0) * L;
}

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
__device__ __forceinline__ void pin_advance(Pin& q) {
  int32_t j = q.j, a = kInf;
  while (j < q.n) {
    const int32_t t = __ldg(q.t + j);
    const int32_t d = (((q.v0 ^ (uint32_t)j) & 1u) == 0u) ? q.dr : q.df;
    if (j + 1 < q.n && __ldg(q.t + j + 1) - t < d) {
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

// Algorithm 1 for one gate and one window (`edit` shifts every gate delay of
// the gate, clamped at 1 ps; 0 without a delay edit).  The output keeps at most one
// edge that may still be cancelled (the last kept one, `pend`): a cancel
// needs the last kept edge to lie after the current time, and once an edge
// has been cancelled the kept edge before it is already in the past, so no
// deeper history is needed.  Edges are handed to `sink` as they become
// final; T1 (time at 1 inside [0, len)) is integrated on the way.
template <int K, class Sink>
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
  for (int i = 0; i < K; ++i) pin_advance(pin[i]);
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
        pin_advance(pin[i]);
      }
    }
    const uint32_t yn = (lut >> col) & 1u;
    if (yn != y) {
      if (pend_on && pend > t) {
        pend_on = false;  // gate inertial filter: cancel the last kept edge
      } else {
        if (pend_on) flush(pend);
        const uint32_t side = (col & ((1u << istar) - 1u)) | ((col >> (istar + 1)) << istar);
        const uint32_t ie = (col >> istar) & 1u;
        pend = t + max(1, __ldg(gd + istar * 32 + (int)(ie * 16u + yn * 8u + side)) + edit);
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

// Appends a thread's output edges to its column of the block's staging
// buffer (element k of the column at [k * NT]); edges past the cap are dropped
// and the thread re-simulates straight to global memory later.
template <int NT>
struct SmemSink {
  int32_t* col;
  int32_t pos;  // edges already staged by this thread's earlier items
  __device__ __forceinline__ void put(int k, int32_t t) {
    if (pos + k < staging_cap<NT>()) col[(pos + k) * NT] = t;
  }
};

struct GlobalSink {
  int32_t* dst;
  long long limit;
  __device__ __forceinline__ void put(int k, int32_t t) {
    if (k < limit) dst[k] = t;
  }
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Load fanin pin pp of item (., w).
__device__ __forceinline__ void load_pin(const JobView& J, int32_t pp, int32_t w, Pin& q) {
  const int32_t net = __ldg(J.fanin_net + pp);
  const int32_t lv = __ldg(J.net_level + net);
  const long long it = (long long)net * J.NW + w + lv;
  const int32_t s = __ldg(J.off + it);
  const int32_t e = __ldg(J.off + it + 1);
  const long long base = __ldg(J.lvl_base + lv);
  q.t = J.times + base + s;
  q.n = e - s;
  if (s < 0 || q.n < 0 || base + e > J.capacity) {
    q.n = 0;  // never read outside the arena (only after an earlier error)
    atomicOr(J.status, kStCorrupt);
  }
  q.j = 0;
  q.a = kInf;
  q.dr = __ldg(J.wire_delay + 2 * pp);
  q.df = __ldg(J.wire_delay + 2 * pp + 1);
  q.v0 = __ldg(J.init + (long long)net * J.NW + w);
}

template <int K, class Sink>
__device__ __forceinline__ void simulate_k(const JobView& J, int32_t g, int32_t w, int32_t p0,
                                           Sink& sink, int32_t& count, int32_t& t1,
                                           uint32_t& y0) {
  Pin pin[K];
#pragma unroll
  for (int i = 0; i < K; ++i) load_pin(J, p0 + i, w, pin[i]);
  const uint32_t lut = __ldg(J.lut + g);
  const int32_t edit = J.gate_delta ? __ldg(J.gate_delta + g) : 0;
  const int32_t len = window_len(J.w0 + w, J.W, J.C, J.L);
  run_gate<K>(pin, lut, J.gate_delay + (long long)p0 * 32, edit, len, sink, count, t1, y0);
}

template <class Sink>
__device__ __forceinline__ void simulate_item(const JobView& J, int32_t g, int32_t w,
                                              Sink& sink, int32_t& count, int32_t& t1,
                                              uint32_t& y0) {
  const int32_t p0 = __ldg(J.fanin_ptr + g);
  switch (__ldg(J.fanin_ptr + g + 1) - p0) {
    case 1: simulate_k<1>(J, g, w, p0, sink, count, t1, y0); break;
    case 2: simulate_k<2>(J, g, w, p0, sink, count, t1, y0); break;
    case 3: simulate_k<3>(J, g, w, p0, sink, count, t1, y0); break;
    default: simulate_k<4>(J, g, w, p0, sink, count, t1, y0); break;
  }
}

// One tile of one job's level: NT threads x IPT items, items in
// gate-major, window-minor order, thread t taking IPT consecutive items
// (consecutive windows of one gate, so its gate metadata is fetched once
// and its records and edges are contiguous).  Simulate, scan the edge
// counts, find the tile's offset by look-back, write records and edges, and
// add the tile's SAIF.  Called by every thread of the block.
template <int NT, int IPT>
__device__ __forceinline__ void propagate_tile(const JobView& J, const SegView& S, int32_t tile) {
  constexpr int NWARP = NT / 32;
  constexpr int TILE = NT * IPT;
  constexpr int kCap = staging_cap<NT>();
  __shared__ int32_t s_scr[kCap * NT];
  __shared__ int32_t s_cmp[kCap * NT];
  __shared__ long long s_wsum[NWARP];
  __shared__ int32_t s_over;
  __shared__ long long s_prefix, s_base;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_over = 0;
    s_base = J.lvl_base[S.level];
  }
  __syncthreads();
  const int32_t r0 = tile * TILE + tid * IPT;  // this thread's first item
  const int32_t n_mine = max(0, min(IPT, S.n_items - r0));
  int32_t cnt[IPT];
  uint32_t y0s = 0;
  int32_t total = 0;
  // SAIF partial sums for the thread's current gate
  int32_t cur_gl = -1;
  long long acc_t1 = 0, acc_tc = 0;
  int32_t gl = 0, w = 0;
  if (n_mine > 0) {
    gl = r0 / J.NW;
    w = r0 - gl * J.NW;
  }
#pragma unroll
  for (int m = 0; m < IPT; ++m) {
    cnt[m] = 0;
    if (m < n_mine) {
      if (gl != cur_gl) {
        if (cur_gl >= 0) {  // gate changed inside the thread's items (small NW)
          const long long n = (long long)J.I + S.gate_begin + cur_gl;
          if (acc_t1) atomicAdd(J.saif_t1 + n, (unsigned long long)acc_t1);
          if (acc_tc) atomicAdd(J.saif_tc + n, (unsigned long long)acc_tc);
        }
        cur_gl = gl;
        acc_t1 = acc_tc = 0;
      }
      SmemSink<NT> sink{s_scr + tid, total};
      int32_t c = 0, t1 = 0;
      uint32_t y0 = 0;
      simulate_item(J, S.gate_begin + gl, w, sink, c, t1, y0);
      cnt[m] = c;
      total += c;
      y0s |= y0 << m;
      acc_t1 += t1;
      acc_tc += c;
      if (++w == J.NW) {
        w = 0;
        ++gl;
      }
    }
  }
  if (total > kCap) s_over = 1;

  // block-wide exclusive scan of the per-thread edge counts
  int32_t incl = total;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long v = lane < NWARP ? s_wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += u;
    }
    if (lane < NWARP) s_wsum[lane] = v;
  }
  __syncthreads();
  const long long excl_local = (warp ? s_wsum[warp - 1] : 0) + incl - total;
  const long long aggregate = s_wsum[NWARP - 1];

  // decoupled look-back: this block's offset among all blocks of the level
  if (warp == 0) {
    long long excl = 0;
    if (tile == 0) {
      if (lane == 0) st_release(S.tile_state, kFlagPrefix | (unsigned long long)aggregate);
    } else {
      if (lane == 0) st_release(S.tile_state + tile, kFlagAggregate | (unsigned long long)aggregate);
      int32_t pos = tile - 1;
      long long spins = 0;
      for (;;) {
        const int32_t idx = pos - lane;
        const unsigned long long word = idx >= 0 ? ld_acquire(S.tile_state + idx) : kFlagPrefix;
        const unsigned long long flag = word & ~kValueMask;
        if (__any_sync(0xffffffffu, flag == 0)) {
          if (++spins > kSpinLimit) {
            if (lane == 0) atomicOr(J.status, kStTimeout);
            break;
          }
          __nanosleep(64);
          continue;
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
        long long val = (long long)(word & kValueMask);
        if (pmask) {
          const int first = __ffs(pmask) - 1;
          if (lane > first) val = 0;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) val += __shfl_xor_sync(0xffffffffu, val, d);
        excl += val;
        if (pmask) break;
        pos -= 32;
      }
      if (lane == 0) st_release(S.tile_state + tile, kFlagPrefix | (unsigned long long)(excl + aggregate));
    }
    if (lane == 0) s_prefix = excl;
  }
  __syncthreads();
  const long long prefix = s_prefix;
  const long long base = s_base;
  const long long my_off = prefix + excl_local;

  // records: offset and start value of every item; a level's record index
  // is linear in the item index
  {
    const long long rec = ((long long)J.I + S.gate_begin) * J.NW + r0;
    long long o = my_off;
#pragma unroll
    for (int m = 0; m < IPT; ++m) {
      if (m < n_mine) {
        J.off[rec + S.level + m] = (int32_t)o;
        J.init[rec + m] = (uint8_t)((y0s >> m) & 1u);
        o += cnt[m];
      }
    }
    if (n_mine > 0 && o > 0x7fffffffll) atomicOr(J.status, kStOffset);
  }
  if (tile == S.n_tiles - 1 && tid == 0) {
    const long long tot = prefix + aggregate;
    if (tot > 0x7fffffffll) atomicOr(J.status, kStOffset);
    J.off[(long long)S.net_end * J.NW + S.level] = (int32_t)tot;
    J.lvl_base[S.level + 1] = base + tot;
    if (base + tot > J.capacity) atomicOr(J.status, kStCapacity);
  }

  // edges
  int32_t* dst = J.times + base + prefix;
  const long long room = J.capacity - base - prefix;  // elements left in the arena
  if (!s_over) {
    for (int k = 0; k < total; ++k) s_cmp[excl_local + k] = s_scr[k * NT + tid];
    __syncthreads();
    const long long n = aggregate < room ? aggregate : (room > 0 ? room : 0);
    for (long long j = tid; j < n; j += NT) dst[j] = s_cmp[j];
  } else if (n_mine > 0) {
    if (total <= kCap) {
      for (int k = 0; k < total; ++k)
        if (excl_local + k < room) dst[excl_local + k] = s_scr[k * NT + tid];
    } else {
      // more edges than the staging column holds: simulate again, straight
      // to the final positions
      int32_t g2 = r0 / J.NW, w2 = r0 - g2 * J.NW;
      long long o = excl_local;
      for (int m = 0; m < n_mine; ++m) {
        GlobalSink gs{dst + o, room - o};
        int32_t c2, t2;
        uint32_t y2;
        simulate_item(J, S.gate_begin + g2, w2, gs, c2, t2, y2);
        o += c2;
        if (++w2 == J.NW) {
          w2 = 0;
          ++g2;
        }
      }
    }
  }

  // SAIF: the thread's last gate; one atomic per warp when the warp agrees
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

template <int NT, int IPT>
__global__ void __launch_bounds__(NT) propagate_kernel(const __grid_constant__ PropParams p) {
  __shared__ int32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(p.tile_counter, 1);
  __syncthreads();
  propagate_tile<NT, IPT>(p.job, p.seg, s_tile);
}

// Several jobs (each at its own level) in one launch: tiles are taken in
// launch order and mapped to (job, level) segments, each segment with its
// own look-back chain.
template <int NT, int IPT>
__global__ void __launch_bounds__(NT) propagate_multi_kernel(const __grid_constant__ MultiParams m) {
  __shared__ JobView s_job;
  __shared__ SegView s_seg;
  __shared__ int32_t s_tile;
  if (threadIdx.x == 0) {
    const int32_t t = atomicAdd(m.tile_counter, 1);
    int32_t lo = 0, hi = m.n_segs - 1;
    while (lo < hi) {  // last segment with tile_begin <= t
      const int32_t mid = (lo + hi + 1) >> 1;
      if (m.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    s_seg = m.segs[lo].seg;
    s_job = m.jobs[m.segs[lo].job];
    s_tile = t - m.segs[lo].tile_begin;
  }
  __syncthreads();
  propagate_tile<NT, IPT>(s_job, s_seg, s_tile);
}

// Host-side launchers of the two propagation kernels for one compiled
// (threads, items per thread) variant.
struct SingleLaunch {
  const PropParams* p;
  cudaStream_t s;
  template <int NT, int IPT>
  void go() { propagate_kernel<NT, IPT><<<p->seg.n_tiles, NT, 0, s>>>(*p); }
};

struct MultiLaunch {
  const MultiParams* m;
  unsigned grid;
  cudaStream_t s;
  template <int NT, int IPT>
  void go() { propagate_multi_kernel<NT, IPT><<<grid, NT, 0, s>>>(*m); }
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
// edge).
struct InputParams {
  const int64_t* __restrict__ edge_ptr;   // [I*C+1]
  const int32_t* __restrict__ edge_time;
  const uint8_t* __restrict__ init_in;    // [I]
  const long long* __restrict__ in_prefix;  // [I] edges of inputs < i in this batch
  uint8_t* init;
  int32_t* off;
  int32_t* times;
  unsigned long long* saif_t1;
  unsigned long long* saif_tc;
  long long total;  // level-0 edges of the batch
  long long* lvl_base;
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
    q.init[(long long)i * q.NW + w] = (uint8_t)v;
    q.off[(long long)i * q.NW + w] = (int32_t)o;
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
    cnt = (int32_t)(b - a);
  }
  if (r == 0) {
    q.off[(long long)q.I * q.NW] = (int32_t)q.total;  // level-0 end slot
    q.lvl_base[0] = 0;
    q.lvl_base[1] = q.total;
  }
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
__global__ void window_counts_kernel(int32_t N, int32_t NW, int32_t w, const int32_t* net_level,
                                     const int32_t* off, const uint8_t* init, int32_t* cnt,
                                     uint8_t* init_out) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const long long it = (long long)n * NW + w + net_level[n];
  cnt[n] = off[it + 1] - off[it];
  init_out[n] = init[(long long)n * NW + w];
}

__global__ void window_gather_kernel(int32_t N, int32_t NW, int32_t w, const int32_t* net_level,
                                     const int32_t* off, const long long* lvl_base,
                                     const int32_t* times, const long long* dst_ptr,
                                     int32_t* out) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int32_t lv = net_level[n];
  const long long it = (long long)n * NW + w + lv;
  const int32_t s = off[it], e = off[it + 1];
  const int32_t* src = times + lvl_base[lv] + s;
  long long d = dst_ptr[n];
  for (int32_t k = 0; k < e - s; ++k) out[d + k] = src[k];
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
