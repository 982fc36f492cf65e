// Stimulus ingest on the device: a raw list of input toggles, (input,
// absolute ps) in any order, as a waveform dump gives them, restructured
// into the per-(input, cycle) layout the re-simulator reads -- each cycle's
// toggles of each input in time order, relative to the cycle start.  The
// paper does this restructuring before the simulation kernels and counts it
// in the application time (Sections 3 and 4).
//
// Steps (all device work, bucket b = input * C + cycle):
//   1. bucket_kernel   validates every event and counts it into its bucket;
//   2. scan_*          exclusive scan of the bucket counts -> edge_ptr;
//   3. scatter_kernel  places every event in its bucket (arbitrary order);
//   4. order_kernel    sorts each bucket's times (insertion sort: buckets
//                      hold a handful of toggles) and checks they differ.
#pragma once

#include <cstdint>

namespace gatspi_dev {
namespace {

constexpr int kIngBadInput = 1;  // input id out of range
constexpr int kIngBadTime = 2;   // time outside [0, C*L)
constexpr int kIngTwice = 4;     // an input toggles twice at the same ps

struct IngestParams {
  const int32_t* __restrict__ ev_input;
  const int64_t* __restrict__ ev_time;
  long long n;  // events
  int32_t I, C, L;
  int32_t* counts;   // [I*C] bucket counts, then fill cursors
  int64_t* edge_ptr; // [I*C+1]
  int32_t* edge_time;
  int32_t* status;
};

__global__ void ingest_bucket_kernel(IngestParams q) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= q.n) return;
  const int32_t i = q.ev_input[e];
  const int64_t t = q.ev_time[e];
  if (i < 0 || i >= q.I) {
    atomicOr(q.status, kIngBadInput);
    return;
  }
  if (t < 0 || t >= (int64_t)q.C * q.L) {
    atomicOr(q.status, kIngBadTime);
    return;
  }
  atomicAdd(q.counts + (long long)i * q.C + (int32_t)(t / q.L), 1);
}

// Exclusive scan of n int32 counts into out[0..n] (int64, out[n] = total),
// in three launches: per-block totals, a scan of those totals by one block,
// and per-block scans offset by them.  kScanItems counts per block.
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanItems = kScanThreads * kScanPer;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long& total) {
  // warp scan, then a scan of the warp totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < kScanThreads / 32 ? sh[lane] : 0;
    long long wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += u;
    }
    if (lane < kScanThreads / 32) sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const long long r = sh[wid] + incl - v;
  total = sh[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_totals_kernel(const int32_t* __restrict__ in, long long n,
                                                                   long long* block_tot) {
  __shared__ long long sh[33];
  const long long b0 = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * kScanPer;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (b0 + k < n) s += in[b0 + k];
  long long tot;
  block_exclusive_scan(s, sh, tot);
  if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

// One block scans all block totals in place (exclusive), looping over them.
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(long long* block_tot, long long nb) {
  __shared__ long long sh[33];
  long long carry = 0;
  for (long long base = 0; base < nb; base += kScanThreads) {
    const long long j = base + threadIdx.x;
    const long long v = j < nb ? block_tot[j] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, sh, tot);
    if (j < nb) block_tot[j] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int32_t* __restrict__ in, long long n,
                                                                  const long long* __restrict__ block_off,
                                                                  int64_t* out) {
  __shared__ long long sh[33];
  const long long b0 = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * kScanPer;
  int32_t v[kScanPer];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = b0 + k < n ? in[b0 + k] : 0;
    s += v[k];
  }
  long long tot;
  long long o = block_off[blockIdx.x] + block_exclusive_scan(s, sh, tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (b0 + k < n) out[b0 + k] = o;
    o += v[k];
  }
  if (b0 <= n - 1 && n - 1 < b0 + kScanPer) out[n] = o;  // the thread holding the last count
}

__global__ void ingest_scatter_kernel(IngestParams q) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= q.n) return;
  const int32_t i = q.ev_input[e];
  const int64_t t = q.ev_time[e];
  if (i < 0 || i >= q.I || t < 0 || t >= (int64_t)q.C * q.L) return;
  const int32_t c = (int32_t)(t / q.L);
  const long long b = (long long)i * q.C + c;
  const int32_t k = atomicAdd(q.counts + b, 1);  // cursors start at 0
  q.edge_time[q.edge_ptr[b] + k] = (int32_t)(t - (int64_t)c * q.L);
}

__global__ void ingest_order_kernel(IngestParams q) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (long long)q.I * q.C) return;
  const int64_t s = q.edge_ptr[b], e = q.edge_ptr[b + 1];
  int32_t* a = q.edge_time;
  for (int64_t j = s + 1; j < e; ++j) {
    const int32_t x = a[j];
    int64_t k = j - 1;
    while (k >= s && a[k] > x) {
      a[k + 1] = a[k];
      --k;
    }
    a[k + 1] = x;
  }
  for (int64_t j = s + 1; j < e; ++j)
    if (a[j] == a[j - 1]) {
      atomicOr(q.status, kIngTwice);
      break;
    }
}

// Checks of a per-cycle stimulus on the device (gatspi_set_stimulus): every
// (input, cycle) slot's edge range lies inside the edge list and does not go
// back, and its times lie in [0, L) and increase strictly.  The first bad
// slot is kept (atomicMin) for the error message.
constexpr int kStimOrder = 8;      // edge_ptr goes back or leaves [0, total]
constexpr int kStimRange = 16;     // a time outside [0, L)
constexpr int kStimIncrease = 32;  // times not strictly increasing in a slot

__global__ void stimulus_check_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ t,
                                      long long nslots, long long total, int32_t L, int32_t* status,
                                      unsigned long long* first_bad) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nslots) return;
  const int64_t a = ptr[k], b = ptr[k + 1];
  int bad = 0;
  if (b < a || a < 0 || b > total) {
    bad = kStimOrder;
  } else {
    int32_t prev = -1;
    for (int64_t e = a; e < b; ++e) {
      const int32_t x = t[e];
      if (x < 0 || x >= L) {
        bad = kStimRange;
        break;
      }
      if (x <= prev) {
        bad = kStimIncrease;
        break;
      }
      prev = x;
    }
  }
  if (bad) {
    atomicOr(status, bad);
    atomicMin(first_bad, (unsigned long long)k);
  }
}

// Edges of each input before cycle c0 and before cycle c1 (the bounds of a
// batch of windows), for the host's batch planning.
__global__ void stimulus_bounds_kernel(int32_t I, int32_t C, int32_t c0, int32_t c1,
                                       const int64_t* __restrict__ ptr, long long* out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  out[2 * i] = ptr[(long long)i * C + c0];
  out[2 * i + 1] = ptr[(long long)i * C + c1];
}

}  // namespace
}  // namespace gatspi_dev
