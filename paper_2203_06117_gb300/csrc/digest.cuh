// Waveform digest kernel of the re-simulator (the check of bit-exactness
// at scale; see gatspi_digest in gatspi.h).  It reads the waveform store the
// propagation kernels in kernels.cuh write.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace gatspi_dev {
namespace {

// Waveform digest (check of bit-exactness at scale): for every (net,
// window) of the batch, a SplitMix64-chained hash of (start value, edge
// times), mixed with the global window index and summed per net (mod 2^64,
// so the order of the sum does not matter).  One warp per (net, tile of
// TW windows); with gate-aligned tiles the window starts come from the tile
// run and a warp scan of the counts, else from the record starts.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct DigestParams {
  const uint16_t* rmeta;
  const int2* tinfo;      // gate-aligned tiling, or null
  const int32_t* rstart;  // linear tiling, or null
  const int32_t* net_level;
  const long long* lvl_base;
  const int32_t* times;
  long long capacity;
  unsigned long long* out;  // [N] internal net order, added to
  int32_t* status;
  int32_t N, NW, w0, TW, T;  // TW, T: windows per tile and tiles per net
};

__global__ void digest_kernel(const DigestParams q) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)q.N * q.T) return;
  const int32_t n = (int32_t)(wid / q.T), t = (int32_t)(wid - (long long)n * q.T);
  const long long base = q.lvl_base[q.net_level[n]];
  const int32_t wb = t * q.TW;
  const int32_t nwin = min(q.TW, q.NW - wb);
  const long long rec0 = (long long)n * q.NW + wb;
  long long run = q.tinfo ? q.tinfo[(long long)n * q.T + t].x : 0;
  unsigned long long acc = 0;
  for (int32_t k0 = 0; k0 < nwin; k0 += 32) {
    const int32_t j = k0 + lane;
    const bool valid = j < nwin;
    const uint32_t m = valid ? q.rmeta[rec0 + j] : 0u;
    const int32_t c = (int32_t)(m & (uint32_t)kMaxCount);
    int32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    const long long start = q.tinfo ? run + incl - c : (valid ? q.rstart[rec0 + j] : 0);
    run += __shfl_sync(0xffffffffu, incl, 31);
    if (valid) {
      unsigned long long h = mix64((unsigned long long)(m >> 15) + 1ull);
      if (start >= 0 && base + start + c <= q.capacity) {
        const int32_t* tp = q.times + base + start;
        for (int32_t e = 0; e < c; ++e) h = mix64(h + 0x9E3779B97F4A7C15ull + (uint32_t)tp[e]);
      } else {
        atomicOr(q.status, kStCorrupt);
      }
      acc += mix64(h ^ mix64((unsigned long long)(q.w0 + wb + j) + 1ull));
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane == 0) atomicAdd(q.out + n, acc);
}

}  // namespace
}  // namespace gatspi_dev
