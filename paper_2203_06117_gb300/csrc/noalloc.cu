// Level propagation into caller-owned buffers without any device allocation
// (gatspi_propagate_level_noalloc in include/gatspi.h).
//
// Some callers cannot call cudaMalloc: code whose device memory is handed
// out by a framework or a pool it does not own, code that must not
// synchronize the device (cudaMalloc and cudaFree may), or code that has
// reserved all memory up front and must not fail for lack of it mid-run.
// They allocate the netlist, delay and waveform buffers themselves and pass
// them in.  The only memory the propagation kernel needs beyond those
// buffers -- the level's counter (edges allocated, tiles done) and the
// launch's tile counter -- lives in a fixed array in this file, so this entry point never
// allocates.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>

#include "gatspi.h"
#include "kernels.cuh"

using namespace gatspi_dev;

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItemsPerThread = 4;
constexpr int kMaxDevices = 64;
constexpr int kScratchWords = 32;

}  // namespace

// Word 0: the level's counter (edges allocated, tiles done); word 1: the
// launch's tile counter; the rest is unused.  Shared by every call on a
// device; each call clears it before its kernel runs.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

namespace {

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the array's name only stands in for the device symbol, so the
// address must come from cudaGetSymbolAddress with the device current.
std::atomic<int> g_state[kMaxDevices];  // 0 = unknown, 1 = busy, 2 = ready
unsigned long long* g_addr[kMaxDevices];

int scratch_address(int device, unsigned long long** out) {
  if (device < 0 || device >= kMaxDevices) return GATSPI_EINVAL;
  for (;;) {
    int s = g_state[device].load(std::memory_order_acquire);
    if (s == 2) {
      *out = g_addr[device];
      return GATSPI_OK;
    }
    if (s == 0 && g_state[device].compare_exchange_strong(s, 1)) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        g_state[device].store(0, std::memory_order_release);
        return GATSPI_ECUDA;
      }
      g_addr[device] = (unsigned long long*)p;
      g_state[device].store(2, std::memory_order_release);
      *out = g_addr[device];
      return GATSPI_OK;
    }
  }
}

int say(const gatspi_level_args* a, int code, const char* msg) {
  if (a && a->err && a->err_len > 0) std::snprintf(a->err, (size_t)a->err_len, "%s", msg);
  return code;
}

}  // namespace

extern "C" int gatspi_propagate_level_noalloc(const gatspi_level_args* a, void* stream) {
  if (!a) return GATSPI_EINVAL;
  if (a->err && a->err_len > 0) a->err[0] = 0;
  if (!a->fanin_ptr || !a->fanin_net || !a->lut || !a->gate_delay || !a->wire_delay || !a->net_level ||
      !a->rmeta || !a->times || !a->lvl_base || !a->saif_t1 || !a->saif_tc || !a->status)
    return say(a, GATSPI_EINVAL, "a device pointer is null");
  if (a->num_inputs < 1 || a->level < 1 || a->gate_begin < 0 || a->gate_end <= a->gate_begin ||
      a->num_windows < 1 || a->first_window < 0 || a->window_cycles < 1 || a->num_cycles < 1 ||
      a->cycle_ps < 1 || a->capacity < 0)
    return say(a, GATSPI_EINVAL, "bad level, gate range, window or cycle argument");
  // the windows must exist, and every window-relative time must stay below
  // 2^31 (the caller keeps the window length plus the longest path delay
  // below that; the window length alone is checked here)
  const long long n_all = ((long long)a->num_cycles + a->window_cycles - 1) / a->window_cycles;
  if ((long long)a->first_window + a->num_windows > n_all)
    return say(a, GATSPI_EINVAL, "first_window + num_windows exceeds the stimulus' windows");
  if ((long long)a->window_cycles * a->cycle_ps >= 0x80000000ll)
    return say(a, GATSPI_EINVAL, "window_cycles * cycle_ps must stay below 2^31 ps");
  const long long items = (long long)(a->gate_end - a->gate_begin) * a->num_windows;
  if (items > GATSPI_NOALLOC_MAX_ITEMS)
    return say(a, GATSPI_ECAPACITY,
               "level too large: more than GATSPI_NOALLOC_MAX_ITEMS (gate, window) items; "
               "use fewer windows per call");
  const long long tiles = level_tiles(a->gate_end - a->gate_begin, a->num_windows, kNoAllocItemsPerThread);
  const bool wide = wide_tiling(a->num_windows, kNoAllocItemsPerThread);
  if (wide && ((uintptr_t)a->tile_info & 7u))
    return say(a, GATSPI_EINVAL, "tile_info must be 8-byte aligned");
  if (wide ? !a->tile_info : !a->rstart)
    return say(a, GATSPI_EINVAL, wide ? "tile_info is null (needed with 64 or more windows)"
                                      : "rstart is null (needed with fewer than 64 windows)");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return say(a, GATSPI_ECUDA, "cudaGetDevice failed");
  unsigned long long* scratch = nullptr;
  int rc = scratch_address(device, &scratch);
  if (rc) return say(a, rc, "cudaGetSymbolAddress of the counter scratch failed");
  cudaStream_t s = (cudaStream_t)stream;
  // the level's counters and the tile counter must start at 0
  if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * kScratchWords, s) != cudaSuccess)
    return say(a, GATSPI_ECUDA, "clearing the counter scratch failed");
  PropParams p{};
  JobView& j = p.job;
  j.fanin_ptr = a->fanin_ptr; j.fanin_net = a->fanin_net; j.lut = a->lut;
  j.gate_delay = a->gate_delay; j.wire_delay = a->wire_delay; j.net_level = a->net_level;
  j.gate_delta = nullptr;
  j.rstart = wide ? nullptr : a->rstart;
  j.tinfo = wide ? (int2*)a->tile_info : nullptr;
  j.T = wide ? (a->num_windows + tile_items_of(kNoAllocItemsPerThread) - 1) / tile_items_of(kNoAllocItemsPerThread) : 0;
  j.rmeta = a->rmeta; j.times = a->times; j.lvl_base = (long long*)a->lvl_base;
  j.capacity = a->capacity;
  j.saif_t1 = (unsigned long long*)a->saif_t1; j.saif_tc = (unsigned long long*)a->saif_tc;
  j.status = a->status;
  j.I = a->num_inputs; j.NW = a->num_windows; j.w0 = a->first_window; j.W = a->window_cycles;
  j.C = a->num_cycles; j.L = a->cycle_ps;
  p.seg.counters = scratch;
  p.seg.level = a->level;
  p.seg.gate_begin = a->gate_begin;
  p.seg.n_items = (int32_t)items;
  p.seg.n_tiles = (int32_t)tiles;
  p.n_tiles = p.seg.n_tiles;
  p.tile_counter = (int32_t*)(scratch + 1);
  SingleLaunch go{&p, s};
  go.go<kNoAllocThreads, kNoAllocItemsPerThread>();
  if (go.err != cudaSuccess)
    return say(a, GATSPI_ECUDA, "enabling the propagation kernel's shared memory on this device failed");
  if (cudaGetLastError() != cudaSuccess) return say(a, GATSPI_ECUDA, "kernel launch failed");
  return GATSPI_OK;
}
