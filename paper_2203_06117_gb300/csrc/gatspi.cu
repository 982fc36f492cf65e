// Host side of the C interface declared in include/gatspi.h: validation,
// levelization, device memory, the level-by-level launch loop over batches
// of windows, SAIF and waveform read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <exception>
#include <new>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gatspi.h"
#include "host_common.h"
#include "kernels.cuh"
#include "digest.cuh"
#include "ingest.cuh"

using namespace gatspi_dev;

namespace {

constexpr int64_t kAlign = 256;

// An NVTX range over a host scope (visible in Nsight Systems / Compute
// timelines; costs nothing when no tool is attached).
struct nvtx_range {
  explicit nvtx_range(const char* name) { nvtxRangePushA(name); }
  ~nvtx_range() { nvtxRangePop(); }
  nvtx_range(const nvtx_range&) = delete;
  nvtx_range& operator=(const nvtx_range&) = delete;
};

int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

struct gatspi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  size_t arena_limit = 0;

  // netlist in internal order (inputs, then gates sorted by level)
  int32_t I = 0, G = 0, N = 0, P = 0, D = 0;
  std::vector<int32_t> gate_ext;   // internal gate -> caller gate
  std::vector<int32_t> net_int;    // caller net -> internal net
  std::vector<int32_t> pin_ext;    // internal pin -> caller pin
  std::vector<int32_t> fanin_ptr, fanin_net, net_level;
  std::vector<uint16_t> lut;
  std::vector<int32_t> lvl_gate_begin;  // [D+2]: gates of level l (l >= 1) are
                                        // lvl_gate_begin[l] .. lvl_gate_begin[l+1]
  std::vector<int32_t> lvl_split;       // [D+2]: the level's gates of at most two
                                        // pins are lvl_gate_begin[l] .. lvl_split[l]
  std::vector<int64_t> fanout;          // pins driven by each internal net
  int32_t max_gate_delay = 0, max_wire_delay = 0;
  bool have_netlist = false, have_delays = false, have_stim = false, have_result = false;

  int32_t* d_fanin_ptr = nullptr;
  int32_t* d_fanin_net = nullptr;
  int32_t* d_net_level = nullptr;
  int32_t* d_gate_desc = nullptr;
  uint16_t* d_lut = nullptr;
  int32_t* d_gate_delay = nullptr;
  int32_t* d_gate_delay_avg = nullptr;  // partial-SDF table (GATSPI_PARTIAL_SDF)
  int32_t* d_wire_delay = nullptr;
  int32_t* d_gate_delta = nullptr;  // delay edit per internal gate, or null
  int32_t max_edit = 0;

  // stimulus (on the device only; the host reads back the few bounds a
  // batch needs)
  int32_t C = 0, L = 0;
  int64_t* d_edge_ptr = nullptr;
  int32_t* d_edge_time = nullptr;
  uint8_t* d_init_in = nullptr;
  size_t cap_edge_ptr = 0, cap_edge_time = 0, cap_init_in = 0;  // elements the buffers hold
  std::vector<uint8_t> init_in;

  // SAIF and status
  unsigned long long* d_t1 = nullptr;
  unsigned long long* d_tc = nullptr;
  unsigned long long* d_digest = nullptr;  // [N] waveform digests (opts.digest)
  bool have_digest = false;
  int32_t* d_status = nullptr;
  // pinned host words the batch's copies use (so a batch can be captured
  // into a CUDA graph): input prefixes, then status and the level end
  long long* h_in_prefix = nullptr;
  long long* h_ret = nullptr;  // [0] status, [1] edges of the batch
  long long* h_bounds = nullptr;  // [2I] edges of each input before a batch's first and end cycle
  long long* d_bounds = nullptr;
  unsigned long long* d_first_bad = nullptr;  // stimulus check: first bad slot
  // the last batch captured into a graph, replayed while nothing it bakes
  // in changes (shape, stimulus, buffers)
  cudaGraphExec_t gexec = nullptr;
  std::vector<long long> gkey;
  int64_t generation = 0;      // bumped by every load/edit/stimulus call
  int eager_nt = 0, eager_ipt = 0;  // a launch shape already run eagerly
  bool eager_pp = false;             // ... and whether with pulse limits
  int eager_feat = 0;                // ... and the features left out
  long long* d_in_prefix = nullptr;
  int64_t total_time = 0;

  // arena, carved per batch
  char* d_arena = nullptr;
  size_t arena_bytes = 0;
  int64_t times_cap_hint = 0;
  int32_t* d_rstart = nullptr;  // linear tiling
  int2* d_tinfo = nullptr;      // gate-aligned tiling
  int32_t batch_T = 0, batch_TW = 0;
  uint16_t* d_rmeta = nullptr;
  unsigned long long* d_counters = nullptr;  // per level: packed tiles done / edges allocated
  int32_t* d_tile_counter = nullptr;
  long long* d_lvl_base = nullptr;
  int32_t* d_times = nullptr;
  int64_t times_cap = 0;
  size_t scratch_bytes = 0;  // counters (zeroed per batch)

  // incremental re-simulation after a delay edit (gatspi_resimulate_edit)
  gatspi_opts last_opts{};         // options of the last gatspi_simulate, launch shape resolved
  bool have_last_opts = false;
  int64_t result_gen = -1;         // generation the resident result belongs to
  bool result_single = false;      // the result is one resident batch with gate-aligned tiles
  int64_t append_ptr = 0;          // first element of times past every stored run
  std::vector<int32_t> delta;      // delay edit per internal gate (empty: none)
  std::vector<int32_t> fo_ptr, fo_gate;  // fanout gates per internal net (built on first use)
  int32_t* d_cone = nullptr;       // cone gate lists, level after level
  long long* d_append = nullptr;   // two words: where a cone launch starts / the next one starts

  // last simulation
  int32_t W = 1, batch_w0 = 0, batch_nw = 0, n_windows = 0, tile = 256;
  int32_t window_limit = 0;          // >0: simulate only the first windows (autotuning)
  int32_t tuned_nt = 0, tuned_ipt = 0;  // autotuned launch shape for this netlist
  gatspi_stats stats{};
  std::vector<cudaEvent_t> ev;
};

namespace {

int fail(gatspi_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

std::string smem_message(int device, cudaError_t e) {
  return "enabling the propagation kernel's shared memory on device " + std::to_string(device) +
         " failed: " + cudaGetErrorString(e);
}

// Entry points run their bodies through this: a C++ exception (a host
// allocation sized by the caller's input, a string operation) must not
// cross the C interface; it becomes a status and a message instead.
template <class F>
int guarded(gatspi_ctx* c, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(c, GATSPI_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, GATSPI_EINVAL, std::string("unexpected error: ") + e.what());
  } catch (...) {
    return fail(c, GATSPI_EINVAL, "unexpected error");
  }
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, GATSPI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Host arrays go to the device on the context's stream, so that every
// later kernel on that stream sees them; a copy from pageable memory is
// staged before the call returns, so the caller may reuse its array.
template <class T>
int upload(gatspi_ctx* ctx, T*& dst, const T* src, size_t n) {
  dfree(dst);
  CK(cudaMalloc(&dst, std::max<size_t>(n, 1) * sizeof(T)));
  if (src && n) CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return GATSPI_OK;
}

void free_netlist(gatspi_ctx* c) {
  dfree(c->d_gate_delta);
  c->max_edit = 0;
  c->delta.clear();
  c->fo_ptr.clear();
  c->fo_gate.clear();
  dfree(c->d_cone);
  dfree(c->d_fanin_ptr); dfree(c->d_fanin_net); dfree(c->d_net_level); dfree(c->d_lut);
  dfree(c->d_gate_desc);
  dfree(c->d_gate_delay); dfree(c->d_gate_delay_avg); dfree(c->d_wire_delay); dfree(c->d_t1); dfree(c->d_tc); dfree(c->d_digest);
  c->have_digest = false;
  dfree(c->d_in_prefix);
  dfree(c->d_bounds);
}

void free_stim(gatspi_ctx* c) {
  dfree(c->d_edge_ptr); dfree(c->d_edge_time); dfree(c->d_init_in);
  c->cap_edge_ptr = c->cap_edge_time = c->cap_init_in = 0;
}

// Copy n elements to a device buffer, reallocating only when it is too small.
template <class T>
int upload_reuse(gatspi_ctx* ctx, T*& dst, size_t& cap, const T* src, size_t n) {
  if (!dst || cap < std::max<size_t>(n, 1)) {
    dfree(dst);
    cap = 0;
    CK(cudaMalloc(&dst, std::max<size_t>(n, 1) * sizeof(T)));
    cap = std::max<size_t>(n, 1);
  }
  if (src && n) CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return GATSPI_OK;
}

void free_arena(gatspi_ctx* c) {
  dfree(c->d_arena);
  c->arena_bytes = 0;
}

// Carve the arena for a batch of NW windows; returns false if it does not fit.
bool plan_batch(gatspi_ctx* c, int32_t NW, int ipt, size_t* need_fixed) {
  const int64_t N = c->N;
  const bool wide = wide_tiling(NW, ipt);
  const int32_t TW = tile_items_of(ipt);
  const int32_t T = wide ? (NW + TW - 1) / TW : 0;
  int64_t off = 0;
  const int64_t o_start = off; off = align_up(off + (wide ? N * T * 8 : N * NW * 4));
  const int64_t o_meta = off; off = align_up(off + N * NW * 2);
  const int64_t o_lvl = off; off = align_up(off + (c->D + 2) * 8);
  const int64_t o_scr = off;
  const int64_t o_cnt = align_up(o_scr + (int64_t)(c->D + 2) * 8);
  off = align_up(o_cnt + 2 * (c->D + 2) * 4);  // two launches' tile counters per level
  c->scratch_bytes = (size_t)(off - o_scr);
  const int64_t o_times = off;
  *need_fixed = (size_t)o_times;
  if ((size_t)o_times + 1024 * 4 > c->arena_bytes) return false;
  char* a = c->d_arena;
  c->d_rstart = wide ? nullptr : (int32_t*)(a + o_start);
  c->d_tinfo = wide ? (int2*)(a + o_start) : nullptr;
  c->batch_T = T;
  c->batch_TW = wide ? TW : 0;
  c->d_rmeta = (uint16_t*)(a + o_meta);
  c->d_lvl_base = (long long*)(a + o_lvl);
  c->d_counters = (unsigned long long*)(a + o_scr);
  c->d_tile_counter = (int32_t*)(a + o_cnt);
  c->d_times = (int32_t*)(a + o_times);
  c->times_cap = (int64_t)((c->arena_bytes - (size_t)o_times) / 4);
  return true;
}

int ensure_arena(gatspi_ctx* ctx, size_t bytes) {
  bytes = std::min(bytes, ctx->arena_limit);
  if (ctx->d_arena && ctx->arena_bytes >= bytes) return GATSPI_OK;
  free_arena(ctx);
  cudaError_t e = cudaMalloc(&ctx->d_arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->d_arena = nullptr;
    return fail(ctx, GATSPI_ENOMEM, std::string("arena allocation of ") + std::to_string(bytes) +
                                        " bytes failed: " + cudaGetErrorString(e));
  }
  ctx->arena_bytes = bytes;
  return GATSPI_OK;
}

// Fixed bytes (everything but edge times) for NW windows.
size_t fixed_bytes(const gatspi_ctx* c, int32_t NW, int ipt) {
  const int64_t N = c->N;
  const int32_t TW = tile_items_of(ipt);
  const int64_t T = (NW + TW - 1) / TW;
  return (size_t)(align_up(wide_tiling(NW, ipt) ? N * T * 8 : N * NW * 4) + align_up(N * NW * 2) + align_up((c->D + 2) * 8) +
                  align_up((int64_t)(c->D + 2) * 8) + align_up(2 * (c->D + 2) * 4) + 4096);
}

// The edit as one delta per internal gate (all zero: empty vector).
int edit_vector(gatspi_ctx* ctx, int32_t n_edits, const int32_t* edit_gate, const int32_t* edit_delta,
                std::vector<int32_t>* out) {
  if (n_edits < 0 || (n_edits > 0 && (!edit_gate || !edit_delta)))
    return fail(ctx, GATSPI_EINVAL, "bad delay edit arrays");
  out->clear();
  if (n_edits == 0) return GATSPI_OK;
  std::vector<int32_t> delta(ctx->G, 0);
  bool any = false;
  for (int32_t k = 0; k < n_edits; ++k) {
    const int32_t g = edit_gate[k];
    if (g < 0 || g >= ctx->G) return fail(ctx, GATSPI_EINVAL, "edit names an unknown gate");
    if (edit_delta[k] < -gatspi_host::kMaxDelay || edit_delta[k] > gatspi_host::kMaxDelay)
      return fail(ctx, GATSPI_EINVAL, "edit delta outside +-2^24 ps");
    delta[ctx->net_int[(size_t)ctx->I + g] - ctx->I] = edit_delta[k];
    any = any || edit_delta[k] != 0;
  }
  if (any) *out = std::move(delta);
  return GATSPI_OK;
}

// Make `delta` the current edit (device copy and host copy).
int apply_edit(gatspi_ctx* ctx, std::vector<int32_t> delta) {
  CK(cudaSetDevice(ctx->device));
  dfree(ctx->d_gate_delta);
  ctx->max_edit = 0;
  ctx->delta.clear();
  if (delta.empty()) return GATSPI_OK;
  int rc;
  if ((rc = upload(ctx, ctx->d_gate_delta, delta.data(), delta.size()))) return rc;
  ctx->max_edit = std::max(0, *std::max_element(delta.begin(), delta.end()));
  ctx->delta = std::move(delta);
  return GATSPI_OK;
}

}  // namespace

extern "C" {

int gatspi_create(gatspi_ctx** out, int device, size_t arena_bytes) {
  return guarded(nullptr, [&]() -> int {
    gatspi_ctx* ctx = nullptr;
    if (!out) return GATSPI_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
      cudaGetLastError();
      return GATSPI_EINVAL;
    }
    ctx = new gatspi_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&ctx->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ret, 2 * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return GATSPI_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    ctx->arena_limit = arena_bytes ? arena_bytes : (size_t)(0.85 * (double)free_b);
    *out = ctx;
    return GATSPI_OK;
  });
}

int gatspi_destroy(gatspi_ctx* ctx) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_netlist(ctx);
    free_stim(ctx);
    free_arena(ctx);
    dfree(ctx->d_status);
    dfree(ctx->d_append);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->h_in_prefix) cudaFreeHost(ctx->h_in_prefix);
    if (ctx->h_bounds) cudaFreeHost(ctx->h_bounds);
    if (ctx->h_ret) cudaFreeHost(ctx->h_ret);
    dfree(ctx->d_first_bad);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return GATSPI_OK;
  });
}

const char* gatspi_last_error(gatspi_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gatspi_load_netlist(gatspi_ctx* ctx, int32_t num_inputs, int32_t num_gates,
                        const int32_t* fanin_ptr, const int32_t* fanin_net, const uint16_t* lut) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    ctx->generation++;
    gatspi_host::Prepared r;
    const std::string why = gatspi_host::prepare_netlist(num_inputs, num_gates, fanin_ptr, fanin_net, lut, &r);
    if (!why.empty()) return fail(ctx, GATSPI_EINVAL, why);
    CK(cudaSetDevice(ctx->device));
    ctx->have_netlist = ctx->have_delays = ctx->have_stim = ctx->have_result = false;
    ctx->tuned_nt = ctx->tuned_ipt = 0;
    free_netlist(ctx);
    ctx->I = r.I; ctx->G = r.G; ctx->N = r.N; ctx->P = r.P; ctx->D = r.D;
    ctx->gate_ext = std::move(r.gate_ext);
    ctx->net_int = std::move(r.net_int);
    ctx->pin_ext = std::move(r.pin_ext);
    ctx->fanin_ptr = std::move(r.fanin_ptr);
    ctx->fanin_net = std::move(r.fanin_net);
    ctx->net_level = std::move(r.net_level);
    ctx->lut = std::move(r.lut);
    ctx->lvl_gate_begin = std::move(r.lvl_gate_begin);
    ctx->lvl_split = std::move(r.lvl_split);
    ctx->fanout = std::move(r.fanout);
    int rc;
    if (!r.gate_desc.empty()) {
      if ((rc = upload(ctx, ctx->d_gate_desc, r.gate_desc.data(), r.gate_desc.size()))) return rc;
    } else {
      dfree(ctx->d_gate_desc);
    }
    if ((rc = upload(ctx, ctx->d_fanin_ptr, ctx->fanin_ptr.data(), ctx->fanin_ptr.size()))) return rc;
    if ((rc = upload(ctx, ctx->d_fanin_net, ctx->fanin_net.data(), ctx->fanin_net.size()))) return rc;
    if ((rc = upload(ctx, ctx->d_net_level, ctx->net_level.data(), ctx->net_level.size()))) return rc;
    if ((rc = upload(ctx, ctx->d_lut, ctx->lut.data(), ctx->lut.size()))) return rc;
    if ((rc = upload<unsigned long long>(ctx, ctx->d_t1, nullptr, ctx->N))) return rc;
    if ((rc = upload<unsigned long long>(ctx, ctx->d_tc, nullptr, ctx->N))) return rc;
    if ((rc = upload<unsigned long long>(ctx, ctx->d_digest, nullptr, ctx->N))) return rc;
    if ((rc = upload<long long>(ctx, ctx->d_in_prefix, nullptr, ctx->I))) return rc;
    if (ctx->h_in_prefix) cudaFreeHost(ctx->h_in_prefix);
    ctx->h_in_prefix = nullptr;
    CK(cudaMallocHost(&ctx->h_in_prefix, sizeof(long long) * std::max<int32_t>(ctx->I, 1)));
    if (ctx->h_bounds) cudaFreeHost(ctx->h_bounds);
    ctx->h_bounds = nullptr;
    CK(cudaMallocHost(&ctx->h_bounds, 2 * sizeof(long long) * std::max<int32_t>(ctx->I, 1)));
    if ((rc = upload<long long>(ctx, ctx->d_bounds, nullptr, 2 * (size_t)ctx->I))) return rc;
    ctx->have_netlist = true;
    return GATSPI_OK;
  });
}

int gatspi_load_delays(gatspi_ctx* ctx, const int32_t* gate_delay, const int32_t* wire_delay) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    ctx->generation++;
    if (!ctx->have_netlist) return fail(ctx, GATSPI_ESTATE, "load a netlist before its delays");
    gatspi_host::Prepared view;  // only the fields prepare_delays reads
    view.G = ctx->G; view.P = ctx->P;
    view.fanin_ptr = ctx->fanin_ptr;
    view.pin_ext = ctx->pin_ext;
    std::vector<int32_t> gd, wd;
    int32_t mg = 0, mw = 0;
    const std::string why = gatspi_host::prepare_delays(view, gate_delay, wire_delay, &gd, &wd, &mg, &mw);
    if (!why.empty()) return fail(ctx, GATSPI_EINVAL, why);
    CK(cudaSetDevice(ctx->device));
    int rc;
    if ((rc = upload(ctx, ctx->d_gate_delay, gd.data(), gd.size()))) return rc;
    if ((rc = upload(ctx, ctx->d_wire_delay, wd.data(), wd.size()))) return rc;
    const std::vector<int32_t> avg = gatspi_host::averaged_delays(ctx->fanin_ptr, ctx->G, gd);
    if ((rc = upload(ctx, ctx->d_gate_delay_avg, avg.data(), avg.size()))) return rc;
    ctx->max_gate_delay = mg;
    ctx->max_wire_delay = mw;
    dfree(ctx->d_gate_delta);
    ctx->max_edit = 0;
    ctx->delta.clear();
    ctx->have_delays = true;
    ctx->have_result = false;
    return GATSPI_OK;
  });
}

int gatspi_set_edit(gatspi_ctx* ctx, int32_t n_edits, const int32_t* edit_gate, const int32_t* edit_delta) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    ctx->generation++;
    if (!ctx->have_delays) return fail(ctx, GATSPI_ESTATE, "load delays before an edit");
    std::vector<int32_t> delta;
    int rc = edit_vector(ctx, n_edits, edit_gate, edit_delta, &delta);
    if (rc) return rc;
    ctx->have_result = false;
    return apply_edit(ctx, std::move(delta));
  });
}

int gatspi_set_stimulus(gatspi_ctx* ctx, int32_t num_cycles, int32_t cycle_ps, const uint8_t* init,
                        const int64_t* edge_ptr, const int32_t* edge_time) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    nvtx_range range("gatspi_set_stimulus");
    ctx->generation++;
    if (!ctx->have_netlist) return fail(ctx, GATSPI_ESTATE, "load a netlist before the stimulus");
    // the arrays' shape on the host; their contents are checked on the device
    if (num_cycles < 1 || cycle_ps < 1) return fail(ctx, GATSPI_EINVAL, "num_cycles and cycle_ps must be >= 1");
    if (!init || !edge_ptr) return fail(ctx, GATSPI_EINVAL, "null stimulus array");
    const int64_t n = (int64_t)ctx->I * num_cycles;
    if (edge_ptr[0] != 0) return fail(ctx, GATSPI_EINVAL, "edge_ptr[0] must be 0");
    const int64_t total = edge_ptr[n];
    if (total < 0) return fail(ctx, GATSPI_EINVAL, "edge_ptr must be non-decreasing");
    if (total > 0 && !edge_time) return fail(ctx, GATSPI_EINVAL, "null edge_time");
    for (int32_t i = 0; i < ctx->I; ++i)
      if (init[i] > 1) return fail(ctx, GATSPI_EINVAL, "initial values must be 0 or 1");
    CK(cudaSetDevice(ctx->device));
    ctx->have_stim = ctx->have_result = false;
    int rc;
    // device buffers are kept and reused while they are large enough
    if ((rc = upload_reuse(ctx, ctx->d_edge_ptr, ctx->cap_edge_ptr, edge_ptr, (size_t)n + 1))) return rc;
    if ((rc = upload_reuse(ctx, ctx->d_edge_time, ctx->cap_edge_time, edge_time, (size_t)total))) return rc;
    if ((rc = upload_reuse(ctx, ctx->d_init_in, ctx->cap_init_in, init, (size_t)ctx->I))) return rc;
    if (!ctx->d_first_bad) CK(cudaMalloc(&ctx->d_first_bad, sizeof(unsigned long long)));
    const unsigned long long none = ~0ull;
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_first_bad, &none, sizeof(none), cudaMemcpyHostToDevice, ctx->stream));
    stimulus_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_edge_ptr, ctx->d_edge_time, n, total, cycle_ps, ctx->d_status, ctx->d_first_bad);
    CK(cudaGetLastError());
    int32_t status = 0;
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&bad, ctx->d_first_bad, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (status) {
      const std::string where = " (input " + std::to_string(bad / (unsigned long long)num_cycles) + " cycle " +
                                std::to_string(bad % (unsigned long long)num_cycles) + ")";
      if (status & kStimOrder) return fail(ctx, GATSPI_EINVAL, "edge_ptr must be non-decreasing" + where);
      if (status & kStimRange) return fail(ctx, GATSPI_EINVAL, "edge time outside [0, cycle_ps)" + where);
      return fail(ctx, GATSPI_EINVAL, "edge times must increase strictly within a cycle" + where);
    }
    ctx->C = num_cycles;
    ctx->L = cycle_ps;
    ctx->init_in.assign(init, init + ctx->I);
    ctx->have_stim = true;
    return GATSPI_OK;
  });
}

int gatspi_set_stimulus_events(gatspi_ctx* ctx, int32_t num_cycles, int32_t cycle_ps, const uint8_t* init,
                               int64_t num_events, const int32_t* ev_input, const int64_t* ev_time) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    nvtx_range range("gatspi_set_stimulus_events");
    ctx->generation++;
    if (!ctx->have_netlist) return fail(ctx, GATSPI_ESTATE, "load a netlist before the stimulus");
    if (num_cycles < 1 || cycle_ps < 1) return fail(ctx, GATSPI_EINVAL, "num_cycles and cycle_ps must be >= 1");
    if (!init || num_events < 0 || (num_events > 0 && (!ev_input || !ev_time)))
      return fail(ctx, GATSPI_EINVAL, "null or negative stimulus arguments");
    for (int32_t i = 0; i < ctx->I; ++i)
      if (init[i] > 1) return fail(ctx, GATSPI_EINVAL, "initial values must be 0 or 1");
    CK(cudaSetDevice(ctx->device));
    ctx->have_stim = ctx->have_result = false;
    const int64_t nb = (int64_t)ctx->I * num_cycles;  // (input, cycle) buckets
    const int64_t n = num_events;
    int32_t* d_in = nullptr;
    int64_t* d_t = nullptr;
    int32_t* d_cnt = nullptr;
    long long* d_blk = nullptr;
    const int64_t nblk = (nb + kScanItems - 1) / kScanItems;
    auto cleanup = [&]() { dfree(d_in); dfree(d_t); dfree(d_cnt); dfree(d_blk); };
    if (cudaMalloc(&d_in, sizeof(int32_t) * std::max<int64_t>(n, 1)) != cudaSuccess ||
        cudaMalloc(&d_t, sizeof(int64_t) * std::max<int64_t>(n, 1)) != cudaSuccess ||
        cudaMalloc(&d_cnt, sizeof(int32_t) * nb) != cudaSuccess ||
        cudaMalloc(&d_blk, sizeof(long long) * std::max<int64_t>(nblk, 1)) != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(ctx, GATSPI_ENOMEM, "stimulus ingest buffers");
    }
    int rc = upload_reuse(ctx, ctx->d_edge_ptr, ctx->cap_edge_ptr, (const int64_t*)nullptr, (size_t)nb + 1);
    if (!rc) rc = upload_reuse(ctx, ctx->d_edge_time, ctx->cap_edge_time, (const int32_t*)nullptr, (size_t)n);
    if (!rc) rc = upload_reuse(ctx, ctx->d_init_in, ctx->cap_init_in, init, (size_t)ctx->I);
    if (rc) {
      cleanup();
      return rc;
    }
    IngestParams q{};
    q.ev_input = d_in; q.ev_time = d_t; q.n = n; q.I = ctx->I; q.C = num_cycles; q.L = cycle_ps;
    q.counts = d_cnt; q.edge_ptr = ctx->d_edge_ptr; q.edge_time = ctx->d_edge_time; q.status = ctx->d_status;
    int32_t status = 0;
    cudaStream_t st = ctx->stream;
    const unsigned eb = (unsigned)std::max<int64_t>(1, (n + 255) / 256);
    const unsigned bb = (unsigned)((nb + 255) / 256);
    cudaError_t e = cudaSuccess;
    do {
      if (n && ((e = cudaMemcpyAsync(d_in, ev_input, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st)) ||
                (e = cudaMemcpyAsync(d_t, ev_time, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st))))
        break;
      if ((e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), st)) ||
          (e = cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * nb, st)))
        break;
      if (n) ingest_bucket_kernel<<<eb, 256, 0, st>>>(q);
      scan_totals_kernel<<<(unsigned)nblk, kScanThreads, 0, st>>>(d_cnt, nb, d_blk);
      scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(d_blk, nblk);
      scan_apply_kernel<<<(unsigned)nblk, kScanThreads, 0, st>>>(d_cnt, nb, d_blk, ctx->d_edge_ptr);
      if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * nb, st))) break;
      if (n) ingest_scatter_kernel<<<eb, 256, 0, st>>>(q);
      ingest_order_kernel<<<bb, 256, 0, st>>>(q);
      if ((e = cudaGetLastError())) break;
      if ((e = cudaMemcpyAsync(&status, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
          (e = cudaStreamSynchronize(st)))
        break;
    } while (0);
    cleanup();
    if (e != cudaSuccess) return fail(ctx, GATSPI_ECUDA, std::string("stimulus ingest: ") + cudaGetErrorString(e));
    if (status & kIngBadInput) return fail(ctx, GATSPI_EINVAL, "an event names an input outside [0, I)");
    if (status & kIngBadTime) return fail(ctx, GATSPI_EINVAL, "an event time lies outside [0, num_cycles * cycle_ps)");
    if (status & kIngTwice) return fail(ctx, GATSPI_EINVAL, "an input toggles twice at the same time");
    ctx->C = num_cycles;
    ctx->L = cycle_ps;
    ctx->init_in.assign(init, init + ctx->I);
    ctx->have_stim = true;
    return GATSPI_OK;
  });
}

}  // extern "C"

namespace {

// The kernels' view of the loaded job and the carved batch.
JobView job_view(const gatspi_ctx* ctx, int32_t nw, int32_t w0, int32_t W, int32_t pulse_g, int32_t pulse_w,
                 int32_t features = 0) {
  JobView job{};
  job.fanin_ptr = ctx->d_fanin_ptr; job.fanin_net = ctx->d_fanin_net; job.lut = ctx->d_lut;
  job.gate_delay = (features & GATSPI_PARTIAL_SDF) ? ctx->d_gate_delay_avg : ctx->d_gate_delay;
  job.wire_delay = ctx->d_wire_delay;
  job.net_level = ctx->d_net_level; job.gate_delta = ctx->d_gate_delta;
  job.gdesc = (const int4*)ctx->d_gate_desc;
  job.rstart = ctx->d_rstart; job.tinfo = ctx->d_tinfo; job.T = ctx->batch_T; job.rmeta = ctx->d_rmeta;
  job.times = ctx->d_times; job.lvl_base = ctx->d_lvl_base;
  job.capacity = ctx->times_cap; job.saif_t1 = ctx->d_t1; job.saif_tc = ctx->d_tc;
  job.status = ctx->d_status;
  job.I = ctx->I; job.NW = nw; job.w0 = w0; job.W = W; job.C = ctx->C; job.L = ctx->L;
  job.pulse_g = pulse_g; job.pulse_w = pulse_w;
  return job;
}

int simulate_impl(gatspi_ctx* ctx, const gatspi_opts* opts) {
  if (!ctx->have_netlist || !ctx->have_delays || !ctx->have_stim)
    return fail(ctx, GATSPI_ESTATE, "load a netlist, its delays and a stimulus first");
  const auto t_start = std::chrono::steady_clock::now();
  CK(cudaSetDevice(ctx->device));
  gatspi_opts o{};
  if (opts) o = *opts;
  const int32_t feat = o.features;
  if (feat < 0 || feat > (GATSPI_NO_INTERCONNECT_FILTER | GATSPI_PARTIAL_SDF))
    return fail(ctx, GATSPI_EINVAL, "features must be a mask of GATSPI_NO_INTERCONNECT_FILTER and GATSPI_PARTIAL_SDF");
  if (o.digest < 0 || o.digest > 1) return fail(ctx, GATSPI_EINVAL, "digest must be 0 or 1");
  if (o.pulse_limits < 0 || o.pulse_limits > 1) return fail(ctx, GATSPI_EINVAL, "pulse_limits must be 0 or 1");
  const int32_t pulse_g = o.pulse_limits ? o.gate_pulse_percent : 100;
  const int32_t pulse_w = o.pulse_limits ? o.wire_pulse_percent : 100;
  if (pulse_g < 0 || pulse_g > 100 || pulse_w < 0 || pulse_w > 100)
    return fail(ctx, GATSPI_EINVAL, "pulse limits must be 0..100 percent");
  // Algorithm 1 as printed unless a limit is below 100 percent
  const bool pp = pulse_g != 100 || pulse_w != 100;
  const int32_t W = o.window_cycles ? o.window_cycles : 1;
  if (W < 1) return fail(ctx, GATSPI_EINVAL, "window_cycles must be >= 1");
  const int nt = o.tile_items ? o.tile_items : 256;
  const int ipt = o.items_per_thread ? o.items_per_thread : 4;
  if ((nt != 128 && nt != 256 && nt != 512) || (ipt != 1 && ipt != 2 && ipt != 4 && ipt != 8) ||
      (nt == 512 && ipt == 8))
    return fail(ctx, GATSPI_EINVAL, "tile_items must be 128, 256 or 512 and items_per_thread 1, 2, 4 or 8 "
                                    "(at most 4 with 512)");
  if (pp && !pulse_variant_compiled(nt, ipt))
    return fail(ctx, GATSPI_EINVAL, "with pulse limits the launch shape must be 256 x 1, 256 x 2, 256 x 4 "
                                    "or 128 x 8 (threads x items_per_thread)");
  if (feat && pp) return fail(ctx, GATSPI_EINVAL, "features need pulse limits of 100 / 100");
  if (feat && !(nt == 256 && (ipt == 1 || ipt == 4)))
    return fail(ctx, GATSPI_EINVAL, "without features the launch shape must be 256 x 4 or 256 x 1");
  const int tile = tile_items_of(ipt);  // items per warp tile
  if (o.batch_windows < 0) return fail(ctx, GATSPI_EINVAL, "batch_windows must be >= 0");
  // every time stays below 2^31: window length plus the longest path
  if (!gatspi_host::horizon_fits(W, ctx->C, ctx->L, ctx->D, ctx->max_gate_delay, ctx->max_wire_delay,
                                 ctx->max_edit))
    return fail(ctx, GATSPI_EINVAL, "window length plus path delays could overflow int32 ps");
  // the segment of windows [wb, we) this call simulates
  const int32_t n_all = (ctx->C + W - 1) / W;
  if (o.first_window < 0 || o.num_windows < 0 || o.first_window >= n_all)
    return fail(ctx, GATSPI_EINVAL, "first_window must lie in [0, " + std::to_string(n_all) +
                                        ") and num_windows must be >= 0");
  const int32_t wb = o.first_window;
  int32_t we = o.num_windows ? (int32_t)std::min<int64_t>(n_all, (int64_t)wb + o.num_windows) : n_all;
  if (ctx->window_limit > 0) we = std::min(we, wb + ctx->window_limit);
  const int32_t n_windows = we - wb;
  int32_t NW = o.batch_windows ? std::min(o.batch_windows, n_windows) : n_windows;
  // per-level item count must fit int32
  int64_t widest = ctx->I;
  for (int32_t l = 1; l <= ctx->D; ++l)
    widest = std::max<int64_t>(widest, ctx->lvl_gate_begin[l + 1] - ctx->lvl_gate_begin[l]);
  while ((int64_t)widest * NW > 0x7fff0000ll && NW > 1) NW = (NW + 1) / 2;

  ctx->W = W;
  ctx->n_windows = n_windows;
  ctx->tile = tile;
  ctx->have_result = false;
  gatspi_stats st{};
  st.levels = ctx->D;
  CK(cudaMemsetAsync(ctx->d_t1, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_tc, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_digest, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
  ctx->have_digest = false;
  const size_t n_ev = (size_t)2 * (ctx->D + 2);
  if (o.time_kernels && ctx->ev.size() < n_ev) {
    for (auto e : ctx->ev) cudaEventDestroy(e);
    ctx->ev.assign(n_ev, nullptr);
    for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
  }
  cudaEvent_t ev_first = o.time_kernels ? ctx->ev[n_ev - 2] : nullptr;
  cudaEvent_t ev_last = o.time_kernels ? ctx->ev[n_ev - 1] : nullptr;
  bool first_recorded = false;

  // size the arena: fixed part + room for edges (grown on overflow)
  auto want_bytes = [&](int32_t nw) {
    const int64_t items = (int64_t)ctx->N * nw;
    int64_t edges = std::max<int64_t>(ctx->times_cap_hint, items * 2 + (1 << 20));
    return fixed_bytes(ctx, nw, ipt) + (size_t)edges * 4;
  };
  while (NW > 1 && fixed_bytes(ctx, NW, ipt) * 2 > ctx->arena_limit) NW = (NW + 1) / 2;

  int32_t w0 = wb;
  int64_t edges_total = 0, rec_bytes = 0;
  while (w0 < we) {
    nvtx_range batch_range("gatspi batch");
    const int32_t nw = std::min(NW, we - w0);
    int rc = ensure_arena(ctx, want_bytes(nw));
    if (rc) return rc;
    size_t fixed = 0;
    if (!plan_batch(ctx, nw, ipt, &fixed)) {
      if (NW == 1) return fail(ctx, GATSPI_ECAPACITY, "arena too small for one window");
      NW = (NW + 1) / 2;
      continue;
    }
    // level 0 from the stimulus: each input's edges in the batch, from the
    // device copy of edge_ptr
    std::vector<long long> in_prefix(ctx->I);
    long long l0 = 0;
    const int32_t c_begin = w0 * W, c_end = std::min((w0 + nw) * W, ctx->C);
    stimulus_bounds_kernel<<<(unsigned)((ctx->I + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->I, ctx->C, c_begin, c_end, ctx->d_edge_ptr, ctx->d_bounds);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_bounds, ctx->d_bounds, 2 * sizeof(long long) * ctx->I, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    st.kernel_launches += 1;
    for (int32_t i = 0; i < ctx->I; ++i) {
      in_prefix[i] = l0;
      l0 += ctx->h_bounds[2 * i + 1] - ctx->h_bounds[2 * i];
    }
    if (l0 > ctx->times_cap || l0 > 0x7fffffffll) {
      if (NW > 1) { NW = (NW + 1) / 2; continue; }
      return fail(ctx, GATSPI_ECAPACITY, "input edges of one window exceed the arena");
    }
    for (int32_t i = 0; i < ctx->I; ++i) ctx->h_in_prefix[i] = in_prefix[i];
    const bool record_first = o.time_kernels && !first_recorded;
    cudaError_t smem_err = cudaSuccess;  // a propagation kernel could not opt in to its shared memory
    // Algorithm 1 as printed or without some features, over gate-aligned
    // tiles: a level's gates of at most two pins run in the pair kernel where
    // it is compiled, when they make enough tiles that a second launch's last
    // partial wave costs less than the pair kernel saves
    const bool split = !pp && ctx->batch_T > 0 && pair_variant_compiled(nt, ipt, feat);
    std::vector<int32_t> pair_gates((size_t)ctx->D + 2, 0);
    int32_t pair_launches = 0, rest_launches = ctx->D;
    if (split) {
      for (int32_t l = 1; l <= ctx->D; ++l) {
        const int32_t np = ctx->lvl_split[l] - ctx->lvl_gate_begin[l];
        if ((int64_t)np * ctx->batch_T < kPairMinTiles) continue;
        pair_gates[l] = np;
        ++pair_launches;
        if (ctx->lvl_split[l] == ctx->lvl_gate_begin[l + 1]) --rest_launches;
      }
    }
    // everything the batch puts on the stream; captured into a CUDA graph
    // and replayed when the same batch comes again (repeated simulations of
    // one stimulus), launched eagerly otherwise.  Timing events are recorded
    // as external events so that a replayed graph still times its kernels.
    auto enqueue = [&](bool capturing) -> cudaError_t {
      cudaError_t e;
      auto rec = [&](cudaEvent_t ev) {
        return capturing ? cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal)
                         : cudaEventRecord(ev, ctx->stream);
      };
      if ((e = cudaMemcpyAsync(ctx->d_in_prefix, ctx->h_in_prefix, sizeof(long long) * ctx->I,
                               cudaMemcpyHostToDevice, ctx->stream)))
        return e;
      if (record_first && (e = rec(ev_first))) return e;
      if ((e = cudaMemsetAsync(ctx->d_counters, 0, ctx->scratch_bytes, ctx->stream))) return e;
      if ((e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream))) return e;
      {
        InputParams q{};
        q.edge_ptr = ctx->d_edge_ptr; q.edge_time = ctx->d_edge_time; q.init_in = ctx->d_init_in;
        q.in_prefix = ctx->d_in_prefix; q.rstart = ctx->d_rstart; q.rmeta = ctx->d_rmeta; q.times = ctx->d_times;
        q.tinfo = ctx->d_tinfo; q.T = ctx->batch_T; q.TW = ctx->batch_TW;
        q.saif_t1 = ctx->d_t1; q.saif_tc = ctx->d_tc; q.total = l0; q.lvl_base = ctx->d_lvl_base;
        q.status = ctx->d_status;
        q.I = ctx->I; q.NW = nw; q.w0 = w0; q.W = W; q.C = ctx->C; q.L = ctx->L;
        q.n_items = ctx->I * nw;
        if (o.time_kernels && (e = rec(ctx->ev[0]))) return e;
        inputs_kernel<<<(q.n_items + 255) / 256, 256, 0, ctx->stream>>>(q);
        if ((e = cudaGetLastError())) return e;
        if (o.time_kernels && (e = rec(ctx->ev[1]))) return e;
      }
      const JobView job = job_view(ctx, nw, w0, W, pulse_g, pulse_w, feat);
      for (int32_t l = 1; l <= ctx->D; ++l) {
        PropParams p{};
        p.job = job;
        p.seg.counters = ctx->d_counters + l;
        p.seg.level = l;
        p.seg.gate_begin = ctx->lvl_gate_begin[l];
        p.seg.n_items = (ctx->lvl_gate_begin[l + 1] - ctx->lvl_gate_begin[l]) * nw;
        p.seg.n_tiles = (int32_t)level_tiles(ctx->lvl_gate_begin[l + 1] - ctx->lvl_gate_begin[l], nw, ipt);
        p.tile_counter = ctx->d_tile_counter + l;
        p.n_tiles = p.seg.n_tiles;
        if (o.time_kernels && (e = rec(ctx->ev[2 * l]))) return e;
        const int32_t n_pair = pair_gates[l];
        if (n_pair > 0) {
          // the level's gates of at most two pins in the pair kernel, the
          // rest after them; both launches count into the level's counter
          PropParams q = p;
          q.n_tiles = n_pair * ctx->batch_T;
          PairLaunch go{&q, ctx->stream};
          if (feat == GATSPI_NO_INTERCONNECT_FILTER) go.go<256, kModeNoWireFilter>();
          else if (feat == GATSPI_PARTIAL_SDF) go.go<256, kModeAvgSdf>();
          else if (feat) go.go<256, kModeNoWireAvgSdf>();
          else if (nt == 128) go.go<128, kModePlain>();
          else go.go<256, kModePlain>();
          if ((e = go.err)) {
            smem_err = e;
            return e;
          }
          if ((e = cudaGetLastError())) return e;
          p.seg.gate_begin = ctx->lvl_split[l];
          p.n_tiles = p.seg.n_tiles - q.n_tiles;
          p.tile_counter = ctx->d_tile_counter + (ctx->D + 2) + l;
        }
        if (p.n_tiles == 0) {
          e = cudaSuccess;  // every gate of the level went to the pair kernel
        } else if (pp) {
          SingleLaunchMode<kModePulse> go{&p, ctx->stream};
          launch_variant_pp(nt, ipt, go);
          e = go.err;
        } else if (feat == GATSPI_NO_INTERCONNECT_FILTER) {
          SingleLaunchMode<kModeNoWireFilter> go{&p, ctx->stream};
          launch_variant_features(ipt, go);
          e = go.err;
        } else if (feat == GATSPI_PARTIAL_SDF) {
          SingleLaunchMode<kModeAvgSdf> go{&p, ctx->stream};
          launch_variant_features(ipt, go);
          e = go.err;
        } else if (feat) {
          SingleLaunchMode<kModeNoWireAvgSdf> go{&p, ctx->stream};
          launch_variant_features(ipt, go);
          e = go.err;
        } else {
          SingleLaunch go{&p, ctx->stream};
          launch_variant(nt, ipt, go);
          e = go.err;
        }
        if (e) {
          smem_err = e;
          return e;
        }
        if ((e = cudaGetLastError())) return e;
        if (o.time_kernels && (e = rec(ctx->ev[2 * l + 1]))) return e;
      }
      if (o.time_kernels && (e = rec(ev_last))) return e;
      if (o.digest) {  // after the timed region: the digest reads every waveform of the batch once
        DigestParams q{};
        q.rmeta = ctx->d_rmeta; q.tinfo = ctx->d_tinfo; q.rstart = ctx->d_rstart;
        q.net_level = ctx->d_net_level; q.lvl_base = ctx->d_lvl_base; q.times = ctx->d_times;
        q.capacity = ctx->times_cap; q.out = ctx->d_digest; q.status = ctx->d_status;
        q.N = ctx->N; q.NW = nw; q.w0 = w0;
        q.TW = ctx->batch_T > 0 ? ctx->batch_TW : 128;
        q.T = (nw + q.TW - 1) / q.TW;
        const long long warps = (long long)q.N * q.T;
        digest_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, ctx->stream>>>(q);
        if ((e = cudaGetLastError())) return e;
      }
      if ((e = cudaMemcpyAsync(&ctx->h_ret[0], ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               ctx->stream)))
        return e;
      return cudaMemcpyAsync(&ctx->h_ret[1], ctx->d_lvl_base + ctx->D + 1, sizeof(long long),
                             cudaMemcpyDeviceToHost, ctx->stream);
    };
    ctx->h_ret[0] = 0;
    // a graph bakes in pointers, sizes and per-batch values: replay it only
    // while all of them are the same
    const std::vector<long long> key = {
        ctx->generation, (long long)(uintptr_t)ctx->d_arena, (long long)ctx->arena_bytes, ctx->times_cap,
        nw, w0, W, nt, ipt, o.digest, o.time_kernels, record_first ? 1 : 0, l0, ctx->batch_T,
        (long long)(uintptr_t)ctx->d_gate_delta, pulse_g, pulse_w, feat};
    bool done = false;
    if (ctx->eager_nt == nt && ctx->eager_ipt == ipt && ctx->eager_pp == pp &&
        ctx->eager_feat == feat) {  // the variant's attributes are set
      if (!(ctx->gexec && ctx->gkey == key)) {
        if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        ctx->gkey.clear();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          const cudaError_t ce = enqueue(true);
          const cudaError_t ee = cudaStreamEndCapture(ctx->stream, &graph);
          if (ce == cudaSuccess && ee == cudaSuccess && graph &&
              cudaGraphInstantiate(&ctx->gexec, graph, 0) == cudaSuccess) {
            ctx->gkey = key;
          } else {
            ctx->gexec = nullptr;
          }
          if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();  // a capture that failed leaves the eager path below
      }
      if (ctx->gexec) {
        CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
        done = true;
      }
    }
    if (!done) {
      const cudaError_t ee = enqueue(false);
      if (ee && smem_err) return fail(ctx, GATSPI_ECUDA, smem_message(ctx->device, smem_err));
      CK(ee);
      ctx->eager_nt = nt;
      ctx->eager_ipt = ipt;
      ctx->eager_pp = pp;
      ctx->eager_feat = feat;
    }
    if (record_first) first_recorded = true;
    st.kernel_launches += 1 + rest_launches + pair_launches + (o.digest ? 1 : 0);
    st.prop_launches += rest_launches + pair_launches;
    st.items += (int64_t)ctx->G * nw;
    CK(cudaStreamSynchronize(ctx->stream));
    const int32_t status = (int32_t)ctx->h_ret[0];
    const long long lvl_end = ctx->h_ret[1];
    if (status & kStTimeout) return fail(ctx, GATSPI_ETIMEOUT, "a device-side wait ran out");
    if (status & (kStCapacity | kStOffset | kStCorrupt)) {
      // undo this batch's SAIF contribution by re-running from scratch
      const bool can_grow = ctx->arena_bytes < ctx->arena_limit;
      if (can_grow && !(status & kStOffset)) {
        ctx->times_cap_hint = std::max<int64_t>(ctx->times_cap_hint, ctx->times_cap) * 2;
      } else if (NW > 1) {
        NW = (NW + 1) / 2;
      } else if (status & kStOffset) {
        return fail(ctx, GATSPI_ECAPACITY,
                    "a net has more than 32767 edges in one window: use fewer cycles per window");
      } else {
        return fail(ctx, GATSPI_ECAPACITY, "waveforms of one window exceed the arena");
      }
      // restart the whole segment: SAIF of earlier batches is kept only
      // if we restart from its first window
      w0 = wb;
      edges_total = 0;
      rec_bytes = 0;
      first_recorded = false;
      st = gatspi_stats{};
      st.levels = ctx->D;
      CK(cudaMemsetAsync(ctx->d_t1, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
      CK(cudaMemsetAsync(ctx->d_tc, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
      CK(cudaMemsetAsync(ctx->d_digest, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
      continue;
    }
    if (o.time_kernels) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, ev_first, ev_last));
      st.device_ms = ms;  // span from the first batch's start to this batch's end
      CK(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
      st.input_ms += ms;
      for (int32_t l = 1; l <= ctx->D; ++l) {
        CK(cudaEventElapsedTime(&ms, ctx->ev[2 * l], ctx->ev[2 * l + 1]));
        st.prop_ms += ms;
      }
    }
    edges_total += lvl_end;
    // record bytes of the batch: a 2-byte meta per record read by every pin
    // and written per gate, plus an 8-byte tile run per (pin or gate, tile)
    // with gate-aligned tiles, or a 4-byte start per record without
    rec_bytes += ctx->batch_T > 0
                     ? ((int64_t)ctx->P + ctx->G) * (2ll * nw + 8ll * ctx->batch_T)
                     : ((int64_t)ctx->P + ctx->G) * 6ll * nw;
    ctx->batch_w0 = w0;
    ctx->batch_nw = nw;
    st.batches++;
    w0 += nw;
  }
  st.windows = n_windows;
  st.batch_windows = NW;
  st.edges = edges_total;
  ctx->total_time = (std::min<int64_t>((int64_t)we * W, ctx->C) - (int64_t)wb * W) * ctx->L;
  // algorithmic bytes: the records' bytes above, plus 4 bytes per edge read
  // by every fanin pin (a pin reads the TC of its driving net) and per edge
  // written by a gate
  {
    std::vector<unsigned long long> tc(ctx->N);
    CK(cudaMemcpy(tc.data(), ctx->d_tc, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost));
    int64_t b = rec_bytes;
    for (int32_t n = 0; n < ctx->N; ++n)
      b += 4ll * (int64_t)tc[n] * (ctx->fanout[n] + (n >= ctx->I ? 1 : 0));
    st.algo_bytes = b;
  }
  st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  st.tile_threads = nt;
  st.items_per_thread = ipt;
  ctx->stats = st;
  ctx->have_result = true;
  ctx->have_digest = o.digest != 0;
  // the last batch stays resident: with one batch it is the whole result,
  // which an edit can then update in place (gatspi_resimulate_edit)
  ctx->result_single = st.batches == 1 && ctx->batch_T > 0 && ctx->window_limit == 0;
  ctx->append_ptr = edges_total;
  ctx->result_gen = ctx->generation;
  return GATSPI_OK;
}

// Pick the launch shape (threads per block x consecutive windows per
// thread) by timing every compiled variant on the first windows of the
// loaded stimulus (about 4*10^8 (gate, window) items, the best of two
// timed runs after a warm-up); cached per netlist.
int autotune(gatspi_ctx* ctx, const gatspi_opts& base) {
  static const int kVariants[][2] = {{256, 1}, {256, 2}, {256, 4}, {256, 8}, {128, 4},
                                     {128, 8}, {512, 1}, {512, 2}, {512, 4}};
  const int32_t W = base.window_cycles ? base.window_cycles : 1;
  const int32_t n_windows = (ctx->C + W - 1) / W;
  const int64_t want = (int64_t)4e8 / std::max<int64_t>(ctx->N, 1);
  ctx->window_limit = (int32_t)std::max<int64_t>(1, std::min<int64_t>(want, n_windows));
  double best = 1e300;
  int bn = 256, bi = 4, rc = GATSPI_OK;
  for (const auto& v : kVariants) {
    gatspi_opts o = base;
    o.tile_items = v[0];
    o.items_per_thread = v[1];
    o.time_kernels = 1;
    double ms = 1e300;
    for (int rep = 0; rep < 3 && rc == GATSPI_OK; ++rep) {
      rc = simulate_impl(ctx, &o);
      if (rep > 0) ms = std::min(ms, ctx->stats.prop_ms);  // the first run warms up
    }
    if (rc != GATSPI_OK) break;
    if (ms < best) {
      best = ms;
      bn = v[0];
      bi = v[1];
    }
  }
  ctx->window_limit = 0;
  ctx->have_result = false;
  if (rc != GATSPI_OK) return rc;
  ctx->tuned_nt = bn;
  ctx->tuned_ipt = bi;
  return GATSPI_OK;
}

}  // namespace

extern "C" {

int gatspi_simulate(gatspi_ctx* ctx, const gatspi_opts* opts) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    nvtx_range range("gatspi_simulate");
    if (!ctx->have_netlist || !ctx->have_delays || !ctx->have_stim)
      return fail(ctx, GATSPI_ESTATE, "load a netlist, its delays and a stimulus first");
    gatspi_opts o{};
    if (opts) o = *opts;
    const bool pp = o.pulse_limits == 1 && (o.gate_pulse_percent != 100 || o.wire_pulse_percent != 100);
    if (o.tile_items == 0 && o.items_per_thread == 0 && !pp && !o.features) {
      if (!ctx->tuned_nt) {
        const int rc = autotune(ctx, o);
        if (rc) return rc;
      }
      o.tile_items = ctx->tuned_nt;
      o.items_per_thread = ctx->tuned_ipt;
    }
    const int rc = simulate_impl(ctx, &o);
    if (rc == GATSPI_OK) {
      ctx->have_last_opts = true;
      ctx->last_opts = o;
      ctx->last_opts.tile_items = ctx->stats.tile_threads;
      ctx->last_opts.items_per_thread = ctx->stats.items_per_thread;
    }
    return rc;
  });
}

int gatspi_resimulate_edit(gatspi_ctx* ctx, int32_t n_edits, const int32_t* edit_gate,
                           const int32_t* edit_delta, gatspi_resim_info* info) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    nvtx_range range("gatspi_resimulate_edit");
    if (!ctx->have_last_opts) return fail(ctx, GATSPI_ESTATE, "simulate once before re-simulating an edit");
    if (!ctx->have_netlist || !ctx->have_delays || !ctx->have_stim)
      return fail(ctx, GATSPI_ESTATE, "load a netlist, its delays and a stimulus first");
    std::vector<int32_t> nd;
    int rc = edit_vector(ctx, n_edits, edit_gate, edit_delta, &nd);
    if (rc) return rc;
    gatspi_resim_info r{};
    const auto t_start = std::chrono::steady_clock::now();
    const bool resident = ctx->have_result && ctx->result_single && ctx->result_gen == ctx->generation;
    const bool current = ctx->have_result;  // the results match the loaded inputs and edit
    // gates whose delays change: the cone's roots
    std::vector<uint8_t> in_cone(ctx->G, 0);
    int32_t roots = 0;
    for (int32_t g = 0; g < ctx->G; ++g) {
      const int32_t a = ctx->delta.empty() ? 0 : ctx->delta[g];
      const int32_t b = nd.empty() ? 0 : nd[g];
      if (a != b) {
        in_cone[g] = 1;
        ++roots;
      }
    }
    ctx->generation++;
    if ((rc = apply_edit(ctx, std::move(nd)))) {
      ctx->have_result = false;
      return rc;
    }
    const gatspi_opts o = ctx->last_opts;
    auto full = [&]() {
      r.mode = 2;
      const int e = simulate_impl(ctx, &o);
      r.cone_gates = ctx->G;
      r.first_level = 1;
      r.levels = ctx->D;
      r.items = (int64_t)ctx->G * ctx->n_windows;
      if (info) *info = r;
      return e;
    };
    if (roots == 0 && current) {  // nothing changes: the results stand
      if (resident) ctx->result_gen = ctx->generation;
      if (info) *info = r;
      return GATSPI_OK;
    }
    // the cone launches carry every feature: without some, run it all again
    if (!resident || o.features) return full();
    // the fanout cone of the changed gates, level by level (gates are sorted
    // by level, so one pass in gate order reaches every cone gate after its
    // fanins)
    if (ctx->fo_ptr.empty()) {
      ctx->fo_ptr.assign((size_t)ctx->N + 1, 0);
      for (int32_t p = 0; p < ctx->P; ++p) ctx->fo_ptr[ctx->fanin_net[p] + 1]++;
      for (int32_t n = 0; n < ctx->N; ++n) ctx->fo_ptr[n + 1] += ctx->fo_ptr[n];
      ctx->fo_gate.assign((size_t)ctx->P, 0);
      std::vector<int32_t> fill(ctx->fo_ptr.begin(), ctx->fo_ptr.end() - 1);
      for (int32_t g = 0; g < ctx->G; ++g)
        for (int32_t p = ctx->fanin_ptr[g]; p < ctx->fanin_ptr[g + 1]; ++p) ctx->fo_gate[fill[ctx->fanin_net[p]]++] = g;
    }
    std::vector<int32_t> list;
    std::vector<int32_t> lvl_off((size_t)ctx->D + 2, 0);  // cone gates of level l: list[lvl_off[l] .. lvl_off[l+1])
    for (int32_t l = 1; l <= ctx->D; ++l) {
      lvl_off[l] = (int32_t)list.size();
      for (int32_t g = ctx->lvl_gate_begin[l]; g < ctx->lvl_gate_begin[l + 1]; ++g) {
        if (!in_cone[g]) continue;
        list.push_back(g);
        const int32_t net = ctx->I + g;
        for (int32_t k = ctx->fo_ptr[net]; k < ctx->fo_ptr[net + 1]; ++k) in_cone[ctx->fo_gate[k]] = 1;
      }
    }
    lvl_off[ctx->D + 1] = (int32_t)list.size();
    const int32_t nw = ctx->batch_nw, T = ctx->batch_T;
    // room for the cone's new runs: at least twice the edges the cone's nets
    // hold now, else the whole batch is simulated again (which also compacts)
    std::vector<unsigned long long> tc(ctx->N);
    CK(cudaMemcpy(tc.data(), ctx->d_tc, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost));
    int64_t old_edges = 0;
    for (int32_t g : list) old_edges += (int64_t)tc[(size_t)ctx->I + g];
    if (ctx->append_ptr + 2 * old_edges + (1 << 16) > ctx->times_cap) return full();
    if (!ctx->d_cone) {
      CK(cudaMalloc(&ctx->d_cone, sizeof(int32_t) * std::max<int32_t>(ctx->G, 1)));
    }
    if (!ctx->d_append) CK(cudaMalloc(&ctx->d_append, 2 * sizeof(long long)));
    CK(cudaMemcpy(ctx->d_cone, list.data(), sizeof(int32_t) * list.size(), cudaMemcpyHostToDevice));
    const long long ap = ctx->append_ptr;
    CK(cudaMemcpy(ctx->d_append, &ap, sizeof(long long), cudaMemcpyHostToDevice));
    const int32_t pulse_g = o.pulse_limits ? o.gate_pulse_percent : 100;
    const int32_t pulse_w = o.pulse_limits ? o.wire_pulse_percent : 100;
    const bool pp = pulse_g != 100 || pulse_w != 100;
    const int nt = o.tile_items, ipt = o.items_per_thread;
    if (ctx->ev.size() < 2) {
      for (auto e : ctx->ev) cudaEventDestroy(e);
      ctx->ev.assign(2, nullptr);
      for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
    }
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream));
    CK(cudaEventRecord(e0, ctx->stream));
    clear_saif_kernel<<<(unsigned)((list.size() + 255) / 256), 256, 0, ctx->stream>>>(
        (int32_t)list.size(), ctx->d_cone, ctx->I, ctx->d_t1, ctx->d_tc);
    CK(cudaGetLastError());
    const JobView job = job_view(ctx, nw, ctx->batch_w0, ctx->W, pulse_g, pulse_w);
    int32_t k = 0;
    for (int32_t l = 1; l <= ctx->D; ++l) {
      const int32_t nc = lvl_off[l + 1] - lvl_off[l];
      if (nc == 0) continue;
      if (r.levels == 0) r.first_level = l;
      CK(cudaMemsetAsync(ctx->d_counters + l, 0, sizeof(unsigned long long), ctx->stream));
      CK(cudaMemsetAsync(ctx->d_tile_counter + l, 0, sizeof(int32_t), ctx->stream));
      PropParams p{};
      p.job = job;
      p.seg.counters = ctx->d_counters + l;
      p.seg.level = l;
      p.seg.gate_begin = ctx->lvl_gate_begin[l];
      p.seg.n_items = nc * nw;
      p.seg.n_tiles = nc * T;
      p.n_tiles = p.seg.n_tiles;
      p.seg.gate_list = ctx->d_cone + lvl_off[l];
      p.seg.append_in = ctx->d_append + (k & 1);
      p.seg.append_out = ctx->d_append + ((k + 1) & 1);
      p.tile_counter = ctx->d_tile_counter + l;
      cudaError_t le = cudaSuccess;
      if (pp) {
        SingleLaunchMode<kModePulse> go{&p, ctx->stream};
        launch_variant_pp(nt, ipt, go);
        le = go.err;
      } else {
        SingleLaunchMode<kModeCone> go{&p, ctx->stream};
        launch_variant_cone(ipt, go);
        le = go.err;
      }
      if (le) return fail(ctx, GATSPI_ECUDA, smem_message(ctx->device, le));
      CK(cudaGetLastError());
      ++k;
      ++r.levels;
      r.items += (int64_t)nc * nw;
    }
    CK(cudaEventRecord(e1, ctx->stream));
    if (o.digest) {
      CK(cudaMemsetAsync(ctx->d_digest, 0, sizeof(unsigned long long) * ctx->N, ctx->stream));
      DigestParams q{};
      q.rmeta = ctx->d_rmeta; q.tinfo = ctx->d_tinfo; q.rstart = ctx->d_rstart;
      q.net_level = ctx->d_net_level; q.lvl_base = ctx->d_lvl_base; q.times = ctx->d_times;
      q.capacity = ctx->times_cap; q.out = ctx->d_digest; q.status = ctx->d_status;
      q.N = ctx->N; q.NW = nw; q.w0 = ctx->batch_w0;
      q.TW = ctx->batch_TW;
      q.T = T;
      const long long warps = (long long)q.N * q.T;
      digest_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, ctx->stream>>>(q);
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(&ctx->h_ret[0], ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&ctx->h_ret[1], ctx->d_append + (k & 1), sizeof(long long), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int32_t status = (int32_t)ctx->h_ret[0];
    if (status & kStTimeout) {
      ctx->have_result = false;
      return fail(ctx, GATSPI_ETIMEOUT, "a device-side wait ran out");
    }
    // a cone that outgrew the append region (or int32 run offsets): the whole
    // batch again, from scratch
    if (status & (kStCapacity | kStOffset | kStCorrupt)) return full();
    ctx->append_ptr = ctx->h_ret[1];
    ctx->result_gen = ctx->generation;
    r.mode = 1;
    r.cone_gates = (int32_t)list.size();
    // figures of this call: the cone's launches
    gatspi_stats st = ctx->stats;
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    st.prop_ms = ms;
    st.device_ms = ms;
    st.input_ms = 0;
    st.kernel_launches = 1 + r.levels + (o.digest ? 1 : 0);
    st.prop_launches = r.levels;
    st.items = r.items;
    CK(cudaMemcpy(tc.data(), ctx->d_tc, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost));
    int64_t edges = 0, bytes = 0;
    for (int32_t n = 0; n < ctx->N; ++n) edges += (int64_t)tc[n];
    for (int32_t g : list) {
      const int32_t pins = ctx->fanin_ptr[g + 1] - ctx->fanin_ptr[g];
      bytes += (int64_t)(pins + 1) * (2ll * nw + 8ll * T) + 4ll * (int64_t)tc[(size_t)ctx->I + g];
      for (int32_t p = ctx->fanin_ptr[g]; p < ctx->fanin_ptr[g + 1]; ++p) bytes += 4ll * (int64_t)tc[ctx->fanin_net[p]];
    }
    st.edges = edges;
    st.algo_bytes = bytes;
    st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    ctx->stats = st;
    if (info) *info = r;
    return GATSPI_OK;
  });
}

int gatspi_saif(gatspi_ctx* ctx, int64_t* t0, int64_t* t1, int64_t* tc) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    if (!ctx->have_result) return fail(ctx, GATSPI_ESTATE, "nothing simulated yet");
    CK(cudaSetDevice(ctx->device));
    std::vector<unsigned long long> a(ctx->N), b(ctx->N);
    CK(cudaMemcpyAsync(a.data(), ctx->d_t1, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b.data(), ctx->d_tc, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int32_t e = 0; e < ctx->N; ++e) {
      const int32_t n = ctx->net_int[e];
      if (t1) t1[e] = (int64_t)a[n];
      if (t0) t0[e] = ctx->total_time - (int64_t)a[n];
      if (tc) tc[e] = (int64_t)b[n];
    }
    return GATSPI_OK;
  });
}

int gatspi_digest(gatspi_ctx* ctx, uint64_t* out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx || !out) return GATSPI_EINVAL;
    if (!ctx->have_digest) return fail(ctx, GATSPI_ESTATE, "no digest: simulate with opts.digest = 1 first");
    CK(cudaSetDevice(ctx->device));
    std::vector<unsigned long long> d(ctx->N);
    CK(cudaMemcpy(d.data(), ctx->d_digest, sizeof(unsigned long long) * ctx->N, cudaMemcpyDeviceToHost));
    for (int32_t e = 0; e < ctx->N; ++e) out[e] = d[ctx->net_int[e]];
    return GATSPI_OK;
  });
}

int gatspi_read_window(gatspi_ctx* ctx, int32_t window, uint8_t* init, int64_t* ptr, int32_t* times,
                       int64_t cap, int64_t* total) {
  return guarded(ctx, [&]() -> int {
    if (!ctx) return GATSPI_EINVAL;
    if (!ctx->have_result) return fail(ctx, GATSPI_ESTATE, "nothing simulated yet");
    if (!init || !ptr) return fail(ctx, GATSPI_EINVAL, "null output array");
    if (window < ctx->batch_w0 || window >= ctx->batch_w0 + ctx->batch_nw)
      return fail(ctx, GATSPI_ESTATE, "window " + std::to_string(window) + " is not in the resident batch [" +
                                          std::to_string(ctx->batch_w0) + ", " +
                                          std::to_string(ctx->batch_w0 + ctx->batch_nw) + ")");
    CK(cudaSetDevice(ctx->device));
    const int32_t N = ctx->N, w = window - ctx->batch_w0;
    int32_t* d_cnt = nullptr;
    uint8_t* d_iv = nullptr;
    long long* d_dst = nullptr;
    int32_t* d_out = nullptr;
    int rc = GATSPI_OK;
    std::vector<int32_t> cnt(N);
    std::vector<uint8_t> iv(N);
    std::vector<long long> dst(N);
    int64_t tot = 0;
    auto cleanup = [&]() { dfree(d_cnt); dfree(d_iv); dfree(d_dst); dfree(d_out); };
    do {
      if (cudaMalloc(&d_cnt, sizeof(int32_t) * N) != cudaSuccess || cudaMalloc(&d_iv, N) != cudaSuccess ||
          cudaMalloc(&d_dst, sizeof(long long) * N) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(ctx, GATSPI_ENOMEM, "read-back buffers");
        break;
      }
      window_counts_kernel<<<(N + 255) / 256, 256, 0, ctx->stream>>>(N, ctx->batch_nw, w, ctx->d_rmeta, d_cnt,
                                                                     d_iv);
      if (cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ctx->stream) ||
          cudaMemcpyAsync(iv.data(), d_iv, N, cudaMemcpyDeviceToHost, ctx->stream) ||
          cudaStreamSynchronize(ctx->stream)) {
        rc = fail(ctx, GATSPI_ECUDA, "read-back copy failed");
        break;
      }
      // caller order
      ptr[0] = 0;
      for (int32_t e = 0; e < N; ++e) {
        const int32_t n = ctx->net_int[e];
        init[e] = iv[n];
        ptr[e + 1] = ptr[e] + cnt[n];
      }
      tot = ptr[N];
      if (total) *total = tot;
      if (!times) break;
      if (cap < tot) {
        rc = fail(ctx, GATSPI_ECAPACITY, "times buffer too small: need " + std::to_string(tot));
        break;
      }
      for (int32_t e = 0; e < N; ++e) dst[ctx->net_int[e]] = ptr[e];
      if (cudaMalloc(&d_out, sizeof(int32_t) * std::max<int64_t>(tot, 1)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(ctx, GATSPI_ENOMEM, "read-back buffers");
        break;
      }
      if (cudaMemcpyAsync(d_dst, dst.data(), sizeof(long long) * N, cudaMemcpyHostToDevice, ctx->stream)) {
        rc = fail(ctx, GATSPI_ECUDA, "read-back copy failed");
        break;
      }
      window_gather_kernel<<<(N + 255) / 256, 256, 0, ctx->stream>>>(N, ctx->batch_nw, w, ctx->d_net_level,
                                                                     ctx->d_rstart, ctx->d_tinfo, ctx->batch_T,
                                                                     ctx->batch_TW, ctx->d_rmeta, ctx->d_lvl_base,
                                                                     ctx->d_times, d_dst, d_out);
      if (cudaMemcpyAsync(times, d_out, sizeof(int32_t) * tot, cudaMemcpyDeviceToHost, ctx->stream) ||
          cudaStreamSynchronize(ctx->stream)) {
        rc = fail(ctx, GATSPI_ECUDA, "read-back copy failed");
        break;
      }
    } while (0);
    cleanup();
    return rc;
  });
}

int gatspi_get_stats(gatspi_ctx* ctx, gatspi_stats* out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx || !out) return GATSPI_EINVAL;
    *out = ctx->stats;
    return GATSPI_OK;
  });
}

}  // extern "C"
