// Multi-job engine (include/gatspi.h, "Multi-job engine"): resident
// netlists, a queue of jobs cut into window parts, admission by device
// memory, and steps that launch one propagation kernel over the next level
// of every admitted part (continuous batching across jobs, netlists and
// levels).
#include <cuda_runtime.h>

#include <algorithm>
#include <exception>
#include <new>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "gatspi.h"
#include "host_common.h"
#include "kernels.cuh"
#include "digest.cuh"

using namespace gatspi_dev;

namespace {

constexpr int64_t kAlign = 256;
int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct ENetlist {
  gatspi_host::Prepared r;
  int32_t max_gate = 0, max_wire = 0;
  int32_t* d_fanin_ptr = nullptr;
  int32_t* d_fanin_net = nullptr;
  int32_t* d_net_level = nullptr;
  int32_t* d_gate_desc = nullptr;
  int32_t* d_gate_delay = nullptr;
  int32_t* d_wire_delay = nullptr;
  uint16_t* d_lut = nullptr;
  double edges_per_item = 2.0;  // observed edges per (net, window), sizes new parts
};

struct EJob {
  int64_t id = 0;
  int32_t net = 0, C = 0, L = 0, W = 1, n_windows = 0, max_edit = 0;
  // each input's edges before cycle c (edge_ptr[i*C + c] for every input i),
  // for the cycles where parts begin or end: all a part's planning needs,
  // without a host copy of the whole edge_ptr
  std::map<int32_t, std::vector<int64_t>> at_cycle;
  int64_t* d_edge_ptr = nullptr;
  int32_t* d_edge_time = nullptr;
  uint8_t* d_init_in = nullptr;
  int32_t* d_gate_delta = nullptr;
  unsigned long long* d_t1 = nullptr;
  unsigned long long* d_tc = nullptr;
  unsigned long long* d_digest = nullptr;  // [N] waveform digests (engine option)
  int32_t parts_total = 0, parts_done = 0;
  int state = GATSPI_JOB_QUEUED;
  std::string err;
  cudaEvent_t done_ev = nullptr;
  bool done_recorded = false;
  cudaEvent_t ready_ev = nullptr;  // the job's uploads are on the device
  bool ready_waited = false;       // the compute stream already waits for it
};

struct PartResult {
  int32_t status;
  int32_t pad;
  long long edges;
};

struct EPart {
  int64_t job = 0;
  int32_t w0 = 0, nw = 0, level = 0, D = 0;
  int64_t edge_hint = 0;
  int64_t level_items = 0;  // (gate, window) items of an average level
  char* mem = nullptr;
  size_t bytes = 0;
  int32_t* rstart = nullptr;  // linear tiling
  int2* tinfo = nullptr;      // gate-aligned tiling
  int32_t T = 0, TW = 0;      // tiles per net and windows per tile (gate-aligned), or 0
  uint16_t* rmeta = nullptr;
  int32_t* times = nullptr;
  long long cap = 0;
  long long* lvl_base = nullptr;
  unsigned long long* counters = nullptr;  // per level: packed tiles done / edges allocated
  int32_t* status = nullptr;
  unsigned long long* t1 = nullptr;
  unsigned long long* tc = nullptr;
  size_t zero_off = 0, zero_bytes = 0;
  int32_t slot = -1;  // pinned result slot
  cudaEvent_t ev = nullptr;
};

}  // namespace

struct gatspi_engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t upload = nullptr;  // job uploads, off the compute stream
  std::string err;
  size_t budget = 0, in_use = 0;
  int64_t step_load = 0;  // average level items of the parts in flight
  gatspi_engine_opts opts{};
  int nt = 256, ipt = 4;
  int tile = 128;  // items per warp tile (linear tiling)
  std::vector<std::unique_ptr<ENetlist>> nets;
  std::map<int64_t, std::unique_ptr<EJob>> jobs;
  int64_t next_job = 1;
  std::deque<std::unique_ptr<EPart>> queued;
  std::vector<std::unique_ptr<EPart>> active;
  std::vector<std::unique_ptr<EPart>> finishing;
  // per-step staging: pinned host ring -> one device buffer
  static constexpr int kRing = 4;
  char* h_stage[kRing] = {};
  cudaEvent_t stage_ev[kRing] = {};
  size_t h_stage_cap = 0;
  int ring = 0;
  char* d_stage = nullptr;
  size_t d_stage_cap = 0;
  int32_t* d_counter = nullptr;  // one tile counter per launch of a step (pair and other launches)
  // pinned per-part result slots
  PartResult* h_results = nullptr;
  std::vector<int32_t> free_slots;
  std::vector<cudaEvent_t> free_events;
  // device time of each step's launches: event pairs in flight, oldest first
  std::deque<std::pair<cudaEvent_t, cudaEvent_t>> step_ev;
  std::vector<cudaEvent_t> spare_ev;
  gatspi_engine_stats stats{};
};

namespace {

int efail(gatspi_engine* e, int code, const std::string& msg) {
  if (e) e->err = msg;
  return code;
}

// As in the single-job interface: no C++ exception crosses the C interface.
template <class F>
int guarded(gatspi_engine* e, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return efail(e, GATSPI_ENOMEM, "host allocation failed");
  } catch (const std::exception& x) {
    return efail(e, GATSPI_EINVAL, std::string("unexpected error: ") + x.what());
  } catch (...) {
    return efail(e, GATSPI_EINVAL, "unexpected error");
  }
}

#define ECK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return efail(eng, GATSPI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <class T>
int eupload(gatspi_engine* eng, T*& dst, const T* src, size_t n) {
  dfree(dst);
  ECK(cudaMalloc(&dst, std::max<size_t>(n, 1) * sizeof(T)));
  if (src && n) ECK(cudaMemcpy(dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return GATSPI_OK;
}

// Stream-ordered allocation and copy on the upload stream (the host buffer
// may be reused as soon as this returns: pageable copies are staged before
// the call returns).  Copies from pageable memory wait for their stream to
// drain first, so they go on a stream of their own: the compute stream
// keeps running while a job is uploaded, and waits for the job's ready
// event only before the job's first kernel.
template <class T>
int eupload_async(gatspi_engine* eng, T*& dst, const T* src, size_t n) {
  ECK(cudaMallocAsync((void**)&dst, std::max<size_t>(n, 1) * sizeof(T), eng->upload));
  if (src && n) ECK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, eng->upload));
  return GATSPI_OK;
}

template <class T>
void dfree_async(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// Lay out one part's device memory; returns the total bytes.
size_t part_layout(const ENetlist& nl, EPart& p, int ipt, char* base) {
  const int64_t N = nl.r.N, D = nl.r.D, NW = p.nw;
  const bool wide = wide_tiling(p.nw, ipt);
  const int32_t TW = tile_items_of(ipt);
  const int32_t T = wide ? (p.nw + TW - 1) / TW : 0;
  int64_t o = 0;
  const int64_t o_start = o; o = align_up(o + (wide ? N * T * 8 : N * NW * 4));
  const int64_t o_meta = o; o = align_up(o + N * NW * 2);
  const int64_t o_lvl = o; o = align_up(o + (D + 2) * 8);
  // zeroed region: level counters, status, part SAIF
  const int64_t o_zero = o;
  const int64_t o_cnt = o; o = align_up(o + (D + 2) * 8);
  const int64_t o_status = o; o = align_up(o + 8);
  const int64_t o_t1 = o; o = align_up(o + N * 8);
  const int64_t o_tc = o; o = align_up(o + N * 8);
  const int64_t zero_end = o;
  const int64_t o_times = o; o = align_up(o + p.edge_hint * 4);
  if (base) {
    p.rstart = wide ? nullptr : (int32_t*)(base + o_start);
    p.tinfo = wide ? (int2*)(base + o_start) : nullptr;
    p.T = T;
    p.TW = wide ? TW : 0;
    p.rmeta = (uint16_t*)(base + o_meta);
    p.lvl_base = (long long*)(base + o_lvl);
    p.counters = (unsigned long long*)(base + o_cnt);
    p.status = (int32_t*)(base + o_status);
    p.t1 = (unsigned long long*)(base + o_t1);
    p.tc = (unsigned long long*)(base + o_tc);
    p.times = (int32_t*)(base + o_times);
    p.cap = p.edge_hint;
    p.zero_off = (size_t)o_zero;
    p.zero_bytes = (size_t)(zero_end - o_zero);
  }
  return (size_t)o;
}

JobView make_view(const ENetlist& nl, const EJob& j, const EPart& p) {
  JobView v{};
  v.fanin_ptr = nl.d_fanin_ptr; v.fanin_net = nl.d_fanin_net; v.lut = nl.d_lut;
  v.gate_delay = nl.d_gate_delay; v.wire_delay = nl.d_wire_delay; v.net_level = nl.d_net_level;
  v.gdesc = (const int4*)nl.d_gate_desc;
  v.gate_delta = j.d_gate_delta;
  v.rstart = p.rstart; v.tinfo = p.tinfo; v.T = p.T; v.rmeta = p.rmeta; v.times = p.times; v.lvl_base = p.lvl_base; v.capacity = p.cap;
  v.saif_t1 = p.t1; v.saif_tc = p.tc; v.status = p.status;
  v.I = nl.r.I; v.NW = p.nw; v.w0 = p.w0; v.W = j.W; v.C = j.C; v.L = j.L;
  return v;
}

void free_job_device(EJob& j, cudaStream_t s) {
  // a job freed before its first kernel: its uploads may still be in flight
  if (j.ready_ev && !j.ready_waited) {
    cudaStreamWaitEvent(s, j.ready_ev, 0);
    j.ready_waited = true;
  }
  dfree_async(j.d_edge_ptr, s); dfree_async(j.d_edge_time, s); dfree_async(j.d_init_in, s);
  dfree_async(j.d_gate_delta, s); dfree_async(j.d_t1, s); dfree_async(j.d_tc, s);
  dfree_async(j.d_digest, s);
  if (j.done_ev) cudaEventDestroy(j.done_ev);
  j.done_ev = nullptr;
  if (j.ready_ev) cudaEventDestroy(j.ready_ev);
  j.ready_ev = nullptr;
}

int fail_job(gatspi_engine* eng, EJob& j, int code, const std::string& why) {
  j.state = GATSPI_JOB_FAILED;
  j.err = why;
  // drop its queued parts
  std::deque<std::unique_ptr<EPart>> keep;
  for (auto& p : eng->queued)
    if (p->job != j.id) keep.push_back(std::move(p));
  eng->queued.swap(keep);
  return efail(eng, code, "job " + std::to_string(j.id) + ": " + why);
}

int stage_reserve(gatspi_engine* eng, size_t bytes) {
  if (bytes > eng->h_stage_cap) {
    ECK(cudaStreamSynchronize(eng->stream));
    size_t cap = std::max<size_t>(bytes, 2 * eng->h_stage_cap);
    for (int k = 0; k < gatspi_engine::kRing; ++k) {
      if (eng->h_stage[k]) cudaFreeHost(eng->h_stage[k]);
      eng->h_stage[k] = nullptr;
      ECK(cudaMallocHost(&eng->h_stage[k], cap));
    }
    dfree(eng->d_stage);
    ECK(cudaMalloc(&eng->d_stage, cap));
    eng->h_stage_cap = eng->d_stage_cap = cap;
  }
  return GATSPI_OK;
}

// Retire parts whose last level has finished on the device.
// Each input's edges before cycle c of job j: captured at submission for
// the planned part bounds; a bound made later (a part split in two) is
// read from the job's device copy of edge_ptr, after its upload.
int bounds_at(gatspi_engine* eng, EJob& j, int32_t c, const std::vector<int64_t>** out) {
  auto it = j.at_cycle.find(c);
  if (it == j.at_cycle.end()) {
    ENetlist& nl = *eng->nets[j.net];
    std::vector<int64_t> v(nl.r.I);
    ECK(cudaMemcpy2DAsync(v.data(), sizeof(int64_t), j.d_edge_ptr + c, sizeof(int64_t) * (size_t)j.C,
                          sizeof(int64_t), (size_t)nl.r.I, cudaMemcpyDeviceToHost, eng->upload));
    ECK(cudaStreamSynchronize(eng->upload));
    it = j.at_cycle.emplace(c, std::move(v)).first;
  }
  *out = &it->second;
  return GATSPI_OK;
}

// Edges of all inputs in cycles [c0, c1) of job j, and optionally each
// input's exclusive prefix of them.
int batch_edges(gatspi_engine* eng, EJob& j, int32_t c0, int32_t c1, int64_t* l0, std::vector<long long>* pre) {
  const std::vector<int64_t>* a = nullptr;
  const std::vector<int64_t>* b = nullptr;
  int rc = bounds_at(eng, j, c0, &a);
  if (!rc) rc = bounds_at(eng, j, c1, &b);
  if (rc) return rc;
  int64_t s = 0;
  if (pre) pre->resize(a->size());
  for (size_t i = 0; i < a->size(); ++i) {
    if (pre) (*pre)[i] = s;
    s += (*b)[i] - (*a)[i];
  }
  *l0 = s;
  return GATSPI_OK;
}

// Add the device time of finished steps to the statistics (`all`: wait for
// the ones still in flight).
int harvest_steps(gatspi_engine* eng, bool all) {
  while (!eng->step_ev.empty()) {
    auto pr = eng->step_ev.front();
    if (all) ECK(cudaEventSynchronize(pr.second));
    const cudaError_t q = cudaEventQuery(pr.second);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return efail(eng, GATSPI_ECUDA, std::string("step event: ") + cudaGetErrorString(q));
    float ms = 0.f;
    ECK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    eng->stats.prop_ms += ms;
    eng->step_ev.pop_front();
    eng->spare_ev.push_back(pr.first);
    eng->spare_ev.push_back(pr.second);
  }
  return GATSPI_OK;
}

int step_event(gatspi_engine* eng, cudaEvent_t* ev) {
  if (!eng->spare_ev.empty()) {
    *ev = eng->spare_ev.back();
    eng->spare_ev.pop_back();
    return GATSPI_OK;
  }
  ECK(cudaEventCreate(ev));
  return GATSPI_OK;
}

int retire(gatspi_engine* eng, bool wait_one) {
  bool waited = false;
  for (size_t k = 0; k < eng->finishing.size();) {
    EPart& p = *eng->finishing[k];
    cudaError_t q = cudaEventQuery(p.ev);
    if (q == cudaErrorNotReady && wait_one && !waited) {
      const auto tw = std::chrono::steady_clock::now();
      ECK(cudaEventSynchronize(p.ev));
      eng->stats.wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tw).count();
      waited = true;
      q = cudaSuccess;
    }
    if (q == cudaErrorNotReady) {
      ++k;
      continue;
    }
    if (q != cudaSuccess) return efail(eng, GATSPI_ECUDA, std::string("part event: ") + cudaGetErrorString(q));
    const PartResult res = eng->h_results[p.slot];
    EJob& j = *eng->jobs.at(p.job);
    ENetlist& nl = *eng->nets[j.net];
    std::unique_ptr<EPart> own = std::move(eng->finishing[k]);
    eng->finishing.erase(eng->finishing.begin() + (long)k);
    eng->free_slots.push_back(p.slot);
    eng->free_events.push_back(p.ev);
    p.ev = nullptr;
    int rc = GATSPI_OK;
    if (j.state == GATSPI_JOB_FAILED) {
      // job already failed: just drop the part
    } else if (res.status & kStTimeout) {
      rc = fail_job(eng, j, GATSPI_ETIMEOUT, "a device-side wait ran out");
    } else if (res.status & (kStCapacity | kStOffset | kStCorrupt)) {
      eng->stats.parts_retried++;
      std::unique_ptr<EPart> again(new EPart());
      again->job = p.job;
      again->D = p.D;
      if ((res.status & kStOffset) && p.nw > 1) {
        // a level overflowed int32 offsets: split the windows
        std::unique_ptr<EPart> b(new EPart());
        const int32_t h = p.nw / 2;
        again->w0 = p.w0; again->nw = h; again->edge_hint = p.edge_hint / 2;
        b->job = p.job; b->D = p.D; b->w0 = p.w0 + h; b->nw = p.nw - h; b->edge_hint = p.edge_hint / 2;
        j.parts_total++;
        eng->queued.push_front(std::move(b));
      } else if (res.status & kStOffset) {
        rc = fail_job(eng, j, GATSPI_ECAPACITY, "a net has more than 32767 edges in one window, or one window's edges exceed the int32 offset range");
      } else {
        again->w0 = p.w0; again->nw = p.nw;
        again->edge_hint = std::max<int64_t>(2 * p.edge_hint, res.edges + 1024);
      }
      if (j.state != GATSPI_JOB_FAILED) eng->queued.push_front(std::move(again));
    } else {
      const int32_t N = nl.r.N;
      saif_add_kernel<<<(N + 255) / 256, 256, 0, eng->stream>>>(N, p.t1, p.tc, j.d_t1, j.d_tc);
      eng->stats.kernel_launches++;
      if (j.d_digest) {  // the part's waveforms, read before its memory is freed below
        DigestParams q{};
        q.rmeta = p.rmeta; q.tinfo = p.tinfo; q.rstart = p.rstart;
        q.net_level = nl.d_net_level; q.lvl_base = p.lvl_base; q.times = p.times;
        q.capacity = p.cap; q.out = j.d_digest; q.status = p.status;
        q.N = N; q.NW = p.nw; q.w0 = p.w0;
        q.TW = p.T > 0 ? p.TW : 128;
        q.T = (p.nw + q.TW - 1) / q.TW;
        const long long warps = (long long)q.N * q.T;
        digest_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, eng->stream>>>(q);
        ECK(cudaGetLastError());
        eng->stats.kernel_launches++;
      }
      const double obs = (double)res.edges / ((double)N * p.nw);
      nl.edges_per_item = std::max(nl.edges_per_item * 0.98, obs * 1.1);
      j.parts_done++;
      eng->stats.parts_done++;
      if (j.parts_done == j.parts_total) {
        if (!j.done_ev) ECK(cudaEventCreateWithFlags(&j.done_ev, cudaEventDisableTiming));
        ECK(cudaEventRecord(j.done_ev, eng->stream));
        j.done_recorded = true;
      }
    }
    ECK(cudaFreeAsync(p.mem, eng->stream));
    eng->in_use -= p.bytes;
    if (rc) return rc;
  }
  return GATSPI_OK;
}

}  // namespace

extern "C" {

int gatspi_engine_create(gatspi_engine** out, int device, size_t arena_bytes, const gatspi_engine_opts* opts) {
  return guarded(nullptr, [&]() -> int {
    if (!out) return GATSPI_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
      cudaGetLastError();
      return GATSPI_EINVAL;
    }
    gatspi_engine_opts o{};
    if (opts) o = *opts;
    if (o.digest < 0 || o.digest > 1 || o.step_items < 0) return GATSPI_EINVAL;
    const int nt = o.tile_items ? o.tile_items : 256;
    const int ipt = o.items_per_thread ? o.items_per_thread : 4;
    if ((nt != 128 && nt != 256 && nt != 512) || (ipt != 1 && ipt != 2 && ipt != 4 && ipt != 8) ||
        (nt == 512 && ipt == 8))
      return GATSPI_EINVAL;
    if (o.max_active < 0 || o.part_items < 0) return GATSPI_EINVAL;
    auto* eng = new gatspi_engine();
    eng->device = device;
    eng->opts = o;
    eng->nt = nt;
    eng->ipt = ipt;
    eng->tile = tile_items_of(ipt);
    if (!eng->opts.max_active) eng->opts.max_active = 1024;
    if (!eng->opts.part_items) eng->opts.part_items = 1ll << 30;
    if (!eng->opts.step_items) eng->opts.step_items = 1ll << 24;  // the best of 2^24..2^28 measured on the batched stream
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&eng->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&eng->upload, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&eng->d_counter, sizeof(int32_t) * (size_t)(2 * (eng->opts.max_active / kMaxSegs + 2))) !=
            cudaSuccess ||
        cudaMallocHost(&eng->h_results, sizeof(PartResult) * (size_t)eng->opts.max_active) != cudaSuccess) {
      cudaGetLastError();
      gatspi_engine_destroy(eng);
      return GATSPI_ECUDA;
    }
    for (int k = 0; k < gatspi_engine::kRing; ++k)
      if (cudaEventCreateWithFlags(&eng->stage_ev[k], cudaEventDisableTiming) != cudaSuccess) {
        gatspi_engine_destroy(eng);
        return GATSPI_ECUDA;
      }
    for (int32_t s = eng->opts.max_active - 1; s >= 0; --s) eng->free_slots.push_back(s);
    // keep freed part memory in the device pool between steps
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    eng->budget = arena_bytes ? arena_bytes : (size_t)(0.85 * (double)free_b);
    *out = eng;
    return GATSPI_OK;
  });
}

int gatspi_engine_destroy(gatspi_engine* eng) {
  return guarded(eng, [&]() -> int {
    if (!eng) return GATSPI_OK;
    cudaSetDevice(eng->device);
    if (eng->stream) cudaStreamSynchronize(eng->stream);
    auto drop = [&](std::unique_ptr<EPart>& p) {
      if (p->mem) cudaFree(p->mem);
      if (p->ev) cudaEventDestroy(p->ev);
    };
    for (auto& p : eng->active) drop(p);
    for (auto& p : eng->finishing) drop(p);
    for (auto& kv : eng->jobs) free_job_device(*kv.second, eng->stream);
    if (eng->stream) cudaStreamSynchronize(eng->stream);
    for (auto& nl : eng->nets) {
      dfree(nl->d_fanin_ptr); dfree(nl->d_fanin_net); dfree(nl->d_net_level); dfree(nl->d_gate_desc);
      dfree(nl->d_gate_delay); dfree(nl->d_wire_delay); dfree(nl->d_lut);
    }
    for (int k = 0; k < gatspi_engine::kRing; ++k) {
      if (eng->h_stage[k]) cudaFreeHost(eng->h_stage[k]);
      if (eng->stage_ev[k]) cudaEventDestroy(eng->stage_ev[k]);
    }
    for (auto e : eng->free_events) cudaEventDestroy(e);
    for (auto& pr : eng->step_ev) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (auto e : eng->spare_ev) cudaEventDestroy(e);
    dfree(eng->d_stage);
    dfree(eng->d_counter);
    if (eng->h_results) cudaFreeHost(eng->h_results);
    if (eng->upload) cudaStreamSynchronize(eng->upload);
    if (eng->upload) cudaStreamDestroy(eng->upload);
    if (eng->stream) cudaStreamDestroy(eng->stream);
    // hand the memory parked in the stream-ordered pool back to the device
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, eng->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    delete eng;
    return GATSPI_OK;
  });
}

const char* gatspi_engine_last_error(gatspi_engine* eng) { return eng ? eng->err.c_str() : "null engine"; }

int gatspi_engine_add_netlist(gatspi_engine* eng, int32_t num_inputs, int32_t num_gates,
                              const int32_t* fanin_ptr, const int32_t* fanin_net, const uint16_t* lut,
                              const int32_t* gate_delay, const int32_t* wire_delay, int32_t* netlist_id) {
  return guarded(eng, [&]() -> int {
    if (!eng || !netlist_id) return GATSPI_EINVAL;
    std::unique_ptr<ENetlist> nl(new ENetlist());
    std::string why = gatspi_host::prepare_netlist(num_inputs, num_gates, fanin_ptr, fanin_net, lut, &nl->r);
    if (!why.empty()) return efail(eng, GATSPI_EINVAL, why);
    std::vector<int32_t> gd, wd;
    why = gatspi_host::prepare_delays(nl->r, gate_delay, wire_delay, &gd, &wd, &nl->max_gate, &nl->max_wire);
    if (!why.empty()) return efail(eng, GATSPI_EINVAL, why);
    ECK(cudaSetDevice(eng->device));
    int rc;
    if ((rc = eupload(eng, nl->d_fanin_ptr, nl->r.fanin_ptr.data(), nl->r.fanin_ptr.size()))) return rc;
    if ((rc = eupload(eng, nl->d_fanin_net, nl->r.fanin_net.data(), nl->r.fanin_net.size()))) return rc;
    if ((rc = eupload(eng, nl->d_net_level, nl->r.net_level.data(), nl->r.net_level.size()))) return rc;
    if ((rc = eupload(eng, nl->d_lut, nl->r.lut.data(), nl->r.lut.size()))) return rc;
    if (!nl->r.gate_desc.empty() &&
        (rc = eupload(eng, nl->d_gate_desc, nl->r.gate_desc.data(), nl->r.gate_desc.size())))
      return rc;
    if ((rc = eupload(eng, nl->d_gate_delay, gd.data(), gd.size()))) return rc;
    if ((rc = eupload(eng, nl->d_wire_delay, wd.data(), wd.size()))) return rc;
    *netlist_id = (int32_t)eng->nets.size();
    eng->nets.push_back(std::move(nl));
    return GATSPI_OK;
  });
}

int gatspi_engine_submit(gatspi_engine* eng, int32_t netlist_id, int32_t num_cycles, int32_t cycle_ps,
                         const uint8_t* init, const int64_t* edge_ptr, const int32_t* edge_time,
                         int32_t window_cycles, int32_t n_edits, const int32_t* edit_gate,
                         const int32_t* edit_delta, int64_t* job_id) {
  return guarded(eng, [&]() -> int {
    if (!eng || !job_id) return GATSPI_EINVAL;
    if (netlist_id < 0 || netlist_id >= (int32_t)eng->nets.size())
      return efail(eng, GATSPI_EINVAL, "unknown netlist id");
    ENetlist& nl = *eng->nets[netlist_id];
    std::string why = gatspi_host::validate_stimulus(nl.r.I, num_cycles, cycle_ps, init, edge_ptr, edge_time);
    if (!why.empty()) return efail(eng, GATSPI_EINVAL, why);
    const int32_t W = window_cycles ? window_cycles : 1;
    if (W < 1) return efail(eng, GATSPI_EINVAL, "window_cycles must be >= 1");
    if (n_edits < 0 || (n_edits > 0 && (!edit_gate || !edit_delta)))
      return efail(eng, GATSPI_EINVAL, "bad delay edit arrays");
    std::vector<int32_t> delta;
    int32_t max_edit = 0;
    if (n_edits > 0) {
      delta.assign(nl.r.G, 0);
      for (int32_t k = 0; k < n_edits; ++k) {
        const int32_t g = edit_gate[k];
        if (g < 0 || g >= nl.r.G) return efail(eng, GATSPI_EINVAL, "edit names an unknown gate");
        if (edit_delta[k] < -gatspi_host::kMaxDelay || edit_delta[k] > gatspi_host::kMaxDelay)
          return efail(eng, GATSPI_EINVAL, "edit delta outside +-2^24 ps");
        delta[nl.r.gate_int[g]] = edit_delta[k];
        max_edit = std::max(max_edit, edit_delta[k]);
      }
    }
    if (!gatspi_host::horizon_fits(W, num_cycles, cycle_ps, nl.r.D, nl.max_gate, nl.max_wire, max_edit))
      return efail(eng, GATSPI_EINVAL, "window length plus path delays could overflow int32 ps");
    ECK(cudaSetDevice(eng->device));
    std::unique_ptr<EJob> j(new EJob());
    j->id = eng->next_job++;
    j->net = netlist_id;
    j->C = num_cycles; j->L = cycle_ps; j->W = W; j->max_edit = max_edit;
    j->n_windows = (num_cycles + W - 1) / W;
    const int64_t n = (int64_t)nl.r.I * num_cycles;
    int rc;
    auto undo = [&](int code) { free_job_device(*j, eng->stream); return code; };
    if ((rc = eupload_async(eng, j->d_edge_ptr, edge_ptr, (size_t)n + 1))) return undo(rc);
    if ((rc = eupload_async(eng, j->d_edge_time, edge_time, (size_t)edge_ptr[n]))) return undo(rc);
    if ((rc = eupload_async(eng, j->d_init_in, init, (size_t)nl.r.I))) return undo(rc);
    if (n_edits > 0 && (rc = eupload_async(eng, j->d_gate_delta, delta.data(), delta.size()))) return undo(rc);
    if ((rc = eupload_async<unsigned long long>(eng, j->d_t1, nullptr, nl.r.N))) return undo(rc);
    if ((rc = eupload_async<unsigned long long>(eng, j->d_tc, nullptr, nl.r.N))) return undo(rc);
    ECK(cudaMemsetAsync(j->d_t1, 0, sizeof(unsigned long long) * nl.r.N, eng->upload));
    ECK(cudaMemsetAsync(j->d_tc, 0, sizeof(unsigned long long) * nl.r.N, eng->upload));
    if (eng->opts.digest) {
      if ((rc = eupload_async<unsigned long long>(eng, j->d_digest, nullptr, nl.r.N))) return undo(rc);
      ECK(cudaMemsetAsync(j->d_digest, 0, sizeof(unsigned long long) * nl.r.N, eng->upload));
    }
    ECK(cudaEventCreateWithFlags(&j->ready_ev, cudaEventDisableTiming));
    ECK(cudaEventRecord(j->ready_ev, eng->upload));
    // cut into parts of at most part_items (gate, window) items and a level
    // item count that fits int32
    int64_t widest = nl.r.I;
    for (int32_t l = 1; l <= nl.r.D; ++l)
      widest = std::max<int64_t>(widest, nl.r.lvl_gate_begin[l + 1] - nl.r.lvl_gate_begin[l]);
    int64_t per = std::max<int64_t>(1, eng->opts.part_items / std::max<int64_t>(nl.r.N, 1));
    per = std::min<int64_t>(per, 0x7fff0000ll / widest);
    per = std::max<int64_t>(per, 1);
    auto capture = [&](int32_t c) {  // the validated caller array, at cycle c
      std::vector<int64_t>& v = j->at_cycle[c];
      v.resize(nl.r.I);
      for (int32_t i = 0; i < nl.r.I; ++i) v[i] = edge_ptr[(size_t)i * num_cycles + c];
    };
    for (int32_t w0 = 0; w0 < j->n_windows; w0 += (int32_t)per) {
      std::unique_ptr<EPart> p(new EPart());
      p->job = j->id;
      p->D = nl.r.D;
      p->w0 = w0;
      p->nw = (int32_t)std::min<int64_t>(per, j->n_windows - w0);
      capture(std::min(w0 * W, num_cycles));
      eng->queued.push_back(std::move(p));
      j->parts_total++;
    }
    capture(num_cycles);
    *job_id = j->id;
    eng->jobs[j->id] = std::move(j);
    return GATSPI_OK;
  });
}

static int engine_step_impl(gatspi_engine* eng, int32_t* active_out, int32_t* queued_out) {
  if (!eng) return GATSPI_EINVAL;
  ECK(cudaSetDevice(eng->device));
  // 1. retire (block on the oldest finishing part only if nothing else can move)
  const bool stuck = eng->active.empty() && !eng->finishing.empty();
  int rc = retire(eng, stuck);
  if (rc) return rc;

  // 2. admit
  std::vector<EPart*> admitted;
  std::vector<std::vector<long long>> prefixes;
  while (!eng->queued.empty() &&
         (int32_t)(eng->active.size() + eng->finishing.size()) < eng->opts.max_active &&
         (eng->active.empty() || eng->step_load < eng->opts.step_items)) {
    EPart& p = *eng->queued.front();
    EJob& j = *eng->jobs.at(p.job);
    if (j.state == GATSPI_JOB_FAILED) {
      eng->queued.pop_front();
      continue;
    }
    ENetlist& nl = *eng->nets[j.net];
    if (!p.edge_hint) {
      // level-0 edges are known; the rest follows the netlist's history
      const int32_t c0 = p.w0 * j.W, c1 = std::min((p.w0 + p.nw) * j.W, j.C);
      int64_t l0 = 0;
      if ((rc = batch_edges(eng, j, c0, c1, &l0, nullptr))) return rc;
      p.edge_hint = l0 + (int64_t)(nl.edges_per_item * (double)nl.r.G * p.nw * 1.25) + 4096;
    }
    const size_t bytes = part_layout(nl, p, eng->ipt, nullptr);
    if (bytes > eng->budget) {
      if (p.nw > 1) {  // split and retry
        std::unique_ptr<EPart> b(new EPart());
        const int32_t h = p.nw / 2;
        b->job = p.job; b->D = p.D; b->w0 = p.w0 + h; b->nw = p.nw - h;
        p.nw = h;
        p.edge_hint = 0;
        j.parts_total++;
        eng->queued.insert(eng->queued.begin() + 1, std::move(b));
        continue;
      }
      return fail_job(eng, j, GATSPI_ECAPACITY, "one window does not fit in the engine's memory budget");
    }
    if (eng->in_use + bytes > eng->budget) break;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, bytes, eng->stream) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    std::unique_ptr<EPart> own = std::move(eng->queued.front());
    eng->queued.pop_front();
    own->mem = (char*)mem;
    own->bytes = bytes;
    part_layout(nl, *own, eng->ipt, own->mem);
    eng->in_use += bytes;
    own->level_items = (int64_t)own->nw * nl.r.G / std::max<int32_t>(nl.r.D, 1);
    eng->step_load += own->level_items;
    eng->stats.bytes_peak = std::max<int64_t>(eng->stats.bytes_peak, (int64_t)eng->in_use);
    ECK(cudaMemsetAsync(own->mem + own->zero_off, 0, own->zero_bytes, eng->stream));
    std::vector<long long> pre;
    int64_t l0 = 0;
    const int32_t c0 = own->w0 * j.W, c1 = std::min((own->w0 + own->nw) * j.W, j.C);
    if ((rc = batch_edges(eng, j, c0, c1, &l0, &pre))) return rc;
    prefixes.push_back(std::move(pre));
    own->level = 0;
    admitted.push_back(own.get());
    eng->active.push_back(std::move(own));
  }

  // 3. stage: input prefixes of admitted parts, then the launch tables
  std::vector<size_t> pre_off(admitted.size());
  size_t bytes = 0;
  for (size_t k = 0; k < admitted.size(); ++k) {
    pre_off[k] = bytes;
    bytes = (size_t)align_up((int64_t)(bytes + prefixes[k].size() * sizeof(long long)));
  }
  std::vector<EPart*> stepping;
  for (auto& p : eng->active)
    if (p->level >= 1 || std::find(admitted.begin(), admitted.end(), p.get()) != admitted.end())
      stepping.push_back(p.get());
  if ((rc = stage_reserve(eng, std::max<size_t>(bytes, 4096)))) return rc;
  const int slot = eng->ring;
  eng->ring = (eng->ring + 1) % gatspi_engine::kRing;
  {
    const auto tw = std::chrono::steady_clock::now();
    ECK(cudaEventSynchronize(eng->stage_ev[slot]));
    eng->stats.wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tw).count();
  }
  char* h = eng->h_stage[slot];
  for (size_t k = 0; k < admitted.size(); ++k)
    std::memcpy(h + pre_off[k], prefixes[k].data(), prefixes[k].size() * sizeof(long long));
  // levels: admitted parts run level 0 (inputs kernel) in this step and
  // level 1 onwards from the next step
  // Each (part, level) segment's gates of at most two pins go to the pair
  // kernel, when the engine's launch shape has one and the step has enough
  // such tiles for a launch of their own; the rest of each level goes to
  // propagate_multi_kernel.  Both parts count into the level's counter.
  const int32_t TW = tile_items_of(eng->ipt);
  auto tiles_per_gate = [&](const EPart* p) {
    return wide_tiling(p->nw, eng->ipt) ? (p->nw + TW - 1) / TW : 0;
  };
  bool split = pair_variant_compiled(eng->nt, eng->ipt, 0);
  if (split) {
    int64_t pair_total = 0;
    for (EPart* p : stepping) {
      if (p->level < 1) continue;
      const ENetlist& nl = *eng->nets[eng->jobs.at(p->job)->net];
      pair_total += (int64_t)(nl.r.lvl_split[p->level] - nl.r.lvl_gate_begin[p->level]) * tiles_per_gate(p);
    }
    split = pair_total >= kPairMinTiles;
  }
  std::vector<MultiSeg> segs, pair_segs;
  std::vector<int32_t> seg_tiles, pair_tiles;  // each segment's tiles in its launch
  int64_t tiles = 0;
  for (EPart* p : stepping) {
    if (p->level < 1) continue;
    EJob& j = *eng->jobs.at(p->job);
    ENetlist& nl = *eng->nets[j.net];
    const int32_t l = p->level;
    MultiSeg s{};
    s.seg.counters = p->counters + l;
    s.seg.level = l;
    s.seg.gate_begin = nl.r.lvl_gate_begin[l];
    s.seg.n_items = (nl.r.lvl_gate_begin[l + 1] - nl.r.lvl_gate_begin[l]) * p->nw;
    s.seg.n_tiles = (int32_t)level_tiles(nl.r.lvl_gate_begin[l + 1] - nl.r.lvl_gate_begin[l], p->nw, eng->ipt);
    s.job = make_view(nl, j, *p);
    s.tile_begin = 0;
    tiles += s.seg.n_tiles;
    eng->stats.items += s.seg.n_items;
    const int32_t T = tiles_per_gate(p);
    const int32_t n_pair = split && T > 0 ? nl.r.lvl_split[l] - nl.r.lvl_gate_begin[l] : 0;
    if (n_pair > 0) {
      pair_segs.push_back(s);
      pair_tiles.push_back(n_pair * T);
      s.seg.gate_begin = nl.r.lvl_split[l];
    }
    const int32_t rest = s.seg.n_tiles - n_pair * T;
    if (rest > 0) {
      segs.push_back(s);
      seg_tiles.push_back(rest);
    }
  }
  if (bytes) ECK(cudaMemcpyAsync(eng->d_stage, h, bytes, cudaMemcpyHostToDevice, eng->stream));
  ECK(cudaEventRecord(eng->stage_ev[slot], eng->stream));

  // 4. launches: the propagation step for parts already past level 0, then
  // level 0 of the admitted parts
  if (tiles > 0) {
    if ((rc = harvest_steps(eng, false))) return rc;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if ((rc = step_event(eng, &ev0)) || (rc = step_event(eng, &ev1))) return rc;
    ECK(cudaEventRecord(ev0, eng->stream));
    // one launch per kMaxSegs segments, each with its own tile counter:
    // the pair launches first, then the others
    const size_t n_pair_launch = (pair_segs.size() + kMaxSegs - 1) / kMaxSegs;
    const size_t n_launch = (segs.size() + kMaxSegs - 1) / kMaxSegs;
    ECK(cudaMemsetAsync(eng->d_counter, 0, sizeof(int32_t) * (n_pair_launch + n_launch), eng->stream));
    for (size_t c = 0; c < n_pair_launch + n_launch; ++c) {
      const bool pair = c < n_pair_launch;
      const std::vector<MultiSeg>& list = pair ? pair_segs : segs;
      const std::vector<int32_t>& ltiles = pair ? pair_tiles : seg_tiles;
      const size_t c0 = pair ? c : c - n_pair_launch;
      MultiParams m{};
      int64_t t = 0;
      for (size_t k = c0 * kMaxSegs; k < list.size() && k < (c0 + 1) * kMaxSegs; ++k) {
        MultiSeg& s = m.segs[m.n_segs++];
        s = list[k];
        s.tile_begin = (int32_t)t;
        t += ltiles[k];
      }
      if (t > 0x7fffff00ll) return efail(eng, GATSPI_ECAPACITY, "too many tiles in one launch");
      m.n_tiles = (int32_t)t;
      m.tile_counter = eng->d_counter + c;
      cudaError_t err;
      if (pair) {
        MultiPairLaunch go{&m, eng->stream};
        if (eng->nt == 128) go.go<128>();
        else go.go<256>();
        err = go.err;
      } else {
        MultiLaunch go{&m, eng->stream};
        launch_variant(eng->nt, eng->ipt, go);
        err = go.err;
      }
      if (err)
        return efail(eng, GATSPI_ECUDA, "enabling the propagation kernel's shared memory on device " +
                                            std::to_string(eng->device) + " failed: " + cudaGetErrorString(err));
      ECK(cudaGetLastError());
      eng->stats.kernel_launches++;
    }
    ECK(cudaEventRecord(ev1, eng->stream));
    eng->step_ev.emplace_back(ev0, ev1);
    eng->stats.steps++;
  }
  for (size_t k = 0; k < admitted.size(); ++k) {
    EPart& p = *admitted[k];
    EJob& j = *eng->jobs.at(p.job);
    ENetlist& nl = *eng->nets[j.net];
    InputParams q{};
    q.edge_ptr = j.d_edge_ptr; q.edge_time = j.d_edge_time; q.init_in = j.d_init_in;
    q.in_prefix = (const long long*)(eng->d_stage + pre_off[k]);
    q.rstart = p.rstart; q.tinfo = p.tinfo; q.T = p.T; q.TW = p.TW; q.rmeta = p.rmeta; q.times = p.times; q.saif_t1 = p.t1; q.saif_tc = p.tc;
    q.lvl_base = p.lvl_base; q.status = p.status;
    int64_t l0 = 0;
    const int32_t c0 = p.w0 * j.W, c1 = std::min((p.w0 + p.nw) * j.W, j.C);
    if ((rc = batch_edges(eng, j, c0, c1, &l0, nullptr))) return rc;
    if (l0 > p.cap) {  // cannot happen: the hint covers level 0
      return fail_job(eng, j, GATSPI_ECAPACITY, "input edges exceed the part's store");
    }
    q.total = l0;
    q.I = nl.r.I; q.NW = p.nw; q.w0 = p.w0; q.W = j.W; q.C = j.C; q.L = j.L;
    q.n_items = nl.r.I * p.nw;
    if (!j.ready_waited) {  // the job's first kernel: its uploads must have landed
      ECK(cudaStreamWaitEvent(eng->stream, j.ready_ev, 0));
      j.ready_waited = true;
    }
    inputs_kernel<<<(q.n_items + 255) / 256, 256, 0, eng->stream>>>(q);
    ECK(cudaGetLastError());
    eng->stats.kernel_launches++;
  }

  // 5. advance; parts past their last level report status and edge count
  for (size_t k = 0; k < eng->active.size();) {
    EPart& p = *eng->active[k];
    p.level++;
    if (p.level > p.D) {
      if (eng->free_slots.empty()) return efail(eng, GATSPI_ESTATE, "no result slot");
      p.slot = eng->free_slots.back();
      eng->free_slots.pop_back();
      if (!eng->free_events.empty()) {
        p.ev = eng->free_events.back();
        eng->free_events.pop_back();
      } else {
        ECK(cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming));
      }
      PartResult* r = eng->h_results + p.slot;
      ECK(cudaMemcpyAsync(&r->status, p.status, sizeof(int32_t), cudaMemcpyDeviceToHost, eng->stream));
      ECK(cudaMemcpyAsync(&r->edges, p.lvl_base + p.D + 1, sizeof(long long), cudaMemcpyDeviceToHost,
                          eng->stream));
      ECK(cudaEventRecord(p.ev, eng->stream));
      eng->step_load -= p.level_items;
      eng->finishing.push_back(std::move(eng->active[k]));
      eng->active.erase(eng->active.begin() + (long)k);
      continue;
    }
    ++k;
  }
  for (auto& kv : eng->jobs) {
    EJob& j = *kv.second;
    if (j.state == GATSPI_JOB_QUEUED && j.parts_done + (int32_t)0 < j.parts_total) {
      for (auto& p : eng->active)
        if (p->job == j.id) { j.state = GATSPI_JOB_RUNNING; break; }
    }
  }
  eng->stats.active = (int32_t)(eng->active.size() + eng->finishing.size());
  eng->stats.queued = (int32_t)eng->queued.size();
  if (active_out) *active_out = eng->stats.active;
  if (queued_out) *queued_out = eng->stats.queued;
  return GATSPI_OK;
}

int gatspi_engine_step(gatspi_engine* eng, int32_t* active_out, int32_t* queued_out) {
  return guarded(eng, [&]() -> int {
    if (!eng) return GATSPI_EINVAL;
    const auto t = std::chrono::steady_clock::now();
    const int rc = engine_step_impl(eng, active_out, queued_out);
    eng->stats.host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
    return rc;
  });
}

int gatspi_engine_drain(gatspi_engine* eng) {
  return guarded(eng, [&]() -> int {
    if (!eng) return GATSPI_EINVAL;
    int rc = GATSPI_OK;
    for (;;) {
      int32_t a = 0, q = 0;
      const int r = gatspi_engine_step(eng, &a, &q);
      if (r && !rc) rc = r;
      if (r == GATSPI_ECUDA) return r;
      if (a == 0 && q == 0) break;
    }
    ECK(cudaStreamSynchronize(eng->stream));
    return rc;
  });
}

int gatspi_engine_poll(gatspi_engine* eng, int64_t job_id, int32_t* state, int64_t* t0, int64_t* t1,
                       int64_t* tc) {
  return guarded(eng, [&]() -> int {
    if (!eng) return GATSPI_EINVAL;
    auto it = eng->jobs.find(job_id);
    if (it == eng->jobs.end()) return efail(eng, GATSPI_EINVAL, "unknown job id");
    EJob& j = *it->second;
    ECK(cudaSetDevice(eng->device));
    if (j.state != GATSPI_JOB_FAILED && j.done_recorded) {
      const cudaError_t q = cudaEventQuery(j.done_ev);
      if (q == cudaSuccess) j.state = GATSPI_JOB_DONE;
      else if (q != cudaErrorNotReady) return efail(eng, GATSPI_ECUDA, cudaGetErrorString(q));
    }
    if (state) *state = j.state;
    if (j.state == GATSPI_JOB_DONE && (t0 || t1 || tc)) {
      const ENetlist& nl = *eng->nets[j.net];
      const int32_t N = nl.r.N;
      std::vector<unsigned long long> a(N), b(N);
      ECK(cudaMemcpy(a.data(), j.d_t1, sizeof(unsigned long long) * N, cudaMemcpyDeviceToHost));
      ECK(cudaMemcpy(b.data(), j.d_tc, sizeof(unsigned long long) * N, cudaMemcpyDeviceToHost));
      const int64_t total = (int64_t)j.C * j.L;
      for (int32_t e = 0; e < N; ++e) {
        const int32_t n = nl.r.net_int[e];
        if (t1) t1[e] = (int64_t)a[n];
        if (t0) t0[e] = total - (int64_t)a[n];
        if (tc) tc[e] = (int64_t)b[n];
      }
    }
    if (j.state == GATSPI_JOB_FAILED) return efail(eng, GATSPI_OK, j.err);
    return GATSPI_OK;
  });
}

int gatspi_engine_digest(gatspi_engine* eng, int64_t job_id, uint64_t* per_net) {
  return guarded(eng, [&]() -> int {
    if (!eng || !per_net) return GATSPI_EINVAL;
    auto it = eng->jobs.find(job_id);
    if (it == eng->jobs.end()) return efail(eng, GATSPI_EINVAL, "unknown job id");
    EJob& j = *it->second;
    ECK(cudaSetDevice(eng->device));
    if (j.state != GATSPI_JOB_FAILED && j.done_recorded && cudaEventQuery(j.done_ev) == cudaSuccess)
      j.state = GATSPI_JOB_DONE;
    cudaGetLastError();
    if (j.state != GATSPI_JOB_DONE) return efail(eng, GATSPI_ESTATE, "job not done");
    if (!j.d_digest) return efail(eng, GATSPI_ESTATE, "the engine was created without digests");
    const ENetlist& nl = *eng->nets[j.net];
    const int32_t N = nl.r.N;
    std::vector<unsigned long long> d(N);
    ECK(cudaMemcpy(d.data(), j.d_digest, sizeof(unsigned long long) * N, cudaMemcpyDeviceToHost));
    for (int32_t e = 0; e < N; ++e) per_net[e] = (uint64_t)d[nl.r.net_int[e]];
    return GATSPI_OK;
  });
}

int gatspi_engine_release(gatspi_engine* eng, int64_t job_id) {
  return guarded(eng, [&]() -> int {
    if (!eng) return GATSPI_EINVAL;
    auto it = eng->jobs.find(job_id);
    if (it == eng->jobs.end()) return efail(eng, GATSPI_EINVAL, "unknown job id");
    EJob& j = *it->second;
    if (j.state != GATSPI_JOB_DONE && j.state != GATSPI_JOB_FAILED)
      return efail(eng, GATSPI_ESTATE, "job still running");
    for (auto& p : eng->active)
      if (p->job == job_id) return efail(eng, GATSPI_ESTATE, "job still has parts in flight");
    for (auto& p : eng->finishing)
      if (p->job == job_id) return efail(eng, GATSPI_ESTATE, "job still has parts in flight");
    ECK(cudaSetDevice(eng->device));
    free_job_device(j, eng->stream);
    eng->jobs.erase(it);
    return GATSPI_OK;
  });
}

int gatspi_engine_get_stats(gatspi_engine* eng, gatspi_engine_stats* out) {
  return guarded(eng, [&]() -> int {
    if (!eng || !out) return GATSPI_EINVAL;
    ECK(cudaSetDevice(eng->device));
    const int rc = harvest_steps(eng, false);
    if (rc) return rc;
    *out = eng->stats;
    return GATSPI_OK;
  });
}

}  // extern "C"
