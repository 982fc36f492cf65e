// Host-side preparation shared by the single-job context and the multi-job
// engine: netlist validation and levelization (Section 3: logic levelization
// before simulation), delay-table validation and reordering, stimulus
// validation.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

namespace gatspi_host {

constexpr int kMaxPins = 4;
constexpr int32_t kMaxDelay = 1 << 24;

// A netlist in the library's internal order: inputs first, then gates sorted
// by level (stable), so each level's gates and nets are contiguous.
struct Prepared {
  int32_t I = 0, G = 0, N = 0, P = 0, D = 0;
  std::vector<int32_t> gate_ext;        // internal gate -> caller gate
  std::vector<int32_t> gate_int;        // caller gate -> internal gate
  std::vector<int32_t> net_int;         // caller net -> internal net
  std::vector<int32_t> pin_ext;         // internal pin -> caller pin
  std::vector<int32_t> fanin_ptr;       // [G+1]
  std::vector<int32_t> fanin_net;       // [P], internal net ids
  std::vector<int32_t> net_level;       // [N]
  std::vector<uint16_t> lut;            // [G]
  std::vector<int32_t> lvl_gate_begin;  // [D+2]: level l >= 1 holds internal
                                        // gates lvl_gate_begin[l] .. [l+1]
  std::vector<int32_t> lvl_split;       // [D+2]: within level l the gates of at
                                        // most two pins come first, up to lvl_split[l]
  std::vector<int64_t> fanout;          // pins driven by each internal net
  // Per internal gate, 8 words the propagation kernel fetches in one go:
  // fanin nets (unused pins repeat pin 0's net), first pin, truth table |
  // pin count << 16, fanin levels as 16-bit pairs.  Empty when a level
  // exceeds 65535 (the kernel then reads the CSR arrays).
  std::vector<int32_t> gate_desc;       // [G*8]
};

// Validate and levelize.  Returns an empty string on success, else why not.
inline std::string prepare_netlist(int32_t I, int32_t G, const int32_t* fanin_ptr,
                                   const int32_t* fanin_net, const uint16_t* lut, Prepared* out) {
  if (I < 1 || G < 0 || (int64_t)I + G > 0x7ffffffe) return "num_inputs must be >= 1 and num_gates >= 0";
  if (!fanin_ptr || (G > 0 && (!fanin_net || !lut))) return "null netlist array";
  if (fanin_ptr[0] != 0) return "fanin_ptr[0] must be 0";
  for (int32_t g = 0; g < G; ++g) {
    const int32_t k = fanin_ptr[g + 1] - fanin_ptr[g];
    if (k < 1 || k > kMaxPins)
      return "gate " + std::to_string(g) + " has " + std::to_string(k) + " pins (1..4 supported)";
  }
  const int32_t P = G ? fanin_ptr[G] : 0;
  std::vector<int32_t> level((size_t)I + G, 0);
  for (int32_t g = 0; g < G; ++g) {
    int32_t lv = 0;
    for (int32_t p = fanin_ptr[g]; p < fanin_ptr[g + 1]; ++p) {
      const int32_t n = fanin_net[p];
      if (n < 0 || n >= I + g)
        return "gate " + std::to_string(g) + " reads net " + std::to_string(n) +
               ": fanin nets must precede the gate's own net";
      lv = std::max(lv, level[n]);
    }
    level[(size_t)I + g] = lv + 1;
  }
  Prepared& r = *out;
  r = Prepared{};
  int32_t D = 0;
  for (int32_t g = 0; g < G; ++g) D = std::max(D, level[(size_t)I + g]);
  r.I = I; r.G = G; r.N = I + G; r.P = P; r.D = D;
  r.lvl_gate_begin.assign(D + 2, 0);
  r.lvl_split.assign(D + 2, 0);
  std::vector<int32_t> pairs(D + 2, 0);  // gates of at most two pins per level
  for (int32_t g = 0; g < G; ++g) {
    r.lvl_gate_begin[level[(size_t)I + g] + 1]++;
    if (fanin_ptr[g + 1] - fanin_ptr[g] <= 2) pairs[level[(size_t)I + g]]++;
  }
  for (int32_t l = 1; l <= D; ++l) r.lvl_gate_begin[l + 1] += r.lvl_gate_begin[l];
  for (int32_t l = 0; l <= D + 1; ++l) r.lvl_split[l] = r.lvl_gate_begin[l] + (l <= D ? pairs[l] : 0);
  // internal order: by level, then gates of at most two pins before the
  // others (each class in the caller's order)
  std::vector<int32_t> fill_pair(r.lvl_gate_begin.begin(), r.lvl_gate_begin.end());
  std::vector<int32_t> fill_rest(r.lvl_split.begin(), r.lvl_split.end());
  r.gate_ext.assign(G, 0);
  r.gate_int.assign(G, 0);
  for (int32_t g = 0; g < G; ++g) {
    const int32_t lv = level[(size_t)I + g];
    const int32_t j = fanin_ptr[g + 1] - fanin_ptr[g] <= 2 ? fill_pair[lv]++ : fill_rest[lv]++;
    r.gate_ext[j] = g;
    r.gate_int[g] = j;
  }
  r.net_int.resize((size_t)I + G);
  for (int32_t i = 0; i < I; ++i) r.net_int[i] = i;
  for (int32_t g = 0; g < G; ++g) r.net_int[(size_t)I + g] = I + r.gate_int[g];
  r.fanin_ptr.assign((size_t)G + 1, 0);
  r.fanin_net.resize(P);
  r.pin_ext.resize(P);
  r.lut.resize(G);
  r.net_level.assign((size_t)I + G, 0);
  r.fanout.assign((size_t)I + G, 0);
  for (int32_t j = 0; j < G; ++j) {
    const int32_t g = r.gate_ext[j];
    const int32_t k = fanin_ptr[g + 1] - fanin_ptr[g];
    r.fanin_ptr[j + 1] = r.fanin_ptr[j] + k;
    for (int32_t i = 0; i < k; ++i) {
      const int32_t pe = fanin_ptr[g] + i, pi = r.fanin_ptr[j] + i;
      r.pin_ext[pi] = pe;
      r.fanin_net[pi] = r.net_int[fanin_net[pe]];
      r.fanout[r.fanin_net[pi]]++;
    }
    r.lut[j] = lut[g];
    r.net_level[(size_t)I + j] = level[(size_t)I + g];
  }
  if (D <= 0xffff) {
    r.gate_desc.assign((size_t)G * 8, 0);
    for (int32_t j = 0; j < G; ++j) {
      int32_t* d = &r.gate_desc[(size_t)j * 8];
      const int32_t p0 = r.fanin_ptr[j], k = r.fanin_ptr[j + 1] - p0;
      int32_t lv[kMaxPins];
      for (int i = 0; i < kMaxPins; ++i) {
        d[i] = r.fanin_net[p0 + (i < k ? i : 0)];
        lv[i] = r.net_level[d[i]];
      }
      d[4] = p0;
      d[5] = (int32_t)((uint32_t)r.lut[j] | ((uint32_t)k << 16));
      d[6] = (int32_t)((uint32_t)lv[0] | ((uint32_t)lv[1] << 16));
      d[7] = (int32_t)((uint32_t)lv[2] | ((uint32_t)lv[3] << 16));
    }
  }
  return "";
}

// Validate the delay tables (used entries in [1, 2^24] ps) and reorder them
// to internal pin order.  Unused side columns are set to 1.
inline std::string prepare_delays(const Prepared& r, const int32_t* gate_delay, const int32_t* wire_delay,
                                  std::vector<int32_t>* gd, std::vector<int32_t>* wd, int32_t* max_gate,
                                  int32_t* max_wire) {
  if (r.P > 0 && (!gate_delay || !wire_delay)) return "null delay array";
  gd->assign((size_t)r.P * 32, 1);
  wd->assign((size_t)r.P * 2, 1);
  int32_t mg = 0, mw = 0;
  for (int32_t j = 0; j < r.G; ++j) {
    const int32_t k = r.fanin_ptr[j + 1] - r.fanin_ptr[j];
    const int32_t ncol = 1 << (k - 1);
    for (int32_t pi = r.fanin_ptr[j]; pi < r.fanin_ptr[j + 1]; ++pi) {
      const int64_t pe = r.pin_ext[pi];
      for (int e = 0; e < 4; ++e)
        for (int s = 0; s < ncol; ++s) {
          const int32_t v = gate_delay[pe * 32 + e * 8 + s];
          if (v < 1 || v > kMaxDelay)
            return "gate delay of pin " + std::to_string(pe) + " outside [1, 2^24] ps";
          mg = std::max(mg, v);
          (*gd)[(size_t)pi * 32 + e * 8 + s] = v;
        }
      for (int e = 0; e < 2; ++e) {
        const int32_t v = wire_delay[pe * 2 + e];
        if (v < 1 || v > kMaxDelay) return "wire delay of pin " + std::to_string(pe) + " outside [1, 2^24] ps";
        mw = std::max(mw, v);
        (*wd)[(size_t)pi * 2 + e] = v;
      }
    }
  }
  *max_gate = mg;
  *max_wire = mw;
  return "";
}

// The partial-SDF table (the paper's variant without full SDF, Section 5,
// Table "features"): every entry of an arc -- its 2 input edges x 2^(n-1)
// COND columns for one output edge -- replaced by their mean, rounded to the
// nearest ps (halves up); unused columns keep the value too.  `gd` is the
// internal-order table [P][2][2][8].
inline std::vector<int32_t> averaged_delays(const std::vector<int32_t>& fanin_ptr, int32_t G,
                                            const std::vector<int32_t>& gd) {
  std::vector<int32_t> out(gd.size(), 1);
  for (int32_t j = 0; j < G; ++j) {
    const int32_t k = fanin_ptr[j + 1] - fanin_ptr[j];
    const int32_t ncol = 1 << (k - 1);
    for (int32_t pi = fanin_ptr[j]; pi < fanin_ptr[j + 1]; ++pi) {
      const int32_t* d = &gd[(size_t)pi * 32];
      int32_t* a = &out[(size_t)pi * 32];
      for (int oe = 0; oe < 2; ++oe) {
        int64_t sum = 0;
        for (int ie = 0; ie < 2; ++ie)
          for (int32_t c = 0; c < ncol; ++c) sum += d[(2 * ie + oe) * 8 + c];
        const int64_t cnt = 2 * (int64_t)ncol;
        const int32_t avg = (int32_t)((sum + cnt / 2) / cnt);
        for (int ie = 0; ie < 2; ++ie)
          for (int c = 0; c < 8; ++c) a[(2 * ie + oe) * 8 + c] = avg;
      }
    }
  }
  return out;
}

// Checks one range of (input, cycle) slots; returns the first bad slot and
// why (0 = fine) in *bad / *kind.
inline void validate_slots(int64_t k0, int64_t k1, int32_t L, const int64_t* edge_ptr, const int32_t* edge_time,
                           int64_t* bad, int* kind) {
  *bad = -1;
  *kind = 0;
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t a = edge_ptr[k], b = edge_ptr[k + 1];
    if (b < a) {
      *bad = k;
      *kind = 1;
      return;
    }
    int32_t prev = -1;
    for (int64_t e = a; e < b; ++e) {
      const int32_t t = edge_time[e];
      if (t < 0 || t >= L || t <= prev) {
        *bad = k;
        *kind = (t < 0 || t >= L) ? 2 : 3;
        return;
      }
      prev = t;
    }
  }
}

// Validates a stimulus; the (input, cycle) slots are checked by up to 16
// host threads (the first bad slot is reported, as a serial scan would).
inline std::string validate_stimulus(int32_t I, int32_t C, int32_t L, const uint8_t* init,
                                     const int64_t* edge_ptr, const int32_t* edge_time) {
  if (C < 1 || L < 1) return "num_cycles and cycle_ps must be >= 1";
  if (!init || !edge_ptr) return "null stimulus array";
  const int64_t n = (int64_t)I * C;
  if (edge_ptr[0] != 0) return "edge_ptr[0] must be 0";
  if (edge_ptr[n] > 0 && !edge_time) return "null edge_time";
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({16, (int64_t)std::thread::hardware_concurrency(),
                                                               n / 65536 + 1}));
  std::vector<int64_t> bad(nt, -1);
  std::vector<int> kind(nt, 0);
  std::vector<std::thread> pool;
  for (int w = 1; w < nt; ++w)
    pool.emplace_back(validate_slots, n * w / nt, n * (w + 1) / nt, L, edge_ptr, edge_time, &bad[w], &kind[w]);
  validate_slots(0, n / nt, L, edge_ptr, edge_time, &bad[0], &kind[0]);
  for (auto& t : pool) t.join();
  for (int w = 0; w < nt; ++w) {
    if (bad[w] < 0) continue;
    const int64_t k = bad[w];
    if (kind[w] == 1) return "edge_ptr must be non-decreasing";
    if (kind[w] == 2)
      return "edge time outside [0, cycle_ps) for input " + std::to_string(k / C) + " cycle " +
             std::to_string(k % C);
    return "edge times must increase strictly within a cycle";
  }
  for (int32_t i = 0; i < I; ++i)
    if (init[i] > 1) return "initial values must be 0 or 1";
  return "";
}

// Longest possible time inside a window: its length plus the longest path.
inline bool horizon_fits(int32_t W, int32_t C, int32_t L, int32_t D, int32_t max_gate, int32_t max_wire,
                         int32_t max_edit = 0) {
  const int64_t h = (int64_t)std::min(W, C) * L + (int64_t)D * ((int64_t)max_gate + max_edit + max_wire);
  return h < 0x7fffffffll;
}

}  // namespace gatspi_host
