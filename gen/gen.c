/*
 * Seeded synthetic inputs for gate-level re-simulation: levelized netlists,
 * SDF-style delay tables and per-cycle input stimulus.
 *
 * This file produces inputs only.  It holds none of the simulation
 * arithmetic (no waveform merge, no delay selection, no filtering); both the
 * CPU oracle and the GPU path consume what it writes.
 *
 * Randomness is counter-based: every draw is SplitMix64's output function
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to a key built from (seed, stream, index), so any
 * element can be regenerated on its own and the result does not depend on
 * call order.  No libm call is made and the file is compiled with
 * -ffp-contract=off, so x86-64 and AArch64 produce identical bytes.
 *
 * Conventions shared with the library interface:
 *   nets 0..I-1 are inputs, gate g drives net I+g, gates are in level order;
 *   pins of gate g are fanin_ptr[g] .. fanin_ptr[g+1]-1 (pin 1 first), pin 1
 *   is the least significant bit of the LUT column index;
 *   lut bit k = Y[k];
 *   gate_delay[p][inEdge][outEdge][side] with 2x2x8 int32 per pin
 *   (1 = rising), side = the other pins' values compressed to n-1 bits;
 *   wire_delay[p][0] = rise, wire_delay[p][1] = fall.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define API __attribute__((visibility("default")))

static inline uint64_t sm64_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* One 64-bit draw for (seed, stream, index). */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t a = sm64_out(seed + 0x9E3779B97F4A7C15ULL * (stream + 1));
  return sm64_out(a ^ (idx * 0xD1B54A32D192ED03ULL + 0x9E3779B97F4A7C15ULL));
}

/* Uniform integer in [lo, hi] (inclusive); the modulo bias is < 2^-40. */
static inline int64_t uni(uint64_t x, int64_t lo, int64_t hi) {
  uint64_t span = (uint64_t)(hi - lo + 1);
  return lo + (int64_t)(x % span);
}

/* Bernoulli with probability permille/1000. */
static inline int bern(uint64_t x, int32_t permille) {
  return (int32_t)(x % 1000ULL) < permille;
}

/* Streams (kept distinct so that draws never collide). */
enum {
  S_CELL = 1, S_PIN = 2, S_QUOTA = 3, S_DUP = 4, S_IOPATH = 5, S_COND = 6,
  S_CONDSEL = 7, S_WIRE = 8, S_INIT = 9, S_STIM = 10
};

/* ------------------------------------------------------------------ cells */

enum {
  C_INV, C_BUF, C_NAND2, C_NOR2, C_AND2, C_OR2, C_XOR2, C_XNOR2, C_AOI21,
  C_OAI21, C_MUX2, C_NAND3, C_NAND4, C_NOR3, C_NOR4, C_AND3, C_AND4, C_OR3,
  C_OR4, C_AOI22, C_OAI22, C_NUM
};

static int cell_pins(int c) {
  switch (c) {
    case C_INV: case C_BUF: return 1;
    case C_AOI21: case C_OAI21: case C_MUX2: case C_NAND3: case C_NOR3:
    case C_AND3: case C_OR3: return 3;
    case C_NAND4: case C_NOR4: case C_AND4: case C_OR4: case C_AOI22:
    case C_OAI22: return 4;
    default: return 2;
  }
}

/* Boolean function of a cell; bit i-1 of x is the value on pin i. */
static int cell_eval(int c, unsigned x) {
  int a = x & 1, b = (x >> 1) & 1, s = (x >> 2) & 1, d = (x >> 3) & 1;
  int all = 0, any = 0, n = cell_pins(c);
  all = ((x & ((1u << n) - 1)) == ((1u << n) - 1));
  any = (x & ((1u << n) - 1)) != 0;
  switch (c) {
    case C_INV: return !a;
    case C_BUF: return a;
    case C_NAND2: case C_NAND3: case C_NAND4: return !all;
    case C_AND2: case C_AND3: case C_AND4: return all;
    case C_NOR2: case C_NOR3: case C_NOR4: return !any;
    case C_OR2: case C_OR3: case C_OR4: return any;
    case C_XOR2: return a ^ b;
    case C_XNOR2: return !(a ^ b);
    case C_AOI21: return !((a && b) || s);          /* pins A1, A2, B */
    case C_OAI21: return !((a || b) && s);
    case C_MUX2: return s ? b : a;                   /* pins A, B, S */
    case C_AOI22: return !((a && b) || (s && d));    /* A1, A2, B1, B2 */
    case C_OAI22: return !((a || b) && (s || d));
  }
  return 0;
}

API int gen_cell_count(void) { return C_NUM; }
API int gen_cell_pins(int c) { return (c >= 0 && c < C_NUM) ? cell_pins(c) : -1; }
API int gen_cell_lut(int c) {
  if (c < 0 || c >= C_NUM) return -1;
  int n = cell_pins(c), lut = 0;
  for (unsigned k = 0; k < (1u << n); ++k) lut |= cell_eval(c, k) << k;
  return lut;
}

static const int TINY_SET[] = {C_INV, C_BUF, C_NAND2, C_NOR2, C_AND2, C_OR2,
                               C_XOR2, C_XNOR2, C_AOI21, C_OAI21, C_MUX2};
static const int MID_SET[] = {C_INV, C_BUF, C_NAND2, C_NOR2, C_AND2, C_OR2,
                              C_XOR2, C_XNOR2, C_AOI21, C_OAI21, C_MUX2,
                              C_NAND3, C_NAND4, C_NOR3, C_NOR4, C_AND3, C_AND4,
                              C_OR3, C_OR4, C_AOI22, C_OAI22};

/* ------------------------------------------------------ fanout quotas */

/* Zipf(1.2) weights k^-1.2 for k = 1..64, tabulated to avoid libm. */
static const double ZIPF12[64] = {
  1.0, 0.43527528164806206, 0.2675805205867436, 0.18946457081379978,
  0.1449559327355391, 0.11647118646192989, 0.09680155905721158, 0.0824692444233059,
  0.0715993349974727, 0.06309573444801933, 0.05627672006216779, 0.050697028491100485,
  0.04605406581088445, 0.04213532588259928, 0.03878738394351254, 0.03589682359365735,
  0.03337807562774001, 0.03116542070683888, 0.029207586990966018, 0.02746401358265295,
  0.025902211566137076, 0.02449586517528923, 0.023223442471487783, 0.02206716335518359,
  0.02101222243523014, 0.020046196466871113, 0.019158587332288392, 0.01834046584088128,
  0.017584191408809388, 0.01688318947040394, 0.01623177325801658, 0.015625000000000003,
  0.015058554051149291, 0.014528651269734849, 0.014031960283392477, 0.013565537275849639,
  0.013126771670787605, 0.012713340653753008, 0.01232317090481261, 0.011954406247375465,
  0.011605380176865748, 0.011274592434758007, 0.010960688952237792, 0.010662444613386975,
  0.010378748387802984, 0.010108590462614413, 0.009851051068273196, 0.009605290744601333,
  0.009370541835906819, 0.009146101038546529, 0.00893132285265437, 0.008725613813089712,
  0.008528427393954558, 0.008339259497040825, 0.008157644447908358, 0.007983151434446263,
  0.007815381332125287, 0.007653963868022941, 0.007498555082351249, 0.007348835051847672,
  0.007204505844172542, 0.007065289676530649, 0.006930927255214929, 0.0068011762757509715};

static int32_t quota_draw(int model, uint64_t x) {
  if (model == 1) {
    /* Geometric with support >= 1 and mean 2.5 (success probability 0.4):
       each trial is one decimal digit drawn from its own counter. */
    int32_t k = 1;
    for (int it = 0; it < 256; ++it) {
      uint64_t digit = sm64_out(x + (uint64_t)it * 0x632BE59BD9B4E019ULL) % 10ULL;
      if (digit < 4) break;
      ++k;
    }
    return k;
  }
  if (model == 2) {
    double total = 0;
    for (int k = 0; k < 64; ++k) total += ZIPF12[k];
    double u = (double)(x >> 11) * (1.0 / 9007199254740992.0) * total;
    double acc = 0;
    for (int k = 0; k < 64; ++k) {
      acc += ZIPF12[k];
      if (u < acc) return k + 1;
    }
    return 64;
  }
  return 1;
}

/* Fenwick tree over int64 weights. */
typedef struct { int64_t* t; int32_t n; } fen_t;
static void fen_add(fen_t* f, int32_t i, int64_t v) {
  for (++i; i <= f->n; i += i & -i) f->t[i] += v;
}
static int64_t fen_prefix(const fen_t* f, int32_t i) {  /* sum of [0, i) */
  int64_t s = 0;
  for (; i > 0; i -= i & -i) s += f->t[i];
  return s;
}
/* smallest index j with prefix(j+1) > target */
static int32_t fen_find(const fen_t* f, int64_t target) {
  int32_t pos = 0, step = 1;
  while (step * 2 <= f->n) step *= 2;
  for (; step > 0; step >>= 1) {
    if (pos + step <= f->n && f->t[pos + step] <= target) {
      pos += step;
      target -= f->t[pos];
    }
  }
  return pos;
}

/*
 * Netlist structure.  Gates per level = G/D with the remainder spread over
 * the first levels; each gate draws its cell uniformly from the set; pin 1
 * comes from level l-1 (so the level is exact), the other pins from any
 * earlier level including the inputs.  With fanout_model 1 (geometric, mean
 * 2.5) or 2 (Zipf(1.2), capped at 64) fanins are drawn with weight equal to
 * the net's remaining fanout quota (uniform once a range has no quota left);
 * with fanout_model 0 they are uniform.  No net appears twice on one gate.
 *
 * fanin_net must hold 4*G entries.  Returns the pin count P, or -1 on bad
 * arguments.
 */
API int64_t gen_netlist(int32_t I, int32_t G, int32_t D, uint64_t seed,
                        int32_t cell_set, int32_t fanout_model,
                        int32_t* fanin_ptr, int32_t* fanin_net,
                        uint8_t* num_pins, uint16_t* lut, uint8_t* cell) {
  if (I < 1 || G < 0 || (G > 0 && D < 1) || (D > G && G > 0)) return -1;
  const int* set = cell_set == 0 ? TINY_SET : MID_SET;
  int nset = cell_set == 0 ? (int)(sizeof TINY_SET / sizeof *TINY_SET)
                           : (int)(sizeof MID_SET / sizeof *MID_SET);
  int32_t N = I + G;
  fen_t f;
  f.n = N;
  f.t = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
  int32_t* quota = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  if (!f.t || !quota) { free(f.t); free(quota); return -1; }
  /* quotas are assigned for every net up front (linear-time Fenwick build) */
  for (int32_t n = 0; n < N; ++n) {
    quota[n] = fanout_model == 0 ? 0 : quota_draw(fanout_model, draw(seed, S_QUOTA, (uint64_t)n));
    f.t[n + 1] += quota[n];
    int32_t parent = (n + 1) + ((n + 1) & -(n + 1));
    if (parent <= N) f.t[parent] += f.t[n + 1];
  }
  int32_t base = D > 0 ? G / D : 0, rem = D > 0 ? G % D : 0;
  int32_t g = 0, prev_begin = 0, prev_end = I;   /* net range of level l-1 */
  int64_t p = 0;
  fanin_ptr[0] = 0;
  for (int32_t l = 1; l <= D; ++l) {
    int32_t cnt = base + (l <= rem ? 1 : 0);
    int32_t lvl_begin_net = I + g;
    for (int32_t j = 0; j < cnt; ++j, ++g) {
      uint64_t cd = draw(seed, S_CELL, (uint64_t)g);
      int c = set[cd % (uint64_t)nset];
      int n = cell_pins(c);
      while (n > lvl_begin_net) {            /* too few earlier nets */
        c = (c == C_INV) ? C_INV : C_BUF;
        n = 1;
      }
      int32_t chosen[4];
      for (int i = 0; i < n; ++i) {
        int32_t lo = i == 0 ? prev_begin : 0;
        int32_t hi = i == 0 ? prev_end : lvl_begin_net;
        int32_t pick = -1;
        for (int attempt = 0; attempt < 32 && pick < 0; ++attempt) {
          uint64_t x = draw(seed, S_PIN, ((uint64_t)g << 8) | ((uint64_t)i << 5) | (uint64_t)attempt);
          int32_t cand;
          int64_t wlo = fanout_model ? fen_prefix(&f, lo) : 0;
          int64_t whi = fanout_model ? fen_prefix(&f, hi) : 0;
          if (fanout_model && whi > wlo)
            cand = fen_find(&f, wlo + (int64_t)(x % (uint64_t)(whi - wlo)));
          else
            cand = lo + (int32_t)(x % (uint64_t)(hi - lo));
          int dup = 0;
          for (int q = 0; q < i; ++q) dup |= chosen[q] == cand;
          if (!dup) pick = cand;
        }
        if (pick < 0) {                      /* deterministic scan fallback */
          uint64_t x = draw(seed, S_DUP, ((uint64_t)g << 3) | (uint64_t)i);
          int32_t start = lo + (int32_t)(x % (uint64_t)(hi - lo));
          for (int32_t s = 0; s < hi - lo && pick < 0; ++s) {
            int32_t cand = lo + (start - lo + s) % (hi - lo);
            int dup = 0;
            for (int q = 0; q < i; ++q) dup |= chosen[q] == cand;
            if (!dup) pick = cand;
          }
        }
        if (pick < 0) { free(f.t); free(quota); return -1; }
        chosen[i] = pick;
        if (fanout_model && quota[pick] > 0) {
          quota[pick] -= 1;
          fen_add(&f, pick, -1);
        }
        fanin_net[p++] = pick;
      }
      num_pins[g] = (uint8_t)n;
      lut[g] = (uint16_t)gen_cell_lut(c);
      cell[g] = (uint8_t)c;
      fanin_ptr[g + 1] = (int32_t)p;
    }
    prev_begin = lvl_begin_net;
    prev_end = I + g;
  }
  free(f.t);
  free(quota);
  return p;
}

/*
 * Delay tables.  Each (pin, output edge) IOPATH delay is uniform in
 * [dlo, dhi]; a non-conditional arc repeats it over input edges and side
 * columns.  A conditional arc draws every (input edge, output edge, side)
 * entry independently.  cond_mode 1: pins of XOR2 and MUX2 cells are
 * conditional; cond_mode 2: each (gate, pin) arc is conditional with
 * probability cond_permille/1000.  Side columns beyond 2^(n-1) are 0.
 * Wire delays are uniform in [wlo, whi] per pin and edge.
 */
API void gen_delays(int32_t G, const int32_t* fanin_ptr, const uint8_t* cell,
                    uint64_t seed, int32_t dlo, int32_t dhi, int32_t wlo,
                    int32_t whi, int32_t cond_mode, int32_t cond_permille,
                    int32_t* gate_delay, int32_t* wire_delay) {
  for (int32_t g = 0; g < G; ++g) {
    int n = fanin_ptr[g + 1] - fanin_ptr[g];
    int ncol = 1 << (n - 1);
    for (int i = 0; i < n; ++i) {
      int64_t p = fanin_ptr[g] + i;
      int32_t io[2];
      io[0] = (int32_t)uni(draw(seed, S_IOPATH, (uint64_t)p * 2), dlo, dhi);
      io[1] = (int32_t)uni(draw(seed, S_IOPATH, (uint64_t)p * 2 + 1), dlo, dhi);
      int cond = 0;
      if (cond_mode == 1) cond = cell[g] == C_XOR2 || cell[g] == C_MUX2;
      if (cond_mode == 2) cond = bern(draw(seed, S_CONDSEL, (uint64_t)p), cond_permille);
      int32_t* d = gate_delay + p * 32;
      for (int ie = 0; ie < 2; ++ie)
        for (int oe = 0; oe < 2; ++oe)
          for (int s = 0; s < 8; ++s) {
            int32_t v = 0;
            if (s < ncol)
              v = cond ? (int32_t)uni(draw(seed, S_COND, (uint64_t)p * 32 + ie * 16 + oe * 8 + s), dlo, dhi)
                       : io[oe];
            d[ie * 16 + oe * 8 + s] = v;
          }
      wire_delay[p * 2 + 0] = (int32_t)uni(draw(seed, S_WIRE, (uint64_t)p * 2), wlo, whi);
      wire_delay[p * 2 + 1] = (int32_t)uni(draw(seed, S_WIRE, (uint64_t)p * 2 + 1), wlo, whi);
    }
  }
}

/* Edges of one (input, cycle), sorted, equal times cancelled in pairs. */
static int stim_edges(uint64_t seed, int64_t key, int32_t p_permille,
                      int32_t q_permille, int32_t narrow_permille, int32_t dmin,
                      int32_t out[3]) {
  uint64_t x0 = draw(seed, S_STIM, (uint64_t)key * 8 + 0);
  uint64_t x1 = draw(seed, S_STIM, (uint64_t)key * 8 + 1);
  uint64_t x2 = draw(seed, S_STIM, (uint64_t)key * 8 + 2);
  uint64_t x3 = draw(seed, S_STIM, (uint64_t)key * 8 + 3);
  uint64_t x4 = draw(seed, S_STIM, (uint64_t)key * 8 + 4);
  uint64_t x5 = draw(seed, S_STIM, (uint64_t)key * 8 + 5);
  int32_t e[3];
  int m = 0;
  if (bern(x0, p_permille)) e[m++] = (int32_t)uni(x1, 0, 199);
  if (bern(x2, q_permille)) {
    int32_t s = (int32_t)uni(x3, 0, 199);
    int32_t w;
    if (dmin > 0 && bern(x5, narrow_permille))
      w = (int32_t)uni(x4, 1, dmin > 2 ? dmin - 1 : 1);
    else
      w = (int32_t)uni(x4, 1, 40);
    e[m++] = s;
    e[m++] = s + w;
  }
  /* sort (at most three) */
  for (int a = 1; a < m; ++a)
    for (int b = a; b > 0 && e[b - 1] > e[b]; --b) {
      int32_t t = e[b]; e[b] = e[b - 1]; e[b - 1] = t;
    }
  int k = 0;
  for (int a = 0; a < m; ++a) {
    if (k > 0 && out[k - 1] == e[a]) { --k; continue; }  /* coincident pair */
    out[k++] = e[a];
  }
  return k;
}

/*
 * Stimulus, pass 1: initial values (Bernoulli(0.5) per input) and the CSR
 * pointer edge_ptr[I*C+1], index i*C+c.  Per (input, cycle): a toggle with
 * probability p at a uniform time in [0, 200); a two-edge pulse with
 * probability q starting uniformly in [0, 200) with width uniform in
 * [1, 40], or, with probability narrow/1000 when dmin[i] > 0, width uniform
 * in [1, dmin[i]-1].  dmin may be NULL.  Returns the number of edges.
 */
API int64_t gen_stimulus_count(int32_t I, int32_t C, uint64_t seed,
                               int32_t p_permille, int32_t q_permille,
                               int32_t narrow_permille, const int32_t* dmin,
                               uint8_t* init, int64_t* edge_ptr) {
  int64_t total = 0;
  edge_ptr[0] = 0;
  for (int32_t i = 0; i < I; ++i) {
    init[i] = (uint8_t)(draw(seed, S_INIT, (uint64_t)i) & 1);
    for (int32_t c = 0; c < C; ++c) {
      int32_t tmp[3];
      total += stim_edges(seed, (int64_t)i * C + c, p_permille, q_permille,
                          narrow_permille, dmin ? dmin[i] : 0, tmp);
      edge_ptr[(int64_t)i * C + c + 1] = total;
    }
  }
  return total;
}

/* Stimulus, pass 2: edge times (relative to the cycle start). */
API void gen_stimulus_fill(int32_t I, int32_t C, uint64_t seed,
                           int32_t p_permille, int32_t q_permille,
                           int32_t narrow_permille, const int32_t* dmin,
                           const int64_t* edge_ptr, int32_t* edge_time) {
  for (int32_t i = 0; i < I; ++i)
    for (int32_t c = 0; c < C; ++c) {
      int32_t tmp[3];
      int64_t key = (int64_t)i * C + c;
      int k = stim_edges(seed, key, p_permille, q_permille, narrow_permille,
                         dmin ? dmin[i] : 0, tmp);
      for (int a = 0; a < k; ++a) edge_time[edge_ptr[key] + a] = tmp[a];
    }
}

/* Raw counter-based draw, exposed for Python-side orchestration. */
API uint64_t gen_draw(uint64_t seed, uint64_t stream, uint64_t idx) {
  return draw(seed, stream, idx);
}
