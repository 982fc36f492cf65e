/*
 * ORACLE -- test infrastructure only.  Only tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code
 * with the GPU library.
 *
 * A plain, slow, event-driven gate-level re-simulator that follows the
 * delay semantics of GATSPI (Zhang et al., DAC'22), Section 3 and
 * Algorithm 1 ("Per-gate, per-cycle parallelism re-simulation"):
 *
 *   - 2-value logic (Section 2: re-simulation for power rarely sees x/z);
 *   - cell function as a truth-table lookup Y[colInd] with pin 1 the least
 *     significant bit of colInd (Algorithm 1, input list and initial value);
 *   - interconnect delay delta_i = [rise, fall] per input pin, chosen by the
 *     direction of the driving edge, with inertial filtering: a pulse
 *     narrower than the delay of its first edge vanishes (Algorithm 1, the
 *     netDelay test inside the next-event search);
 *   - multiple-simultaneous-input switching: every pin whose delayed edge
 *     arrives at the same time switches before the output is re-evaluated
 *     (Algorithm 1, the pin loop after the next event is found);
 *   - the gate delay is read from the switching pin's table d_i, indexed by
 *     that pin's edge, the output edge and the other pins' values (the COND
 *     column) (Algorithm 1; Fig. "WaveformLUTSDF");
 *   - gate inertial filtering with PATHPULSEPERCENT = 100: a new output edge
 *     closer than gateDelay to the last kept output edge cancels that edge
 *     instead of being added (Algorithm 1, output update; Section 3 text).
 *     Other PATHPULSEPERCENT values replace gateDelay in that test by
 *     percent/100 of it, as Section 3 says they may; the same percentage may
 *     be set for the interconnect test (osim_set_pulse, default 100/100).
 *
 * The simulator is structured unlike the level-by-level sweep of the paper:
 * every window is simulated with one global event queue ordered by time.
 * The two inertial rules are stated here in their event form:
 *
 *   wire:  the paper drops the pulse (e_j, e_j+1) when
 *          t_{j+1} - t_j < delta(e_j).  That is exactly "e_j's delayed
 *          arrival t_j + delta(e_j) is still in the future when e_{j+1}
 *          happens", so a net edge at time t cancels the pin's in-flight
 *          arrival if it is later than t, and then schedules nothing.
 *   gate:  the paper cancels the last kept output edge E when
 *          t_o - E < gateDelay with t_o = t + gateDelay, i.e. when E > t:
 *          E has not happened yet.  Equality keeps both edges.
 *
 * With a pulse limit of pct percent (0..100) the tests read
 *   wire:  drop the pair when 100 (t_{j+1} - t_j) < pct delta(e_j), or when
 *          the second edge's delayed arrival would not come after the
 *          first's (a pulse of zero or negative width after the delay);
 *   gate:  cancel E when 100 (t_o - E) < pct gateDelay, or t_o <= E.
 * Either test can only hit an arrival or output edge that is still in the
 * future (the limit never exceeds the delay), so both stay causal.  Below
 * 100 percent several of a pin's arrivals, or of a gate's kept output
 * edges, can be in flight at once: the wire test always concerns the pin's
 * latest edge (and after a drop the next edge is not tested, as the pair
 * scan of Algorithm 1 restarts behind the dropped pair), while the gate test
 * concerns the last kept output edge, and a cancel exposes the one kept
 * before it (a stack: the output pointer moves back by one).  At 100 percent
 * this reduces to the rules above.
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   - a pin whose next edge is its last one is never filtered;
 *   - filtering repeats until the next edge survives (not one skip per
 *     step);
 *   - with several pins switching at once, the highest-index pin selects
 *     the delay table, the side column holds the other pins' values after
 *     the switch, and the row is 2*inEdge + outEdge (1 = rising);
 *   - a window of W cycles starts from the settled (zero-delay) values of
 *     its initial input values, runs on its own time axis [0, W*L), and
 *     keeps edges that land after W*L (counted in TC, not integrated into
 *     T1);
 *   - all delays are at least 1 ps.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define API __attribute__((visibility("default")))
#define NONE (-1)

enum { K_ARRIVAL = 0, K_NETEDGE = 1 };

/* Planted-mistake switches, used only by the test that checks the pins'
   sensitivity.  They exist only in a separate test build compiled with
   OSIM_PLANTED_MISTAKES (liboracle_planted.so); in the oracle itself every
   #ifdef OSIM_PLANTED_MISTAKES block below is compiled out and osim_create
   rejects a mistake number other than 0. */
enum {
  M_NONE = 0,
  M_WIRE_RISE_FALL_SWAPPED = 1,
  M_WIRE_CANCEL_ON_EQUAL = 2,
  M_GATE_CANCEL_ON_EQUAL = 3,
  M_MSI_LOWEST_PIN = 4,
  M_SIDE_BEFORE_SWITCH = 5,
  M_ROW_TRANSPOSED = 6,
  M_T1_UNCLIPPED = 7,
  M_WINDOW_INIT_FROM_CYCLE0 = 8,
  M_NO_WIRE_FILTER = 9,
  M_NO_GATE_FILTER = 10,
  M_OUT_DELAY_FROM_OLD_Y = 11,
  M_GATE_STACK_DEPTH_ONE = 12,
  M_WIRE_CROSSING_KEPT = 13,
  M_SIDE_LOW_BITS = 14
};

typedef struct { uint64_t key; int64_t seq; } event_t;

typedef struct {
  int32_t I, G, N, P, C, L, W, mutation;
  int32_t pulse_gate, pulse_wire;  /* pulse limits, percent of the delay */
  const int32_t *fanin_ptr, *fanin_net, *gate_delay, *wire_delay, *edge_time;
  const int32_t* caller_gate_delay;  /* the table passed in (gate_delay may point at avg_delay) */
  int32_t* avg_delay;                /* arcs averaged over COND columns and input edges, or NULL */
  const uint16_t* lut;
  const uint8_t* init;
  const int64_t* edge_ptr;
  int32_t *gate_of_pin, *fo_ptr, *fo_pin;
  /* window state */
  uint8_t *netval, *pinval, *vs;
  int32_t *arr_time, *last_time;
  int32_t *arr_src, *arr_delay;   /* latest kept edge of each pin: its time, its delay */
  int64_t *arr_seq, *last_seq;
  event_t* heap;
  int64_t heap_n, heap_cap;
  uint8_t* cancelled;   /* per event: 1 cancelled, 2 fired (output edges) */
  int64_t* below;       /* per output-edge event: the gate's kept edge before it */
  int32_t* seq_time;    /* per event: its time */
  int64_t seq_n, seq_cap;
  int32_t *log_net, *log_time;
  int64_t log_n, log_cap;
  /* results of the last window */
  uint8_t* res_init;
  int64_t* res_ptr;
  int32_t* res_times;
  int64_t* res_t1;
  int32_t res_len;   /* simulated time of the window, ps */
  int32_t res_window;
} osim_t;

static int grow(void** p, int64_t* cap, int64_t need, size_t elem) {
  if (need <= *cap) return 0;
  int64_t nc = *cap ? *cap : 1024;
  while (nc < need) nc *= 2;
  void* q = realloc(*p, (size_t)nc * elem);
  if (!q) return -1;
  *p = q;
  *cap = nc;
  return 0;
}

/* At equal times arrivals sort before net edges. */
static int kind_bit(const osim_t* s, int kind) {
#ifdef OSIM_PLANTED_MISTAKES
  if (s->mutation == M_WIRE_CANCEL_ON_EQUAL) return !kind;  /* net edges first */
#endif
  (void)s;
  return kind;
}

static uint64_t mkkey(const osim_t* s, int32_t t, int kind, int32_t id) {
  return ((uint64_t)(uint32_t)t << 33) | ((uint64_t)kind_bit(s, kind) << 32) | (uint32_t)id;
}

static int heap_push(osim_t* s, int32_t t, int kind, int32_t id, int64_t seq) {
  if (grow((void**)&s->heap, &s->heap_cap, s->heap_n + 1, sizeof(event_t))) return -1;
  event_t e = {mkkey(s, t, kind, id), seq};
  int64_t i = s->heap_n++;
  while (i > 0) {
    int64_t par = (i - 1) / 2;
    if (s->heap[par].key < e.key || (s->heap[par].key == e.key && s->heap[par].seq < e.seq)) break;
    s->heap[i] = s->heap[par];
    i = par;
  }
  s->heap[i] = e;
  return 0;
}

static int lt(const event_t* a, const event_t* b) {
  return a->key < b->key || (a->key == b->key && a->seq < b->seq);
}

static event_t heap_pop(osim_t* s) {
  event_t top = s->heap[0];
  event_t last = s->heap[--s->heap_n];
  int64_t i = 0, n = s->heap_n;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    const event_t* best = &last;
    if (l < n && lt(&s->heap[l], best)) { m = l; best = &s->heap[l]; }
    if (r < n && lt(&s->heap[r], best)) { m = r; best = &s->heap[r]; }
    if (m == i) break;
    s->heap[i] = s->heap[m];
    i = m;
  }
  if (n > 0) s->heap[i] = last;
  return top;
}

static int64_t new_seq(osim_t* s, int32_t t) {
  if (s->seq_n + 1 > s->seq_cap) {
    int64_t cap = s->seq_cap;
    if (grow((void**)&s->cancelled, &cap, s->seq_n + 1, 1)) return -1;
    /* the other per-event arrays grow in lockstep */
    void* a = realloc(s->below, sizeof(int64_t) * (size_t)cap);
    if (!a) return -1;
    s->below = (int64_t*)a;
    void* b = realloc(s->seq_time, sizeof(int32_t) * (size_t)cap);
    if (!b) return -1;
    s->seq_time = (int32_t*)b;
    s->seq_cap = cap;
  }
  s->cancelled[s->seq_n] = 0;
  s->below[s->seq_n] = NONE;
  s->seq_time[s->seq_n] = t;
  return s->seq_n++;
}

API void osim_destroy(osim_t* s) {
  if (!s) return;
  free(s->gate_of_pin); free(s->fo_ptr); free(s->fo_pin);
  free(s->netval); free(s->pinval); free(s->vs);
  free(s->arr_time); free(s->last_time); free(s->arr_seq); free(s->last_seq);
  free(s->arr_src); free(s->arr_delay);
  free(s->heap); free(s->cancelled); free(s->below); free(s->seq_time);
  free(s->log_net); free(s->log_time);
  free(s->res_init); free(s->res_ptr); free(s->res_times); free(s->res_t1);
  free(s->avg_delay);
  free(s);
}

/*
 * Create a simulator over caller-owned arrays (they must outlive it):
 * netlist (I inputs, G gates, CSR fanin with fanin_net[p] < I+g for pins of
 * gate g), truth tables, delay tables gate_delay[P][2][2][8] and
 * wire_delay[P][2], stimulus (C cycles of L ps, initial input values and
 * edge lists per (input, cycle)), and the window length W in cycles.
 * Returns NULL on bad arguments.
 */
API osim_t* osim_create(int32_t I, int32_t G, const int32_t* fanin_ptr,
                        const int32_t* fanin_net, const uint16_t* lut,
                        const int32_t* gate_delay, const int32_t* wire_delay,
                        int32_t C, int32_t L, const uint8_t* init,
                        const int64_t* edge_ptr, const int32_t* edge_time,
                        int32_t W, int32_t mutation) {
  if (I < 0 || G < 0 || C < 0 || L < 1 || W < 1) return NULL;
#ifndef OSIM_PLANTED_MISTAKES
  if (mutation != M_NONE) return NULL;
#endif
  osim_t* s = (osim_t*)calloc(1, sizeof(osim_t));
  if (!s) return NULL;
  s->I = I; s->G = G; s->N = I + G; s->C = C; s->L = L; s->W = W;
  s->mutation = mutation;
  s->pulse_gate = 100;
  s->pulse_wire = 100;
  s->fanin_ptr = fanin_ptr; s->fanin_net = fanin_net; s->lut = lut;
  s->gate_delay = gate_delay; s->wire_delay = wire_delay;
  s->caller_gate_delay = gate_delay;
  s->init = init; s->edge_ptr = edge_ptr; s->edge_time = edge_time;
  s->P = G ? fanin_ptr[G] : 0;
  int32_t N = s->N, P = s->P;
  s->gate_of_pin = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
  s->fo_ptr = (int32_t*)calloc((size_t)N + 1, sizeof(int32_t));
  s->fo_pin = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
  s->netval = (uint8_t*)malloc((size_t)N + 1);
  s->pinval = (uint8_t*)malloc((size_t)P + 1);
  s->vs = (uint8_t*)malloc((size_t)G + 1);
  s->arr_time = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
  s->arr_seq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P + 1));
  s->arr_src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
  s->arr_delay = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
  s->last_time = (int32_t*)malloc(sizeof(int32_t) * (size_t)(G + 1));
  s->last_seq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
  s->res_init = (uint8_t*)malloc((size_t)N + 1);
  s->res_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
  s->res_t1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
  if (!s->gate_of_pin || !s->fo_ptr || !s->fo_pin || !s->netval || !s->pinval ||
      !s->vs || !s->arr_time || !s->arr_seq || !s->arr_src || !s->arr_delay || !s->last_time || !s->last_seq ||
      !s->res_init || !s->res_ptr || !s->res_t1) {
    osim_destroy(s);
    return NULL;
  }
  for (int32_t g = 0; g < G; ++g) {
    int32_t n = fanin_ptr[g + 1] - fanin_ptr[g];
    if (n < 1 || n > 4) { osim_destroy(s); return NULL; }
    for (int32_t p = fanin_ptr[g]; p < fanin_ptr[g + 1]; ++p) {
      if (fanin_net[p] < 0 || fanin_net[p] >= I + g) { osim_destroy(s); return NULL; }
      s->gate_of_pin[p] = g;
      s->fo_ptr[fanin_net[p] + 1]++;
    }
  }
  for (int32_t n = 0; n < N; ++n) s->fo_ptr[n + 1] += s->fo_ptr[n];
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N + 1));
  if (!fill) { osim_destroy(s); return NULL; }
  memcpy(fill, s->fo_ptr, sizeof(int32_t) * (size_t)N);
  for (int32_t p = 0; p < P; ++p) s->fo_pin[fill[fanin_net[p]]++] = p;
  free(fill);
  s->res_window = -1;
  return s;
}

/*
 * Pulse limits (PATHPULSEPERCENT) of the gate and interconnect inertial
 * tests, each 0..100 percent of the delay (100 = Algorithm 1 as printed;
 * 0 = transport delay, where only pulses of zero or negative width after
 * the delay vanish).  Returns 0, or -1 for a value out of range.
 */
API int32_t osim_set_pulse(osim_t* s, int32_t gate_percent, int32_t wire_percent) {
  if (gate_percent < 0 || gate_percent > 100 || wire_percent < 0 || wire_percent > 100) return -1;
  s->pulse_gate = gate_percent;
  s->pulse_wire = wire_percent;
  return 0;
}

/*
 * Full SDF delays (1, the default) or the partial-SDF variant of the
 * paper's feature comparison (0; Section 5, Table "features"): every
 * input-pin-to-output arc keeps only an average rise and an average fall
 * delay of the output, each the mean of the arc's delays over all COND
 * columns and both input edges, rounded to the nearest ps (halves up).  The
 * averaged values replace the whole table of the arc, so the simulation
 * itself is unchanged.  Returns 0, or -1 on a bad value or no memory.
 */
API int32_t osim_set_full_sdf(osim_t* s, int32_t full) {
  if (full != 0 && full != 1) return -1;
  if (full) {
    s->gate_delay = s->caller_gate_delay;
    return 0;
  }
  if (!s->avg_delay) {
    s->avg_delay = (int32_t*)malloc(sizeof(int32_t) * 32 * (size_t)(s->P + 1));
    if (!s->avg_delay) return -1;
  }
  for (int32_t g = 0; g < s->G; ++g) {
    const int32_t n = s->fanin_ptr[g + 1] - s->fanin_ptr[g];
    const int32_t ncol = 1 << (n - 1);
    for (int32_t p = s->fanin_ptr[g]; p < s->fanin_ptr[g + 1]; ++p) {
      const int32_t* d = s->caller_gate_delay + (int64_t)p * 32;
      int32_t* a = s->avg_delay + (int64_t)p * 32;
      for (int out_edge = 0; out_edge < 2; ++out_edge) {
        int64_t sum = 0;
        for (int in_edge = 0; in_edge < 2; ++in_edge)
          for (int32_t c = 0; c < ncol; ++c) sum += d[(2 * in_edge + out_edge) * 8 + c];
        const int64_t cnt = 2 * (int64_t)ncol;
        const int32_t avg = (int32_t)((sum + cnt / 2) / cnt);
        for (int in_edge = 0; in_edge < 2; ++in_edge)
          for (int32_t c = 0; c < 8; ++c) a[(2 * in_edge + out_edge) * 8 + c] = avg;
      }
    }
  }
  s->gate_delay = s->avg_delay;
  return 0;
}

API int32_t osim_num_windows(const osim_t* s) {
  return (s->C + s->W - 1) / s->W;
}

/* Column index of gate g from the gate-side pin values (pin 1 = bit 0). */
static uint32_t col_index(const osim_t* s, int32_t g) {
  uint32_t col = 0;
  for (int32_t p = s->fanin_ptr[g]; p < s->fanin_ptr[g + 1]; ++p)
    col |= (uint32_t)s->pinval[p] << (p - s->fanin_ptr[g]);
  return col;
}

/* The other pins' bits of col, with pin i's bit removed. */
static uint32_t side_column(uint32_t col, int i) {
  return (col & ((1u << i) - 1u)) | ((col >> (i + 1)) << i);
}

static int log_edge(osim_t* s, int32_t net, int32_t t) {
  if (s->log_n + 1 > s->log_cap) {
    if (grow((void**)&s->log_net, &s->log_cap, s->log_n + 1, sizeof(int32_t))) return -1;
    /* log_time grows in lockstep with log_net */
    void* q = realloc(s->log_time, sizeof(int32_t) * (size_t)s->log_cap);
    if (!q) return -1;
    s->log_time = (int32_t*)q;
  }
  s->log_net[s->log_n] = net;
  s->log_time[s->log_n] = t;
  s->log_n++;
  return 0;
}

/* A net edge at time t on net n: record it, then update every fanout pin. */
static int net_edge(osim_t* s, int32_t n, int32_t t) {
  s->netval[n] ^= 1;
  if (log_edge(s, n, t)) return -1;
  int rising = s->netval[n];
  for (int32_t k = s->fo_ptr[n]; k < s->fo_ptr[n + 1]; ++k) {
    int32_t p = s->fo_pin[k];
    int32_t delta = rising ? s->wire_delay[2 * p] : s->wire_delay[2 * p + 1];
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_WIRE_RISE_FALL_SWAPPED) delta = rising ? s->wire_delay[2 * p + 1] : s->wire_delay[2 * p];
#endif
    /* the pin's latest edge was kept and its arrival is still ahead */
    int pending = s->arr_seq[p] != NONE && s->arr_time[p] > t;
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_WIRE_CANCEL_ON_EQUAL) pending = s->arr_seq[p] != NONE && s->arr_time[p] >= t;
    if (s->mutation == M_NO_WIRE_FILTER) pending = 0;
#endif
    int drop = 0;
    if (pending) {
      /* the pulse (latest edge, this edge) is narrower than the limit, or
         would arrive with zero or negative width; at 100 percent every
         pending arrival qualifies, since pending means t - t_prev < delta */
      int64_t width = (int64_t)t - s->arr_src[p];
      int crossed = (int64_t)t + delta <= s->arr_time[p];
#ifdef OSIM_PLANTED_MISTAKES
      if (s->mutation == M_WIRE_CROSSING_KEPT) crossed = 0;
#endif
      drop = 100 * width < (int64_t)s->pulse_wire * s->arr_delay[p] || crossed;
#ifdef OSIM_PLANTED_MISTAKES
      if (s->mutation == M_WIRE_CANCEL_ON_EQUAL) drop = 1;
#endif
    }
    if (drop) {
      /* the pulse vanishes: cancel the earlier edge's arrival, schedule
         nothing, and leave the next edge untested */
      s->cancelled[s->arr_seq[p]] = 1;
      s->arr_seq[p] = NONE;
    } else {
      int64_t q = new_seq(s, t + delta);
      if (q < 0 || heap_push(s, t + delta, K_ARRIVAL, p, q)) return -1;
      s->arr_seq[p] = q;
      s->arr_time[p] = t + delta;
      s->arr_src[p] = t;
      s->arr_delay[p] = delta;
    }
  }
  return 0;
}

/* All arrivals at gate g at time t have been applied; re-evaluate. */
static int gate_eval(osim_t* s, int32_t g, int32_t t, int istar, uint32_t col_before) {
  uint32_t col = col_index(s, g);
  int y = (s->lut[g] >> col) & 1;
  if (y == s->vs[g]) return 0;
  /* delay of the new output edge: the switching pin's arc */
  int32_t p = s->fanin_ptr[g] + istar;
  int in_edge = s->pinval[p];
  int out_edge = y;
  uint32_t side = side_column(col, istar);
  int row = 2 * in_edge + out_edge;
#ifdef OSIM_PLANTED_MISTAKES
  if (s->mutation == M_OUT_DELAY_FROM_OLD_Y) row = 2 * in_edge + s->vs[g];
  if (s->mutation == M_SIDE_BEFORE_SWITCH) side = side_column(col_before, istar);
  if (s->mutation == M_SIDE_LOW_BITS) side = col & ((1u << (s->fanin_ptr[g + 1] - s->fanin_ptr[g] - 1)) - 1u);
  if (s->mutation == M_ROW_TRANSPOSED) row = 2 * out_edge + in_edge;
#else
  (void)col_before;
#endif
  int32_t d = s->gate_delay[(int64_t)p * 32 + row * 8 + side];
  int64_t top = s->last_seq[g];
  int cancel = 0;
  if (top != NONE) {
    /* the last kept output edge E is still ahead (kept edges that fired
       have left the stack) */
    int64_t E = s->last_time[g];
    int64_t to = (int64_t)t + d;
    cancel = 100 * (to - E) < (int64_t)s->pulse_gate * d || to <= E;
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_GATE_CANCEL_ON_EQUAL) cancel = E >= t;
#endif
  }
#ifdef OSIM_PLANTED_MISTAKES
  if (s->mutation == M_NO_GATE_FILTER) cancel = 0;
#endif
  if (cancel) {
    /* the new edge would come too soon after E: cancel E instead, and the
       kept edge before it (if still ahead) becomes the last kept one */
    s->cancelled[top] = 1;
    int64_t b = s->below[top];
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_GATE_STACK_DEPTH_ONE) b = NONE;
#endif
    if (b != NONE && s->cancelled[b] == 0) {
      s->last_seq[g] = b;
      s->last_time[g] = s->seq_time[b];
    } else {
      s->last_seq[g] = NONE;
    }
  } else {
    int64_t q = new_seq(s, t + d);
    if (q < 0 || heap_push(s, t + d, K_NETEDGE, s->I + g, q)) return -1;
    s->below[q] = top;
    s->last_seq[g] = q;
    s->last_time[g] = t + d;
  }
  s->vs[g] = (uint8_t)y;
  return 0;
}

/*
 * Simulate window w (cycles [w*W, min((w+1)*W, C))).  Returns the number of
 * edges recorded over all nets, or -1 on error.  Results are kept until the
 * next call and read with osim_get / osim_t1.
 */
API int64_t osim_run_window(osim_t* s, int32_t w) {
  int32_t I = s->I, G = s->G, N = s->N;
  int32_t c0 = w * s->W, c1 = c0 + s->W;
  if (w < 0 || c0 >= s->C) return -1;
  if (c1 > s->C) c1 = s->C;
  s->heap_n = 0; s->seq_n = 0; s->log_n = 0;
  /* initial (settled) values: inputs from the stimulus, gates by zero-delay
     evaluation in net order (fanins always have lower ids) */
  for (int32_t i = 0; i < I; ++i) {
    int64_t before = s->edge_ptr[(int64_t)i * s->C + c0] - s->edge_ptr[(int64_t)i * s->C];
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_WINDOW_INIT_FROM_CYCLE0) before = 0;
#endif
    s->netval[i] = (uint8_t)(s->init[i] ^ (before & 1));
  }
  for (int32_t g = 0; g < G; ++g) {
    for (int32_t p = s->fanin_ptr[g]; p < s->fanin_ptr[g + 1]; ++p) {
      s->pinval[p] = s->netval[s->fanin_net[p]];
      s->arr_seq[p] = NONE;
    }
    s->netval[I + g] = (uint8_t)((s->lut[g] >> col_index(s, g)) & 1);
    s->vs[g] = s->netval[I + g];
    s->last_seq[g] = NONE;
    s->last_time[g] = 0;
  }
  memcpy(s->res_init, s->netval, (size_t)N);
  /* input edges on the window's time axis */
  for (int32_t i = 0; i < I; ++i)
    for (int32_t c = c0; c < c1; ++c) {
      int64_t a = s->edge_ptr[(int64_t)i * s->C + c], b = s->edge_ptr[(int64_t)i * s->C + c + 1];
      for (int64_t e = a; e < b; ++e) {
        int32_t te = (c - c0) * s->L + s->edge_time[e];
        int64_t q = new_seq(s, te);
        if (q < 0 || heap_push(s, te, K_NETEDGE, i, q)) return -1;
      }
    }
  /* event loop: at equal times arrivals come before net edges (key order) */
  while (s->heap_n > 0) {
    event_t e = heap_pop(s);
    if (s->cancelled[e.seq]) continue;
    int32_t t = (int32_t)(e.key >> 33);
    int kind = kind_bit(s, (int)((e.key >> 32) & 1));
    int32_t id = (int32_t)(e.key & 0xffffffffu);
    if (kind == K_NETEDGE) {
      /* a gate's output edge fires: it is the oldest of its kept edges
         still ahead, so it leaves the bottom of the gate's stack */
      s->cancelled[e.seq] = 2;
      if (id >= I && s->last_seq[id - I] == e.seq) s->last_seq[id - I] = NONE;
      if (net_edge(s, id, t)) return -1;
      continue;
    }
    /* gather every arrival at this gate at this time (pins of one gate are
       contiguous, and the key orders them by pin) */
    int32_t g = s->gate_of_pin[id];
    uint32_t col_before = col_index(s, g);
    int istar = -1, ilow = 99;
    event_t cur = e;
    for (;;) {
      int32_t p = (int32_t)(cur.key & 0xffffffffu);
      if (!s->cancelled[cur.seq]) {
        int i = p - s->fanin_ptr[g];
        s->pinval[p] ^= 1;
        if (s->arr_seq[p] == cur.seq) s->arr_seq[p] = NONE;
        if (i > istar) istar = i;
        if (i < ilow) ilow = i;
      }
      if (s->heap_n == 0) break;
      const event_t* nx = &s->heap[0];
      if ((int32_t)(nx->key >> 33) != t || kind_bit(s, (int)((nx->key >> 32) & 1)) != K_ARRIVAL) break;
      if (s->gate_of_pin[(int32_t)(nx->key & 0xffffffffu)] != g) break;
      cur = heap_pop(s);
    }
#ifdef OSIM_PLANTED_MISTAKES
    if (s->mutation == M_MSI_LOWEST_PIN) istar = ilow;
#else
    (void)ilow;
#endif
    if (gate_eval(s, g, t, istar, col_before)) return -1;
  }
  /* group the time-ordered log by net (stable counting sort) */
  memset(s->res_ptr, 0, sizeof(int64_t) * (size_t)(N + 1));
  for (int64_t k = 0; k < s->log_n; ++k) s->res_ptr[s->log_net[k] + 1]++;
  for (int32_t n = 0; n < N; ++n) s->res_ptr[n + 1] += s->res_ptr[n];
  free(s->res_times);
  s->res_times = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->log_n + 1));
  if (!s->res_times) return -1;
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
  if (!fill) return -1;
  memcpy(fill, s->res_ptr, sizeof(int64_t) * (size_t)(N + 1));
  for (int64_t k = 0; k < s->log_n; ++k) s->res_times[fill[s->log_net[k]]++] = s->log_time[k];
  free(fill);
  /* T1 over [0, len): time at value 1 */
  s->res_len = (c1 - c0) * s->L;
  for (int32_t n = 0; n < N; ++n) {
    int v = s->res_init[n];
    int64_t t1 = 0, prev = 0;
    for (int64_t k = s->res_ptr[n]; k < s->res_ptr[n + 1]; ++k) {
      int64_t t = s->res_times[k];
      if (t > s->res_len) t = s->res_len;
#ifdef OSIM_PLANTED_MISTAKES
      if (s->mutation == M_T1_UNCLIPPED) t = s->res_times[k];
#endif
      if (v) t1 += t - prev;
      prev = t;
      v ^= 1;
    }
    if (v && prev < s->res_len) t1 += s->res_len - prev;
    s->res_t1[n] = t1;
  }
  s->res_window = w;
  return s->log_n;
}

/* Copy the last window's waveforms: init[N], ptr[N+1], times[ptr[N]]. */
API void osim_get(const osim_t* s, uint8_t* init, int64_t* ptr, int32_t* times) {
  memcpy(init, s->res_init, (size_t)s->N);
  memcpy(ptr, s->res_ptr, sizeof(int64_t) * (size_t)(s->N + 1));
  if (s->res_ptr[s->N] > 0) memcpy(times, s->res_times, sizeof(int32_t) * (size_t)s->res_ptr[s->N]);
}

/* Last window's per-net time at 1 (T1) and its length in ps. */
API int32_t osim_t1(const osim_t* s, int64_t* t1) {
  memcpy(t1, s->res_t1, sizeof(int64_t) * (size_t)s->N);
  return s->res_len;
}

/*
 * SAIF over windows [w0, w1): T1 and TC per net summed over the windows
 * (T0 = simulated time - T1).  Returns the simulated time, or -1.
 */
API int64_t osim_saif(osim_t* s, int32_t w0, int32_t w1, int64_t* t1, int64_t* tc) {
  memset(t1, 0, sizeof(int64_t) * (size_t)s->N);
  memset(tc, 0, sizeof(int64_t) * (size_t)s->N);
  int64_t total = 0;
  for (int32_t w = w0; w < w1; ++w) {
    if (osim_run_window(s, w) < 0) return -1;
    for (int32_t n = 0; n < s->N; ++n) {
      t1[n] += s->res_t1[n];
      tc[n] += s->res_ptr[n + 1] - s->res_ptr[n];
    }
    total += s->res_len;
  }
  return total;
}
