/*
 * gatspi.h -- C interface of a GB300 (sm_103a) gate-level re-simulator with
 * the delay semantics of GATSPI (Zhang, Ren, Sridharan, Khailany, "GATSPI:
 * GPU Accelerated Gate-Level Simulation for Power Improvement", DAC 2022).
 *
 * What it computes (Section 3, Algorithm 1): input waveforms of the primary
 * and pseudo-primary inputs are given per clock cycle ("re-simulation",
 * Section 1); every combinational gate's output waveform is derived level by
 * level, in parallel over the gates of a level and over independent windows
 * of cycles, with
 *   - cell functions as truth tables Y[colInd], pin 1 = least significant
 *     bit of colInd;
 *   - per-pin interconnect delays [rise, fall] with inertial filtering of
 *     pulses narrower than the delay of their first edge;
 *   - multiple-simultaneous-input switching (all pins arriving at the same
 *     time switch before the output is re-evaluated);
 *   - gate delays read from the switching pin's table, indexed by its edge,
 *     the output edge and the other pins' values (SDF COND);
 *   - gate inertial filtering with PATHPULSEPERCENT = 100 (or other pulse
 *     limits for the gate and interconnect tests, gatspi_opts);
 * and every net is reduced to SAIF figures T0 / T1 / TC (Section 3: the
 * simulator produces SAIF files for power analysis).
 *
 * Conventions
 *   - Nets 0..I-1 are inputs; gate g (0-based) drives net I+g.  Every fanin
 *     net of gate g has a smaller id than I+g (this is how acyclicity is
 *     checked).  Gates need not be sorted by level: the library levelizes.
 *   - Pins of gate g are fanin_ptr[g] .. fanin_ptr[g+1]-1 (pin 1 first),
 *     1 to 4 pins per gate.
 *   - Times are int32 picoseconds.  A window of W cycles is simulated on its
 *     own time axis [0, W*L) starting from the zero-delay settled values of
 *     the inputs' values at the window start; edges that land after W*L are
 *     kept and counted in TC, while T0/T1 integrate only over [0, W*L).
 *   - Values are 0/1 (2-value simulation, Section 2).
 *
 * Ownership and errors
 *   - Host arrays passed in are owned by the caller and copied before the
 *     call returns.  The library owns all device memory it uses.
 *   - Every call returns GATSPI_OK (0) or a negative status; the message of
 *     the last failure is returned by gatspi_last_error().
 *   - A context is bound to one CUDA device and is not thread-safe.
 *   - Calls out of order (for example gatspi_simulate before a netlist, its
 *     delays and a stimulus were loaded) return GATSPI_ESTATE.
 */
#ifndef GATSPI_H
#define GATSPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GATSPI_OK 0
#define GATSPI_EINVAL (-1)    /* bad argument (message says which) */
#define GATSPI_ENOMEM (-2)    /* device or host allocation failed */
#define GATSPI_ECAPACITY (-3) /* waveforms do not fit, even one window per batch */
#define GATSPI_ECUDA (-4)     /* a CUDA call failed */
#define GATSPI_ETIMEOUT (-5)  /* a bounded device-side wait ran out (no kernel waits today) */
#define GATSPI_ESTATE (-6)    /* call out of order */

typedef struct gatspi_ctx gatspi_ctx;

/* Options of one gatspi_simulate call.  Zero means "default" everywhere. */
typedef struct gatspi_opts {
  int32_t window_cycles; /* W: cycles per independent window (default 1) */
  int32_t batch_windows; /* windows resident on the device at once; 0 = all
                            that fit in the arena (halved on overflow) */
  int32_t tile_items;    /* threads per block of the propagation kernel:
                            128, 256 or 512 (0 with items_per_thread 0:
                            autotuned -- every variant is timed on a sample
                            of the stimulus at the first call for a netlist
                            and the fastest is kept; 0 otherwise: 256) */
  int32_t time_kernels;  /* 1 = time every propagation launch with CUDA
                            events on the library's stream (read back with
                            gatspi_get_stats) */
  int32_t items_per_thread; /* consecutive windows of one gate per thread:
                               1, 2, 4 or 8 (at most 4 with 512 threads);
                               0 = autotuned (see tile_items) or 4 */
  int32_t digest;        /* 1 = also reduce every (net, window) waveform to a
                            per-net 64-bit digest (gatspi_digest) */
  int32_t pulse_limits;  /* 1 = the two pulse limits below apply; 0 = both
                            100 percent (Algorithm 1 as printed) */
  int32_t gate_pulse_percent; /* PATHPULSEPERCENT of the gate inertial test
                            (Section 3: Algorithm 1 assumes 100 and other
                            values edit its output test), 0..100: the last
                            kept output edge E is cancelled when
                            100 (t_o - E) < percent * gateDelay or t_o <= E;
                            0 is transport delay */
  int32_t wire_pulse_percent; /* the same for the interconnect test, 0..100:
                            a pulse (t_j, t_j+1) on a pin is dropped when
                            100 (t_j+1 - t_j) < percent * delta(e_j), or when
                            its delayed edges would not stay in order.  With
                            pulse limits the launch shape is 256 threads x 4
                            windows unless tile_items / items_per_thread ask
                            for 256 x 1, 256 x 2 or 128 x 8 (no autotuning) */
  int32_t first_window;  /* simulate windows [first_window, first_window +
                            num_windows) only: a segment of a long stimulus
                            (Section 4: a testbench too long for device
                            memory runs in shorter segments whose results are
                            combined).  Window indices and times stay global,
                            so the SAIF figures (T0, T1, TC) and the digests
                            of consecutive segments add up to those of the
                            whole run, and a run can resume at any window */
  int32_t num_windows;   /* 0 = through the last window */
  int32_t features;      /* 0 = Algorithm 1 with every feature.  The paper's
                            variants without some features, to measure their
                            cost (Section 5, Table "features"), as a mask:
                            GATSPI_NO_INTERCONNECT_FILTER deletes the
                            interconnect inertial test (two consecutive edges
                            of a pin whose delayed arrivals would cross or
                            coincide still cancel as a pair, which keeps
                            every pin's arrivals in time order);
                            GATSPI_PARTIAL_SDF gives every arc one delay per
                            output edge, the mean of its table over all COND
                            columns and both input edges, rounded to the
                            nearest ps (halves up), computed from the delays
                            loaded (a delay edit then shifts it).  Needs pulse
                            limits of 100 / 100; the launch shape is 256
                            threads x 4 windows (or x 1); no cone
                            re-simulation (gatspi_resimulate_edit runs the
                            whole simulation again) */
} gatspi_opts;

#define GATSPI_NO_INTERCONNECT_FILTER 1
#define GATSPI_PARTIAL_SDF 2

/* Figures of the last gatspi_simulate call. */
typedef struct gatspi_stats {
  double prop_ms;          /* summed propagation-kernel time (time_kernels) */
  double input_ms;         /* summed input-restructuring kernel time */
  double wall_ms;          /* host wall time of gatspi_simulate */
  double device_ms;        /* device time from the first to the last kernel
                              of the call, CUDA events (time_kernels) */
  int64_t kernel_launches; /* kernels of this library launched */
  int64_t prop_launches;   /* propagation-kernel launches */
  int64_t items;           /* (gate, window) items simulated */
  int64_t edges;           /* waveform store entries used, all nets and windows: the
                              edge count at 100 percent; with pulse limits it also
                              counts the unused rest of each tile's claim */
  int64_t algo_bytes;      /* algorithmic bytes of the propagation kernels:
                              per (gate, window) item and fanin pin a 2-byte
                              record read, per item a 2-byte record written;
                              per (pin or gate, tile of 32 * items_per_thread
                              windows) an 8-byte tile run read or written
                              (with at least 16 * items_per_thread windows
                              per batch; else a 4-byte start per record);
                              4 bytes per edge read by each fanin pin and per
                              edge written */
  int32_t batches;         /* device batches of windows */
  int32_t windows;         /* windows simulated */
  int32_t batch_windows;   /* windows per batch actually used */
  int32_t levels;          /* logic depth D */
  int32_t tile_threads;    /* launch shape used: threads per block ... */
  int32_t items_per_thread; /* ... and consecutive windows per thread */
} gatspi_stats;

/*
 * Create a context on CUDA device `device`.  `arena_bytes` caps the device
 * memory used for waveforms (0 = 85% of the device memory free now).
 * Errors: EINVAL (bad device), ECUDA.
 */
int gatspi_create(gatspi_ctx** out, int device, size_t arena_bytes);

/* Free every device and host resource of the context (NULL is allowed). */
int gatspi_destroy(gatspi_ctx* ctx);

/* Message of the last failed call on this context ("" if none). */
const char* gatspi_last_error(gatspi_ctx* ctx);

/*
 * Load the combinational netlist (Section 3: the netlist, its levelization
 * and the cell truth tables of Fig. "WaveformLUTSDF").
 *   num_inputs  I >= 1 primary/pseudo-primary inputs (nets 0..I-1)
 *   num_gates   G >= 0
 *   fanin_ptr   int32 [G+1], fanin_ptr[0] = 0, non-decreasing, 1..4 pins/gate
 *   fanin_net   int32 [P = fanin_ptr[G]], fanin_net[p] < I + g for pins of g
 *   lut         uint16 [G], bit k = output for column index k (pin 1 = bit 0)
 * Replaces any previous netlist and drops loaded delays, stimulus and
 * results.  Errors: EINVAL (pin count, net id or cycle), ENOMEM, ECUDA.
 */
int gatspi_load_netlist(gatspi_ctx* ctx, int32_t num_inputs, int32_t num_gates,
                        const int32_t* fanin_ptr, const int32_t* fanin_net,
                        const uint16_t* lut);

/*
 * Load (or replace, for a delay edit) the delays of the loaded netlist
 * (Algorithm 1 inputs delta_i and d_i; SDF IOPATH / COND / INTERCONNECT).
 *   gate_delay  int32 [P][2 inEdge][2 outEdge][8 side]: delay of an output
 *               edge caused by pin p (1 = rising), with `side` the other
 *               pins' values in pin order compressed to n-1 bits; columns
 *               >= 2^(n-1) are ignored
 *   wire_delay  int32 [P][2]: interconnect delay to pin p for a rising /
 *               falling edge of the driving net
 * All used entries must be >= 1 ps.  Errors: ESTATE (no netlist), EINVAL.
 */
int gatspi_load_delays(gatspi_ctx* ctx, const int32_t* gate_delay, const int32_t* wire_delay);

/*
 * Set (n_edits > 0) or clear (n_edits = 0) a delay edit on the loaded
 * delays without reloading them: gate edit_gate[k] (caller numbering) has
 * every gate delay shifted by edit_delta[k] ps, clamped at 1 ps -- the
 * re-timing of a cell resize in a glitch-optimization loop (Section 4).
 * The arrays are copied.  Errors: ESTATE (no delays), EINVAL.
 */
int gatspi_set_edit(gatspi_ctx* ctx, int32_t n_edits, const int32_t* edit_gate,
                    const int32_t* edit_delta);

/*
 * Set the input stimulus: C cycles of L ps.
 *   init       uint8 [I], value of each input at time 0 of cycle 0
 *   edge_ptr   int64 [I*C+1], edges of input i in cycle c are
 *              edge_time[edge_ptr[i*C+c] .. edge_ptr[i*C+c+1])
 *   edge_time  int32, strictly increasing within each (i, c), in [0, L);
 *              each edge toggles the input
 * The stimulus is copied to the device once.  Errors: ESTATE (no netlist),
 * EINVAL (ordering, range), ENOMEM, ECUDA.
 */
int gatspi_set_stimulus(gatspi_ctx* ctx, int32_t num_cycles, int32_t cycle_ps,
                        const uint8_t* init, const int64_t* edge_ptr, const int32_t* edge_time);

/*
 * Set the input stimulus from a raw list of toggles, restructured on the
 * device.  A waveform dump gives each input's changes as (input, time)
 * pairs; cycle-parallel re-simulation needs them grouped per (input, cycle)
 * in time order, relative to the cycle start -- the restructuring the paper
 * does before its simulation kernels and counts in the application time
 * (Sections 3 and 4).  Here the grouping runs on the GPU: a histogram of
 * (input, cycle) buckets, an exclusive scan, a scatter, and a sort of each
 * bucket's times.  The result is the same stimulus gatspi_set_stimulus
 * takes (C cycles of L ps).
 *   init        uint8 [I], value of each input at time 0
 *   num_events  number of toggles (0 is allowed)
 *   ev_input    int32 [num_events], the toggling input, in [0, I)
 *   ev_time     int64 [num_events], ps from the start of cycle 0, in
 *               [0, C*L); the events may come in any order
 * Every event toggles its input.  The arrays are copied.  Errors: ESTATE
 * (no netlist), EINVAL (an input id or a time out of range, an input that
 * toggles twice at the same ps, bad init), ENOMEM, ECUDA.
 */
int gatspi_set_stimulus_events(gatspi_ctx* ctx, int32_t num_cycles, int32_t cycle_ps, const uint8_t* init,
                               int64_t num_events, const int32_t* ev_input, const int64_t* ev_time);

/*
 * Simulate every window (Algorithm 1 for every gate and window, level by
 * level; output storage claimed from the produced edge counts in the
 * same pass, where Section 3 counts, scans and stores in two) and accumulate SAIF.  Synchronous.  `opts` may be NULL.
 * Errors: ESTATE, EINVAL (options, or times that could overflow int32),
 * ECAPACITY, ETIMEOUT, ECUDA.
 */
int gatspi_simulate(gatspi_ctx* ctx, const gatspi_opts* opts);

/* What gatspi_resimulate_edit did. */
typedef struct gatspi_resim_info {
  int32_t mode;        /* 0: no gate's delays changed, nothing ran; 1: only
                          the fanout cone of the changed gates ran; 2: the
                          whole simulation ran again */
  int32_t cone_gates;  /* gates simulated again */
  int32_t first_level; /* lowest level simulated again (0 with mode 0) */
  int32_t levels;      /* levels with a launch */
  int64_t items;       /* (gate, window) items simulated again */
} gatspi_resim_info;

/*
 * Set a delay edit (same arrays and rules as gatspi_set_edit; it replaces
 * the current edit) and bring the last simulation's results up to date --
 * the glitch-optimization loop of Section 4: re-simulate, resize cells,
 * re-simulate.  Only gates whose delays change, and the gates in their
 * fanout cone, can get new waveforms, so when the last gatspi_simulate kept
 * every window in one resident batch (with at least 64 windows: gate-aligned
 * tiles) and nothing else was loaded since, only the cone is simulated again,
 * level by level, reading the other gates' waveforms where they are; the
 * cone's new waveforms go to free arena space after everything stored, and
 * its nets' SAIF (and digest, if the last run made one) is recomputed.
 * Otherwise -- several batches, a stimulus, netlist or delay load since, or
 * too little free arena for the cone -- it runs gatspi_simulate again with the
 * last call's options.  Either way, SAIF, digest and resident waveforms are
 * those of a full gatspi_simulate with the new edit.  Synchronous.
 * gatspi_get_stats afterwards describes the cone's launches (mode 1).
 * `info` may be NULL.  Errors: ESTATE (nothing simulated), EINVAL (edits),
 * and those of gatspi_simulate.
 */
int gatspi_resimulate_edit(gatspi_ctx* ctx, int32_t n_edits, const int32_t* edit_gate,
                           const int32_t* edit_delta, gatspi_resim_info* info);

/*
 * SAIF of the last simulation, per net in the caller's net numbering:
 *   t0, t1  int64 [I+G], time at 0 / 1 in ps summed over windows
 *   tc      int64 [I+G], number of edges (toggle count)
 * Any pointer may be NULL.  Errors: ESTATE (nothing simulated).
 */
int gatspi_saif(gatspi_ctx* ctx, int64_t* t0, int64_t* t1, int64_t* tc);

/*
 * Per-net digest of every waveform of the last gatspi_simulate run with
 * opts.digest = 1 (the check of bit-exactness at scale: one number per net
 * covers all its windows).  For net n and window w (global index) with
 * start value v and edge times t_1..t_c:
 *   h = mix(v + 1);  h = mix(h + 0x9E3779B97F4A7C15 + (uint32)t_k) for k = 1..c;
 *   digest[n] = sum over windows of mix(h ^ mix(w + 1))   (mod 2^64)
 * where mix is the SplitMix64 output function (Steele, Lea, Flood 2014):
 *   z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) *
 *   0x94D049BB133111EB; z ^ z >> 31.
 * The sum is order-free, so windows may be reduced in any order.  out is
 * [I+G] in the caller's net order.  Errors: ESTATE (no digest computed).
 */
int gatspi_digest(gatspi_ctx* ctx, uint64_t* out);

/*
 * Waveforms of every net in window `window` of the last simulation.  Only
 * windows of the last device batch are resident (all windows when they fit
 * in one batch); others return ESTATE.
 *   init   uint8 [I+G]  value at the window start
 *   ptr    int64 [I+G+1] edges of net n are times[ptr[n] .. ptr[n+1])
 *   times  int32 [cap]   window-relative edge times; may be NULL to size it
 *   total  out: number of edges (ptr[I+G])
 * Returns ECAPACITY if cap < total (init and ptr are still filled).
 */
int gatspi_read_window(gatspi_ctx* ctx, int32_t window, uint8_t* init, int64_t* ptr,
                       int32_t* times, int64_t cap, int64_t* total);

/* Figures of the last gatspi_simulate call.  Errors: EINVAL (NULL). */
int gatspi_get_stats(gatspi_ctx* ctx, gatspi_stats* out);


/* ------------------------------------------------------------------------
 * File formats (host only: no context, no device).  The input waveforms of a
 * re-simulation usually come from a VCD dump of an earlier simulation
 * (Section 1: the waveforms of the sequential elements are known), and the
 * results go to power analysis as a SAIF file (Section 3).
 * ---------------------------------------------------------------------- */

/*
 * Read the input waveforms of `num_names` 1-bit signals from a VCD file.
 * names[k] is a signal's reference name or its dot-separated path from the
 * top scope ("top.u1.a"); it must match exactly one 1-bit $var.  A
 * signal's first value, at time 0, is its initial value (init[k]); every
 * time step, time 0 included, whose final value differs from the value
 * before it is a toggle, written as (ev_input = k, ev_time = time in ps) in
 * file (time) order -- the arrays gatspi_set_stimulus_events takes.
 * Several changes of one signal in one time step count only by their final
 * value (a zero-width glitch is no toggle).  Supported:
 * $timescale of 1, 10 or 100 s, ms, us, ns or ps; $scope/$upscope; scalar
 * changes and 1-bit vectors ("b1 id"); $dumpvars, $dumpall and $dumpon
 * blocks (ordinary changes) and $dumpoff blocks (their x values are
 * ignored; the values after $dumpon count as changes at that time).
 * Other x/z values of a requested signal are rejected (2-value
 * simulation, Section 2).
 * `cap` is the size of ev_input / ev_time; *num_events receives the total.
 * Errors: EINVAL (file, syntax, names, x/z, a first value after time 0),
 * ECAPACITY (cap < total: call again with larger arrays).  A message goes
 * to err (err_len bytes, may be NULL).
 */
int gatspi_vcd_read(const char* path, int32_t num_names, const char* const* names, uint8_t* init,
                    int32_t* ev_input, int64_t* ev_time, int64_t cap, int64_t* num_events, char* err,
                    int32_t err_len);

/*
 * Write SAIF (version 2.0, backward, TIMESCALE 1 ps) for `num_nets` nets of
 * one instance `design`: per net T0, T1 and TC as gatspi_saif returns them
 * (TX and IG are 0: 2-value simulation).  Names are written as SAIF
 * identifiers, every character other than a letter, a digit or '_' escaped
 * with a backslash.  Errors: EINVAL (arguments, file).
 */
int gatspi_saif_write(const char* path, const char* design, int64_t duration_ps, int32_t num_nets,
                      const char* const* net_names, const int64_t* t0, const int64_t* t1, const int64_t* tc,
                      char* err, int32_t err_len);

/* ------------------------------------------------------------------------
 * Multi-job engine: batched and served re-simulation.
 *
 * Many jobs (netlist + stimulus + optional delay edit) run together: each
 * job is cut into parts (windows), parts are admitted while their waveform
 * store fits in the engine's device-memory budget, and every step launches
 * one propagation kernel covering the next logic level of every admitted
 * part, whatever its netlist or level (continuous batching).  A part that
 * finishes frees its memory at once, so waiting parts join mid-flight.
 * Each part's results are bit-identical to a plain gatspi_simulate of the
 * same job: parts never share counters or waveform stores.
 * The paper runs one design at a time (Section 3); its glitch-optimization
 * loop (Section 4) re-simulates after delay edits, which is the workload
 * the edits below serve.
 * ---------------------------------------------------------------------- */
typedef struct gatspi_engine gatspi_engine;

typedef struct gatspi_engine_opts {
  int32_t tile_items;  /* threads per block for every launch: 128, 256, 512;
                          0 = 256 */
  int32_t max_active;  /* parts in flight at once; 0 = 1024 */
  int64_t part_items;  /* max (gate, window) items of one part; 0 = 2^30 */
  int32_t items_per_thread; /* 1, 2, 4, 8 (at most 4 with 512 threads);
                               0 = 4 */
  int32_t digest;      /* 1: every job also reduces its waveforms to per-net
                          digests (gatspi_engine_digest); 0 = off */
  int64_t step_items;  /* admission stops while the parts in flight hold
                          this many (gate, window) items per level on
                          average: enough to fill the GPU in one launch,
                          few enough that a step's levels stay in L2;
                          0 = 2^24 */
} gatspi_engine_opts;

typedef struct gatspi_engine_stats {
  int64_t steps;          /* propagation launches (one per step) */
  int64_t kernel_launches;
  int64_t parts_done;
  int64_t parts_retried;  /* parts re-run with a larger waveform store */
  int64_t items;          /* (gate, window) items simulated */
  int64_t bytes_peak;     /* largest device bytes held by admitted parts */
  int32_t active;         /* parts in flight now */
  int32_t queued;         /* parts waiting for admission now */
  double host_ms;         /* host time spent inside gatspi_engine_step */
  double wait_ms;         /* of which blocked waiting for the device */
  double prop_ms;         /* device time of the steps' propagation launches
                             (CUDA events around each step's launches; steps
                             still in flight are counted once they finish) */
} gatspi_engine_stats;

/* Job states reported by gatspi_engine_poll. */
#define GATSPI_JOB_QUEUED 0
#define GATSPI_JOB_RUNNING 1
#define GATSPI_JOB_DONE 2
#define GATSPI_JOB_FAILED 3

/* Create an engine on `device` holding at most `arena_bytes` of waveform
 * stores (0 = 85% of free memory).  `opts` may be NULL.
 * Errors: EINVAL, ECUDA. */
int gatspi_engine_create(gatspi_engine** out, int device, size_t arena_bytes,
                         const gatspi_engine_opts* opts);

/* Wait for the device, then free everything (NULL is allowed). */
int gatspi_engine_destroy(gatspi_engine* eng);

const char* gatspi_engine_last_error(gatspi_engine* eng);

/* Make a netlist and its delays resident (same arrays and rules as
 * gatspi_load_netlist + gatspi_load_delays); *netlist_id receives its id.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int gatspi_engine_add_netlist(gatspi_engine* eng, int32_t num_inputs, int32_t num_gates,
                              const int32_t* fanin_ptr, const int32_t* fanin_net,
                              const uint16_t* lut, const int32_t* gate_delay,
                              const int32_t* wire_delay, int32_t* netlist_id);

/* Queue a job on a resident netlist: a stimulus (same arrays and rules as
 * gatspi_set_stimulus, copied before return), windows of window_cycles
 * cycles (0 = 1), and an optional delay edit scoped to this job: gate
 * edit_gate[k] (caller numbering) has every gate delay shifted by
 * edit_delta[k] ps, clamped at 1 ps (a cell-resize step of a
 * glitch-optimization loop).  *job_id receives the job's id.
 * Errors: EINVAL (ids, stimulus, edits), ENOMEM, ECUDA. */
int gatspi_engine_submit(gatspi_engine* eng, int32_t netlist_id, int32_t num_cycles,
                         int32_t cycle_ps, const uint8_t* init, const int64_t* edge_ptr,
                         const int32_t* edge_time, int32_t window_cycles, int32_t n_edits,
                         const int32_t* edit_gate, const int32_t* edit_delta, int64_t* job_id);

/* One engine step: retire finished parts, admit queued parts that fit, and
 * launch one level of every admitted part.  Returns without waiting for the
 * device except when a retired part's status must be read.  *active and
 * *queued (may be NULL) receive the parts in flight and waiting.
 * Errors: ETIMEOUT, ECAPACITY (a part cannot fit even alone), ECUDA. */
int gatspi_engine_step(gatspi_engine* eng, int32_t* active, int32_t* queued);

/* Step until every queued job is done. */
int gatspi_engine_drain(gatspi_engine* eng);

/* State of a job, and its SAIF when done (t0, t1, tc: int64 [I+G] in the
 * caller's net numbering; any may be NULL).  Errors: EINVAL (unknown id). */
int gatspi_engine_poll(gatspi_engine* eng, int64_t job_id, int32_t* state, int64_t* t0,
                       int64_t* t1, int64_t* tc);

/* Per-net waveform digests of a finished job (uint64 [I+G], caller's net
 * numbering), with the definition of gatspi_digest over all of the job's
 * windows (window indices are the job's own).  The check of bit-exactness
 * at scale for batched and served jobs (Section 4 compares SAIF and
 * spot-checks waveforms).  Needs an engine created with digest = 1.
 * Errors: EINVAL (unknown id, NULL), ESTATE (job not done, or no digests). */
int gatspi_engine_digest(gatspi_engine* eng, int64_t job_id, uint64_t* per_net);

/* Forget a finished job and free its device memory.  Errors: EINVAL,
 * ESTATE (job not finished). */
int gatspi_engine_release(gatspi_engine* eng, int64_t job_id);

int gatspi_engine_get_stats(gatspi_engine* eng, gatspi_engine_stats* out);

/* ------------------------------------------------------------------------
 * Allocation-free level propagation.  (The paper has no counterpart: this
 * is an interface for embedding, not part of the method.)
 *
 * Some callers cannot call cudaMalloc: code whose device memory comes from
 * a framework or pool it does not own, code that must not synchronize the
 * device (allocation and release may), and code that reserved all memory up
 * front and must not fail for lack of it mid-run.  This entry point runs the
 * propagation kernel for ONE logic level of ONE job into buffers the caller
 * allocated, and allocates nothing itself: the kernel's only extra memory
 * (the level's counter of edges allocated and tiles done, and the launch's
 * tile counter) is a fixed array of 32 words (256 bytes) held by every device
 * that loads the library until the process exits.
 *
 * Buffer layout (the one gatspi_simulate uses internally), for a batch of
 * NW = num_windows windows starting at window first_window:
 *   - nets 0..I-1 are inputs, then gates in level order: all gates of level
 *     l are contiguous, gate_begin..gate_end-1 of this call are exactly the
 *     gates of `level` (0-based gate indices), and gate g drives net I+g;
 *     fanin_ptr/fanin_net/lut/gate_delay/wire_delay are as in
 *     gatspi_load_netlist / gatspi_load_delays (fanin nets in this order);
 *     net_level[n] is the level of net n (inputs 0);
 *   - rmeta[n*NW + w] (uint16): bit 15 the value of net n at the start of
 *     window w, bits 0-14 its number of edges in the window;
 *   - where the edges of (n, w) start, relative to lvl_base[level(n)]:
 *     with NW >= 64 the kernel works on tiles of one gate x 128 windows and
 *     tile_info[2*(n*T + t)], tile_info[2*(n*T + t) + 1] (int32, 8-byte
 *     aligned, T =
 *     ceil(NW / 128)) are the first edge and the edge count of tile t of
 *     net n, whose edges are one run in window order, so window w starts at
 *     its tile's first edge plus the counts of the tile's earlier windows
 *     (rstart is unused and may be NULL); with fewer windows, rstart[n*NW +
 *     w] (int32) is the first edge of (n, w) (tile_info may be NULL);
 *   - times[lvl_base[l] + ...] (int32): window-relative edge times,
 *     `capacity` elements in all; lvl_base (int64, D+2 entries).  A level's
 *     tiles may appear in any order inside its range of times;
 *   - saif_t1 / saif_tc (uint64 [N]): time at 1 and toggle count, added to;
 *   - status (int32): error bits are ORed in (1 capacity, 2 wait timeout,
 *     4 corrupt record, 8 offset overflow: a level's edges beyond int32 or
 *     a record beyond 32767 edges); clear it before the first call.
 * The call reads levels < `level` and lvl_base[level]; it writes the records
 * and edges of `level`, lvl_base[level + 1], and the SAIF of its gates.
 *
 * The work is queued on `stream` (NULL = default stream) and not waited
 * for.  The first call on a device looks up the scratch array's device
 * address; make that first call before any stream capture on the device.
 * Every call on a device shares the scratch array, which keeps the last
 * call's contents (each call clears it first): calls that may overlap on
 * the GPU -- on different streams without ordering -- race and give wrong
 * results.  Levels of one job must run in order anyway.
 * Window w of the batch is global window first_window + w, cycles
 * [(first_window + w) * window_cycles, ...) clipped to num_cycles, on its own
 * time axis; first_window + num_windows must not exceed ceil(num_cycles /
 * window_cycles).  Every time is int32 ps: the caller must keep the window
 * length (window_cycles * cycle_ps) plus the longest path delay below 2^31
 * (the window length alone is checked).
 * Errors: EINVAL (null pointer, bad range, windows past the stimulus,
 * window length of 2^31 ps or more), ECAPACITY (more than
 * GATSPI_NOALLOC_MAX_ITEMS (gate, window) items in the level: use fewer
 * windows per call), ECUDA.  A message is written to err/err_len when given.
 * ---------------------------------------------------------------------- */
#define GATSPI_NOALLOC_MAX_ITEMS 2147418112LL /* 0x7fff0000 */

typedef struct gatspi_level_args {
  const int32_t* fanin_ptr;
  const int32_t* fanin_net;
  const uint16_t* lut;
  const int32_t* gate_delay;
  const int32_t* wire_delay;
  const int32_t* net_level;
  int32_t* rstart;
  int32_t* tile_info;
  uint16_t* rmeta;
  int32_t* times;
  int64_t* lvl_base;
  int64_t capacity;
  uint64_t* saif_t1;
  uint64_t* saif_tc;
  int32_t* status;
  int32_t num_inputs;
  int32_t level;
  int32_t gate_begin;
  int32_t gate_end;
  int32_t num_windows;
  int32_t first_window;
  int32_t window_cycles;
  int32_t num_cycles;
  int32_t cycle_ps;
  int32_t err_len;
  char* err;
} gatspi_level_args;

int gatspi_propagate_level_noalloc(const gatspi_level_args* args, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GATSPI_H */
