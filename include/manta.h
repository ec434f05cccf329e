/*
 * manta.h -- C ABI of the B300 (sm_103a) microsimulation library.
 *
 * The library runs the per-timestep update of the MANTA traffic
 * microsimulator (Yedavalli, Kumar, Waddell, arXiv 2007.03614, Section II-D):
 * every on-network vehicle looks up its leader in a byte-per-metre lane map
 * ("traffic atlas"), scanning ahead along its precomputed route; applies the
 * Intelligent Driver Model (Eq. 1) with the lane-change rule (Eq. 2) and the
 * gap-acceptance rule (Eqs. 3-4) and the intersection controls of Section
 * II-D (case 1 flashing red, case 2 green) plus fixed-time signals; advances
 * at dt; and writes itself into a double-buffered next-step map.  Departing
 * trips are injected and arrivals retired in the same step.
 *
 * Conventions for every call:
 *  - Status: each call returns a manta_status and sets a thread-local message
 *    readable with manta_last_error().
 *  - Ownership: every input array is caller-owned HOST memory, copied during
 *    the call; the library keeps no caller pointer.  Every output array is
 *    caller-owned host memory of the stated length.
 *  - Device memory: the library allocates and owns all device memory of a
 *    simulation (cudaMalloc); manta_destroy frees it.
 *  - Streams: work is enqueued on the cudaStream_t given to manta_create
 *    (NULL = the legacy default stream).  manta_step returns without waiting;
 *    calls that return data (manta_stats, manta_edge_counters, manta_snapshot,
 *    manta_lane_map) synchronise that stream.
 *  - Device errors: a bounded wait that ran out (grid barrier) or an index
 *    check that failed sets a sticky error word on the device; the next
 *    synchronising call returns MANTA_E_TIMEOUT or MANTA_E_DEVICE and every
 *    later manta_step does nothing.
 *  - Threads: a simulation handle must not be used from two threads at once.
 */
#ifndef MANTA_H
#define MANTA_H

#include <stdint.h>

#if defined(__GNUC__)
#define MANTA_API __attribute__((visibility("default")))
#else
#define MANTA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct manta_sim manta_sim;

typedef enum {
  MANTA_OK = 0,
  MANTA_E_INVALID = -1,   /* bad argument or configuration                       */
  MANTA_E_ROUTE = -2,     /* empty, out-of-range or non-contiguous route          */
  MANTA_E_STATE = -3,     /* call not allowed in the current state                */
  MANTA_E_OOM = -4,       /* device allocation failed                              */
  MANTA_E_CUDA = -5,      /* a CUDA runtime call failed                            */
  MANTA_E_TIMEOUT = -6,   /* a device-side bounded wait ran out                    */
  MANTA_E_DEVICE = -7     /* a device-side index check failed                      */
} manta_status;

/* Node control types (Section II-D "case 1" / "case 2", plus fixed-time signals). */
enum { MANTA_NODE_GREEN = 0, MANTA_NODE_STOP = 1, MANTA_NODE_SIGNAL = 2 };

/* Model configuration.  Lengths in metres (= cells, cell_m must be 1),
 * times in seconds or steps of dt as named.  Defaults: manta_default_config. */
typedef struct {
  float dt;                 /* time step, Section II-D: 0.5 s                                   */
  float cell_m;             /* lane-map cell length t_m, Section II-D: 1 m (only 1 supported)  */
  int32_t veh_len_cells;    /* vehicle length L in cells: 5                                     */
  int32_t horizon_cells;    /* leader-scan horizon H in cells (>= 16): 256                      */
  int32_t n_classes;        /* road classes (1..8); edge_class < n_classes                      */
  float v0f[8];             /* desired speed v0 = speed limit x v0f[class] (Eq. 1): 1           */
  float T[8];               /* time headway T (Eq. 1), s: 1.5                                   */
  float a[8];               /* maximum acceleration a (Eq. 1), m/s^2: 1.0                       */
  float b[8];               /* comfortable deceleration b (Eq. 1), m/s^2: 2.0                   */
  float s0[8];              /* jam distance s0 (Eq. 1), m: 2.0                                  */
  float lc_x0_m;            /* critical distance x0 of Eq. 2: 1 m                               */
  float lc_len_scale_m;     /* length scale of Eq. 2's exponent: 1 m (the literal equation)     */
  float alpha_lo, alpha_hi; /* anticipation-time range of Eqs. 3-4: 0.05, 0.40 s                */
  float g_low, g_high;      /* desired lead/lag gap below / above g_speed_split: 3.0, 7.5 m     */
  float g_speed_split;      /* 25 mph = 11.176 m/s                                              */
  int32_t stop_dwell_steps; /* flashing-red stop before proceeding, Section IV-C: 4 (= 2 s)     */
  float stop_v_eps;         /* speed below which a vehicle counts as stopped: 0.1 m/s           */
  int32_t stats_window_steps; /* per-edge speed statistics window: 600 steps (5 min)            */
  int32_t n_stats_windows;  /* windows kept per edge: 96                                        */
  int32_t idm_textbook;     /* 0: Eq. 1 as printed; 1: s* = s0 + max(0, vT + v dv / 2 sqrt(ab)) */
  int64_t t0_step;          /* absolute step index of the first manta_step (t = t0_step * dt)   */
  uint64_t seed;            /* seed of the counter-based random numbers (Eqs. 2-4)              */
  float speed_sigma_frac;   /* Section IV-B per-driver speed limits: sigma_s / s, the spread of
                               observed speeds at speed limit s as a fraction of s (the paper
                               takes sigma_s from Uber data; this is its synthetic stand-in).
                               A driver's limit on the edge of route entry r is
                               s * max(0.25, 1 + 2 sigma_frac z), z the counter-based normal of
                               (seed, trip id, r, stream 4); v0 = that limit x v0f[class].
                               0 (the default): every driver uses the edge's limit.  0..1.    */
} manta_config;

typedef struct {
  int64_t step;             /* absolute index of the next step to run                  */
  int64_t loaded, departed, arrived, on_network, waiting;
  uint64_t vehicle_updates; /* vehicle-steps updated (one per on-network vehicle and step) */
  uint64_t cells_scanned;   /* lane-map cells examined by leader scans                 */
  uint64_t clamps;          /* updates clamped to the leader's rear / a stop line      */
  uint64_t lane_changes;    /* lane changes applied                                    */
  uint64_t lc_evals;        /* gap-acceptance evaluations (Eqs. 3-4)                   */
  uint64_t route_reads;     /* route entries read by leader scans crossing a node       */
  uint64_t lc_cells_scanned; /* lane-map cells read by the lane-change scans (Section II-D:
                                own-lane leader and target-lane lead for a discretionary
                                change, then the lateral-overlap window, the lead and the
                                lag of the gap acceptance, Eqs. 3-4), each scan counted from
                                its first cell to its hit or its end                         */
} manta_stats_t;

/* Fills *cfg with the defaults listed above. */
MANTA_API void manta_default_config(manta_config *cfg);

/* Builds a simulation on the current CUDA device from a directed road network
 * (Section II-A: edges with lanes, length and speed limit; Section II-D: node
 * control).  Arrays (host memory, copied):
 *   edge_src, edge_dst [n_edges]   node ids in [0, n_nodes)
 *   edge_lanes [n_edges]           1..8
 *   edge_length_m [n_edges]        > 0; the edge gets max(L + ceil(max s0) + 1,
 *                                  round(length / cell_m)) cells (Section II-D)
 *   edge_speed_limit_mps [n_edges] > 0
 *   edge_class [n_edges]           < cfg->n_classes
 *   node_type [n_nodes]            MANTA_NODE_*
 *   node_cycle_steps, node_offset_steps [n_nodes]  signal cycle (1..32767) and
 *                                  offset in steps; read for signal nodes only
 *   edge_green_start, edge_green_len [n_edges]  green window of an in-edge
 *                                  within its head node's cycle: green iff
 *                                  ((k - offset) mod cycle) in [start, start+len)
 *   conn_lane_mask                 NULL = every lane may take every turn; else,
 *                                  for each in-edge e in id order and each
 *                                  out-edge e2 of e's head node in ascending
 *                                  id, a bitmask of e's lanes allowed to
 *                                  continue onto e2 (non-empty)
 *   cuda_stream                    cudaStream_t for all work, or NULL
 * Errors: MANTA_E_INVALID (bad array/config), MANTA_E_OOM, MANTA_E_CUDA.
 * On success *out owns the simulation; release it with manta_destroy. */
MANTA_API manta_status manta_create(int32_t n_nodes, int32_t n_edges, const int32_t *edge_src, const int32_t *edge_dst,
                          const uint8_t *edge_lanes, const float *edge_length_m,
                          const float *edge_speed_limit_mps, const uint8_t *edge_class,
                          const uint8_t *node_type, const int32_t *node_cycle_steps,
                          const int32_t *node_offset_steps, const int16_t *edge_green_start,
                          const int16_t *edge_green_len, const uint32_t *conn_lane_mask,
                          const manta_config *cfg, void *cuda_stream, manta_sim **out);

/* Loads the trips (Section II-C routes, Section II-D departure times), once,
 * before the first manta_step.  Trip i (its vehicle id) follows edges
 * route_edges[route_off[i] .. route_off[i+1]) and may depart at absolute step
 * ceil(depart_time_s[i] / dt) or later (seconds on the same clock as
 * t0_step * dt).  route_off has n_trips + 1 entries, route_off[0] = 0.
 * Departures enter lane 0 of the first edge at x = 0, v = 0.
 * Errors: MANTA_E_ROUTE (empty route, edge out of range, consecutive edges not
 * sharing a node), MANTA_E_INVALID, MANTA_E_STATE (already loaded), MANTA_E_OOM. */
MANTA_API manta_status manta_load_trips(manta_sim *sim, int64_t n_trips, const int64_t *route_off,
                              const int32_t *route_edges, const float *depart_time_s);

/* Incident lane closure: lane `lane` of `edge` is closed during absolute steps
 * [k0, k1) (a later call for the same lane replaces the window).  While
 * closed, the lane holds a stationary obstacle from mid-edge (cell C_e / 2)
 * on, so vehicles behind it stop short of it unless they change lanes (the
 * closure makes that change mandatory, with the Eq. 2 probability taken at the
 * distance to the obstacle); no vehicle changes into the lane, enters it from
 * upstream or departs onto it.  Must be called before manta_load_trips.
 * Errors: MANTA_E_INVALID, MANTA_E_STATE (trips already loaded), MANTA_E_CUDA. */
MANTA_API manta_status manta_set_lane_closure(manta_sim *sim, int32_t edge, int32_t lane, int64_t k0, int64_t k1);

/* Enqueues n_steps >= 0 time steps (Section II-D update) on the stream and
 * returns.  A device error from earlier work is reported here only if it is
 * already known on the host; otherwise at the next synchronising call.
 * Errors: MANTA_E_STATE (no trips loaded or a sticky device error),
 * MANTA_E_CUDA. */
MANTA_API manta_status manta_step(manta_sim *sim, int64_t n_steps);

/* Synchronises the stream and returns the scalar counters: the step clock,
 * trips loaded / departed / arrived / on the network / waiting (Section II-D
 * departures and arrivals), vehicle updates (Section V-B's workload: one per
 * on-network vehicle and step), lane-map cells examined by leader scans
 * (the atlas look-ups of Section II-D), clamps, lane changes and
 * gap-acceptance evaluations (Eqs. 2-4), and route entries read by scans
 * crossing a node. */
MANTA_API manta_status manta_stats(manta_sim *sim, manta_stats_t *out);

/* Synchronises and copies per-edge counters: entries and exits since the
 * start [n_edges], and, for statistics window `window` (window w covers steps
 * t0_step + [w, w+1) * stats_window_steps), the per-edge sum of end-of-step
 * speeds in units of 2^-20 m/s (truncated per vehicle-step) and the number of
 * vehicle-steps (link speeds of Sections IV-A/B).  Any pointer may be NULL. */
MANTA_API manta_status manta_edge_counters(manta_sim *sim, uint32_t *entries, uint32_t *exits, uint64_t *speed_sum_fx,
                                 uint32_t *speed_cnt, int32_t window);

/* Synchronises and copies the on-network vehicles in ascending id into arrays
 * of capacity `cap`: front position in cells from the start of the edge,
 * speed, edge, lane, id, stop dwell counter, position in the route -- the
 * per-vehicle state the update of Section II-D carries from step to step
 * (Eq. 1 position and speed; lane; the Section IV-C stop dwell).  A test and
 * inspection hook.  *n_out receives the count; MANTA_E_INVALID if cap is too
 * small.  Pointers may be NULL. */
MANTA_API manta_status manta_snapshot(manta_sim *sim, int64_t cap, int64_t *n_out, float *x, float *v, int32_t *edge,
                            uint8_t *lane, uint32_t *id, uint8_t *dwell, int32_t *route_pos);

/* Test hook: puts n waiting trips directly on the network, as if each had
 * driven to the stated place, so that a run can start from a dense traffic
 * state instead of an empty network.  The paper has no counterpart (its runs
 * start empty, Section II-D); the hook gives the same state as the same
 * placements in the CPU oracle.  Placement i puts trip trip[i] on route
 * entry route_pos[i] of its route (0 = its first edge), lane lane[i], front
 * position x[i] cells from the start of that edge (0 <= x < cells), speed
 * v[i] >= 0, dwell counter 0; its front cell of the current lane map gets its
 * speed code.  A placed trip leaves its departure queue (the queue's other
 * trips keep their order), counts as departed and adds an entry on its edge.
 * Host arrays [n], copied.  Call once, after manta_load_trips and before the
 * first step.  Errors: MANTA_E_STATE (no trips, already stepped or placed),
 * MANTA_E_INVALID (a trip out of range or listed twice, a route position out
 * of range; or a lane, position or cell not valid -- two placements on one
 * cell, or a cell already taken -- which leaves the simulation unusable),
 * MANTA_E_OOM, MANTA_E_CUDA.  The caller keeps the usual invariant of a lane:
 * front cells at least veh_len_cells apart. */
MANTA_API manta_status manta_place(manta_sim *sim, int64_t n, const int64_t *trip, const int32_t *route_pos,
                                   const uint8_t *lane, const float *x, const float *v);

/* Synchronises and copies the current lane map in canonical layout: edges in
 * id order, lanes in order, one byte per cell (0xFF empty, else the speed code
 * round(8 v) saturated at 254).  *n_out = total bytes; MANTA_E_INVALID if cap
 * is too small. */
MANTA_API manta_status manta_lane_map(manta_sim *sim, uint8_t *out, int64_t cap, int64_t *n_out);

/* Synchronises and returns the cumulative device time, in milliseconds, of
 * the four phases of the step kernel as seen by its first block: [0] lane-
 * change decisions, [1] lane-change apply, [2] leader scans / IDM / map
 * writes, [3] merges, departures and arrivals.  Each includes the wait at
 * the grid barrier that ends it.  A profiling aid. */
MANTA_API manta_status manta_phase_times(manta_sim *sim, double *ms4);

/* ---- launch shapes and autotuning ------------------------------------
 * The step kernel exists in several launch shapes (threads per block,
 * minimum blocks per SM: the second sets the register budget).  Every shape
 * computes the same results bit for bit; only speed differs with the
 * workload.  A new simulation uses shape 0.  (No counterpart in the paper:
 * these concern only how the step kernel is launched.) */
MANTA_API int32_t manta_variant_count(void);
/* Threads per block and minimum blocks per SM of shape v (either pointer may
 * be NULL); MANTA_E_INVALID if v is out of range. */
MANTA_API manta_status manta_variant_info(int32_t v, int32_t *threads, int32_t *min_blocks_per_sm);
/* Selects the shape used by later manta_step calls and graph captures. */
MANTA_API manta_status manta_set_variant(manta_sim *sim, int32_t v);
/* Shape in use, or -1 for NULL. */
MANTA_API int32_t manta_get_variant(const manta_sim *sim);
/* Autotuner: runs `rounds` rounds in which every shape advances the
 * simulation by `trial_steps` steps (in alternating order from round to
 * round), timed with CUDA events on the sim's stream, and selects the shape
 * with the least device time per vehicle update; returns it in *chosen.
 * ms (optional, manta_variant_count() floats) receives each shape's score:
 * milliseconds per million vehicle updates, or milliseconds per round if
 * some shape's trials saw no vehicle.  The simulation really advances by
 * rounds x count x trial_steps steps: tune on the live run, whose results
 * do not depend on the shapes chosen.  Synchronises the stream; device
 * errors are reported as by manta_stats. */
MANTA_API manta_status manta_autotune(manta_sim *sim, int64_t trial_steps, int32_t rounds, int32_t *chosen,
                                      float *ms);

/* ---- CUDA graphs -------------------------------------------------------
 * manta_graph_capture records the launches that advance the simulation by
 * n_steps steps (barrier resets and cooperative step launches, in the shape
 * selected now) into an executable CUDA graph, without running them; the
 * sim must have been created on a non-default stream.  Every
 * manta_graph_launch replays them on the sim's stream, asynchronously, and
 * advances the simulation by n_steps: the kernels take their first step
 * index from device memory, so replays continue where the previous work
 * left off.  Replays and manta_step calls may be mixed.  The graph refers
 * to the simulation and must be destroyed before it.  (No counterpart in
 * the paper.)  Errors: MANTA_E_INVALID for NULL arguments, n_steps < 1 or a
 * sim on the default stream; MANTA_E_STATE before manta_load_trips or after
 * a device error; MANTA_E_CUDA if capture or instantiation fails (nothing
 * was launched then). */
typedef struct manta_graph manta_graph;
MANTA_API manta_status manta_graph_capture(manta_sim *sim, int64_t n_steps, manta_graph **out);
MANTA_API manta_status manta_graph_launch(manta_graph *graph);
/* Releases the graph (NULL is a no-op). */
MANTA_API void manta_graph_destroy(manta_graph *graph);

/* ---- checkpoints ------------------------------------------------------
 * manta_checkpoint_save copies the simulation's whole mutable device state
 * (lane maps, vehicle records, lists, queues, request and stop slots,
 * permits, statistics, control block) into a new device buffer,
 * asynchronously on the sim's stream; manta_checkpoint_restore copies it
 * back, and the run continues from the saved step as if it had never left
 * it (results are bit-identical).  Checkpoints belong to the simulation they
 * were taken from and must be destroyed before it.  They serve the
 * checkpointed adjoint below (re-running segments of a run) and resuming a
 * run; the paper has no counterpart.  Errors: MANTA_E_INVALID for NULL
 * arguments or a checkpoint of another simulation; MANTA_E_STATE before
 * manta_load_trips or after a device error; MANTA_E_OOM if the device
 * buffer cannot be allocated. */
typedef struct manta_checkpoint manta_checkpoint;
MANTA_API manta_status manta_checkpoint_save(manta_sim *sim, manta_checkpoint **out);
MANTA_API manta_status manta_checkpoint_restore(manta_sim *sim, const manta_checkpoint *ckpt);
/* Step index of the saved state, or -1 for NULL. */
MANTA_API int64_t manta_checkpoint_step(const manta_checkpoint *ckpt);
/* Device bytes held by the checkpoint. */
MANTA_API int64_t manta_checkpoint_bytes(const manta_checkpoint *ckpt);
MANTA_API void manta_checkpoint_destroy(manta_checkpoint *ckpt);

/* ---- event tape and adjoint (calibration of Eq. 1's parameters) --------
 * manta_tape_start makes the next n_steps steps (from the current one)
 * record, per trip and step, the continuous state entering the step and
 * the discrete events of it: leader gap and speed (or stop line), the
 * ballistic branch, the clamp, the node outcome (crossed, held, arrived)
 * and the statistics cell of the speed sample taken after it.  The tape
 * holds n_steps x n_trips records of 40 bytes in device memory (reused by
 * later calls); recording stops by itself after n_steps steps, or at
 * manta_tape_stop.  The simulation itself is unchanged by recording.
 *
 * With every event held fixed, the run is a smooth map of the per-class
 * IDM parameters theta = (v0f, T, a, b, s0) for each road class.
 *
 * manta_adjoint: reverse sweep over the recorded segment (all its steps
 * must have been run), with the sim's own parameters.  All pointers are
 * device pointers to binary64 arrays:
 *   seed [n_stats_windows x n_edges]: dLoss/d(one speed sample) of each
 *        statistics cell (window * n_edges + edge), e.g. dLoss/d(mean) / count;
 *   lam_x, lam_v [n_trips]: in, the adjoint of every trip's position and
 *        speed after the segment (zero after the last segment); out, the
 *        adjoint of the state entering it;
 *   grad [5 x n_classes]: dLoss/dtheta is added, index 5 * class + j with j
 *        over (v0f, T, a, b, s0).
 * Asynchronous on the sim's stream.
 *
 * manta_replay: forward replay of the recorded segment with the events held
 * fixed and parameters theta (host, binary64, 5 x n_classes in the order
 * above), for finite differences.  Device arrays: x, v [n_trips] binary64
 * and present [n_trips] (0/1) carry every trip's state into and out of the
 * segment (all zero before the first); sums [n_stats_windows x n_edges]
 * binary64 accumulates the replayed speed of every sample.  Asynchronous on
 * the sim's stream.
 *
 * Both are reproducible bit for bit: the gradient is summed per thread, per
 * block in a fixed tree and over blocks in block order, and replayed speeds
 * are summed exactly in 128-bit fixed point before one rounding to binary64,
 * so no result depends on the order in which GPU threads run.  Each keeps a
 * small device scratch buffer in the simulation, allocated on its first call
 * (the adjoint: 320 bytes per 256 trips; the replay: 16 bytes per statistics
 * cell) and freed by manta_destroy.
 *
 * Both return MANTA_E_STATE when no tape was recorded or its segment has
 * not been run completely, MANTA_E_OOM when the scratch buffer cannot be
 * allocated. */
/* One record of the event tape (40 bytes): index (k - k0) * n_trips + trip
 * for step k of the recorded segment [k0, k0 + n_steps).  flags: bit 0 on
 * the network at the start of the step; bits 1-2 kind (0 free road, 1
 * interacting with gap s and leader speed vL, 2 stopped in place); bit 3
 * v + acc dt >= 0 (else the ballistic step stops the vehicle); bits 4-5
 * clamp (0 none, 1 old position kept, 2 set to bnd); bits 6-8 outcome (0
 * stayed on its edge, 1 crossed the node, 2 held at its old position, 3
 * held at the stop line, 4 arrived); bits 12-15 road class.  sample is the
 * statistics cell (window * n_edges + edge) of the speed sample taken after
 * the step, or 0xFFFFFFFF. */
typedef struct {
  float x, v, s, vL, bnd, lim;
  uint32_t cells, flags, sample, pad;
} manta_tape_record;
MANTA_API manta_status manta_tape_start(manta_sim *sim, int64_t n_steps);
MANTA_API manta_status manta_tape_stop(manta_sim *sim);
/* Copies the recorded segment (n_steps x n_trips records, synchronising the
 * sim's stream) to host memory of capacity `cap` records; *n_out receives
 * the number copied.  MANTA_E_INVALID if cap is too small. */
MANTA_API manta_status manta_tape_copy(manta_sim *sim, manta_tape_record *out, int64_t cap, int64_t *n_out);
MANTA_API manta_status manta_adjoint(manta_sim *sim, const double *seed, double *lam_x, double *lam_v, double *grad);
MANTA_API manta_status manta_replay(manta_sim *sim, const double *theta, double *x, double *v, uint8_t *present,
                                    double *sums);

/* Bytes of the canonical lane map (sum over edges of cells x lanes). */
MANTA_API int64_t manta_lane_map_bytes(const manta_sim *sim);

/* Releases every device and host resource of the simulation (NULL is a no-op). */
MANTA_API void manta_destroy(manta_sim *sim);

/* Message of the last failing call on this thread ("" if none). */
MANTA_API const char *manta_last_error(void);

/* Self-test of the device grid barrier's bounded wait: launches a small
 * cooperative kernel in which one block never arrives, with a wait limit of
 * about `limit_ms` milliseconds; returns MANTA_E_TIMEOUT when every waiting
 * block gave up and returned (the expected outcome), MANTA_OK if the wait
 * did not run out.  The context stays usable. */
MANTA_API manta_status manta_selftest_barrier_timeout(int32_t limit_ms, void *cuda_stream);

/* ---- test hooks for failure detection (no counterpart in the paper) ----
 * 1 if this build of the library checks the indices of the step kernel's
 * device writes (compiled with MANTA_CHECK_BOUNDS), else 0.  In a checked
 * build every write of the step kernel into the lane maps, vehicle records,
 * per-step lists, per-lane slots and statistics is checked against its
 * array's capacity; a failing check skips the write, records the first
 * failing site, and ends the launch at the next grid barrier; the next
 * synchronising call returns MANTA_E_DEVICE (with the site in the message)
 * and the simulation stops, while the CUDA context stays usable.  The
 * product build compiles the checks away. */
MANTA_API int32_t manta_debug_checks(void);
/* Lowers the capacity the checked build allows for writes into a lane-map
 * buffer to `bytes` (the buffers themselves stay as they are), so that a
 * test can make an index check fail on an access that is in bounds.  No
 * effect on a build without checks.  Errors: MANTA_E_INVALID. */
MANTA_API manta_status manta_debug_limit_map(manta_sim *sim, int64_t bytes);
/* Host-side fault injection on the calling thread: from now on, the nth
 * device allocation (kind 0) or the nth host-to-device copy (kind 1) that
 * the library makes fails as the CUDA call would (nth = 0 turns it off).
 * The call that meets the fault returns MANTA_E_OOM or MANTA_E_CUDA;
 * manta_destroy then releases everything allocated so far.
 * Errors: MANTA_E_INVALID for another kind or nth < 0. */
MANTA_API manta_status manta_debug_fail_nth(int32_t kind, int64_t nth);

/* Runs a whole small simulation without allocating any device memory, for
 * callers that cannot call cudaMalloc: host applications whose device memory
 * is wholly reserved by their own pool allocator (a cudaMalloc from a library
 * would fail, or fragment their pool), or real-time loops that must not
 * stall on the driver's allocator.  The paper has no counterpart: it only
 * concerns how device memory is obtained.
 *
 * Arguments are those of manta_create, manta_load_trips (host arrays,
 * copied), the number of steps, and the outputs of manta_stats and
 * manta_snapshot (host arrays of capacity `cap`).  It returns the same
 * results, bit for bit, as manta_create + manta_load_trips + manta_step +
 * manta_stats + manta_snapshot on the same inputs.
 *
 * All device state lives in one static device array of 8 MiB that every GPU
 * loading this library keeps until the process exits (enough for e.g. a
 * 10x10 grid with 1,000 trips).  A network and trip table needing more is
 * rejected with MANTA_E_INVALID and a message naming the limit.  Every call
 * reuses the same array and resets what must start empty; two calls that
 * overlap on the GPU (other threads, other streams) race on it and must not
 * be issued.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the life of the process;
 * a cudaDeviceReset invalidates it, so do not call this function after one.
 * cuda_stream must belong to the current device (MANTA_E_INVALID otherwise).
 *
 * The call uploads its inputs from pageable host memory, synchronises
 * cuda_stream several times and returns only when the results are on the
 * host: issue it outside any stream capture. */
MANTA_API manta_status manta_run_noalloc(
    int32_t n_nodes, int32_t n_edges, const int32_t *edge_src, const int32_t *edge_dst, const uint8_t *edge_lanes,
    const float *edge_length_m, const float *edge_speed_limit_mps, const uint8_t *edge_class,
    const uint8_t *node_type, const int32_t *node_cycle_steps, const int32_t *node_offset_steps,
    const int16_t *edge_green_start, const int16_t *edge_green_len, const uint32_t *conn_lane_mask,
    const manta_config *cfg, int64_t n_trips, const int64_t *route_off, const int32_t *route_edges,
    const float *depart_time_s, int64_t n_steps, void *cuda_stream, manta_stats_t *stats_out, int64_t cap,
    int64_t *n_out, float *x, float *v, int32_t *edge, uint8_t *lane, uint32_t *id, uint8_t *dwell,
    int32_t *route_pos);

#ifdef __cplusplus
}
#endif
#endif /* MANTA_H */
