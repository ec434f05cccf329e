/*
 * manta_oracle.c -- plain, slow, single-threaded CPU oracle of the MANTA
 * per-timestep microsimulation update (arXiv 2007.03614, Section II-D).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the two meet
 * only in the seeded input generators and in the numbers they print.
 *
 * Arithmetic: strict IEEE binary32 for every quantity the paper's model
 * computes (compiled with -ffp-contract=off -fno-fast-math, SSE2), so that
 * every float operation is one correctly rounded binary op.  No
 * transcendental function is evaluated on the per-step path; the Eq. 2
 * probability table is computed once on the host in double.
 *
 * What it computes, per step k (every phase reads only what earlier phases
 * wrote; no result depends on the order vehicles are visited):
 *
 *  A. Lane-change decision on the lane map M_k        (Section II-D, Eqs. 2-4)
 *  B. Lane-change apply, in place: M_k -> M_k'        (Section II-D)
 *  C. Departure requests: queue heads due by step k whose entry cells on
 *     lane 0 are free in M_k'                        (Section II-D departures; Section II-D case 2 capacity)
 *  D. Leader scan along the route on M_k' (lane-map lookup of neighbouring
 *     cells), IDM acceleration (Eq. 1, delta = 4) with the driver's own
 *     speed limit on the edge (Section IV-B, off unless speed_sigma_frac > 0),
 *     ballistic "double integration" at dt, clamp behind the leader
 *                                                   (Section II-D, Eq. 1)
 *  E. Merge resolution: per target lane the lowest vehicle id among crossing
 *     and departure requests wins                      (Section II-D capacity rule)
 *  F. Apply outcomes: crossings, held vehicles, departures, arrivals
 *  G. Next lane map M_{k+1}: one byte per vehicle at its front cell holding
 *     its speed code; every other byte empty        (Section II-D traffic atlas)
 *  H. Statistics: counters, per-edge entries/exits, per-edge speed sums in
 *     fixed windows                                     (Section IV-A/B link speeds)
 *  I. Flashing-red (stop) permits for step k+1: round robin over in-lanes,
 *     2 s stop first                                (Section II-D case 1, Section IV-C)
 *
 * Pins (tests/): free-flow lone vehicle vs the IDM ODE closed form and vs a
 * float64 replay; ring-road equilibrium vs the IDM steady-state relation;
 * conservation; no-overlap / per-lane FIFO; hand-traced merge, signal, stop
 * and lane-change cases; a naive list-based implementation on tiny
 * networks; SplitMix64 reference outputs; the moments of the per-driver
 * limits and a lone driver's terminal speed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#include <math.h>

#define OR_API __attribute__((visibility("default")))

#define EMPTY 0xFFu
#define NODE_GREEN 0
#define NODE_STOP 1
#define NODE_SIGNAL 2
#define NONE_ID 0xFFFFFFFFu

typedef struct {
  float dt, cell_m;
  int32_t veh_len_cells, horizon_cells, n_classes;
  float v0f[8], T[8], a[8], b[8], s0[8];
  float lc_x0_m, lc_len_scale_m;
  float alpha_lo, alpha_hi;
  float g_low, g_high, g_speed_split;
  int32_t stop_dwell_steps;
  float stop_v_eps;
  int32_t stats_window_steps, n_stats_windows;
  int32_t idm_textbook;
  int64_t t0_step;
  uint64_t seed;
  float speed_sigma_frac;
} oracle_config;

typedef struct {
  int64_t step, loaded, departed, arrived, on_network, waiting;
  uint64_t vehicle_updates, cells_scanned, clamps, lane_changes, lc_evals, route_reads;
  uint64_t lc_cells_scanned;   /* lane-map cells read by the lane-change scans (step 3) */
} oracle_stats_t;

typedef struct {
  int32_t e, l;            /* edge, lane                                  */
  float x, v;              /* front bumper position in cells, speed m/s   */
  int64_t r;               /* index into route_edges of the current edge  */
  uint8_t dwell;           /* consecutive stopped steps at a stop line    */
  uint8_t status;          /* 0 waiting, 1 on network, 2 arrived          */
} veh_t;

typedef struct {
  oracle_config cfg;
  int32_t N, E;
  int32_t *src, *dst, *C, *nl, *cls;
  float *lim;
  uint8_t *ntype; int32_t *ncyc, *noff; int16_t *gs, *gl;
  int64_t *lane_base;       /* first lane index of each edge                */
  int64_t n_lanes;
  int64_t *row_off;         /* byte offset of lane 0 of each edge in a map  */
  int64_t map_bytes;
  uint8_t *map_cur, *map_nxt;
  int64_t *out_off; int32_t *out_e;         /* out-edges per node, ascending id */
  int64_t *conn_off; uint32_t *conn;       /* lane masks per (in, out) pair    */
  int64_t *inl_off; int64_t *inl;          /* in-lanes of each node, (edge, lane) order */
  uint32_t *permit; int32_t *rr;
  int64_t *clo_k0, *clo_k1;                /* closure window [k0, k1) of each lane, empty if k0 >= k1 */
  int stepped;
  float *mtab; int32_t mtab_n;             /* Eq. 2 probability by distance in cells */
  /* trips */
  int64_t NT;
  int64_t *route_off; int32_t *route; uint8_t *rmask;
  int64_t *dstep;
  veh_t *V;
  int64_t *q_off, *q_trip, *q_head;       /* departure queues per first edge   */
  int64_t *on; int64_t n_on;               /* on-network trip ids               */
  int loaded;
  int64_t k;
  oracle_stats_t st;
  uint32_t *entry, *exitc;
  uint64_t *ssum; uint32_t *scnt;
  /* scratch */
  int32_t *lc_tgt;
  uint32_t *best;
  /* optional event tape of steps [tp_k0, tp_k0 + tp_len), arrays [step][trip]
   * owned by the caller: the state entering each step and the events of it
   * (see oracle_set_tape) */
  int64_t tp_k0, tp_len;
  float *tp_x, *tp_v, *tp_s, *tp_vL, *tp_bnd, *tp_lim;
  int32_t *tp_C, *tp_flags;
  int64_t *tp_sample;
} osim;

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 (Steele, Lea, Flood 2014) applied
 * to a key built from (seed, vehicle id, step, stream).                     */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t rkey(uint64_t seed, uint64_t id, int64_t k, uint64_t stream) {
  return splitmix64(seed ^ (id * 0x9E3779B97F4A7C15ULL) ^ ((uint64_t)k * 0xC2B2AE3D27D4EB4FULL) ^ stream);
}
/* Uniform on [0,1): the top 24 bits scaled by 2^-24 (exact in binary32). */
static float rng_u(uint64_t seed, uint64_t id, int64_t k, uint64_t stream) {
  return (float)(uint32_t)(rkey(seed, id, k, stream) >> 40) * 5.9604644775390625e-8f;
}
/* Standard normal approximated by the Irwin-Hall sum of twelve uniforms,
 * summed exactly in integers, centred, converted once and scaled by 2^-24.  */
static float rng_n(uint64_t seed, uint64_t id, int64_t k, uint64_t s) {
  int32_t acc = 0;
  for (uint64_t j = 0; j < 12; ++j) acc += (int32_t)(uint32_t)(rkey(seed, id, k, 16 * s + j) >> 40);
  return (float)(acc - 100663296) * 5.9604644775390625e-8f;
}

OR_API uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }
OR_API float oracle_rng_u(uint64_t seed, uint64_t id, int64_t k, uint64_t stream) { return rng_u(seed, id, k, stream); }
OR_API float oracle_rng_n(uint64_t seed, uint64_t id, int64_t k, uint64_t s) { return rng_n(seed, id, k, s); }

/* Speed byte of the lane map: 1/8 m/s resolution, rounded, saturating at 254. */
static uint8_t speed_code(float v) {
  int c = (int)(v * 8.0f + 0.5f);
  return (uint8_t)(c > 254 ? 254 : c);
}
static float speed_decode(uint8_t c) { return (float)c * 0.125f; }

static uint8_t *row(osim *S, uint8_t *map, int32_t e, int32_t l) { return map + S->row_off[e] + (int64_t)l * S->C[e]; }

static int is_green(const osim *S, int32_t e, int64_t k) {
  int32_t n = S->dst[e];
  if (S->ntype[n] != NODE_SIGNAL) return 1;
  int64_t cyc = S->ncyc[n];
  int64_t m = (k - (int64_t)S->noff[n]) % cyc;
  if (m < 0) m += cyc;
  return m >= S->gs[e] && m < (int64_t)S->gs[e] + S->gl[e];
}

/* Incident lane closure: lane l of edge e is closed at step k; from mid-edge
 * (cell C_e / 2) on it holds a stationary obstacle. */
/* Section IV-B: a driver's own speed limit on the edge of route entry r.  The
 * paper samples each driver's maximum speed per edge from a normal law around
 * the edge's limit s with standard deviation 2 sigma_s; here sigma_s is
 * speed_sigma_frac x s (the paper's sigma_s comes from Uber data), the
 * normal draw is stream 4 of the trip's numbers keyed by r, and the result is
 * floored at s / 4.  With speed_sigma_frac = 0 every driver uses s.        */
static float driver_limit(const osim *S, int32_t e, int64_t id, int64_t r) {
  const float s = S->lim[e];
  const float f = S->cfg.speed_sigma_frac;
  if (!(f > 0.0f)) return s;
  const float z = rng_n(S->cfg.seed, (uint64_t)id, r, 4);
  float q = 1.0f + (2.0f * f) * z;
  if (q < 0.25f) q = 0.25f;
  return s * q;
}

static int lane_closed(const osim *S, int32_t e, int32_t l, int64_t k) {
  int64_t g = S->lane_base[e] + l;
  return S->clo_k0[g] <= k && k < S->clo_k1[g];
}

static void set_err(char *err, int errlen, const char *msg) {
  if (err && errlen > 0) { strncpy(err, msg, (size_t)errlen - 1); err[errlen - 1] = 0; }
}

OR_API void oracle_destroy(osim *S) {
  if (!S) return;
  free(S->src); free(S->dst); free(S->C); free(S->nl); free(S->cls); free(S->lim);
  free(S->ntype); free(S->ncyc); free(S->noff); free(S->gs); free(S->gl);
  free(S->lane_base); free(S->row_off); free(S->map_cur); free(S->map_nxt);
  free(S->out_off); free(S->out_e); free(S->conn_off); free(S->conn);
  free(S->inl_off); free(S->inl); free(S->permit); free(S->rr); free(S->mtab);
  free(S->clo_k0); free(S->clo_k1);
  free(S->route_off); free(S->route); free(S->rmask); free(S->dstep); free(S->V);
  free(S->q_off); free(S->q_trip); free(S->q_head); free(S->on);
  free(S->entry); free(S->exitc); free(S->ssum); free(S->scnt); free(S->lc_tgt); free(S->best);
  free(S);
}

/* Build the simulation from the network arrays (Section II-A: directed edges
 * with lanes, length and speed limit; node control per Section II-D).       */
OR_API osim *oracle_create(int32_t n_nodes, int32_t n_edges, const int32_t *edge_src, const int32_t *edge_dst,
                           const uint8_t *edge_lanes, const float *edge_length_m, const float *edge_speed,
                           const uint8_t *edge_class, const uint8_t *node_type, const int32_t *node_cycle,
                           const int32_t *node_offset, const int16_t *green_start, const int16_t *green_len,
                           const uint32_t *conn_lane_mask, const oracle_config *cfg, char *err, int errlen) {
  if (!cfg || n_nodes <= 0 || n_edges <= 0 || !edge_src || !edge_dst || !edge_lanes || !edge_length_m ||
      !edge_speed || !edge_class || !node_type) { set_err(err, errlen, "null or empty input"); return NULL; }
  if (cfg->cell_m != 1.0f || !(cfg->dt > 0.0f) || cfg->veh_len_cells < 1 || cfg->horizon_cells < 16 ||
      cfg->n_classes < 1 || cfg->n_classes > 8 || cfg->stats_window_steps < 1 || cfg->n_stats_windows < 1) {
    set_err(err, errlen, "bad config"); return NULL;
  }
  osim *S = (osim *)calloc(1, sizeof(osim));
  S->cfg = *cfg; S->N = n_nodes; S->E = n_edges;
  const int32_t N = n_nodes, E = n_edges, L = cfg->veh_len_cells;
  S->src = malloc(4 * (size_t)E); S->dst = malloc(4 * (size_t)E); S->C = malloc(4 * (size_t)E);
  S->nl = malloc(4 * (size_t)E); S->cls = malloc(4 * (size_t)E); S->lim = malloc(4 * (size_t)E);
  S->gs = calloc((size_t)E, 2); S->gl = calloc((size_t)E, 2);
  S->ntype = malloc((size_t)N); S->ncyc = calloc((size_t)N, 4); S->noff = calloc((size_t)N, 4);
  float s0max = 0.0f;
  for (int c = 0; c < cfg->n_classes; ++c) {
    if (!(cfg->a[c] > 0.0f) || !(cfg->b[c] > 0.0f) || !(cfg->T[c] >= 0.0f) || !(cfg->s0[c] >= 0.0f) || !(cfg->v0f[c] > 0.0f)) {
      set_err(err, errlen, "bad class parameters"); oracle_destroy(S); return NULL;
    }
    if (cfg->s0[c] > s0max) s0max = cfg->s0[c];
  }
  if (!(cfg->speed_sigma_frac >= 0.0f) || !(cfg->speed_sigma_frac <= 1.0f)) {
    set_err(err, errlen, "speed_sigma_frac out of range"); oracle_destroy(S); return NULL;
  }
  const int32_t cmin = L + (int32_t)ceilf(s0max) + 1;
  for (int32_t n = 0; n < N; ++n) {
    if (node_type[n] > 2) { set_err(err, errlen, "bad node type"); oracle_destroy(S); return NULL; }
    S->ntype[n] = node_type[n];
    if (node_type[n] == NODE_SIGNAL) {
      if (!node_cycle || !node_offset || node_cycle[n] <= 0 || node_cycle[n] > 32767) {
        set_err(err, errlen, "bad signal cycle"); oracle_destroy(S); return NULL;
      }
      S->ncyc[n] = node_cycle[n]; S->noff[n] = node_offset[n];
    }
  }
  S->lane_base = malloc(8 * ((size_t)E + 1)); S->row_off = malloc(8 * ((size_t)E + 1));
  int64_t lanes = 0, bytes = 0;
  int32_t maxC = 0;
  for (int32_t e = 0; e < E; ++e) {
    if (edge_src[e] < 0 || edge_src[e] >= N || edge_dst[e] < 0 || edge_dst[e] >= N || edge_lanes[e] < 1 ||
        edge_lanes[e] > 8 || edge_class[e] >= cfg->n_classes || !(edge_speed[e] > 0.0f) ||
        !(edge_length_m[e] > 0.0f) || edge_length_m[e] > 1.0e6f) {
      set_err(err, errlen, "bad edge"); oracle_destroy(S); return NULL;
    }
    S->src[e] = edge_src[e]; S->dst[e] = edge_dst[e]; S->nl[e] = edge_lanes[e]; S->cls[e] = edge_class[e];
    S->lim[e] = edge_speed[e];
    /* Section II-D: a segment of length l becomes l / t_m one-metre cells. */
    int64_t c = llround((double)edge_length_m[e] / (double)cfg->cell_m);
    if (c < cmin) c = cmin;
    S->C[e] = (int32_t)c;
    if (c > maxC) maxC = (int32_t)c;
    S->lane_base[e] = lanes; S->row_off[e] = bytes;
    lanes += edge_lanes[e]; bytes += c * edge_lanes[e];
    if (node_type[edge_dst[e]] == NODE_SIGNAL) {
      if (!green_start || !green_len) { set_err(err, errlen, "signal windows missing"); oracle_destroy(S); return NULL; }
      S->gs[e] = green_start[e]; S->gl[e] = green_len[e];
    }
  }
  S->lane_base[E] = lanes; S->row_off[E] = bytes;
  S->n_lanes = lanes; S->map_bytes = bytes;
  S->map_cur = malloc((size_t)bytes); S->map_nxt = malloc((size_t)bytes);
  memset(S->map_cur, EMPTY, (size_t)bytes); memset(S->map_nxt, EMPTY, (size_t)bytes);
  /* out-edges per node in ascending edge id; lane masks per (in-edge, out-edge) */
  S->out_off = calloc((size_t)N + 1, 8); S->out_e = malloc(4 * (size_t)E);
  for (int32_t e = 0; e < E; ++e) S->out_off[S->src[e] + 1]++;
  for (int32_t n = 0; n < N; ++n) S->out_off[n + 1] += S->out_off[n];
  {
    int64_t *f = malloc(8 * (size_t)N);
    memcpy(f, S->out_off, 8 * (size_t)N);
    for (int32_t e = 0; e < E; ++e) S->out_e[f[S->src[e]]++] = e;
    free(f);
  }
  S->conn_off = malloc(8 * ((size_t)E + 1));
  int64_t nc = 0;
  for (int32_t e = 0; e < E; ++e) { S->conn_off[e] = nc; int32_t n = S->dst[e]; nc += S->out_off[n + 1] - S->out_off[n]; }
  S->conn_off[E] = nc;
  S->conn = malloc(4 * (size_t)(nc ? nc : 1));
  for (int32_t e = 0; e < E; ++e) {
    uint32_t all = (1u << S->nl[e]) - 1u;
    for (int64_t j = S->conn_off[e]; j < S->conn_off[e + 1]; ++j) {
      uint32_t m = conn_lane_mask ? (conn_lane_mask[j] & all) : all;
      if (!m) { set_err(err, errlen, "lane mask with no lane"); oracle_destroy(S); return NULL; }
      S->conn[j] = m;
    }
  }
  /* in-lanes of every node, ordered by (edge id, lane) */
  S->inl_off = calloc((size_t)N + 1, 8);
  for (int32_t e = 0; e < E; ++e) S->inl_off[S->dst[e] + 1] += S->nl[e];
  for (int32_t n = 0; n < N; ++n) S->inl_off[n + 1] += S->inl_off[n];
  S->inl = malloc(8 * (size_t)(lanes ? lanes : 1));
  {
    int64_t *f = malloc(8 * (size_t)N);
    memcpy(f, S->inl_off, 8 * (size_t)N);
    for (int32_t e = 0; e < E; ++e)
      for (int32_t l = 0; l < S->nl[e]; ++l) S->inl[f[S->dst[e]]++] = S->lane_base[e] + l;
    free(f);
  }
  S->permit = malloc(4 * (size_t)N); S->rr = calloc((size_t)N, 4);
  S->clo_k0 = calloc((size_t)(lanes ? lanes : 1), 8); S->clo_k1 = calloc((size_t)(lanes ? lanes : 1), 8);
  for (int32_t n = 0; n < N; ++n) S->permit[n] = NONE_ID;
  /* Eq. 2: m(x) = 1 for x <= x0, exp(-((x - x0)/lambda)^2) beyond; x = distance
     in metres to the end of the edge.  Evaluated once here in double. */
  S->mtab_n = maxC + 1;
  S->mtab = malloc(4 * (size_t)S->mtab_n);
  for (int32_t d = 0; d < S->mtab_n; ++d) {
    double xm = (double)d * (double)cfg->cell_m, x0 = (double)cfg->lc_x0_m, lam = (double)cfg->lc_len_scale_m;
    double m = xm <= x0 ? 1.0 : exp(-((xm - x0) / lam) * ((xm - x0) / lam));
    S->mtab[d] = (float)m;
  }
  S->entry = calloc((size_t)E, 4); S->exitc = calloc((size_t)E, 4);
  S->ssum = calloc((size_t)E * (size_t)cfg->n_stats_windows, 8);
  S->scnt = calloc((size_t)E * (size_t)cfg->n_stats_windows, 4);
  S->best = malloc(4 * (size_t)(lanes ? lanes : 1));
  for (int64_t g = 0; g < lanes; ++g) S->best[g] = NONE_ID;
  S->k = cfg->t0_step;
  S->st.step = cfg->t0_step;
  return S;
}

static uint32_t lane_mask(const osim *S, int32_t e, int32_t e2) {
  int32_t n = S->dst[e];
  for (int64_t j = S->out_off[n]; j < S->out_off[n + 1]; ++j)
    if (S->out_e[j] == e2) return S->conn[S->conn_off[e] + (j - S->out_off[n])];
  return 0;
}

/* Trips: route edge lists (Section II-C) and departure times (Section II-D). */
OR_API int oracle_load_trips(osim *S, int64_t n, const int64_t *route_off, const int32_t *route_edges,
                             const float *depart_time_s, char *err, int errlen) {
  if (!S) return -1;
  if (S->loaded) { set_err(err, errlen, "trips already loaded"); return -3; }
  if (n < 0 || (n > 0 && (!route_off || !route_edges || !depart_time_s)) || n > 0xFFFFFFFELL) {
    set_err(err, errlen, "bad trip arrays"); return -1;
  }
  if (n > 0 && route_off[0] != 0) { set_err(err, errlen, "route_off[0] != 0"); return -2; }
  for (int64_t j = 0; j < n; ++j) {
    if (route_off[j + 1] <= route_off[j]) { set_err(err, errlen, "empty route"); return -2; }
    for (int64_t q = route_off[j]; q < route_off[j + 1]; ++q) {
      int32_t e = route_edges[q];
      if (e < 0 || e >= S->E) { set_err(err, errlen, "route edge out of range"); return -2; }
      if (q + 1 < route_off[j + 1]) {
        int32_t e2 = route_edges[q + 1];
        if (e2 < 0 || e2 >= S->E || S->dst[e] != S->src[e2]) { set_err(err, errlen, "route not contiguous"); return -2; }
      }
    }
    if (!(depart_time_s[j] == depart_time_s[j])) { set_err(err, errlen, "NaN departure time"); return -1; }
  }
  S->NT = n;
  int64_t nr = n ? route_off[n] : 0;
  S->route_off = malloc(8 * ((size_t)n + 1)); S->route = malloc(4 * (size_t)(nr ? nr : 1));
  S->rmask = malloc((size_t)(nr ? nr : 1));
  S->route_off[0] = 0;
  for (int64_t j = 0; j < n; ++j) S->route_off[j + 1] = route_off[j + 1];
  for (int64_t q = 0; q < nr; ++q) S->route[q] = route_edges[q];
  for (int64_t j = 0; j < n; ++j)
    for (int64_t q = route_off[j]; q < route_off[j + 1]; ++q)
      S->rmask[q] = (q + 1 < route_off[j + 1]) ? (uint8_t)lane_mask(S, route_edges[q], route_edges[q + 1]) : 0xFF;
  S->dstep = malloc(8 * (size_t)(n ? n : 1));
  S->V = calloc((size_t)(n ? n : 1), sizeof(veh_t));
  for (int64_t j = 0; j < n; ++j) S->dstep[j] = (int64_t)ceil((double)depart_time_s[j] / (double)S->cfg.dt);
  /* departure queues per first edge, ordered by (departure step, id) */
  S->q_off = calloc((size_t)S->E + 1, 8); S->q_head = calloc((size_t)S->E, 8);
  S->q_trip = malloc(8 * (size_t)(n ? n : 1));
  for (int64_t j = 0; j < n; ++j) S->q_off[S->route[S->route_off[j]] + 1]++;
  for (int32_t e = 0; e < S->E; ++e) S->q_off[e + 1] += S->q_off[e];
  {
    int64_t *f = malloc(8 * (size_t)S->E);
    memcpy(f, S->q_off, 8 * (size_t)S->E);
    for (int64_t j = 0; j < n; ++j) S->q_trip[f[S->route[S->route_off[j]]]++] = j;
    free(f);
  }
  for (int32_t e = 0; e < S->E; ++e) {
    /* insertion sort per queue by (dstep, id): queues are short and ids already ascending */
    int64_t lo = S->q_off[e], hi = S->q_off[e + 1];
    for (int64_t a = lo + 1; a < hi; ++a) {
      int64_t t = S->q_trip[a], b = a - 1;
      while (b >= lo && (S->dstep[S->q_trip[b]] > S->dstep[t])) { S->q_trip[b + 1] = S->q_trip[b]; --b; }
      S->q_trip[b + 1] = t;
    }
    S->q_head[e] = lo;
  }
  S->on = malloc(8 * (size_t)(n ? n : 1));
  S->lc_tgt = malloc(4 * (size_t)(n ? n : 1));
  S->n_on = 0;
  S->loaded = 1;
  S->st.loaded = n;
  S->st.waiting = n;
  return 0;
}

/* --------------------------------------------------------- lane change -- */
/* first occupied cell of lane row `rw` in [lo, hi] scanning upward (-1 if
 * none); every cell read is added to *cnt when cnt is not NULL */
static int32_t first_up(const uint8_t *rw, int32_t lo, int32_t hi, uint64_t *cnt) {
  for (int32_t c = lo; c <= hi; ++c) {
    if (cnt) ++*cnt;
    if (rw[c] != EMPTY) return c;
  }
  return -1;
}
static int32_t first_down(const uint8_t *rw, int32_t hi, int32_t lo, uint64_t *cnt) {
  for (int32_t c = hi; c >= lo; --c) {
    if (cnt) ++*cnt;
    if (rw[c] != EMPTY) return c;
  }
  return -1;
}

/* Returns the target lane or -1.  Mandatory vs discretionary per Section
 * II-D; probability of attempting a mandatory change per Eq. 2; critical
 * lead/lag gaps per Eqs. 3 and 4.  Every lane-map cell its scans read is
 * counted in lc_cells_scanned.                                            */
static int32_t lc_decide(osim *S, int64_t id) {
  const oracle_config *cf = &S->cfg;
  veh_t *V = &S->V[id];
  const int32_t e = V->e, l = V->l, nl = S->nl[e], Ce = S->C[e], L = cf->veh_len_cells, H = cf->horizon_cells;
  if (nl < 2) return -1;
  const int64_t k = S->k;
  const int32_t dir = (k & 1) ? -1 : 1;
  const int32_t lt = l + dir;
  if (lt < 0 || lt >= nl) return -1;
  if (lane_closed(S, e, lt, k)) return -1;              /* never into a closed lane */
  const int32_t cell = (int32_t)floorf(V->x);
  const int has_next = (V->r + 1 < S->route_off[id + 1]);
  uint32_t mask = has_next ? S->rmask[V->r] : 0xFFu;
  if (has_next) {
    /* lanes whose continuation on the next edge is closed are not allowed either */
    const int32_t e2 = S->route[V->r + 1];
    uint32_t open = 0;
    for (int32_t q = 0; q < nl; ++q) {
      const int32_t q2 = q < S->nl[e2] - 1 ? q : S->nl[e2] - 1;
      if (!lane_closed(S, e2, q2, k)) open |= 1u << q;
    }
    if (mask & open) mask &= open;
  }
  const int ok_l = (mask >> l) & 1, ok_lt = (mask >> lt) & 1;
  const int32_t obst = Ce / 2;
  const int closed_here = lane_closed(S, e, l, k) && cell < obst;
  int mandatory = 0;
  if (closed_here) {
    mandatory = 2;                                       /* leave the closed lane before the obstacle */
  } else if (has_next && !ok_l) {
    /* distance to the nearest allowed lane on each side */
    int32_t dp = 99, dm = 99;
    for (int32_t q = l + 1; q < nl; ++q) if ((mask >> q) & 1) { dp = q - l; break; }
    for (int32_t q = l - 1; q >= 0; --q) if ((mask >> q) & 1) { dm = l - q; break; }
    int toward = (dir > 0) ? (dp < 99 && dp <= dm) : (dm < 99 && dm <= dp);
    if (!toward) return -1;
    mandatory = 1;
  } else if (!ok_lt) {
    return -1;
  }
  const float v = V->v;
  uint64_t *lcc = &S->st.lc_cells_scanned;   /* cells read by the scans below */
  uint8_t *tr = row(S, S->map_cur, e, lt);
  if (mandatory) {
    /* Eq. 2 probability at the distance to the end of the edge (or to the obstacle) */
    int32_t dist = mandatory == 2 ? obst - 1 - cell : Ce - 1 - cell;
    float u1 = rng_u(cf->seed, (uint64_t)id, k, 0);
    if (!(u1 < S->mtab[dist])) return -1;
  } else {
    /* discretionary: a slower leader ahead in the own lane and more room
     * ahead in the target lane (a stopped vehicle has no slower leader) */
    if (!(v > 0.0f)) return -1;
    uint8_t *orw = row(S, S->map_cur, e, l);
    int32_t hi = cell + H < Ce - 1 ? cell + H : Ce - 1;
    int32_t co = first_up(orw, cell + 1, hi, lcc);
    if (co < 0) return -1;
    if (!(speed_decode(orw[co]) < v)) return -1;
    int32_t own_gap = co - L - cell;
    int32_t ca = first_up(tr, cell + L, hi, lcc);
    if (ca >= 0 && !(ca - L - cell > own_gap)) return -1;
  }
  S->st.lc_evals++;
  /* gap acceptance in the target lane */
  {
    int32_t lo = cell - L + 1 < 0 ? 0 : cell - L + 1;
    int32_t hi = cell + L - 1 > Ce - 1 ? Ce - 1 : cell + L - 1;
    if (first_up(tr, lo, hi, lcc) >= 0) return -1;       /* lateral overlap */
  }
  int32_t hi = cell + H < Ce - 1 ? cell + H : Ce - 1;
  int32_t ca = first_up(tr, cell + L, hi, lcc);
  int32_t cb = first_down(tr, cell - L, cell - H < 0 ? 0 : cell - H, lcc);
  const float g = v < cf->g_speed_split ? cf->g_low : cf->g_high;
  const float alpha = cf->alpha_lo + (cf->alpha_hi - cf->alpha_lo) * rng_u(cf->seed, (uint64_t)id, 0, 3);
  if (ca >= 0) {
    float va = speed_decode(tr[ca]);
    float eps_a = rng_n(cf->seed, (uint64_t)id, k, 1);
    float gl = g + alpha * v;           /* Eq. 3 with alpha_a = alpha_i */
    gl = gl + alpha * (v - va);
    float glead = fmaxf(g, gl) + eps_a;
    if (!((float)(ca - L - cell) >= glead)) return -1;
  }
  if (cb >= 0) {
    float vb = speed_decode(tr[cb]);
    float eps_b = rng_n(cf->seed, (uint64_t)id, k, 2);
    float gg = g + alpha * v;           /* Eq. 4 with alpha_b = alpha_i */
    gg = gg + alpha * (v - vb);
    float glag = fmaxf(g, gg) + eps_b;
    if (!((float)(cell - L - cb) >= glag)) return -1;
  }
  return lt;
}

/* ---------------------------------------------------------- leader scan -- */
enum { SC_FREE = 0, SC_LEADER = 1, SC_VIRTUAL = 2 };
typedef struct {
  int kind;
  int64_t cL;          /* route-relative leader front cell                  */
  float vL;
  int reached_own;     /* scan reached the own edge's end node (not last edge) */
  int stop_only;       /* ... and was held there only by a stop sign        */
} scan_t;

/* Walk the lane map from the cell ahead of the vehicle along its route, at
 * most H cells, looking for the first occupied byte (Section II-D: the
 * leader is found by looking up neighbouring cells).  Nodes on the way act
 * as a stationary virtual leader at their stop line when they hold the
 * vehicle: red signal or stop sign without permit (own node); red signal or
 * stop sign (later nodes).  A lane not allowed for the next edge does not
 * hold the vehicle: it only makes the lane change mandatory (Eq. 2), and a
 * vehicle still in such a lane at the node continues into lane
 * min(l, lanes - 1) of the next edge.               */
static scan_t leader_scan(osim *S, int64_t id) {
  const oracle_config *cf = &S->cfg;
  veh_t *V = &S->V[id];
  const int32_t L = cf->veh_len_cells, H = cf->horizon_cells;
  const int64_t cell = (int64_t)floorf(V->x);
  const int64_t limit = cell + H, rend = S->route_off[id + 1];
  scan_t res; memset(&res, 0, sizeof(res));
  int64_t base = 0, p = cell + 1, r = V->r;
  int32_t se = V->e, sl = V->l;
  int own = 1;
  for (;;) {
    const int64_t segC = S->C[se];
    const uint8_t *rw = row(S, S->map_cur, se, sl);
    /* a closed own lane holds an obstacle from mid-edge on, for vehicles behind it */
    const int64_t obst = (own && lane_closed(S, se, sl, S->k) && cell < segC / 2) ? segC / 2 : -1;
    while (p < base + segC) {
      if (p > limit) { res.kind = SC_FREE; S->st.cells_scanned += (uint64_t)H; return res; }
      if (p == obst) {
        res.kind = SC_VIRTUAL; res.cL = obst + L - 1; res.vL = 0.0f;
        S->st.cells_scanned += (uint64_t)(obst - 1 - cell);
        return res;
      }
      uint8_t byte = rw[p - base];
      if (byte != EMPTY) {
        res.kind = SC_LEADER; res.cL = p; res.vL = speed_decode(byte);
        S->st.cells_scanned += (uint64_t)(p - cell);
        return res;
      }
      ++p;
    }
    const int64_t B = base + segC;
    if (B > limit) { res.kind = SC_FREE; S->st.cells_scanned += (uint64_t)H; return res; }
    if (r + 1 >= rend) { res.kind = SC_FREE; S->st.cells_scanned += (uint64_t)(B - 1 - cell); return res; }
    S->st.route_reads++;
    const int32_t n = S->dst[se], e2 = S->route[r + 1];
    int blocked = 0;
    if (S->ntype[n] == NODE_SIGNAL && !is_green(S, se, S->k)) blocked = 1;
    {
      const int32_t l2 = sl < S->nl[e2] - 1 ? sl : S->nl[e2] - 1;
      if (lane_closed(S, e2, l2, S->k)) blocked = 1;       /* no entry into a closed lane */
    }
    if (own) {
      int stop_np = (S->ntype[n] == NODE_STOP) && (S->permit[n] != (uint32_t)id);
      res.reached_own = 1;
      res.stop_only = stop_np;
      if (stop_np) blocked = 1;
    } else if (S->ntype[n] == NODE_STOP) {
      blocked = 1;
    }
    if (blocked) {
      res.kind = SC_VIRTUAL; res.cL = B + L - 1; res.vL = 0.0f;
      S->st.cells_scanned += (uint64_t)(B - 1 - cell);
      return res;
    }
    ++r; base = B;
    sl = sl < S->nl[e2] - 1 ? sl : S->nl[e2] - 1;
    se = e2; own = 0;
  }
}

/* ------------------------------------------------------------------ step -- */
typedef struct { int64_t id; float xn, vn; uint8_t dwn; int kind; int64_t tgt_lane; int32_t e2, l2; } upd_t;

/* Event tape for the calibration adjoint (test infrastructure): for every
 * trip and every step k in [k0, k0 + len), element (k - k0) * n_trips + id
 * receives the state entering the step (x, v), the leader gap s and speed vL
 * when the vehicle is interacting, the clamp bound, the edge's speed limit
 * and cells, and flags = present | kind << 1 | ballistic << 3 | clamp << 4 |
 * outcome << 6 | class << 9, with kind 0 free / 1 interacting / 2 stopped in
 * place, ballistic 1 when v + acc dt >= 0, clamp 0 none / 1 old position
 * kept / 2 bound, outcome 0 stayed / 1 crossed / 2 held at its old position
 * / 3 held at the stop line / 4 arrived; sample = window * E + edge of the
 * speed sample taken after the step, or -1.  Entries of trips not on the
 * network stay as the caller initialised them (flags 0).  NULL x disables. */
OR_API void oracle_set_tape(osim *S, int64_t k0, int64_t len, float *x, float *v, float *s, float *vL, float *bnd,
                            float *lim, int32_t *C, int32_t *flags, int64_t *sample) {
  S->tp_k0 = k0; S->tp_len = x ? len : 0;
  S->tp_x = x; S->tp_v = v; S->tp_s = s; S->tp_vL = vL; S->tp_bnd = bnd; S->tp_lim = lim;
  S->tp_C = C; S->tp_flags = flags; S->tp_sample = sample;
}

OR_API int oracle_step(osim *S, int64_t n_steps, char *err, int errlen) {
  if (!S) return -1;
  if (!S->loaded) { set_err(err, errlen, "no trips loaded"); return -3; }
  const oracle_config *cf = &S->cfg;
  const int32_t L = cf->veh_len_cells;
  const float dt = cf->dt;
  S->stepped = 1;
  upd_t *U = malloc(sizeof(upd_t) * (size_t)(S->NT ? S->NT : 1));
  int64_t *dep = malloc(sizeof(int64_t) * (size_t)S->E);  /* requesting trip per edge, -1 none */
  for (int64_t it = 0; it < n_steps; ++it) {
    const int64_t k = S->k;
    /* A: lane-change decisions on M_k */
    for (int64_t q = 0; q < S->n_on; ++q) S->lc_tgt[q] = lc_decide(S, S->on[q]);
    /* B: apply (all changers move the same direction this step) */
    for (int64_t q = 0; q < S->n_on; ++q) {
      if (S->lc_tgt[q] < 0) continue;
      veh_t *V = &S->V[S->on[q]];
      int32_t cell = (int32_t)floorf(V->x);
      uint8_t *a = row(S, S->map_cur, V->e, V->l), *b = row(S, S->map_cur, V->e, S->lc_tgt[q]);
      b[cell] = a[cell]; a[cell] = EMPTY;
      V->l = S->lc_tgt[q];
      S->st.lane_changes++;
    }
    /* C: departure requests on M_k' */
    for (int32_t e = 0; e < S->E; ++e) {
      dep[e] = -1;
      if (S->q_head[e] >= S->q_off[e + 1]) continue;
      int64_t j = S->q_trip[S->q_head[e]];
      if (S->dstep[j] > k) continue;
      if (lane_closed(S, e, 0, k)) continue;
      int32_t need = L + (int32_t)ceilf(cf->s0[S->cls[e]]);
      if (need > S->C[e]) need = S->C[e];
      uint8_t *rw = row(S, S->map_cur, e, 0);
      if (first_up(rw, 0, need - 1, NULL) >= 0) continue;
      dep[e] = j;
    }
    /* D: leader scan, IDM (Eq. 1), ballistic integration, clamp */
    const int64_t n_start = S->n_on;
    for (int64_t q = 0; q < n_start; ++q) {
      const int64_t id = S->on[q];
      veh_t *V = &S->V[id];
      const int32_t e = V->e, p = S->cls[e], Ce = S->C[e];
      const float x = V->x, v = V->v;
      const int32_t cell = (int32_t)floorf(x);
      scan_t sc = leader_scan(S, id);
      const float a = cf->a[p], b = cf->b[p], T = cf->T[p], s0 = cf->s0[p];
      const float lim = driver_limit(S, e, id, V->r);
      const float v0 = lim * cf->v0f[p];
      float xn, vn;
      int stop_in_place = 0;
      float acc = 0.0f;
      const float r1 = v / v0, r2 = r1 * r1, r4 = r2 * r2;   /* (v/v0)^delta, delta = 4 */
      if (sc.kind == SC_FREE) {
        acc = a * (1.0f - r4);
      } else {
        const float s = (float)(sc.cL - cell - L);
        if (s <= 0.0f) stop_in_place = 1;
        else {
          const float dv = v - sc.vL;
          const float dyn = (v * dv) / (2.0f * sqrtf(a * b));
          float ss;
          if (cf->idm_textbook) ss = s0 + fmaxf(0.0f, v * T + dyn);
          else ss = (s0 + v * T) + dyn;
          const float qq = ss / s;
          acc = a * ((1.0f - r4) - qq * qq);
        }
      }
      int t_ball = 0, t_clamp = 0;   /* events of the step, for the tape */
      float t_bnd = 0.0f;
      if (stop_in_place) { xn = x; vn = 0.0f; }
      else {
        /* "double integrating": ballistic update (position with the mean speed over dt) */
        const float vt = v + acc * dt;
        float xt, vv;
        if (vt >= 0.0f) { xt = x + (v * dt + (0.5f * acc) * (dt * dt)); vv = vt; t_ball = 1; }
        else { xt = x - (v * v) / (2.0f * acc); vv = 0.0f; }
        int has_bound = 0; int64_t bnd = 0;
        if (sc.kind != SC_FREE) { has_bound = 1; bnd = sc.cL - L; }
        if (V->r + 1 < S->route_off[id + 1]) {
          int64_t cap = (int64_t)Ce + S->C[S->route[V->r + 1]] - 1;   /* at most one node per step */
          if (!has_bound || cap < bnd) { has_bound = 1; bnd = cap; }
        }
        if (has_bound && xt > (float)bnd) {
          xn = fmaxf(x, (float)bnd); vn = 0.0f; S->st.clamps++;
          t_bnd = (float)bnd; t_clamp = x > t_bnd ? 1 : 2;
        }
        else { xn = xt; vn = vv; }
      }
      /* stop-sign dwell: held at the stop line by the stop sign alone */
      uint8_t dwn = 0;
      {
        const int last = !(V->r + 1 < S->route_off[id + 1]);
        const int32_t zone = Ce - 1 - ((int32_t)ceilf(s0) + 2);
        if (!last && sc.reached_own && sc.stop_only && (int32_t)floorf(xn) >= zone && vn < cf->stop_v_eps)
          dwn = V->dwell < 255 ? (uint8_t)(V->dwell + 1) : 255;
      }
      if (S->tp_len > 0 && k >= S->tp_k0 && k < S->tp_k0 + S->tp_len) {
        const size_t ti = (size_t)(k - S->tp_k0) * (size_t)S->NT + (size_t)id;
        const int32_t kind = sc.kind == SC_FREE ? 0 : (stop_in_place ? 2 : 1);
        S->tp_x[ti] = x; S->tp_v[ti] = v;
        S->tp_s[ti] = sc.kind == SC_FREE ? 0.0f : (float)(sc.cL - cell - L);
        S->tp_vL[ti] = sc.kind == SC_FREE ? 0.0f : sc.vL;
        S->tp_bnd[ti] = t_bnd; S->tp_lim[ti] = lim; S->tp_C[ti] = Ce;
        S->tp_flags[ti] = 1 | (kind << 1) | (t_ball << 3) | (t_clamp << 4) | ((int32_t)S->cls[e] << 9);
        S->tp_sample[ti] = -1;
      }
      upd_t *u = &U[q];
      u->id = id; u->xn = xn; u->vn = vn; u->dwn = dwn; u->kind = 0; u->tgt_lane = -1;
      (void)cell;
      if (xn >= (float)Ce) {
        if (!(V->r + 1 < S->route_off[id + 1])) u->kind = 2;          /* arrival */
        else {
          int32_t e2 = S->route[V->r + 1];
          int32_t l2 = V->l < S->nl[e2] - 1 ? V->l : S->nl[e2] - 1;
          u->kind = 1; u->e2 = e2; u->l2 = l2; u->tgt_lane = S->lane_base[e2] + l2;
        }
      }
    }
    /* E: per target lane the lowest id wins */
    for (int64_t q = 0; q < n_start; ++q)
      if (U[q].kind == 1 && (uint32_t)U[q].id < S->best[U[q].tgt_lane]) S->best[U[q].tgt_lane] = (uint32_t)U[q].id;
    for (int32_t e = 0; e < S->E; ++e)
      if (dep[e] >= 0 && (uint32_t)dep[e] < S->best[S->lane_base[e]]) S->best[S->lane_base[e]] = (uint32_t)dep[e];
    /* F: apply outcomes; G: write M_{k+1} and empty M_k'; H: statistics */
    const int64_t w = (k - cf->t0_step) / cf->stats_window_steps;
    const int in_window = (k >= cf->t0_step) && w < cf->n_stats_windows;
    int64_t n_new = 0;
    for (int64_t q = 0; q < n_start; ++q) {
      upd_t *u = &U[q];
      veh_t *V = &S->V[u->id];
      const int32_t cell = (int32_t)floorf(V->x);
      row(S, S->map_cur, V->e, V->l)[cell] = EMPTY;
      const int taped = S->tp_len > 0 && k >= S->tp_k0 && k < S->tp_k0 + S->tp_len;
      const size_t ti = taped ? (size_t)(k - S->tp_k0) * (size_t)S->NT + (size_t)u->id : 0;
      int32_t outcome = 0;
      if (u->kind == 2) {
        S->exitc[V->e]++; S->st.arrived++; V->status = 2;
        if (taped) S->tp_flags[ti] |= 4 << 6;
        continue;
      }
      if (u->kind == 1) {
        if (S->best[u->tgt_lane] == (uint32_t)u->id) {
          outcome = 1;
          const int32_t n = S->dst[V->e];
          if (S->ntype[n] == NODE_STOP && S->permit[n] == (uint32_t)u->id) S->permit[n] = NONE_ID;
          S->exitc[V->e]++; S->entry[u->e2]++;
          V->x = u->xn - (float)S->C[V->e];
          V->e = u->e2; V->l = u->l2; V->r++; V->v = u->vn; V->dwell = 0;
        } else {
          const float held = fmaxf(V->x, (float)(S->C[V->e] - 1));
          outcome = held == V->x ? 2 : 3;
          V->x = held; V->v = 0.0f; V->dwell = u->dwn;
        }
      } else {
        V->x = u->xn; V->v = u->vn; V->dwell = u->dwn;
      }
      S->on[n_new++] = u->id;
      if (in_window) {
        S->ssum[(size_t)w * S->E + V->e] += (uint64_t)(V->v * 1048576.0f);
        S->scnt[(size_t)w * S->E + V->e]++;
      }
      if (taped) {
        S->tp_flags[ti] |= outcome << 6;
        S->tp_sample[ti] = in_window ? (int64_t)w * S->E + V->e : -1;
      }
    }
    for (int32_t e = 0; e < S->E; ++e) {
      if (dep[e] < 0) continue;
      int64_t j = dep[e];
      if (S->best[S->lane_base[e]] != (uint32_t)j) continue;
      veh_t *V = &S->V[j];
      V->e = e; V->l = 0; V->x = 0.0f; V->v = 0.0f; V->r = S->route_off[j]; V->dwell = 0; V->status = 1;
      S->q_head[e]++;
      S->entry[e]++; S->st.departed++;
      S->on[n_new++] = j;
    }
    for (int64_t q = 0; q < n_start; ++q) if (U[q].kind == 1) S->best[U[q].tgt_lane] = NONE_ID;
    for (int32_t e = 0; e < S->E; ++e) if (dep[e] >= 0) S->best[S->lane_base[e]] = NONE_ID;
    S->n_on = n_new;
    for (int64_t q = 0; q < n_new; ++q) {
      veh_t *V = &S->V[S->on[q]];
      row(S, S->map_nxt, V->e, V->l)[(int32_t)floorf(V->x)] = speed_code(V->v);
    }
    { uint8_t *t = S->map_cur; S->map_cur = S->map_nxt; S->map_nxt = t; }
    S->st.vehicle_updates += (uint64_t)n_start;
    /* I: stop-sign permits for step k+1 (round robin over in-lanes) */
    int any_stop = 0;
    for (int32_t n = 0; n < S->N && !any_stop; ++n) any_stop = S->ntype[n] == NODE_STOP;
    if (any_stop) {
      /* head (largest front cell) of every lane after the step */
      int64_t *head = malloc(8 * (size_t)(S->n_lanes ? S->n_lanes : 1));
      for (int64_t g = 0; g < S->n_lanes; ++g) head[g] = -1;
      for (int64_t q = 0; q < S->n_on; ++q) {
        veh_t *V = &S->V[S->on[q]];
        int64_t g = S->lane_base[V->e] + V->l;
        if (head[g] < 0 || S->V[head[g]].x < V->x) head[g] = S->on[q];
      }
      for (int32_t n = 0; n < S->N; ++n) {
        if (S->ntype[n] != NODE_STOP || S->permit[n] != NONE_ID) continue;
        int64_t m = S->inl_off[n + 1] - S->inl_off[n];
        for (int64_t t = 0; t < m; ++t) {
          int64_t idx = (S->rr[n] + t) % m;
          int64_t h = head[S->inl[S->inl_off[n] + idx]];
          if (h >= 0 && S->V[h].dwell >= cf->stop_dwell_steps) {
            S->permit[n] = (uint32_t)h; S->rr[n] = (int32_t)((idx + 1) % m); break;
          }
        }
      }
      free(head);
    }
    S->k = k + 1;
  }
  free(U); free(dep);
  S->st.step = S->k;
  S->st.on_network = S->n_on;
  S->st.waiting = S->st.loaded - S->st.departed;
  return 0;
}

OR_API void oracle_stats(osim *S, oracle_stats_t *out) {
  S->st.step = S->k; S->st.on_network = S->n_on; S->st.waiting = S->st.loaded - S->st.departed;
  *out = S->st;
}

OR_API void oracle_edge_counters(osim *S, uint32_t *entries, uint32_t *exits, uint64_t *speed_sum,
                                 uint32_t *speed_cnt, int32_t window) {
  if (entries) memcpy(entries, S->entry, 4 * (size_t)S->E);
  if (exits) memcpy(exits, S->exitc, 4 * (size_t)S->E);
  if (window >= 0 && window < S->cfg.n_stats_windows) {
    if (speed_sum) memcpy(speed_sum, S->ssum + (size_t)window * S->E, 8 * (size_t)S->E);
    if (speed_cnt) memcpy(speed_cnt, S->scnt + (size_t)window * S->E, 4 * (size_t)S->E);
  }
}

/* On-network vehicles in ascending id. Returns the count (or -1 if cap too small). */
OR_API int64_t oracle_snapshot(osim *S, int64_t cap, float *x, float *v, int32_t *edge, uint8_t *lane,
                               uint32_t *id, uint8_t *dwell, int32_t *route_pos) {
  if (S->n_on > cap) return -1;
  int64_t c = 0;
  for (int64_t j = 0; j < S->NT; ++j) {
    if (S->V[j].status != 1) continue;
    veh_t *V = &S->V[j];
    if (x) x[c] = V->x;
    if (v) v[c] = V->v;
    if (edge) edge[c] = V->e;
    if (lane) lane[c] = (uint8_t)V->l;
    if (id) id[c] = (uint32_t)j;
    if (dwell) dwell[c] = V->dwell;
    if (route_pos) route_pos[c] = (int32_t)(V->r - S->route_off[j]);
    ++c;
  }
  return c;
}

/* The current lane map, edges in id order, lanes in order, C_e bytes each. */
OR_API int64_t oracle_lane_map(osim *S, uint8_t *out, int64_t cap) {
  if (cap < S->map_bytes) return -1;
  memcpy(out, S->map_cur, (size_t)S->map_bytes);
  return S->map_bytes;
}

OR_API int32_t oracle_edge_cells(osim *S, int32_t e) { return (e >= 0 && e < S->E) ? S->C[e] : -1; }
OR_API uint32_t oracle_permit(osim *S, int32_t n) { return (n >= 0 && n < S->N) ? S->permit[n] : NONE_ID; }

/* Test hook: put a waiting trip on the network at (route position, lane, x, v),
 * marking the lane map; returns 0 or a negative code.                      */
OR_API int oracle_place(osim *S, int64_t id, int32_t route_pos, int32_t lane, float x, float v) {
  if (!S || id < 0 || id >= S->NT || S->V[id].status != 0) return -1;
  int64_t r = S->route_off[id] + route_pos;
  if (route_pos < 0 || r >= S->route_off[id + 1]) return -1;
  int32_t e = S->route[r];
  if (lane < 0 || lane >= S->nl[e] || !(x >= 0.0f) || x >= (float)S->C[e] || !(v >= 0.0f)) return -1;
  uint8_t *rw = row(S, S->map_cur, e, lane);
  int32_t cell = (int32_t)floorf(x);
  if (rw[cell] != EMPTY) return -2;
  veh_t *V = &S->V[id];
  V->e = e; V->l = lane; V->x = x; V->v = v; V->r = r; V->dwell = 0; V->status = 1;
  rw[cell] = speed_code(v);
  /* the trip leaves its departure queue */
  int32_t e0 = S->route[S->route_off[id]];
  for (int64_t q = S->q_head[e0]; q < S->q_off[e0 + 1]; ++q)
    if (S->q_trip[q] == id) {
      for (int64_t z = q; z > S->q_head[e0]; --z) S->q_trip[z] = S->q_trip[z - 1];
      S->q_trip[S->q_head[e0]] = id; S->q_head[e0]++;
      break;
    }
  S->on[S->n_on++] = id;
  S->st.departed++;
  S->entry[e]++;
  return 0;
}

/* Test hook: oracle_place for placements 0 .. n-1 in order; returns -1 - i for
 * the first placement i that fails, else 0.                                */
OR_API int64_t oracle_place_many(osim *S, int64_t n, const int64_t *id, const int32_t *route_pos, const uint8_t *lane,
                                 const float *x, const float *v) {
  for (int64_t i = 0; i < n; ++i)
    if (oracle_place(S, id[i], route_pos[i], (int32_t)lane[i], x[i], v[i]) != 0) return -1 - i;
  return 0;
}

/* Invariants after a step: every lane's front cells at least L apart, map bytes
 * exactly the vehicles' speed codes, conservation. Returns 0 or an error code. */
OR_API int oracle_check(osim *S, char *msg, int len) {
  const int32_t L = S->cfg.veh_len_cells;
  int64_t marked = 0;
  for (int64_t b = 0; b < S->map_bytes; ++b) marked += S->map_cur[b] != EMPTY;
  if (marked != S->n_on) { set_err(msg, len, "map byte count != on-network count"); return 1; }
  for (int64_t q = 0; q < S->n_on; ++q) {
    veh_t *V = &S->V[S->on[q]];
    int32_t cell = (int32_t)floorf(V->x);
    if (cell < 0 || cell >= S->C[V->e]) { set_err(msg, len, "vehicle outside its edge"); return 2; }
    if (row(S, S->map_cur, V->e, V->l)[cell] != speed_code(V->v)) { set_err(msg, len, "map byte != speed code"); return 3; }
  }
  for (int32_t e = 0; e < S->E; ++e)
    for (int32_t l = 0; l < S->nl[e]; ++l) {
      uint8_t *rw = row(S, S->map_cur, e, l);
      int32_t last = -1000000;
      for (int32_t c = 0; c < S->C[e]; ++c)
        if (rw[c] != EMPTY) { if (c - last < L) { set_err(msg, len, "fronts closer than L"); return 4; } last = c; }
    }
  if (S->st.departed != S->st.arrived + S->n_on) { set_err(msg, len, "departed != arrived + on"); return 5; }
  uint64_t se = 0, sx = 0;
  for (int32_t e = 0; e < S->E; ++e) { se += S->entry[e]; sx += S->exitc[e]; }
  if ((int64_t)(se - sx) != S->n_on) { set_err(msg, len, "sum(entry) - sum(exit) != on"); return 6; }
  return 0;
}

OR_API int64_t oracle_map_bytes(osim *S) { return S->map_bytes; }

/* Close lane `lane` of edge `edge` during steps [k0, k1) (replaces an earlier
 * window of that lane).  Only before the first step. */
OR_API int oracle_set_lane_closure(osim *S, int32_t edge, int32_t lane, int64_t k0, int64_t k1) {
  if (!S || edge < 0 || edge >= S->E || lane < 0 || lane >= S->nl[edge] || k1 < k0) return -1;
  if (S->stepped) return -3;
  int64_t g = S->lane_base[edge] + lane;
  S->clo_k0[g] = k0; S->clo_k1[g] = k1;
  return 0;
}
