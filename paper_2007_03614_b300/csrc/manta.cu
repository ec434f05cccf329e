// manta.cu -- host side of the C ABI declared in include/manta.h.
//
// Validation, lane-map layout, departure queues and every device allocation
// live here; the per-step work is the persistent kernel in step_kernel.cuh.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "manta.h"
#include "sim.cuh"
#include <cstddef>
#include "step_kernel.cuh"
#include "adjoint.cuh"

namespace {

thread_local std::string g_err;

manta_status fail(manta_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

constexpr int32_t kStepsPerLaunch = 2048;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per grid barrier wait
// lane-map padding after the last row: the first leader-scan batch is fetched
// whole (kFirstChunks 16-byte chunks) before its row's end is known, and may
// start at the last row's last chunk
constexpr uint64_t kMapPad = 16 * kFirstChunks > 64 ? 16 * kFirstChunks : 64;

// Marks the first route entry of every trip in a bitmap.
__global__ void trip_start_kernel(const uint32_t *roff, uint32_t n, uint32_t *bits) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t q = roff[j];
    atomicOr(bits + (q >> 5), 1u << (q & 31));
  }
}

// Turns the raw route edges into route entries, in place: entry q becomes
// edge | (lane mask toward the next edge of the trip) << 24, and bit q of
// nclo is set when that next edge has a closure window.  The edge bits of an
// entry are the same before and after, so reading a neighbour's entry while
// it is being rewritten is safe.  The first failing entry (edge out of range,
// or not followed by an edge leaving its head node) goes to *bad.
__global__ void route_kernel(uint32_t *route, uint64_t nr, const uint32_t *start_bits, uint32_t E,
                             const uint32_t *esrc, const EdgeMeta *em, const uint32_t *out_off, const uint32_t *out_e,
                             const uint32_t *conn_off, const uint32_t *conn, uint32_t *nclo,
                             unsigned long long *bad) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nr; q += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t raw = (int32_t)route[q];
    if (raw < 0 || (uint32_t)raw >= E) { atomicMin(bad, (unsigned long long)q); continue; }
    const uint32_t e = (uint32_t)raw;
    const bool last = q + 1 == nr || ((start_bits[(q + 1) >> 5] >> ((q + 1) & 31)) & 1u);
    uint32_t mask = 0xFFu;
    if (!last) {
      const uint32_t e2 = route[q + 1] & MANTA_EDGE_MASK;
      const uint32_t nd = em[e].dst & ~MANTA_CLOSABLE;
      int64_t idx = -1;
      if (e2 < E && esrc[e2] == nd)
        for (uint32_t z = out_off[nd]; z < out_off[nd + 1]; ++z)
          if (out_e[z] == e2) { idx = (int64_t)(z - out_off[nd]); break; }
      if (idx < 0) { atomicMin(bad, (unsigned long long)q); continue; }
      mask = conn[conn_off[e] + (uint32_t)idx];
      if (em[e2].dst & MANTA_CLOSABLE) atomicOr(nclo + (q >> 5), 1u << (q & 31));
    }
    route[q] = e | (mask << MANTA_EDGE_BITS);
  }
}

__global__ void prime_kernel(Params p, uint32_t hi, int cb) {
  uint32_t *dep = cb ? p.dep1 : p.dep0;
  const uint32_t gsz = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gsz) {
    const uint32_t e = p.due_edge[i];
    const bool first = atomicAdd(p.pending + e, 1u) == 0u;
    const uint32_t at = warp_append(&p.ctl->n_dep[cb], first);
    if (first) dep[at] = e;
  }
}

// Puts placement i (trip trip[i] at absolute route entry rabs[i], lane, x, v)
// on the network in vehicle slot i and active-list position i: the vehicle
// record, its front cell in the current lane map (claimed with a compare-
// and-swap on the aligned word, so two placements on one cell are caught)
// and the entry count of its edge.  The lowest failing index goes to *bad.
__global__ void place_kernel(Params p, const uint32_t *trip, const uint32_t *rabs, const uint8_t *lane,
                             const float *xs, const float *vs, uint32_t n, int cb, unsigned long long *bad) {
  uint8_t *cur = cb ? p.atlas1 : p.atlas0;
  uint32_t *act = p.act0;                      // act_sel is 0 before the first step
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t j = trip[i], r = rabs[i], l = lane[i];
    const float x = xs[i], v = vs[i];
    const uint32_t e = p.route[r] & MANTA_EDGE_MASK;
    const EdgeMeta em = load_em(p, e);
    const uint32_t C = cells_of(em.cnl);
    if ((int)l >= lanes_of(em.cnl) || !(x >= 0.0f) || !(x < __uint2float_rn(C))) {
      atomicMin(bad, (unsigned long long)i);
      continue;
    }
    const uint32_t off = em.row0 + l * stride_of(C) + (uint32_t)(int)floorf(x);
    unsigned *word = reinterpret_cast<unsigned *>(cur + (off & ~3u));
    const unsigned sh = 8u * (off & 3u);
    bool ok = false;
    unsigned old = *word;
    for (int tries = 0; tries < 16; ++tries) {      // at most 4 placements share a word
      if (((old >> sh) & 0xFFu) != MANTA_EMPTY) break;
      const unsigned nw = (old & ~(0xFFu << sh)) | ((unsigned)speed_code(v) << sh);
      const unsigned got = atomicCAS(word, old, nw);
      if (got == old) { ok = true; break; }
      old = got;
    }
    if (!ok) { atomicMin(bad, (unsigned long long)i); continue; }
    Veh w;
    w.x = x; w.v = v; w.id = j; w.rc = r; w.rend = p.route_off[j + 1u]; w.e = e;
    w.ld = ld_for_entry(p, r, l); w.pcell = MANTA_NONE; w.em = em;
    w.em.lim = driver_limit(p, em.lim, j, r);
    store_veh(p.vs[0], i, w);
    p.vs[0].nx[i] = r + 1u < w.rend ? p.route[r + 1u] : 0u;
    act[i] = i;
    atomicAdd(p.entry + e, 1u);
  }
}

__global__ void barrier_selftest_kernel(Ctl *ctl, uint64_t limit_ns) {
  __shared__ int s_ok;
  if (blockIdx.x == 0) return;   // this block never arrives
  unsigned target = 0;
  grid_sync(ctl, target, limit_ns, &s_ok);
}

}  // namespace

struct manta_sim {
  manta_config cfg;
  cudaStream_t stream = nullptr;
  int32_t N = 0, E = 0;
  std::vector<uint32_t> cells, lanes, row0, lane_base;
  std::vector<int32_t> esrc, edst;
  std::vector<int64_t> out_off, conn_off;
  std::vector<int32_t> out_e;
  std::vector<uint32_t> conn;
  uint64_t atlas_bytes = 0, canon_bytes = 0;
  uint32_t n_lanes = 0;
  std::vector<void *> allocs;
  Params P;
  bool loaded = false, primed = false, dead = false;
  int64_t k = 0, n_trips = 0;
  uint32_t prime_hi = 0;
  std::vector<uint32_t> route_off_h;
  // host copies kept from manta_load_trips for manta_place: departure queues
  // (offsets by first edge, trips in (step, id) order), trips in departure
  // order, departure steps and first edges
  std::vector<uint32_t> q_off_h, q_trip_h, dorder_h, first_h;
  std::vector<int64_t> dstep_h;
  bool placed = false;
  std::vector<EdgeMeta> em_h;
  std::vector<long long> clo_k0, clo_k1;
  int grid[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // co-resident grid size of every launch shape
  int variant = 0;                          // launch shape used by manta_step
  // event tape (calibration): device records, capacity, recorded segment
  TapeRec *tape = nullptr;
  size_t tape_cap = 0;
  int64_t tape_k0 = 0;
  int32_t tape_len = 0;
  // scratch of the adjoint (per-block parts of the gradient) and of the
  // replay (128-bit fixed-point sums per statistics cell), allocated on first use
  double *adj_part = nullptr;
  size_t adj_part_cap = 0;
  unsigned long long *rep_acc = nullptr;
  size_t rep_acc_cap = 0;
};

// Launch shapes of the step kernel (threads per block, minimum blocks per
// SM); the second number sets the register budget.  All shapes compute the
// same results bit for bit; manta_autotune picks the fastest on the live run.
struct StepVariant {
  int threads, min_blocks;
  const void *fn;
};
static const StepVariant kVariants[] = {
    {384, 1, (const void *)manta_step_kernel<384, 1>},
    {256, 1, (const void *)manta_step_kernel<256, 1>},
    {256, 2, (const void *)manta_step_kernel<256, 2>},
    {192, 2, (const void *)manta_step_kernel<192, 2>},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// Static device memory for manta_run_noalloc: every device that loads the
// library holds these bytes until the process exits.
#define MANTA_NOALLOC_ARENA_BYTES (8u << 20)
static __device__ __align__(256) unsigned char g_noalloc_arena[MANTA_NOALLOC_ARENA_BYTES];

namespace {

// While set (only inside manta_run_noalloc, on the calling thread), device
// arrays are carved from the static arena instead of being allocated.
struct Arena {
  unsigned char *base;
  size_t cap, used;
  bool overflow;
};
thread_local Arena *t_arena = nullptr;

// Host-side fault injection (manta_debug_fail_nth): on this thread, the nth
// device allocation or host-to-device copy made by the library from now on
// fails as the CUDA call would have (0: off).
thread_local int64_t t_fail_alloc = 0, t_fail_copy = 0;
bool injected(int64_t &countdown) {
  if (countdown <= 0) return false;
  return --countdown == 0;
}
cudaError_t dev_malloc(void **p, size_t bytes) {
  if (injected(t_fail_alloc)) { *p = nullptr; return cudaErrorMemoryAllocation; }
  return cudaMalloc(p, bytes);
}
cudaError_t h2d_async(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (injected(t_fail_copy)) return cudaErrorInvalidValue;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}

template <class T>
T *dalloc(manta_sim *S, size_t n, bool *ok) {
  void *p = nullptr;
  if (n == 0) n = 1;
  if (injected(t_fail_alloc)) {
    *ok = false;
    return nullptr;
  }
  if (t_arena) {
    const size_t off = (t_arena->used + 255u) & ~(size_t)255u;
    if (off + n * sizeof(T) > t_arena->cap) {
      t_arena->overflow = true;
      *ok = false;
      return nullptr;
    }
    t_arena->used = off + n * sizeof(T);
    return reinterpret_cast<T *>(t_arena->base + off);
  }
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *ok = false;
    return nullptr;
  }
  S->allocs.push_back(p);
  return static_cast<T *>(p);
}

template <class T>
bool upload(manta_sim *S, T *dst, const std::vector<T> &src) {
  if (src.empty()) return true;
  return h2d_async(dst, src.data(), src.size() * sizeof(T), S->stream) == cudaSuccess;
}

manta_status check_cfg(const manta_config *c) {
  if (!c) return fail(MANTA_E_INVALID, "config is NULL");
  if (c->cell_m != 1.0f) return fail(MANTA_E_INVALID, "cell_m must be 1");
  if (!(c->dt > 0.0f) || !(c->dt < 60.0f)) return fail(MANTA_E_INVALID, "dt out of range");
  if (c->veh_len_cells < 1 || c->veh_len_cells > 100) return fail(MANTA_E_INVALID, "veh_len_cells out of range");
  if (c->horizon_cells < 16 || c->horizon_cells > (1 << 20)) return fail(MANTA_E_INVALID, "horizon_cells out of range");
  if (c->n_classes < 1 || c->n_classes > 8) return fail(MANTA_E_INVALID, "n_classes out of range");
  for (int i = 0; i < c->n_classes; ++i)
    if (!(c->a[i] > 0.0f) || !(c->b[i] > 0.0f) || !(c->T[i] >= 0.0f) || !(c->s0[i] >= 0.0f) ||
        !(c->s0[i] < 100.0f) || !(c->v0f[i] > 0.0f))
      return fail(MANTA_E_INVALID, "bad class parameters");
  if (c->stop_dwell_steps < 1 || c->stop_dwell_steps > 255) return fail(MANTA_E_INVALID, "stop_dwell_steps out of range");
  if (c->stats_window_steps < 1 || c->n_stats_windows < 1) return fail(MANTA_E_INVALID, "bad statistics windows");
  if (c->t0_step < 0 || c->t0_step > (int64_t)1 << 40) return fail(MANTA_E_INVALID, "t0_step out of range");
  if (!(c->lc_len_scale_m > 0.0f)) return fail(MANTA_E_INVALID, "lc_len_scale_m must be > 0");
  if (!(c->speed_sigma_frac >= 0.0f) || !(c->speed_sigma_frac <= 1.0f))
    return fail(MANTA_E_INVALID, "speed_sigma_frac out of range");
  return MANTA_OK;
}

uint32_t stride16(uint32_t c) { return (c + 15u) & ~15u; }

}  // namespace

extern "C" {

void manta_default_config(manta_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->dt = 0.5f;
  c->cell_m = 1.0f;
  c->veh_len_cells = 5;
  c->horizon_cells = 256;
  c->n_classes = 3;
  for (int i = 0; i < 8; ++i) { c->v0f[i] = 1.0f; c->T[i] = 1.5f; c->a[i] = 1.0f; c->b[i] = 2.0f; c->s0[i] = 2.0f; }
  c->lc_x0_m = 1.0f;
  c->lc_len_scale_m = 1.0f;
  c->alpha_lo = 0.05f;
  c->alpha_hi = 0.40f;
  c->g_low = 3.0f;
  c->g_high = 7.5f;
  c->g_speed_split = 11.176f;
  c->stop_dwell_steps = 4;
  c->stop_v_eps = 0.1f;
  c->stats_window_steps = 600;
  c->n_stats_windows = 96;
  c->idm_textbook = 0;
  c->t0_step = 0;
  c->seed = 1;
  c->speed_sigma_frac = 0.0f;
}

const char *manta_last_error(void) { return g_err.c_str(); }

void manta_destroy(manta_sim *S) {
  if (!S) return;
  cudaStreamSynchronize(S->stream);
  for (void *p : S->allocs) cudaFree(p);
  if (S->tape) cudaFree(S->tape);
  if (S->adj_part) cudaFree(S->adj_part);
  if (S->rep_acc) cudaFree(S->rep_acc);
  delete S;
}

manta_status manta_create(int32_t n_nodes, int32_t n_edges, const int32_t *edge_src, const int32_t *edge_dst,
                          const uint8_t *edge_lanes, const float *edge_length_m,
                          const float *edge_speed_limit_mps, const uint8_t *edge_class,
                          const uint8_t *node_type, const int32_t *node_cycle_steps,
                          const int32_t *node_offset_steps, const int16_t *edge_green_start,
                          const int16_t *edge_green_len, const uint32_t *conn_lane_mask,
                          const manta_config *cfg, void *cuda_stream, manta_sim **out) {
  g_err.clear();
  if (!out) return fail(MANTA_E_INVALID, "out is NULL");
  *out = nullptr;
  manta_status st = check_cfg(cfg);
  if (st != MANTA_OK) return st;
  if (n_nodes <= 0 || n_edges <= 0) return fail(MANTA_E_INVALID, "empty network");
  if (n_edges > (int32_t)MANTA_EDGE_MASK) return fail(MANTA_E_INVALID, "too many edges (max 2^24 - 1)");
  if (!edge_src || !edge_dst || !edge_lanes || !edge_length_m || !edge_speed_limit_mps || !edge_class || !node_type)
    return fail(MANTA_E_INVALID, "required network array is NULL");
  const int32_t N = n_nodes, E = n_edges, L = cfg->veh_len_cells;
  float s0max = 0.0f;
  for (int i = 0; i < cfg->n_classes; ++i) s0max = std::max(s0max, cfg->s0[i]);
  const uint32_t cmin = (uint32_t)(L + (int)std::ceil(s0max) + 1);
  for (int32_t n = 0; n < N; ++n) {
    if (node_type[n] > 2) return fail(MANTA_E_INVALID, "node_type out of range at node " + std::to_string(n));
    if (node_type[n] == MANTA_NODE_SIGNAL &&
        (!node_cycle_steps || !node_offset_steps || node_cycle_steps[n] < 1 || node_cycle_steps[n] > 32767))
      return fail(MANTA_E_INVALID, "signal node without a cycle in 1..32767 at node " + std::to_string(n));
  }
  manta_sim *S = new manta_sim();
  S->cfg = *cfg;
  S->stream = static_cast<cudaStream_t>(cuda_stream);
  S->N = N;
  S->E = E;
  S->cells.resize(E); S->lanes.resize(E); S->row0.resize(E); S->lane_base.resize(E + 1);
  S->esrc.assign(edge_src, edge_src + E); S->edst.assign(edge_dst, edge_dst + E);
  std::vector<EdgeMeta> em(E);
  std::vector<EdgeSig> es(E);
  uint64_t bytes = 0, canon = 0;
  uint32_t lanes_total = 0, maxC = 0;
  for (int32_t e = 0; e < E; ++e) {
    const float len = edge_length_m[e], lim = edge_speed_limit_mps[e];
    if (edge_src[e] < 0 || edge_src[e] >= N || edge_dst[e] < 0 || edge_dst[e] >= N || edge_lanes[e] < 1 ||
        edge_lanes[e] > 8 || edge_class[e] >= cfg->n_classes || !(lim > 0.0f) || !(len > 0.0f) || !(len <= 1.0e6f)) {
      delete S;
      return fail(MANTA_E_INVALID, "bad edge " + std::to_string(e));
    }
    // Section II-D: one cell per t_m = 1 m of length
    int64_t c = std::llround((double)len / (double)cfg->cell_m);
    if (c < (int64_t)cmin) c = cmin;
    S->cells[e] = (uint32_t)c;
    S->lanes[e] = edge_lanes[e];
    maxC = std::max(maxC, (uint32_t)c);
    S->row0[e] = (uint32_t)bytes;
    S->lane_base[e] = lanes_total;
    bytes += (uint64_t)stride16((uint32_t)c) * edge_lanes[e];
    canon += (uint64_t)c * edge_lanes[e];
    lanes_total += edge_lanes[e];
    if (bytes > 0xFFFFFF00ull) { delete S; return fail(MANTA_E_INVALID, "lane map larger than 4 GB"); }
    em[e].row0 = S->row0[e];
    em[e].cnl = (uint32_t)c | ((uint32_t)edge_lanes[e] << 24) | ((uint32_t)edge_class[e] << 28);
    em[e].lim = lim;
    em[e].dst = (uint32_t)edge_dst[e];
    es[e] = EdgeSig{0, 0, 0, 0};
    const int32_t n = edge_dst[e];
    if (node_type[n] == MANTA_NODE_SIGNAL) {
      if (!edge_green_start || !edge_green_len) { delete S; return fail(MANTA_E_INVALID, "signal windows are NULL"); }
      const int32_t cyc = node_cycle_steps[n];
      int64_t off = (int64_t)node_offset_steps[n] % cyc;
      if (off < 0) off += cyc;
      es[e].cyc = (int16_t)cyc;
      es[e].off = (int16_t)off;
      es[e].gs = edge_green_start[e];
      es[e].gl = edge_green_len[e];
    }
  }
  S->lane_base[E] = lanes_total;
  S->n_lanes = lanes_total;
  S->atlas_bytes = bytes;
  S->canon_bytes = canon;
  // out-edges per node (ascending id) and lane masks per (in-edge, out-edge)
  S->out_off.assign(N + 1, 0);
  for (int32_t e = 0; e < E; ++e) S->out_off[edge_src[e] + 1]++;
  for (int32_t n = 0; n < N; ++n) S->out_off[n + 1] += S->out_off[n];
  S->out_e.resize(E);
  {
    std::vector<int64_t> f(S->out_off.begin(), S->out_off.end() - 1);
    for (int32_t e = 0; e < E; ++e) S->out_e[f[edge_src[e]]++] = e;
  }
  S->conn_off.assign(E + 1, 0);
  for (int32_t e = 0; e < E; ++e) {
    const int32_t n = edge_dst[e];
    S->conn_off[e + 1] = S->conn_off[e] + (S->out_off[n + 1] - S->out_off[n]);
  }
  S->conn.resize(S->conn_off[E]);
  for (int32_t e = 0; e < E; ++e) {
    const uint32_t all = (1u << S->lanes[e]) - 1u;
    for (int64_t j = S->conn_off[e]; j < S->conn_off[e + 1]; ++j) {
      const uint32_t m = conn_lane_mask ? (conn_lane_mask[j] & all) : all;
      if (!m) { delete S; return fail(MANTA_E_INVALID, "lane mask with no lane for in-edge " + std::to_string(e)); }
      S->conn[j] = m;
    }
  }
  // request and stop-line slots numbered node by node: the in-lanes of node n
  // are slots [nin_off[n], nin_off[n + 1]) in (edge id, lane) order, and lane
  // l of edge e is slot rslot[e] + l; stop-node list
  std::vector<uint32_t> nin_off(N + 1, 0), rslot(E);
  for (int32_t e = 0; e < E; ++e) nin_off[edge_dst[e] + 1] += S->lanes[e];
  for (int32_t n = 0; n < N; ++n) nin_off[n + 1] += nin_off[n];
  {
    std::vector<uint32_t> f(nin_off.begin(), nin_off.end() - 1);
    for (int32_t e = 0; e < E; ++e) {
      rslot[e] = f[edge_dst[e]];
      f[edge_dst[e]] += S->lanes[e];
    }
  }
  std::vector<uint32_t> stops;
  for (int32_t n = 0; n < N; ++n)
    if (node_type[n] == MANTA_NODE_STOP) stops.push_back((uint32_t)n);
  // Eq. 2 probability of a mandatory change by distance to the end of the edge
  std::vector<float> mtab(maxC + 1);
  for (uint32_t d = 0; d <= maxC; ++d) {
    const double xm = (double)d * cfg->cell_m, x0 = cfg->lc_x0_m, lam = cfg->lc_len_scale_m;
    mtab[d] = (float)(xm <= x0 ? 1.0 : std::exp(-((xm - x0) / lam) * ((xm - x0) / lam)));
  }
  std::vector<uint32_t> esrc_u(E);
  for (int32_t e = 0; e < E; ++e) esrc_u[e] = (uint32_t)edge_src[e];
  // in-lane range of each edge's tail node: a departure's competitors
  std::vector<uint2> src_in(E);
  for (int32_t e = 0; e < E; ++e) src_in[e] = make_uint2(nin_off[edge_src[e]], nin_off[edge_src[e] + 1]);
  std::vector<uint32_t> lane_base_e(S->lane_base.begin(), S->lane_base.end() - 1);
  std::vector<uint8_t> ntype(node_type, node_type + N);
  // device allocations
  bool ok = true;
  Params &P = S->P;
  memset(&P, 0, sizeof(P));
  EdgeMeta *d_em = dalloc<EdgeMeta>(S, E, &ok);
  EdgeSig *d_es = dalloc<EdgeSig>(S, E, &ok);
  uint8_t *d_nt = dalloc<uint8_t>(S, N, &ok);
  uint32_t *d_esrc = dalloc<uint32_t>(S, E, &ok);
  uint2 *d_src_in = dalloc<uint2>(S, E, &ok);
  uint32_t *d_lb = dalloc<uint32_t>(S, E, &ok);
  uint32_t *d_nin_off = dalloc<uint32_t>(S, N + 1, &ok);
  uint32_t *d_rslot = dalloc<uint32_t>(S, E, &ok);
  uint32_t *d_stops = dalloc<uint32_t>(S, stops.size(), &ok);
  float *d_mtab = dalloc<float>(S, mtab.size(), &ok);
  // kMapPad padding bytes: a first scan batch may run past the last row
  P.atlas0 = dalloc<uint8_t>(S, bytes + kMapPad, &ok);
  P.atlas1 = dalloc<uint8_t>(S, bytes + kMapPad, &ok);
  P.permit = dalloc<uint32_t>(S, N, &ok);
  P.rr = dalloc<uint32_t>(S, N, &ok);
  P.req_key = dalloc<unsigned long long>(S, lanes_total, &ok);
  P.req_tgt = dalloc<uint32_t>(S, lanes_total, &ok);
  P.slot_td = dalloc<uint32_t>(S, lanes_total, &ok);
  P.slot_id = dalloc<uint32_t>(S, lanes_total, &ok);
  P.entry = dalloc<uint32_t>(S, E, &ok);
  P.exitc = dalloc<uint32_t>(S, E, &ok);
  P.lstat = dalloc<LinkStat>(S, (size_t)E * cfg->n_stats_windows, &ok);
  P.pending = dalloc<uint32_t>(S, E, &ok);
  P.q_pos = dalloc<uint32_t>(S, E, &ok);
  P.dep_key = dalloc<unsigned long long>(S, E, &ok);
  P.dep0 = dalloc<uint32_t>(S, E, &ok);
  P.dep1 = dalloc<uint32_t>(S, E, &ok);
  P.dep_info = dalloc<uint32_t>(S, 8 * (size_t)E, &ok);
  P.ctl = dalloc<Ctl>(S, 1, &ok);
  if (!ok) { manta_destroy(S); return fail(MANTA_E_OOM, "device allocation failed in manta_create"); }
  bool cp = upload(S, d_em, em) && upload(S, d_es, es) && upload(S, d_nt, ntype) && upload(S, d_esrc, esrc_u) &&
            upload(S, d_src_in, src_in) &&
            upload(S, d_lb, lane_base_e) && upload(S, d_nin_off, nin_off) && upload(S, d_rslot, rslot) &&
            upload(S, d_stops, stops) && upload(S, d_mtab, mtab);
  cp = cp && cudaMemsetAsync(P.atlas0, 0xFF, bytes + kMapPad, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.atlas1, 0xFF, bytes + kMapPad, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.permit, 0xFF, sizeof(uint32_t) * N, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.rr, 0, sizeof(uint32_t) * N, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.req_key, 0, sizeof(unsigned long long) * std::max<uint32_t>(lanes_total, 1), S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.slot_td, 0, sizeof(uint32_t) * std::max<uint32_t>(lanes_total, 1), S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.entry, 0, sizeof(uint32_t) * E, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.exitc, 0, sizeof(uint32_t) * E, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.lstat, 0, sizeof(LinkStat) * (size_t)E * cfg->n_stats_windows, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.pending, 0, sizeof(uint32_t) * E, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.q_pos, 0, sizeof(uint32_t) * E, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.dep_key, 0, sizeof(unsigned long long) * E, S->stream) == cudaSuccess &&
       cudaMemsetAsync(P.ctl, 0, sizeof(Ctl), S->stream) == cudaSuccess;
  if (!cp || cudaStreamSynchronize(S->stream) != cudaSuccess) {
    std::string m = cudaGetErrorString(cudaGetLastError());
    manta_destroy(S);
    return fail(MANTA_E_CUDA, "upload failed in manta_create: " + m);
  }
  S->em_h = em;
  S->clo_k0.assign(lanes_total ? lanes_total : 1, 0);
  S->clo_k1.assign(lanes_total ? lanes_total : 1, 0);
  long long *d_ck0 = dalloc<long long>(S, lanes_total, &ok);
  long long *d_ck1 = dalloc<long long>(S, lanes_total, &ok);
  if (!ok) {
    manta_destroy(S);
    return fail(MANTA_E_OOM, "device allocation failed in manta_create");
  }
  if (!upload(S, d_ck0, S->clo_k0) || !upload(S, d_ck1, S->clo_k1)) {
    manta_destroy(S);
    return fail(MANTA_E_CUDA, "upload failed in manta_create");
  }
  P.clo_k0 = d_ck0; P.clo_k1 = d_ck1;
  P.em = d_em; P.es = d_es; P.ntype = d_nt; P.esrc = d_esrc; P.src_in = d_src_in; P.lane_base = d_lb;
  P.nin_off = d_nin_off; P.rslot = d_rslot; P.stop_nodes = d_stops; P.mtab = d_mtab;
  P.dt = cfg->dt; P.L = cfg->veh_len_cells; P.H = cfg->horizon_cells;
  for (int i = 0; i < 8; ++i) {
    P.T[i] = cfg->T[i]; P.a[i] = cfg->a[i]; P.b[i] = cfg->b[i]; P.s0[i] = cfg->s0[i]; P.v0f[i] = cfg->v0f[i];
    P.s0c[i] = (int32_t)std::ceil(cfg->s0[i]);
  }
  P.alpha_lo = cfg->alpha_lo; P.alpha_hi = cfg->alpha_hi; P.g_low = cfg->g_low; P.g_high = cfg->g_high;
  P.g_split = cfg->g_speed_split; P.stop_eps = cfg->stop_v_eps; P.stop_dwell = cfg->stop_dwell_steps;
  P.win_steps = cfg->stats_window_steps; P.n_win = cfg->n_stats_windows; P.textbook = cfg->idm_textbook;
  P.t0 = cfg->t0_step; P.seed = cfg->seed; P.sigma_frac = cfg->speed_sigma_frac;
  P.E = (uint32_t)E; P.N = (uint32_t)N; P.n_stop = (uint32_t)stops.size(); P.mtab_n = (uint32_t)mtab.size();
  P.wait_limit_ns = kWaitLimitNs;
  P.cap_map = bytes + kMapPad;
  P.cap_lanes = lanes_total;
  S->k = cfg->t0_step;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int v = 0; v < kNumVariants; ++v) {
    const StepVariant &sv = kVariants[v];
    const size_t smem = step_smem_bytes(sv.threads);
    int per_sm = 0;
    if (cudaFuncSetAttribute(sv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sv.fn, sv.threads, smem) != cudaSuccess ||
        per_sm < 1) {
      manta_destroy(S);
      return fail(MANTA_E_CUDA, "occupancy query failed");
    }
    S->grid[v] = sms * per_sm;
  }
  *out = S;
  return MANTA_OK;
}

manta_status manta_load_trips(manta_sim *S, int64_t n, const int64_t *route_off, const int32_t *route_edges,
                              const float *depart_time_s) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (S->loaded) return fail(MANTA_E_STATE, "trips already loaded");
  if (n < 0 || n > 0x7FFFFFFE) return fail(MANTA_E_INVALID, "n_trips out of range");
  if (n > 0 && (!route_off || !route_edges || !depart_time_s)) return fail(MANTA_E_INVALID, "trip array is NULL");
  if (n > 0 && route_off[0] != 0) return fail(MANTA_E_ROUTE, "route_off[0] != 0");
  const int64_t nr = n > 0 ? route_off[n] : 0;
  if (nr < 0 || nr > 0xFFFFFFF0ll) return fail(MANTA_E_ROUTE, "too many route entries");
  // per trip on the host: route bounds, first edge, departure step; the
  // route entries themselves are checked and converted on the device
  std::vector<uint32_t> roff((size_t)n + 1), first((size_t)n);
  std::vector<int64_t> dstep((size_t)n);
  const double dt = S->cfg.dt;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t a = route_off[j], b = route_off[j + 1];
    if (b <= a || b > nr) return fail(MANTA_E_ROUTE, "empty or unordered route of trip " + std::to_string(j));
    roff[j] = (uint32_t)a;
    const int32_t e = route_edges[a];
    if (e < 0 || e >= S->E) return fail(MANTA_E_ROUTE, "route edge out of range in trip " + std::to_string(j));
    first[j] = (uint32_t)e;
    const float t = depart_time_s[j];
    if (!(t == t) || std::fabs((double)t / dt) > 2.0e9) return fail(MANTA_E_INVALID, "bad departure time of trip " + std::to_string(j));
    dstep[j] = (int64_t)std::ceil((double)t / dt);
  }
  roff[n] = (uint32_t)nr;
  auto first_edge = [&](uint32_t j) { return first[j]; };
  // trips in departure-step order (ties by id): a counting sort when the
  // steps span a modest range, else a stable comparison sort
  std::vector<uint32_t> dorder((size_t)n);
  {
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (int64_t j = 0; j < n; ++j) { lo = std::min(lo, dstep[j]); hi = std::max(hi, dstep[j]); }
    if (n > 0 && hi - lo < 4 * n + 1024) {
      std::vector<uint32_t> cnt((size_t)(hi - lo) + 2, 0u);
      for (int64_t j = 0; j < n; ++j) cnt[(size_t)(dstep[j] - lo) + 1]++;
      for (size_t i = 1; i < cnt.size(); ++i) cnt[i] += cnt[i - 1];
      for (int64_t j = 0; j < n; ++j) dorder[cnt[(size_t)(dstep[j] - lo)]++] = (uint32_t)j;
    } else {
      std::iota(dorder.begin(), dorder.end(), 0u);
      std::stable_sort(dorder.begin(), dorder.end(), [&](uint32_t a, uint32_t b) { return dstep[a] < dstep[b]; });
    }
  }
  // departure queues per first edge, ordered by (step, id): a stable counting
  // sort by first edge of the trips in departure-step order
  std::vector<uint32_t> q_off(S->E + 1, 0);
  for (int64_t j = 0; j < n; ++j) q_off[first_edge((uint32_t)j) + 1]++;
  for (int32_t e = 0; e < S->E; ++e) q_off[e + 1] += q_off[e];
  std::vector<uint32_t> order((size_t)n);
  {
    std::vector<uint32_t> at(q_off.begin(), q_off.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      const uint32_t j = dorder[i];
      order[at[first_edge(j)]++] = j;
    }
  }
  std::vector<int32_t> due_step((size_t)n);
  std::vector<uint32_t> due_edge((size_t)n);
  uint32_t prime_hi = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t d = dstep[dorder[i]];
    due_step[i] = (int32_t)std::max<int64_t>(std::min<int64_t>(d, INT32_MAX), INT32_MIN);
    due_edge[i] = first_edge(dorder[i]);
    if (d <= S->k) prime_hi = (uint32_t)(i + 1);
  }
  Params &P = S->P;
  bool ok = true;
  const size_t nbits = ((size_t)nr + 31) / 32 + 1;   // bitmaps over route entries
  uint32_t *d_nclo = dalloc<uint32_t>(S, nbits, &ok);
  uint32_t *d_starts = dalloc<uint32_t>(S, nbits, &ok);
  uint32_t *d_route = dalloc<uint32_t>(S, (size_t)nr, &ok);
  // out-edges of every node and lane masks per (in-edge, out-edge), for the route conversion
  std::vector<uint32_t> h_out_off(S->out_off.begin(), S->out_off.end()), h_out_e(S->out_e.begin(), S->out_e.end());
  std::vector<uint32_t> h_conn_off(S->conn_off.begin(), S->conn_off.end());
  uint32_t *d_out_off = dalloc<uint32_t>(S, h_out_off.size(), &ok);
  uint32_t *d_out_e = dalloc<uint32_t>(S, h_out_e.size(), &ok);
  uint32_t *d_conn_off = dalloc<uint32_t>(S, h_conn_off.size(), &ok);
  uint32_t *d_conn = dalloc<uint32_t>(S, S->conn.size(), &ok);
  unsigned long long *d_bad = dalloc<unsigned long long>(S, 1, &ok);
  uint32_t *d_roff = dalloc<uint32_t>(S, roff.size(), &ok);
  uint32_t *d_qoff = dalloc<uint32_t>(S, q_off.size(), &ok);
  uint32_t *d_qtrip = dalloc<uint32_t>(S, order.size(), &ok);
  int32_t *d_due = dalloc<int32_t>(S, due_step.size(), &ok);
  uint32_t *d_due_e = dalloc<uint32_t>(S, due_edge.size(), &ok);
  const size_t NT = (size_t)std::max<int64_t>(n, 1);
  for (int b = 0; b < 2; ++b) {
    P.vs[b].xv = dalloc<float2>(S, NT, &ok);
    P.vs[b].idr = dalloc<uint4>(S, NT, &ok);
    P.vs[b].ld = dalloc<uint32_t>(S, NT, &ok);
    P.vs[b].pc = dalloc<uint32_t>(S, NT, &ok);
    P.vs[b].em = dalloc<uint4>(S, NT, &ok);
    P.vs[b].nx = dalloc<uint32_t>(S, NT, &ok);
  }
  P.act0 = dalloc<uint32_t>(S, NT, &ok); P.act1 = dalloc<uint32_t>(S, NT, &ok);
  P.lcm = dalloc<LcMove>(S, NT, &ok);
  P.p3a = dalloc<uint32_t>(S, NT, &ok);
  // candidate overflow regions, for every launch shape: at most NT list
  // entries and NT + E merge-phase items (requests and departures) per step
  size_t NC = 1;
  for (int v = 0; v < kNumVariants; ++v) {
    const uint32_t gsz = (uint32_t)S->grid[v] * (uint32_t)kVariants[v].threads;
    NC = std::max(NC, (size_t)S->grid[v] * lc_overflow(kVariants[v].threads, gsz / 2u, gsz, (uint32_t)NT,
                                                       (uint32_t)(NT + (size_t)S->E)));
  }
  P.lcq = dalloc<Veh>(S, NC, &ok); P.lcq_pos = dalloc<uint32_t>(S, NC, &ok);
  P.cap_slots = (uint32_t)NT;
  P.cap_list = (uint32_t)NT;
  P.cap_lcq = (uint32_t)NC;
  P.req = dalloc<uint32_t>(S, NT, &ok); P.arr = dalloc<uint32_t>(S, NT, &ok);
  P.req_x = dalloc<float>(S, NT, &ok); P.req_v = dalloc<float>(S, NT, &ok); P.req_dw = dalloc<uint32_t>(S, NT, &ok);
  P.req_g = dalloc<uint32_t>(S, NT, &ok); P.req_t = dalloc<uint32_t>(S, NT, &ok);
  P.req_e2 = dalloc<uint32_t>(S, NT, &ok); P.req_n = dalloc<uint32_t>(S, NT, &ok);
  if (!ok) return fail(MANTA_E_OOM, "device allocation failed in manta_load_trips");
  bool cp = upload(S, d_roff, roff) && upload(S, d_qoff, q_off) && upload(S, d_qtrip, order) &&
            upload(S, d_due, due_step) && upload(S, d_due_e, due_edge) && upload(S, d_out_off, h_out_off) &&
            upload(S, d_out_e, h_out_e) && upload(S, d_conn_off, h_conn_off) && upload(S, d_conn, S->conn);
  cp = cp && (nr == 0 || h2d_async(d_route, route_edges, (size_t)nr * 4, S->stream) == cudaSuccess);
  cp = cp && cudaMemsetAsync(d_nclo, 0, nbits * 4, S->stream) == cudaSuccess &&
       cudaMemsetAsync(d_starts, 0, nbits * 4, S->stream) == cudaSuccess &&
       cudaMemsetAsync(d_bad, 0xFF, sizeof(unsigned long long), S->stream) == cudaSuccess;
  if (!cp) return fail(MANTA_E_CUDA, "upload failed in manta_load_trips");
  if (nr > 0) {
    const int bt = (int)std::min<int64_t>((n + 255) / 256, 4096);
    trip_start_kernel<<<bt, 256, 0, S->stream>>>(d_roff, (uint32_t)n, d_starts);
    const int br = (int)std::min<int64_t>((nr + 255) / 256, 65536);
    route_kernel<<<br, 256, 0, S->stream>>>(d_route, (uint64_t)nr, d_starts, (uint32_t)S->E, P.esrc, P.em, d_out_off,
                                           d_out_e, d_conn_off, d_conn, d_nclo, d_bad);
    unsigned long long bad = ~0ull;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
        cudaStreamSynchronize(S->stream) != cudaSuccess)
      return fail(MANTA_E_CUDA, "route conversion failed in manta_load_trips");
    if (bad != ~0ull) {
      const int64_t j = (int64_t)(std::upper_bound(roff.begin(), roff.end() - 1, (uint32_t)bad) - roff.begin()) - 1;
      return fail(MANTA_E_ROUTE, "route of trip " + std::to_string(j) +
                                     " has an edge out of range or is not contiguous");
    }
  }
  Ctl c0;
  memset(&c0, 0, sizeof(c0));
  c0.due_pos = prime_hi;
  c0.due_hi = prime_hi;
  c0.k_next = S->k;
  cp = cp && h2d_async(P.ctl, &c0, sizeof(c0), S->stream) == cudaSuccess;
  if (!cp) return fail(MANTA_E_CUDA, "upload failed in manta_load_trips");
  P.nclo = d_nclo;
  P.route = d_route; P.route_off = d_roff; P.q_off = d_qoff; P.q_trip = d_qtrip;
  P.due_step = d_due; P.due_edge = d_due_e; P.n_trips = (uint32_t)n;
  S->q_off_h = std::move(q_off);
  S->q_trip_h = std::move(order);
  S->dorder_h = std::move(dorder);
  S->first_h = std::move(first);
  S->dstep_h = std::move(dstep);
  S->route_off_h = std::move(roff);
  S->n_trips = n;
  S->prime_hi = prime_hi;
  // trips already due at the first step join their queues
  if (prime_hi > 0) {
    const int cb = (int)(S->k & 1);
    const int blocks = (int)std::min<uint32_t>((prime_hi + kBlock - 1) / kBlock, 4096u);
    prime_kernel<<<blocks, kBlock, 0, S->stream>>>(P, prime_hi, cb);
    if (cudaGetLastError() != cudaSuccess) return fail(MANTA_E_CUDA, "prime kernel launch failed");
  }
  if (cudaStreamSynchronize(S->stream) != cudaSuccess)
    return fail(MANTA_E_CUDA, std::string("manta_load_trips: ") + cudaGetErrorString(cudaGetLastError()));
  S->loaded = true;
  return MANTA_OK;
}

manta_status manta_place(manta_sim *S, int64_t n, const int64_t *trip, const int32_t *route_pos, const uint8_t *lane,
                         const float *x, const float *v) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (!S->loaded) return fail(MANTA_E_STATE, "no trips loaded");
  if (S->placed || S->k != S->cfg.t0_step) return fail(MANTA_E_STATE, "placement runs once, before the first step");
  if (S->dead) return fail(MANTA_E_STATE, "simulation stopped after an error");
  if (n < 0 || n > S->n_trips) return fail(MANTA_E_INVALID, "placement count out of range");
  if (n > 0 && (!trip || !route_pos || !lane || !x || !v)) return fail(MANTA_E_INVALID, "placement array is NULL");
  const size_t NT = (size_t)S->n_trips;
  std::vector<uint8_t> is_placed(NT, 0);
  std::vector<uint32_t> h_trip((size_t)n), h_rabs((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t j = trip[i];
    if (j < 0 || j >= S->n_trips || is_placed[(size_t)j])
      return fail(MANTA_E_INVALID, "placement " + std::to_string(i) + ": trip out of range or placed twice");
    is_placed[(size_t)j] = 1;
    const int64_t r = (int64_t)S->route_off_h[(size_t)j] + route_pos[i];
    if (route_pos[i] < 0 || r >= (int64_t)S->route_off_h[(size_t)j + 1])
      return fail(MANTA_E_INVALID, "placement " + std::to_string(i) + ": route position out of range");
    if (!(v[i] >= 0.0f) || !(v[i] < 1.0e4f))
      return fail(MANTA_E_INVALID, "placement " + std::to_string(i) + ": speed out of range");
    h_trip[(size_t)i] = (uint32_t)j;
    h_rabs[(size_t)i] = (uint32_t)r;
  }
  // Departure queues: the placed trips of each first edge move to its front,
  // in placement order, and the queue head starts past them.
  const int32_t E = S->E;
  std::vector<uint32_t> qpos(E, 0);
  for (int64_t i = 0; i < n; ++i) qpos[S->first_h[h_trip[(size_t)i]]]++;
  {
    std::vector<uint32_t> at(E), rest(E);
    for (int32_t e = 0; e < E; ++e) { at[e] = S->q_off_h[e]; rest[e] = S->q_off_h[e] + qpos[e]; }
    std::vector<uint32_t> q2(S->q_trip_h.size());
    for (int64_t i = 0; i < n; ++i) {
      const uint32_t j = h_trip[(size_t)i];
      q2[at[S->first_h[j]]++] = j;
    }
    for (int32_t e = 0; e < E; ++e)
      for (uint32_t q = S->q_off_h[e]; q < S->q_off_h[e + 1]; ++q)
        if (!is_placed[S->q_trip_h[q]]) q2[rest[e]++] = S->q_trip_h[q];
    S->q_trip_h.swap(q2);
  }
  // Trips that join departure queues when due: the unplaced ones, in
  // departure order; the freed tail is never due.
  std::vector<int32_t> due_step(NT, INT32_MAX);
  std::vector<uint32_t> due_edge(NT, 0u);
  uint32_t m = 0, prime_hi = 0;
  for (size_t i = 0; i < NT; ++i) {
    const uint32_t j = S->dorder_h[i];
    if (is_placed[j]) continue;
    const int64_t d = S->dstep_h[j];
    due_step[m] = (int32_t)std::max<int64_t>(std::min<int64_t>(d, INT32_MAX), INT32_MIN);
    due_edge[m] = S->first_h[j];
    ++m;
    if (d <= S->k) prime_hi = m;
  }
  Params &P = S->P;
  bool ok = true;
  uint32_t *d_trip = dalloc<uint32_t>(S, (size_t)n, &ok);
  uint32_t *d_rabs = dalloc<uint32_t>(S, (size_t)n, &ok);
  uint8_t *d_lane = dalloc<uint8_t>(S, (size_t)n, &ok);
  float *d_x = dalloc<float>(S, (size_t)n, &ok);
  float *d_v = dalloc<float>(S, (size_t)n, &ok);
  unsigned long long *d_bad = dalloc<unsigned long long>(S, 1, &ok);
  if (!ok) return fail(MANTA_E_OOM, "device allocation failed in manta_place");
  const int cb = (int)(S->k & 1);
  Ctl c0;
  memset(&c0, 0, sizeof(c0));
  c0.due_pos = prime_hi;
  c0.due_hi = prime_hi;
  c0.k_next = S->k;
  c0.n_act[cb] = (uint32_t)n;
  c0.cnt[CNT_DEP] = (unsigned long long)n;
  const bool cp =
      upload(S, d_trip, h_trip) && upload(S, d_rabs, h_rabs) &&
      (n == 0 || cudaMemcpyAsync(d_lane, lane, (size_t)n, cudaMemcpyHostToDevice, S->stream) == cudaSuccess) &&
      (n == 0 || cudaMemcpyAsync(d_x, x, 4 * (size_t)n, cudaMemcpyHostToDevice, S->stream) == cudaSuccess) &&
      (n == 0 || cudaMemcpyAsync(d_v, v, 4 * (size_t)n, cudaMemcpyHostToDevice, S->stream) == cudaSuccess) &&
      cudaMemsetAsync(d_bad, 0xFF, sizeof(unsigned long long), S->stream) == cudaSuccess &&
      upload(S, const_cast<uint32_t *>(P.q_trip), S->q_trip_h) &&
      upload(S, P.q_pos, qpos) &&
      upload(S, const_cast<int32_t *>(P.due_step), due_step) &&
      upload(S, const_cast<uint32_t *>(P.due_edge), due_edge) &&
      cudaMemsetAsync(P.pending, 0, sizeof(uint32_t) * (size_t)E, S->stream) == cudaSuccess &&
      cudaMemcpyAsync(P.ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, S->stream) == cudaSuccess;
  S->placed = true;
  if (!cp) { S->dead = true; return fail(MANTA_E_CUDA, "upload failed in manta_place"); }
  if (prime_hi > 0) {
    const int blocks = (int)std::min<uint32_t>((prime_hi + kBlock - 1) / kBlock, 4096u);
    prime_kernel<<<blocks, kBlock, 0, S->stream>>>(P, prime_hi, cb);
  }
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 4096);
    place_kernel<<<blocks, kBlock, 0, S->stream>>>(P, d_trip, d_rabs, d_lane, d_x, d_v, (uint32_t)n, cb, d_bad);
  }
  unsigned long long bad = ~0ull;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
      cudaStreamSynchronize(S->stream) != cudaSuccess) {
    S->dead = true;
    return fail(MANTA_E_CUDA, "placement kernels failed in manta_place");
  }
  if (bad != ~0ull) {
    S->dead = true;
    return fail(MANTA_E_INVALID, "placement " + std::to_string(bad) +
                                     ": lane, position or cell not valid (the simulation is unusable)");
  }
  return MANTA_OK;
}

manta_status manta_set_lane_closure(manta_sim *S, int32_t edge, int32_t lane, int64_t k0, int64_t k1) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (S->loaded) return fail(MANTA_E_STATE, "lane closures must be set before manta_load_trips");
  if (edge < 0 || edge >= S->E || lane < 0 || lane >= (int32_t)S->lanes[edge] || k1 < k0)
    return fail(MANTA_E_INVALID, "bad lane closure");
  const uint32_t g = S->lane_base[edge] + (uint32_t)lane;
  S->clo_k0[g] = k0;
  S->clo_k1[g] = k1;
  S->em_h[edge].dst |= MANTA_CLOSABLE;
  bool ok = cudaMemcpyAsync((void *)(S->P.clo_k0 + g), &S->clo_k0[g], sizeof(long long), cudaMemcpyHostToDevice, S->stream) == cudaSuccess &&
            cudaMemcpyAsync((void *)(S->P.clo_k1 + g), &S->clo_k1[g], sizeof(long long), cudaMemcpyHostToDevice, S->stream) == cudaSuccess &&
            cudaMemcpyAsync((void *)(S->P.em + edge), &S->em_h[edge], sizeof(EdgeMeta), cudaMemcpyHostToDevice, S->stream) == cudaSuccess &&
            cudaStreamSynchronize(S->stream) == cudaSuccess;
  if (!ok) return fail(MANTA_E_CUDA, "upload of a lane closure failed");
  return MANTA_OK;
}

namespace {
manta_status sync_and_check(manta_sim *S, Ctl *c) {
  cudaError_t e = cudaStreamSynchronize(S->stream);
  if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  if (cudaMemcpy(c, S->P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MANTA_E_CUDA, "reading the control block failed");
  if (c->err == 1) { S->dead = true; return fail(MANTA_E_TIMEOUT, "a device grid-barrier wait ran out"); }
  if (c->err != 0) {
    S->dead = true;
    return fail(MANTA_E_DEVICE, "a device index check failed (site " + std::to_string(c->err_info) + ")");
  }
  return MANTA_OK;
}
}  // namespace

namespace {
// Enqueues the launches for n_steps steps on the sim's stream: per launch of
// at most kStepsPerLaunch steps, a reset of the barrier's arrival counter and
// one cooperative launch.  With from_ctl the kernel takes its first step
// index from the control block (which every launch advances), so the same
// launches can be captured once and replayed.
manta_status enqueue_steps(manta_sim *S, int64_t n_steps, bool from_ctl) {
  const StepVariant &sv = kVariants[S->variant];
  int64_t k = S->k;
  while (n_steps > 0) {
    const int32_t chunk = (int32_t)std::min<int64_t>(n_steps, kStepsPerLaunch);
    Params P = S->P;
    P.k0 = k;
    P.k_from_ctl = from_ctl ? 1 : 0;
    P.n_steps = chunk;
    void *args[] = {&P};
    cudaError_t e = cudaMemsetAsync(&S->P.ctl->bar_count, 0, sizeof(unsigned), S->stream);
    if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("barrier reset: ") + cudaGetErrorString(e));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(S->grid[S->variant]);
    lc.blockDim = dim3(sv.threads);
    lc.dynamicSmemBytes = step_smem_bytes(sv.threads);
    lc.stream = S->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelExC(&lc, sv.fn, args);
    if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    k += chunk;
    n_steps -= chunk;
  }
  return MANTA_OK;
}
manta_status check_steppable(const manta_sim *S) {
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (!S->loaded) return fail(MANTA_E_STATE, "no trips loaded");
  if (S->dead) return fail(MANTA_E_STATE, "simulation stopped after a device error");
  return MANTA_OK;
}
}  // namespace

manta_status manta_step(manta_sim *S, int64_t n_steps) {
  g_err.clear();
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  if (n_steps < 0) return fail(MANTA_E_INVALID, "n_steps < 0");
  st = enqueue_steps(S, n_steps, false);
  if (st == MANTA_OK) S->k += n_steps;
  return st;
}

int32_t manta_variant_count(void) { return kNumVariants; }

manta_status manta_variant_info(int32_t v, int32_t *threads, int32_t *min_blocks_per_sm) {
  g_err.clear();
  if (v < 0 || v >= kNumVariants) return fail(MANTA_E_INVALID, "variant out of range");
  if (threads) *threads = kVariants[v].threads;
  if (min_blocks_per_sm) *min_blocks_per_sm = kVariants[v].min_blocks;
  return MANTA_OK;
}

manta_status manta_set_variant(manta_sim *S, int32_t v) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (v < 0 || v >= kNumVariants) return fail(MANTA_E_INVALID, "variant out of range");
  S->variant = v;
  return MANTA_OK;
}

int32_t manta_get_variant(const manta_sim *S) { return S ? S->variant : -1; }

manta_status manta_autotune(manta_sim *S, int64_t trial_steps, int32_t rounds, int32_t *chosen, float *ms) {
  g_err.clear();
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  if (trial_steps < 1 || rounds < 1) return fail(MANTA_E_INVALID, "trial_steps and rounds must be >= 1");
  // device time and vehicle updates of every shape's trials; the load of
  // the live run changes from trial to trial, so shapes are ranked by time
  // per vehicle update, and the order of the shapes alternates by round
  std::vector<double> tms(kNumVariants, 0.0), upd(kNumVariants, 0.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(MANTA_E_CUDA, "event creation failed");
  }
  Ctl c;
  st = sync_and_check(S, &c);
  unsigned long long u0 = c.cnt[CNT_UPD];
  for (int r = 0; r < rounds && st == MANTA_OK; ++r) {
    for (int j = 0; j < kNumVariants && st == MANTA_OK; ++j) {
      const int v = (r & 1) ? kNumVariants - 1 - j : j;
      S->variant = v;
      cudaEventRecord(e0, S->stream);
      st = enqueue_steps(S, trial_steps, false);
      if (st != MANTA_OK) break;
      S->k += trial_steps;
      cudaEventRecord(e1, S->stream);
      st = sync_and_check(S, &c);
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      tms[v] += t;
      upd[v] += (double)(c.cnt[CNT_UPD] - u0);
      u0 = c.cnt[CNT_UPD];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MANTA_OK) return st;
  // milliseconds per million vehicle updates (per round when a shape saw none)
  std::vector<double> score(kNumVariants);
  bool any_empty = false;
  for (int v = 0; v < kNumVariants; ++v) any_empty = any_empty || upd[v] <= 0.0;
  for (int v = 0; v < kNumVariants; ++v) score[v] = any_empty ? tms[v] / rounds : tms[v] / (upd[v] * 1e-6);
  int best = 0;
  for (int v = 1; v < kNumVariants; ++v)
    if (score[v] < score[best]) best = v;
  S->variant = best;
  if (chosen) *chosen = best;
  if (ms)
    for (int v = 0; v < kNumVariants; ++v) ms[v] = (float)score[v];
  return MANTA_OK;
}

struct manta_graph {
  manta_sim *sim;
  int64_t n_steps;
  cudaGraphExec_t exec;
};

manta_status manta_graph_capture(manta_sim *S, int64_t n_steps, manta_graph **out) {
  g_err.clear();
  if (!out) return fail(MANTA_E_INVALID, "out is NULL");
  *out = nullptr;
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  if (n_steps < 1) return fail(MANTA_E_INVALID, "n_steps < 1");
  if (!S->stream) return fail(MANTA_E_INVALID, "graph capture needs a created (non-default) stream");
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(MANTA_E_CUDA, "stream capture could not begin");
  st = enqueue_steps(S, n_steps, true);
  const cudaError_t ee = cudaStreamEndCapture(S->stream, &g);
  if (st != MANTA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ee != cudaSuccess || !g) return fail(MANTA_E_CUDA, std::string("stream capture: ") + cudaGetErrorString(ee));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(MANTA_E_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
  *out = new manta_graph{S, n_steps, ex};
  return MANTA_OK;
}

manta_status manta_graph_launch(manta_graph *G) {
  g_err.clear();
  if (!G) return fail(MANTA_E_INVALID, "graph is NULL");
  manta_status st = check_steppable(G->sim);
  if (st != MANTA_OK) return st;
  const cudaError_t e = cudaGraphLaunch(G->exec, G->sim->stream);
  if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  G->sim->k += G->n_steps;
  return MANTA_OK;
}

void manta_graph_destroy(manta_graph *G) {
  if (!G) return;
  cudaGraphExecDestroy(G->exec);
  delete G;
}


manta_status manta_stats(manta_sim *S, manta_stats_t *out) {
  g_err.clear();
  if (!S || !out) return fail(MANTA_E_INVALID, "NULL argument");
  memset(out, 0, sizeof(*out));
  out->step = S->k;
  out->loaded = S->n_trips;
  out->waiting = S->n_trips;
  if (!S->loaded) return MANTA_OK;
  Ctl c;
  manta_status st = sync_and_check(S, &c);
  if (st != MANTA_OK) return st;
  out->departed = (int64_t)c.cnt[CNT_DEP];
  out->arrived = (int64_t)c.cnt[CNT_ARR];
  out->on_network = (int64_t)c.cnt[CNT_DEP] - (int64_t)c.cnt[CNT_ARR];
  out->waiting = S->n_trips - out->departed;
  out->vehicle_updates = c.cnt[CNT_UPD];
  out->cells_scanned = c.cnt[CNT_SCAN];
  out->clamps = c.cnt[CNT_CLAMP];
  out->lane_changes = c.cnt[CNT_LC];
  out->lc_evals = c.cnt[CNT_LCE];
  out->route_reads = c.cnt[CNT_RR];
  out->lc_cells_scanned = c.cnt[CNT_LCS];
  return MANTA_OK;
}

manta_status manta_edge_counters(manta_sim *S, uint32_t *entries, uint32_t *exits, uint64_t *speed_sum_fx,
                                 uint32_t *speed_cnt, int32_t window) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if ((speed_sum_fx || speed_cnt) && (window < 0 || window >= S->cfg.n_stats_windows))
    return fail(MANTA_E_INVALID, "window out of range");
  Ctl c;
  manta_status st = sync_and_check(S, &c);
  if (st != MANTA_OK && st != MANTA_E_TIMEOUT && st != MANTA_E_DEVICE) return st;
  const size_t E = (size_t)S->E;
  bool ok = true;
  if (entries) ok = ok && cudaMemcpy(entries, S->P.entry, 4 * E, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (exits) ok = ok && cudaMemcpy(exits, S->P.exitc, 4 * E, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (speed_sum_fx || speed_cnt) {
    std::vector<LinkStat> ls(E);
    ok = ok && cudaMemcpy(ls.data(), S->P.lstat + (size_t)window * E, sizeof(LinkStat) * E, cudaMemcpyDeviceToHost) ==
                   cudaSuccess;
    for (size_t e = 0; ok && e < E; ++e) {
      if (speed_sum_fx) speed_sum_fx[e] = ls[e].sum;
      if (speed_cnt) speed_cnt[e] = ls[e].cnt;
    }
  }
  if (!ok) return fail(MANTA_E_CUDA, "copy of edge counters failed");
  return st;
}

manta_status manta_snapshot(manta_sim *S, int64_t cap, int64_t *n_out, float *x, float *v, int32_t *edge,
                            uint8_t *lane, uint32_t *id, uint8_t *dwell, int32_t *route_pos) {
  g_err.clear();
  if (!S || !n_out) return fail(MANTA_E_INVALID, "NULL argument");
  *n_out = 0;
  if (!S->loaded) return MANTA_OK;
  Ctl c;
  manta_status st = sync_and_check(S, &c);
  if (st != MANTA_OK) return st;
  const uint32_t len = c.n_act[S->k & 1];
  const int64_t live = (int64_t)c.cnt[CNT_DEP] - (int64_t)c.cnt[CNT_ARR];
  *n_out = live;
  if (live > cap) return fail(MANTA_E_INVALID, "snapshot capacity too small");
  if (live == 0) return MANTA_OK;
  const Params &P = S->P;
  const uint32_t sel = c.act_sel[S->k & 1];
  std::vector<uint32_t> act(len);
  std::vector<float2> hxv(len);
  std::vector<uint4> hidr(len);
  std::vector<uint32_t> hld(len);
  const VehSet &R = P.vs[sel];
  if (len > 0 &&
      (cudaMemcpy(act.data(), sel ? P.act1 : P.act0, 4ull * len, cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(hxv.data(), R.xv, sizeof(float2) * len, cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(hidr.data(), R.idr, sizeof(uint4) * len, cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(hld.data(), R.ld, 4ull * len, cudaMemcpyDeviceToHost) != cudaSuccess))
    return fail(MANTA_E_CUDA, "copy of vehicle state failed");
  // live list positions (an entry is its own position, a requester's marked)
  std::vector<uint32_t> pos;
  pos.reserve(len);
  for (uint32_t i = 0; i < len; ++i)
    if (act[i] != MANTA_NONE) pos.push_back(i);
  if ((int64_t)pos.size() != live) return fail(MANTA_E_DEVICE, "active list and counters disagree");
  std::sort(pos.begin(), pos.end(), [&](uint32_t a, uint32_t b) { return hidr[a].x < hidr[b].x; });
  for (size_t q = 0; q < pos.size(); ++q) {
    const uint32_t i = pos[q];
    if (x) x[q] = hxv[i].x;
    if (v) v[q] = hxv[i].y;
    if (edge) edge[q] = (int32_t)hidr[i].w;
    if (lane) lane[q] = (uint8_t)(hld[i] & 0xFu);
    if (id) id[q] = hidr[i].x;
    if (dwell) dwell[q] = (uint8_t)((hld[i] >> 8) & 0xFFu);
    if (route_pos) route_pos[q] = (int32_t)(hidr[i].y - S->route_off_h[hidr[i].x]);
  }
  return MANTA_OK;
}

manta_status manta_phase_times(manta_sim *S, double *ms4) {
  g_err.clear();
  if (!S || !ms4) return fail(MANTA_E_INVALID, "NULL argument");
  for (int q = 0; q < 4; ++q) ms4[q] = 0.0;
  if (!S->loaded) return MANTA_OK;
  Ctl c;
  manta_status st = sync_and_check(S, &c);
  for (int q = 0; q < 4; ++q) ms4[q] = (double)c.phase_ns[q] * 1e-6;
  return st;
}

int64_t manta_lane_map_bytes(const manta_sim *S) { return S ? (int64_t)S->canon_bytes : 0; }

manta_status manta_lane_map(manta_sim *S, uint8_t *out, int64_t cap, int64_t *n_out) {
  g_err.clear();
  if (!S || !n_out || !out) return fail(MANTA_E_INVALID, "NULL argument");
  *n_out = (int64_t)S->canon_bytes;
  if (cap < (int64_t)S->canon_bytes) return fail(MANTA_E_INVALID, "lane map capacity too small");
  Ctl c;
  if (S->loaded) {
    manta_status st = sync_and_check(S, &c);
    if (st != MANTA_OK) return st;
  } else if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
    return fail(MANTA_E_CUDA, "stream synchronisation failed");
  }
  std::vector<uint8_t> buf(S->atlas_bytes);
  const uint8_t *src = (S->k & 1) ? S->P.atlas1 : S->P.atlas0;
  if (cudaMemcpy(buf.data(), src, S->atlas_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MANTA_E_CUDA, "copy of the lane map failed");
  uint64_t o = 0;
  for (int32_t e = 0; e < S->E; ++e)
    for (uint32_t l = 0; l < S->lanes[e]; ++l) {
      memcpy(out + o, buf.data() + S->row0[e] + (uint64_t)l * stride16(S->cells[e]), S->cells[e]);
      o += S->cells[e];
    }
  return MANTA_OK;
}

manta_status manta_selftest_barrier_timeout(int32_t limit_ms, void *cuda_stream) {
  g_err.clear();
  if (limit_ms < 1 || limit_ms > 10000) return fail(MANTA_E_INVALID, "limit_ms out of range");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Ctl *c = nullptr;
  if (cudaMalloc(&c, sizeof(Ctl)) != cudaSuccess) return fail(MANTA_E_OOM, "selftest allocation failed");
  cudaMemsetAsync(c, 0, sizeof(Ctl), s);
  barrier_selftest_kernel<<<2, 32, 0, s>>>(c, (uint64_t)limit_ms * 1000000ull);
  cudaError_t e = cudaStreamSynchronize(s);
  Ctl h;
  memset(&h, 0, sizeof(h));
  if (e == cudaSuccess) e = cudaMemcpy(&h, c, sizeof(Ctl), cudaMemcpyDeviceToHost);
  cudaFree(c);
  if (e != cudaSuccess) return fail(MANTA_E_CUDA, cudaGetErrorString(e));
  if (h.err == 1) return fail(MANTA_E_TIMEOUT, "barrier wait ran out as expected");
  return MANTA_OK;
}

int32_t manta_debug_checks(void) {
#ifdef MANTA_CHECK_BOUNDS
  return 1;
#else
  return 0;
#endif
}

manta_status manta_debug_limit_map(manta_sim *S, int64_t bytes) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (bytes < 0 || (uint64_t)bytes > S->atlas_bytes + kMapPad) return fail(MANTA_E_INVALID, "bytes out of range");
  S->P.cap_map = (uint64_t)bytes;
  return MANTA_OK;
}

manta_status manta_debug_fail_nth(int32_t kind, int64_t nth) {
  g_err.clear();
  if (nth < 0) return fail(MANTA_E_INVALID, "nth < 0");
  if (kind == 0) t_fail_alloc = nth;
  else if (kind == 1) t_fail_copy = nth;
  else return fail(MANTA_E_INVALID, "kind must be 0 (device allocation) or 1 (host-to-device copy)");
  return MANTA_OK;
}

manta_status manta_run_noalloc(int32_t n_nodes, int32_t n_edges, const int32_t *edge_src, const int32_t *edge_dst,
                               const uint8_t *edge_lanes, const float *edge_length_m,
                               const float *edge_speed_limit_mps, const uint8_t *edge_class,
                               const uint8_t *node_type, const int32_t *node_cycle_steps,
                               const int32_t *node_offset_steps, const int16_t *edge_green_start,
                               const int16_t *edge_green_len, const uint32_t *conn_lane_mask,
                               const manta_config *cfg, int64_t n_trips, const int64_t *route_off,
                               const int32_t *route_edges, const float *depart_time_s, int64_t n_steps,
                               void *cuda_stream, manta_stats_t *stats_out, int64_t cap, int64_t *n_out, float *x,
                               float *v, int32_t *edge, uint8_t *lane, uint32_t *id, uint8_t *dwell,
                               int32_t *route_pos) {
  g_err.clear();
  if (!stats_out || !n_out) return fail(MANTA_E_INVALID, "stats_out and n_out are required");
  if (n_steps < 0) return fail(MANTA_E_INVALID, "n_steps < 0");
  // One-time set-up per device: the device address of the static arena.
  static std::mutex mu;
  static void *addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(MANTA_E_CUDA, "no current CUDA device");
  // the kernels run on cuda_stream: it must belong to the device whose arena
  // address is used (the legacy default stream follows the current device)
  if (cuda_stream) {
    int sdev = -1;
    cudaError_t e = cudaStreamGetDevice(static_cast<cudaStream_t>(cuda_stream), &sdev);
    if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("cudaStreamGetDevice: ") + cudaGetErrorString(e));
    if (sdev != dev) return fail(MANTA_E_INVALID, "cuda_stream belongs to device " + std::to_string(sdev) +
                                                      ", not the current device " + std::to_string(dev));
  }
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&addr[dev], g_noalloc_arena);
      if (e != cudaSuccess) {
        addr[dev] = nullptr;
        return fail(MANTA_E_CUDA, std::string("cudaGetSymbolAddress of the static arena: ") + cudaGetErrorString(e));
      }
    }
    base = addr[dev];
  }
  Arena arena{static_cast<unsigned char *>(base), MANTA_NOALLOC_ARENA_BYTES, 0, false};
  manta_sim *S = nullptr;
  t_arena = &arena;
  manta_status st = manta_create(n_nodes, n_edges, edge_src, edge_dst, edge_lanes, edge_length_m,
                                 edge_speed_limit_mps, edge_class, node_type, node_cycle_steps, node_offset_steps,
                                 edge_green_start, edge_green_len, conn_lane_mask, cfg, cuda_stream, &S);
  if (st == MANTA_OK) st = manta_load_trips(S, n_trips, route_off, route_edges, depart_time_s);
  t_arena = nullptr;
  if (arena.overflow) {
    if (S) manta_destroy(S);
    return fail(MANTA_E_INVALID, "network and trips need more device memory than the " +
                                     std::to_string(MANTA_NOALLOC_ARENA_BYTES >> 20) +
                                     " MiB static arena of manta_run_noalloc");
  }
  if (st == MANTA_OK) st = manta_step(S, n_steps);
  if (st == MANTA_OK) st = manta_stats(S, stats_out);
  if (st == MANTA_OK) st = manta_snapshot(S, cap, n_out, x, v, edge, lane, id, dwell, route_pos);
  const std::string msg = g_err;
  if (S) manta_destroy(S);
  g_err = msg;
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoints
namespace {
// Every device array whose content carries over from one step to the next
// (the rest is rewritten within each step before it is read, or is input).
std::vector<std::pair<void *, size_t>> mutable_state(const manta_sim *S) {
  const Params &P = S->P;
  const size_t E = (size_t)S->E, N = (size_t)S->N, G = (size_t)std::max<uint32_t>(S->n_lanes, 1);
  const size_t W = (size_t)S->cfg.n_stats_windows, NT = (size_t)std::max<int64_t>(S->n_trips, 1);
  const size_t map = (size_t)S->atlas_bytes + kMapPad;
  return {{P.atlas0, map}, {P.atlas1, map}, {P.permit, 4 * N}, {P.rr, 4 * N},
          {P.req_key, 8 * G}, {P.req_tgt, 4 * G}, {P.slot_td, 4 * G}, {P.slot_id, 4 * G},
          {P.entry, 4 * E}, {P.exitc, 4 * E}, {P.lstat, sizeof(LinkStat) * E * W},
          {P.pending, 4 * E}, {P.q_pos, 4 * E}, {P.dep_key, 8 * E}, {P.dep0, 4 * E}, {P.dep1, 4 * E},
          {P.ctl, sizeof(Ctl)}, {P.act0, 4 * NT}, {P.act1, 4 * NT},
          {P.vs[0].xv, 8 * NT}, {P.vs[0].idr, 16 * NT}, {P.vs[0].ld, 4 * NT}, {P.vs[0].pc, 4 * NT},
          {P.vs[0].em, 16 * NT}, {P.vs[1].xv, 8 * NT}, {P.vs[1].idr, 16 * NT}, {P.vs[1].ld, 4 * NT},
          {P.vs[1].pc, 4 * NT}, {P.vs[1].em, 16 * NT}, {P.vs[0].nx, 4 * NT}, {P.vs[1].nx, 4 * NT}};
}
}  // namespace

struct manta_checkpoint {
  const manta_sim *sim;
  int64_t k;
  size_t bytes;
  unsigned char *buf;
};

manta_status manta_checkpoint_save(manta_sim *S, manta_checkpoint **out) {
  g_err.clear();
  if (!out) return fail(MANTA_E_INVALID, "out is NULL");
  *out = nullptr;
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  const auto parts = mutable_state(S);
  size_t total = 0;
  for (const auto &q : parts) total += (q.second + 255u) & ~(size_t)255u;
  unsigned char *buf = nullptr;
  if (dev_malloc((void **)&buf, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(MANTA_E_OOM, "checkpoint allocation failed");
  }
  size_t off = 0;
  for (const auto &q : parts) {
    if (cudaMemcpyAsync(buf + off, q.first, q.second, cudaMemcpyDeviceToDevice, S->stream) != cudaSuccess) {
      cudaFree(buf);
      return fail(MANTA_E_CUDA, "checkpoint copy failed");
    }
    off += (q.second + 255u) & ~(size_t)255u;
  }
  *out = new manta_checkpoint{S, S->k, total, buf};
  return MANTA_OK;
}

manta_status manta_checkpoint_restore(manta_sim *S, const manta_checkpoint *c) {
  g_err.clear();
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  if (!c || c->sim != S) return fail(MANTA_E_INVALID, "checkpoint is NULL or belongs to another simulation");
  const auto parts = mutable_state(S);
  size_t off = 0;
  for (const auto &q : parts) {
    if (cudaMemcpyAsync(q.first, c->buf + off, q.second, cudaMemcpyDeviceToDevice, S->stream) != cudaSuccess)
      return fail(MANTA_E_CUDA, "checkpoint copy failed");
    off += (q.second + 255u) & ~(size_t)255u;
  }
  S->k = c->k;
  return MANTA_OK;
}

int64_t manta_checkpoint_step(const manta_checkpoint *c) { return c ? c->k : -1; }
int64_t manta_checkpoint_bytes(const manta_checkpoint *c) { return c ? (int64_t)c->bytes : 0; }

void manta_checkpoint_destroy(manta_checkpoint *c) {
  if (!c) return;
  cudaFree(c->buf);
  delete c;
}

// ---------------------------------------------------------------- event tape and adjoint
manta_status manta_tape_start(manta_sim *S, int64_t n_steps) {
  g_err.clear();
  manta_status st = check_steppable(S);
  if (st != MANTA_OK) return st;
  if (n_steps < 1 || n_steps > (1 << 30)) return fail(MANTA_E_INVALID, "n_steps out of range");
  if ((double)n_steps * (double)std::max<int64_t>(S->n_trips, 1) * (double)sizeof(TapeRec) > 1.0e15)
    return fail(MANTA_E_INVALID, "tape larger than 1 PB: record fewer steps per segment");
  const size_t need = (size_t)n_steps * (size_t)std::max<int64_t>(S->n_trips, 1);
  if (need > S->tape_cap) {
    cudaStreamSynchronize(S->stream);
    if (S->tape) cudaFree(S->tape);
    S->tape = nullptr;
    S->tape_cap = 0;
    if (dev_malloc((void **)&S->tape, need * sizeof(TapeRec)) != cudaSuccess) {
      cudaGetLastError();
      S->tape = nullptr;
      return fail(MANTA_E_OOM, "tape allocation failed");
    }
    S->tape_cap = need;
  }
  if (cudaMemsetAsync(S->tape, 0, need * sizeof(TapeRec), S->stream) != cudaSuccess)
    return fail(MANTA_E_CUDA, "tape reset failed");
  S->tape_k0 = S->k;
  S->tape_len = (int32_t)n_steps;
  S->P.tape = S->tape;
  S->P.tape_k0 = S->k;
  S->P.tape_len = (int32_t)n_steps;
  return MANTA_OK;
}

manta_status manta_tape_stop(manta_sim *S) {
  g_err.clear();
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  S->P.tape = nullptr;
  return MANTA_OK;
}

namespace {
IdmTheta theta_of(const manta_config &c) {
  IdmTheta t;
  for (int i = 0; i < 8; ++i) {
    t.v0f[i] = c.v0f[i]; t.T[i] = c.T[i]; t.a[i] = c.a[i]; t.b[i] = c.b[i]; t.s0[i] = c.s0[i];
  }
  return t;
}
manta_status check_tape(const manta_sim *S) {
  if (!S) return fail(MANTA_E_INVALID, "sim is NULL");
  if (!S->tape || S->tape_len < 1) return fail(MANTA_E_STATE, "no tape recorded");
  if (S->k < S->tape_k0 + S->tape_len) return fail(MANTA_E_STATE, "the tape segment has not been fully stepped");
  return MANTA_OK;
}
}  // namespace

static_assert(sizeof(TapeRec) == sizeof(manta_tape_record), "tape record layout");
static_assert(offsetof(TapeRec, C) == offsetof(manta_tape_record, cells), "tape record layout");
static_assert(offsetof(TapeRec, sample) == offsetof(manta_tape_record, sample), "tape record layout");

manta_status manta_tape_copy(manta_sim *S, manta_tape_record *out, int64_t cap, int64_t *n_out) {
  g_err.clear();
  if (!S || !out || !n_out) return fail(MANTA_E_INVALID, "NULL argument");
  if (!S->tape || S->tape_len < 1) return fail(MANTA_E_STATE, "no tape recorded");
  const int64_t n = (int64_t)S->tape_len * std::max<int64_t>(S->n_trips, 1);
  if (cap < n) return fail(MANTA_E_INVALID, "capacity too small for the tape");
  if (cudaStreamSynchronize(S->stream) != cudaSuccess ||
      cudaMemcpy(out, S->tape, (size_t)n * sizeof(TapeRec), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MANTA_E_CUDA, "tape copy failed");
  *n_out = n;
  return MANTA_OK;
}

manta_status manta_adjoint(manta_sim *S, const double *seed, double *lam_x, double *lam_v, double *grad) {
  g_err.clear();
  manta_status st = check_tape(S);
  if (st != MANTA_OK) return st;
  if (!seed || !lam_x || !lam_v || !grad) return fail(MANTA_E_INVALID, "NULL argument");
  const uint32_t n = (uint32_t)std::max<int64_t>(S->n_trips, 1);
  const int blocks = (int)std::min<uint32_t>((n + kAdjBlock - 1u) / kAdjBlock, 4096u);
  if (S->adj_part_cap < (size_t)blocks * 40) {
    if (S->adj_part) { cudaStreamSynchronize(S->stream); cudaFree(S->adj_part); }
    S->adj_part = nullptr;
    S->adj_part_cap = 0;
    if (dev_malloc((void **)&S->adj_part, (size_t)blocks * 40 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      S->adj_part = nullptr;
      return fail(MANTA_E_OOM, "adjoint scratch allocation failed");
    }
    S->adj_part_cap = (size_t)blocks * 40;
  }
  adjoint_kernel<<<blocks, kAdjBlock, 0, S->stream>>>(S->tape, S->tape_len, (uint32_t)S->n_trips, (double)S->cfg.dt,
                                                      theta_of(S->cfg), seed, lam_x, lam_v, S->adj_part);
  adjoint_grad_kernel<<<1, 64, 0, S->stream>>>(S->adj_part, blocks, grad, 5 * S->cfg.n_classes);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
  return MANTA_OK;
}

manta_status manta_replay(manta_sim *S, const double *theta, double *x, double *v, uint8_t *present, double *sums) {
  g_err.clear();
  manta_status st = check_tape(S);
  if (st != MANTA_OK) return st;
  if (!theta || !x || !v || !present || !sums) return fail(MANTA_E_INVALID, "NULL argument");
  IdmTheta th;
  memset(&th, 0, sizeof(th));
  for (int c = 0; c < S->cfg.n_classes && c < 8; ++c) {
    th.v0f[c] = theta[5 * c]; th.T[c] = theta[5 * c + 1]; th.a[c] = theta[5 * c + 2];
    th.b[c] = theta[5 * c + 3]; th.s0[c] = theta[5 * c + 4];
  }
  const uint32_t n = (uint32_t)std::max<int64_t>(S->n_trips, 1);
  const int blocks = (int)std::min<uint32_t>((n + 255u) / 256u, 4096u);
  const size_t cells = (size_t)S->cfg.n_stats_windows * (size_t)S->E;
  if (S->rep_acc_cap < 2 * cells) {
    if (S->rep_acc) { cudaStreamSynchronize(S->stream); cudaFree(S->rep_acc); }
    S->rep_acc = nullptr;
    S->rep_acc_cap = 0;
    if (dev_malloc((void **)&S->rep_acc, 2 * cells * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      S->rep_acc = nullptr;
      return fail(MANTA_E_OOM, "replay scratch allocation failed");
    }
    S->rep_acc_cap = 2 * cells;
  }
  if (cudaMemsetAsync(S->rep_acc, 0, 2 * cells * sizeof(unsigned long long), S->stream) != cudaSuccess)
    return fail(MANTA_E_CUDA, "replay scratch reset failed");
  replay_kernel<<<blocks, 256, 0, S->stream>>>(S->tape, S->tape_len, (uint32_t)S->n_trips, (double)S->cfg.dt, th,
                                               x, v, present, S->rep_acc);
  const int sb = (int)std::min<size_t>((cells + 255) / 256, 4096);
  replay_sums_kernel<<<sb, 256, 0, S->stream>>>(S->rep_acc, cells, sums);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MANTA_E_CUDA, std::string("replay launch: ") + cudaGetErrorString(e));
  return MANTA_OK;
}
