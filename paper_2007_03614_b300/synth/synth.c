/*
 * synth.c -- seeded synthetic road networks and trip tables.
 *
 * Input generation only: this file holds none of the simulation's arithmetic.
 * It stands in for the paper's data pipeline (Section II-A street network,
 * Section II-B demand, Section II-C routing), none of whose data sets exist
 * here.  Both the CPU oracle and the CUDA library consume what it writes.
 *
 *  - Lattice networks: nodes on an nx x ny lattice, two directed edges per kept
 *    segment.  Rows/columns are classed local / arterial / freeway; local
 *    segments are deleted at random; the largest connected component is kept
 *    (every node reaches every other node, Section II-A).  Segment lengths are
 *    lognormal and clamped.  Fixed-time signals sit at arterial crossings.
 *    A per-(in-edge, out-edge) lane mask encodes which lanes may take a turn.
 *  - Trips: uniform OD node pairs or a gravity model over rectangular zones with
 *    origins/destinations sampled uniformly inside the zone (Section II-B);
 *    departure times uniform or truncated-normal (Section II-D).
 *  - Routes: Dijkstra shortest free-flow travel time (integer milliseconds,
 *    ties to the lower edge id), one tree per distinct origin node, computed
 *    only for the OD pairs needed (Section II-C), parallel over origins.
 *
 * Sequential random numbers come from SplitMix64 (Steele, Lea, Flood 2014).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYNTH_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ RNG -- */
typedef struct { uint64_t s; } rng_t;
static uint64_t rng_next(rng_t *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_normal(rng_t *r) {
  /* Box-Muller on two uniforms in (0,1]. */
  double u1 = 1.0 - rng_u01(r), u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
static uint64_t rng_below(rng_t *r, uint64_t n) { return n ? rng_next(r) % n : 0; }

/* -------------------------------------------------------------- network -- */
typedef struct {
  int32_t n_nodes, n_edges;
  int32_t *edge_src, *edge_dst;
  uint8_t *edge_lanes, *edge_class;
  float *edge_length_m, *edge_speed_mps;
  uint8_t *node_type;
  int32_t *node_cycle, *node_offset;
  int16_t *edge_green_start, *edge_green_len;
  int64_t n_conn;
  uint32_t *conn_lane_mask;
  int32_t *node_i, *node_j;       /* lattice coordinates of each kept node */
  uint8_t *edge_dir;              /* 0 +i, 1 +j, 2 -i, 3 -j                */
  uint8_t *node_trip_ok;          /* 1 if trips may start or end at the node */
} synth_net;

typedef struct {
  int32_t nx, ny;
  int32_t arterial_every, freeway_every;   /* 0 disables the class        */
  double  local_keep;                      /* keep probability, local      */
  double  len_median_m, len_sigma, len_min_m, len_max_m;
  float   speed_mps[3];                    /* local, arterial, freeway     */
  uint8_t lanes[3];
  int32_t signal_cycle_steps, signal_green_steps;
  int32_t signals_at;     /* 0 none, 1 arterial x arterial (incl. freeway rows excluded), 2 interior nodes */
  int32_t all_stop;       /* 1: every node is a flashing red (stop) node       */
  int32_t limited_access; /* 1: local streets pass over freeways (no junction);
                             only arterial and freeway crossings are interchanges */
  uint64_t seed;
} synth_lattice_params;

static int seg_class(const synth_lattice_params *p, int32_t line) {
  if (p->freeway_every > 0 && line % p->freeway_every == 0) return 2;
  if (p->arterial_every > 0 && line % p->arterial_every == 0) return 1;
  return 0;
}

SYNTH_API void synth_net_free(synth_net *n) {
  if (!n) return;
  free(n->edge_src); free(n->edge_dst); free(n->edge_lanes); free(n->edge_class);
  free(n->edge_length_m); free(n->edge_speed_mps); free(n->node_type);
  free(n->node_cycle); free(n->node_offset); free(n->edge_green_start);
  free(n->edge_green_len); free(n->conn_lane_mask); free(n->node_i); free(n->node_j);
  free(n->edge_dir); free(n->node_trip_ok); free(n);
}

SYNTH_API synth_net *synth_lattice(const synth_lattice_params *p) {
  const int32_t nx = p->nx, ny = p->ny;
  const int64_t NN = (int64_t)nx * ny;
  /* segments: horizontal h(i,j) between (i,j),(i+1,j); vertical v(i,j) between (i,j),(i,j+1) */
  const int64_t NH = (int64_t)(nx - 1) * ny, NV = (int64_t)nx * (ny - 1);
  uint8_t *keep = (uint8_t *)malloc((size_t)(NH + NV));
  float *slen = (float *)malloc(sizeof(float) * (size_t)(NH + NV));
  uint8_t *scls = (uint8_t *)malloc((size_t)(NH + NV));
  rng_t r = { p->seed * 0x9E3779B97F4A7C15ULL + 12345 };
  for (int64_t s = 0; s < NH + NV; ++s) {
    int32_t line = s < NH ? (int32_t)((s) / (nx - 1)) /* row j */ : (int32_t)((s - NH) % nx) /* col i */;
    int c = seg_class(p, line);
    scls[s] = (uint8_t)c;
    double u = rng_u01(&r);
    keep[s] = (c > 0) ? 1 : (u < p->local_keep);
    double z = rng_normal(&r);
    double L = p->len_median_m * exp(p->len_sigma * z);
    if (L < p->len_min_m) L = p->len_min_m;
    if (L > p->len_max_m) L = p->len_max_m;
    slen[s] = (float)L;
  }
  /* Per node and direction (0 +i, 1 +j, 2 -i, 3 -j): neighbour node and
     segment.  With limited access a local street crossing a freeway becomes
     one overpass segment that skips the freeway node. */
  const int64_t NSEG = NH + NV + 2 * (int64_t)nx * ny / 1 + 1;
  slen = (float *)realloc(slen, sizeof(float) * (size_t)NSEG);
  scls = (uint8_t *)realloc(scls, (size_t)NSEG);
  int64_t nseg = NH + NV;
  int64_t *nbn = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)NN);
  int64_t *nbs = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)NN);
  for (int64_t v = 0; v < NN; ++v) {
    int32_t i = (int32_t)(v % nx), j = (int32_t)(v / nx);
    int64_t sg[4], nb[4];
    sg[0] = i + 1 < nx ? (int64_t)j * (nx - 1) + i : -1;       nb[0] = v + 1;
    sg[1] = j + 1 < ny ? NH + (int64_t)j * nx + i : -1;        nb[1] = v + nx;
    sg[2] = i > 0 ? (int64_t)j * (nx - 1) + (i - 1) : -1;      nb[2] = v - 1;
    sg[3] = j > 0 ? NH + (int64_t)(j - 1) * nx + i : -1;       nb[3] = v - nx;
    for (int d = 0; d < 4; ++d) {
      const int ok = sg[d] >= 0 && keep[sg[d]];
      nbn[v * 4 + d] = ok ? nb[d] : -1;
      nbs[v * 4 + d] = ok ? sg[d] : -1;
    }
  }
  uint8_t *trip_ok = (uint8_t *)malloc((size_t)NN);
  for (int64_t v = 0; v < NN; ++v) {
    int32_t i = (int32_t)(v % nx), j = (int32_t)(v / nx);
    trip_ok[v] = !(p->limited_access && (seg_class(p, i) == 2 || seg_class(p, j) == 2));
  }
  if (p->limited_access) {
    for (int64_t v = 0; v < NN; ++v) {
      int32_t i = (int32_t)(v % nx), j = (int32_t)(v / nx);
      /* freeway row j crossed by a local column i, or freeway column i crossed by a local row j */
      for (int axis = 0; axis < 2; ++axis) {
        const int fw = axis == 0 ? seg_class(p, j) == 2 : seg_class(p, i) == 2;
        const int loc = axis == 0 ? seg_class(p, i) == 0 : seg_class(p, j) == 0;
        if (!fw || !loc) continue;
        const int dp = axis == 0 ? 1 : 0, dm = dp + 2;        /* +j/-j across a row, +i/-i across a column */
        const int64_t up = nbn[v * 4 + dp], dn = nbn[v * 4 + dm];
        const int64_t su = nbs[v * 4 + dp], sd = nbs[v * 4 + dm];
        nbn[v * 4 + dp] = nbn[v * 4 + dm] = -1;
        nbs[v * 4 + dp] = nbs[v * 4 + dm] = -1;
        if (up >= 0) { nbn[up * 4 + dm] = -1; nbs[up * 4 + dm] = -1; }
        if (dn >= 0) { nbn[dn * 4 + dp] = -1; nbs[dn * 4 + dp] = -1; }
        if (up >= 0 && dn >= 0) {
          const int64_t o = nseg++;
          slen[o] = slen[su] + slen[sd];
          scls[o] = 0;
          nbn[dn * 4 + dp] = up; nbs[dn * 4 + dp] = o;
          nbn[up * 4 + dm] = dn; nbs[up * 4 + dm] = o;
        }
      }
    }
  }
  /* largest connected component by BFS */
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)NN);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)NN);
  for (int64_t v = 0; v < NN; ++v) comp[v] = -1;
  int32_t ncomp = 0, best = -1; int64_t best_size = 0;
  for (int64_t s0 = 0; s0 < NN; ++s0) {
    if (comp[s0] >= 0) continue;
    int64_t qh = 0, qt = 0; queue[qt++] = (int32_t)s0; comp[s0] = ncomp;
    while (qh < qt) {
      int32_t v = queue[qh++];
      for (int d = 0; d < 4; ++d) {
        const int64_t w = nbn[(int64_t)v * 4 + d];
        if (w >= 0 && comp[w] < 0) { comp[w] = ncomp; queue[qt++] = (int32_t)w; }
      }
    }
    if (qt > best_size) { best_size = qt; best = ncomp; }
    ++ncomp;
  }
  int32_t *nid = (int32_t *)malloc(sizeof(int32_t) * (size_t)NN);
  int32_t nn = 0;
  for (int64_t v = 0; v < NN; ++v) nid[v] = comp[v] == best ? nn++ : -1;
  /* count edges in a fixed order: by source node, then direction 0..3 */
  int64_t ne = 0;
  for (int pass = 0; pass < 2; ++pass) {
    synth_net *out = NULL;
    if (pass == 1) {
      out = (synth_net *)calloc(1, sizeof(synth_net));
      out->n_nodes = nn; out->n_edges = (int32_t)ne;
      out->edge_src = (int32_t *)malloc(4 * (size_t)ne); out->edge_dst = (int32_t *)malloc(4 * (size_t)ne);
      out->edge_lanes = (uint8_t *)malloc((size_t)ne); out->edge_class = (uint8_t *)malloc((size_t)ne);
      out->edge_dir = (uint8_t *)malloc((size_t)ne);
      out->edge_length_m = (float *)malloc(4 * (size_t)ne); out->edge_speed_mps = (float *)malloc(4 * (size_t)ne);
      out->edge_green_start = (int16_t *)calloc((size_t)ne, 2); out->edge_green_len = (int16_t *)calloc((size_t)ne, 2);
      out->node_type = (uint8_t *)calloc((size_t)nn, 1);
      out->node_cycle = (int32_t *)calloc((size_t)nn, 4); out->node_offset = (int32_t *)calloc((size_t)nn, 4);
      out->node_i = (int32_t *)malloc(4 * (size_t)nn); out->node_j = (int32_t *)malloc(4 * (size_t)nn);
      out->node_trip_ok = (uint8_t *)malloc((size_t)nn);
    }
    int64_t e = 0;
    for (int64_t v = 0; v < NN; ++v) {
      if (nid[v] < 0) continue;
      int32_t i = (int32_t)(v % nx), j = (int32_t)(v / nx);
      if (pass == 1) { out->node_i[nid[v]] = i; out->node_j[nid[v]] = j; out->node_trip_ok[nid[v]] = trip_ok[v]; }
      for (int d = 0; d < 4; ++d) {
        const int64_t w = nbn[v * 4 + d], sgi = nbs[v * 4 + d];
        if (w < 0 || nid[w] < 0) continue;
        if (pass == 1) {
          int c = scls[sgi];
          out->edge_src[e] = nid[v]; out->edge_dst[e] = nid[w];
          out->edge_class[e] = (uint8_t)c; out->edge_lanes[e] = p->lanes[c];
          out->edge_speed_mps[e] = p->speed_mps[c]; out->edge_length_m[e] = slen[sgi];
          out->edge_dir[e] = (uint8_t)d;
        }
        ++e;
      }
    }
    if (pass == 0) { ne = e; continue; }
    /* node control */
    for (int32_t n = 0; n < nn; ++n) {
      int32_t i = out->node_i[n], j = out->node_j[n];
      int sig = 0;
      if (p->signals_at == 1) {
        int ci = seg_class(p, i), cj = seg_class(p, j);
        sig = (ci == 1 && cj == 1);
      } else if (p->signals_at == 2) {
        sig = (i > 0 && j > 0 && i < nx - 1 && j < ny - 1);
      }
      if (p->all_stop) out->node_type[n] = 1;
      else if (sig) {
        out->node_type[n] = 2;
        out->node_cycle[n] = p->signal_cycle_steps;
        out->node_offset[n] = 0;
      }
    }
    /* signal windows per in-edge: +-j approaches (north-south) first, +-i second */
    for (int64_t k = 0; k < ne; ++k) {
      int32_t n = out->edge_dst[k];
      if (out->node_type[n] != 2) continue;
      int ns = (out->edge_dir[k] == 1 || out->edge_dir[k] == 3);
      out->edge_green_start[k] = (int16_t)(ns ? 0 : p->signal_green_steps);
      out->edge_green_len[k] = (int16_t)p->signal_green_steps;
    }
    /* lane masks per (in-edge, out-edge of its head node), out-edges in ascending edge id */
    int64_t *out_off = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t k = 0; k < ne; ++k) out_off[out->edge_src[k] + 1]++;
    for (int32_t n = 0; n < nn; ++n) out_off[n + 1] += out_off[n];
    /* edges are emitted grouped by source node in ascending order, so out-edges
       of node n are the contiguous id range [out_off[n], out_off[n+1]). */
    int64_t nc = 0;
    for (int64_t k = 0; k < ne; ++k) { int32_t n = out->edge_dst[k]; nc += out_off[n + 1] - out_off[n]; }
    out->n_conn = nc;
    out->conn_lane_mask = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nc ? nc : 1));
    int64_t c = 0;
    for (int64_t k = 0; k < ne; ++k) {
      int32_t n = out->edge_dst[k];
      int nl = out->edge_lanes[k];
      uint32_t all = (1u << nl) - 1u;
      for (int64_t k2 = out_off[n]; k2 < out_off[n + 1]; ++k2) {
        int turn = ((int)out->edge_dir[k2] - (int)out->edge_dir[k] + 4) % 4;  /* 0 straight, 1 left, 2 U, 3 right */
        uint32_t m;
        if (turn == 0) m = all;
        else if (turn == 3) m = 1u;                 /* right turn from the curb lane */
        else m = 1u << (nl - 1);                    /* left turn / U-turn from the median lane */
        out->conn_lane_mask[c++] = m;
      }
    }
    free(out_off);
    free(keep); free(slen); free(scls); free(comp); free(queue); free(nid);
    free(nbn); free(nbs); free(trip_ok);
    return out;
  }
  return NULL;
}

/* ------------------------------------------------------------ routing -- */
typedef struct { int64_t d; int32_t v; } hent;
typedef struct { hent *a; int64_t n, cap; } heap_t;
static void heap_push(heap_t *h, int64_t d, int32_t v) {
  if (h->n == h->cap) { h->cap = h->cap ? 2 * h->cap : 1024; h->a = (hent *)realloc(h->a, sizeof(hent) * (size_t)h->cap); }
  int64_t i = h->n++;
  while (i > 0) {
    int64_t pnt = (i - 1) >> 1;
    hent q = h->a[pnt];
    if (q.d < d || (q.d == d && q.v <= v)) break;
    h->a[i] = q; i = pnt;
  }
  h->a[i].d = d; h->a[i].v = v;
}
static hent heap_pop(heap_t *h) {
  hent top = h->a[0];
  hent last = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= h->n) break;
    if (c + 1 < h->n && (h->a[c + 1].d < h->a[c].d || (h->a[c + 1].d == h->a[c].d && h->a[c + 1].v < h->a[c].v))) ++c;
    if (last.d < h->a[c].d || (last.d == h->a[c].d && last.v <= h->a[c].v)) break;
    h->a[i] = h->a[c]; i = c;
  }
  if (h->n) h->a[i] = last;
  return top;
}

typedef struct {
  int64_t n_trips;
  int32_t *origin, *dest;
  float *depart_time_s;
  int64_t *route_off;
  int32_t *route_edges;
  int64_t n_route_edges;
  int64_t n_unroutable;
} synth_trips;

SYNTH_API void synth_trips_free(synth_trips *t) {
  if (!t) return;
  free(t->origin); free(t->dest); free(t->depart_time_s); free(t->route_off); free(t->route_edges); free(t);
}

/* Route every trip: Dijkstra from each distinct origin (integer ms weights,
   lexicographic (dist, node) settle order, ties in the predecessor broken to
   the lower edge id), early exit once every destination of that origin is
   settled. */
static void route_all(int32_t n_nodes, int32_t n_edges, const int32_t *esrc, const int32_t *edst,
                      const float *len, const float *spd, synth_trips *t, int n_threads) {
  int64_t *out_off = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  int32_t *out_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_edges);
  int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_edges);
  for (int32_t e = 0; e < n_edges; ++e) {
    out_off[esrc[e] + 1]++;
    int64_t ms = llround((double)len[e] / (double)spd[e] * 1000.0);
    w[e] = ms < 1 ? 1 : ms;
  }
  for (int32_t n = 0; n < n_nodes; ++n) out_off[n + 1] += out_off[n];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_nodes);
  memcpy(fill, out_off, sizeof(int64_t) * (size_t)n_nodes);
  for (int32_t e = 0; e < n_edges; ++e) out_e[fill[esrc[e]]++] = e;  /* ascending edge id per node */
  free(fill);
  /* group trips by origin */
  const int64_t nt = t->n_trips;
  int64_t *ooff = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  int64_t *otrip = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt ? nt : 1));
  for (int64_t k = 0; k < nt; ++k) ooff[t->origin[k] + 1]++;
  for (int32_t n = 0; n < n_nodes; ++n) ooff[n + 1] += ooff[n];
  int64_t *of2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_nodes);
  memcpy(of2, ooff, sizeof(int64_t) * (size_t)n_nodes);
  for (int64_t k = 0; k < nt; ++k) otrip[of2[t->origin[k]]++] = k;
  free(of2);
  int32_t *origins = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
  int32_t n_orig = 0;
  for (int32_t n = 0; n < n_nodes; ++n) if (ooff[n + 1] > ooff[n]) origins[n_orig++] = n;
  int32_t *rlen = (int32_t *)calloc((size_t)(nt ? nt : 1), sizeof(int32_t));
  /* per-trip route buffers: each thread appends into its own growable array */
  int nthr = n_threads > 0 ? n_threads : 1;
  int32_t **tbuf = (int32_t **)calloc((size_t)nthr, sizeof(int32_t *));
  int64_t *tcap = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
  int64_t *tlen = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
  int64_t *tpos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt ? nt : 1));  /* position in its thread buffer */
  int32_t *towner = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
  int64_t unroutable = 0;
#pragma omp parallel num_threads(nthr) reduction(+ : unroutable)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_nodes);
    int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
    uint32_t *stamp = (uint32_t *)calloc((size_t)n_nodes, sizeof(uint32_t));
    uint32_t *tgt = (uint32_t *)calloc((size_t)n_nodes, sizeof(uint32_t));
    uint8_t *done = (uint8_t *)calloc((size_t)n_nodes, 1);
    heap_t h = { 0, 0, 0 };
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
    uint32_t epoch = 0;
#pragma omp for schedule(dynamic, 4)
    for (int32_t oi = 0; oi < n_orig; ++oi) {
      int32_t o = origins[oi];
      ++epoch;
      int64_t need = 0;
      for (int64_t q = ooff[o]; q < ooff[o + 1]; ++q) {
        int32_t d = t->dest[otrip[q]];
        if (tgt[d] != epoch) { tgt[d] = epoch; ++need; }
      }
      h.n = 0;
      stamp[o] = epoch; dist[o] = 0; pred[o] = -1; done[o] = 0;
      heap_push(&h, 0, o);
      while (h.n && need > 0) {
        hent top = heap_pop(&h);
        int32_t u = top.v;
        if (done[u] && stamp[u] == epoch) continue;
        if (top.d != dist[u]) continue;
        done[u] = 1;
        if (tgt[u] == epoch) --need;
        for (int64_t q = out_off[u]; q < out_off[u + 1]; ++q) {
          int32_t e = out_e[q], v = edst[e];
          int64_t nd = top.d + w[e];
          if (stamp[v] != epoch) { stamp[v] = epoch; done[v] = 0; dist[v] = nd; pred[v] = e; heap_push(&h, nd, v); }
          else if (!done[v]) {
            if (nd < dist[v]) { dist[v] = nd; pred[v] = e; heap_push(&h, nd, v); }
            else if (nd == dist[v] && e < pred[v]) pred[v] = e;
          }
        }
      }
      for (int64_t q = ooff[o]; q < ooff[o + 1]; ++q) {
        int64_t trip = otrip[q];
        int32_t d = t->dest[trip];
        towner[trip] = tid;
        if (stamp[d] != epoch || !done[d] || d == o) { rlen[trip] = 0; tpos[trip] = 0; ++unroutable; continue; }
        int32_t m = 0, x = d;
        while (x != o) { int32_t e = pred[x]; tmp[m++] = e; x = esrc[e]; }
        if (tlen[tid] + m > tcap[tid]) {
          int64_t nc = tcap[tid] ? tcap[tid] : (1 << 20);
          while (nc < tlen[tid] + m) nc *= 2;
          tbuf[tid] = (int32_t *)realloc(tbuf[tid], sizeof(int32_t) * (size_t)nc); tcap[tid] = nc;
        }
        for (int32_t z = 0; z < m; ++z) tbuf[tid][tlen[tid] + z] = tmp[m - 1 - z];
        tpos[trip] = tlen[tid]; tlen[tid] += m; rlen[trip] = m;
      }
    }
    free(dist); free(pred); free(stamp); free(tgt); free(done); free(h.a); free(tmp);
  }
  t->route_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt + 1));
  t->route_off[0] = 0;
  for (int64_t k = 0; k < nt; ++k) t->route_off[k + 1] = t->route_off[k] + rlen[k];
  t->n_route_edges = t->route_off[nt];
  t->route_edges = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t->n_route_edges ? t->n_route_edges : 1));
#pragma omp parallel for num_threads(nthr) schedule(static)
  for (int64_t k = 0; k < nt; ++k)
    if (rlen[k]) memcpy(t->route_edges + t->route_off[k], tbuf[towner[k]] + tpos[k], sizeof(int32_t) * (size_t)rlen[k]);
  t->n_unroutable = unroutable;
  for (int z = 0; z < nthr; ++z) free(tbuf[z]);
  free(tbuf); free(tcap); free(tlen); free(tpos); free(towner); free(rlen);
  free(out_off); free(out_e); free(w); free(ooff); free(otrip); free(origins);
}

typedef struct {
  int64_t n_trips;
  int32_t od_model;            /* 0 uniform node pairs, 1 gravity over zones */
  int32_t zones_x, zones_y, pool_per_zone;
  double  spacing_km, beta_km, zone_mass_sigma;
  int32_t depart_model;        /* 0 uniform [lo,hi), 1 truncated normal, 2 two-component mixture */
  double  t_lo_s, t_hi_s, mean_s, sd_s, mean2_s, sd2_s, w2;
  uint64_t seed;
  int32_t n_threads;
} synth_trip_params;

SYNTH_API synth_trips *synth_make_trips(const synth_net *net, const synth_trip_params *p) {
  synth_trips *t = (synth_trips *)calloc(1, sizeof(synth_trips));
  const int64_t nt = p->n_trips;
  t->n_trips = nt;
  t->origin = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
  t->dest = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
  t->depart_time_s = (float *)malloc(sizeof(float) * (size_t)(nt ? nt : 1));
  rng_t r = { p->seed * 0xD1B54A32D192ED03ULL + 777 };
  const int32_t nn = net->n_nodes;
  /* trip ends only at nodes flagged for it (not on limited-access freeways) */
  int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
  int32_t n_ends = 0;
  for (int32_t n = 0; n < nn; ++n)
    if (!net->node_trip_ok || net->node_trip_ok[n]) ends[n_ends++] = n;
  if (p->od_model == 0) {
    /* uniform OD; with pool_per_zone > 0 the origins come from that many
       uniformly drawn nodes (one shortest-path tree per pool node) */
    int32_t *opool = NULL;
    int32_t np_ = 0;
    if (p->pool_per_zone > 0 && p->pool_per_zone < n_ends) {
      np_ = p->pool_per_zone;
      opool = (int32_t *)malloc(sizeof(int32_t) * (size_t)np_);
      for (int32_t q = 0; q < np_; ++q) opool[q] = ends[rng_below(&r, (uint64_t)n_ends)];
    }
    for (int64_t k = 0; k < nt; ++k) {
      int32_t o = opool ? opool[rng_below(&r, (uint64_t)np_)] : ends[rng_below(&r, (uint64_t)n_ends)], d;
      do { d = ends[rng_below(&r, (uint64_t)n_ends)]; } while (d == o && n_ends > 1);
      t->origin[k] = o; t->dest[k] = d;
    }
    free(opool);
  } else {
    /* zones: rectangular blocks of the lattice */
    int32_t maxi = 0, maxj = 0;
    for (int32_t n = 0; n < nn; ++n) { if (net->node_i[n] > maxi) maxi = net->node_i[n]; if (net->node_j[n] > maxj) maxj = net->node_j[n]; }
    const int32_t ZX = p->zones_x, ZY = p->zones_y, NZ = ZX * ZY;
    int32_t *zone = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    int64_t *zoff = (int64_t *)calloc((size_t)NZ + 1, sizeof(int64_t));
    for (int32_t q = 0; q < n_ends; ++q) {
      const int32_t n = ends[q];
      int32_t zx = (int32_t)((int64_t)net->node_i[n] * ZX / (maxi + 1));
      int32_t zy = (int32_t)((int64_t)net->node_j[n] * ZY / (maxj + 1));
      zone[n] = zy * ZX + zx; zoff[zone[n] + 1]++;
    }
    for (int32_t z = 0; z < NZ; ++z) zoff[z + 1] += zoff[z];
    int32_t *znodes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    int64_t *zf = (int64_t *)malloc(sizeof(int64_t) * (size_t)NZ);
    memcpy(zf, zoff, sizeof(int64_t) * (size_t)NZ);
    for (int32_t q = 0; q < n_ends; ++q) znodes[zf[zone[ends[q]]]++] = ends[q];
    free(zf);
    /* origin pools: pool_per_zone nodes drawn uniformly from each zone */
    int32_t P = p->pool_per_zone;
    int32_t *pool = (int32_t *)malloc(sizeof(int32_t) * (size_t)NZ * (size_t)P);
    double *mass = (double *)malloc(sizeof(double) * (size_t)NZ);
    double *cx = (double *)malloc(sizeof(double) * (size_t)NZ), *cy = (double *)malloc(sizeof(double) * (size_t)NZ);
    for (int32_t z = 0; z < NZ; ++z) {
      int64_t cnt = zoff[z + 1] - zoff[z];
      for (int32_t q = 0; q < P; ++q) pool[(int64_t)z * P + q] = cnt ? znodes[zoff[z] + (int64_t)rng_below(&r, (uint64_t)cnt)] : -1;
      mass[z] = cnt ? exp(p->zone_mass_sigma * rng_normal(&r)) : 0.0;
      cx[z] = ((z % ZX) + 0.5) * (double)(maxi + 1) / ZX * p->spacing_km;
      cy[z] = ((z / ZX) + 0.5) * (double)(maxj + 1) / ZY * p->spacing_km;
    }
    /* joint OD table, cumulative for inverse-CDF sampling */
    double *cum = (double *)malloc(sizeof(double) * (size_t)NZ * (size_t)NZ);
    double acc = 0.0;
    for (int32_t a = 0; a < NZ; ++a)
      for (int32_t b = 0; b < NZ; ++b) {
        double dx = cx[a] - cx[b], dy = cy[a] - cy[b];
        acc += mass[a] * mass[b] * exp(-sqrt(dx * dx + dy * dy) / p->beta_km);
        cum[(int64_t)a * NZ + b] = acc;
      }
    for (int64_t k = 0; k < nt; ++k) {
      double u = rng_u01(&r) * acc;
      int64_t lo = 0, hi = (int64_t)NZ * NZ - 1;
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (cum[mid] > u) hi = mid; else lo = mid + 1; }
      int32_t za = (int32_t)(lo / NZ), zb = (int32_t)(lo % NZ);
      int32_t o = pool[(int64_t)za * P + (int64_t)rng_below(&r, (uint64_t)P)];
      int64_t cnt = zoff[zb + 1] - zoff[zb];
      int32_t d;
      int tries = 0;
      do { d = znodes[zoff[zb] + (int64_t)rng_below(&r, (uint64_t)cnt)]; } while (d == o && ++tries < 64);
      if (d == o) d = ends[(rng_below(&r, (uint64_t)n_ends))];
      t->origin[k] = o; t->dest[k] = d;
    }
    free(zone); free(zoff); free(znodes); free(pool); free(mass); free(cx); free(cy); free(cum);
  }
  for (int64_t k = 0; k < nt; ++k) {
    double s;
    if (p->depart_model == 0) s = p->t_lo_s + (p->t_hi_s - p->t_lo_s) * rng_u01(&r);
    else {
      do {
        int second = (p->depart_model == 2) && (rng_u01(&r) < p->w2);
        s = second ? p->mean2_s + p->sd2_s * rng_normal(&r) : p->mean_s + p->sd_s * rng_normal(&r);
      } while (s < p->t_lo_s || s >= p->t_hi_s);
    }
    t->depart_time_s[k] = (float)s;
  }
  free(ends);
  route_all(nn, net->n_edges, net->edge_src, net->edge_dst, net->edge_length_m, net->edge_speed_mps, t,
            p->n_threads);
  return t;
}
