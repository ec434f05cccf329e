// sim.cuh -- device-side layout of a simulation (internal to libmanta).
//
// HBM layout (all device memory owned by one manta_sim):
//   lane map      two buffers; lane l of edge e is a 16-byte aligned row of
//                 C_e bytes at row0[e] + l * stride(C_e), stride = round_up(C_e, 16);
//                 padding bytes stay 0xFF.  One byte per 1 m cell: 0xFF empty,
//                 else the speed code of the vehicle whose front is there.
//   edge tables   EdgeMeta (16 B) and EdgeSig (8 B) per edge, read-only.
//   vehicle SoA   by slot: x, v, id, rc (route cursor), rend, e, ld (lane |
//                 dwell << 8 | lane-change target << 16), pcell (its cell in
//                 the other map buffer, cleared at the start of the next step).
//   lists         active slots (double buffered), free slots, lane changers,
//                 crossing requesters, arrivals, departure edges (double
//                 buffered); appended with warp-aggregated atomics (the order
//                 of a list never changes a result).
//   request slots per lane: key = (step + 1) << 32 | vehicle id and target lane,
//                 read by competitors; the lowest id wins (no atomics).
#pragma once
#include <stdint.h>

#define MANTA_EMPTY 0xFFu
#define MANTA_NONE 0xFFFFFFFFu
#define MANTA_EDGE_BITS 24
#define MANTA_EDGE_MASK 0x00FFFFFFu

struct EdgeMeta {
  uint32_t row0;   // byte offset of lane 0, cell 0 in a lane-map buffer
  uint32_t cnl;    // cells | lanes << 24 | class << 28
  float lim;       // speed limit, m/s
  uint32_t dst;    // head node
};

struct EdgeSig {   // signal window of this in-edge at its head node
  int16_t cyc;     // 0: head node is not a signal
  int16_t off;     // offset mod cycle
  int16_t gs, gl;  // green window [gs, gs + gl) within the cycle
};

enum {
  CNT_UPD = 0, CNT_SCAN, CNT_CLAMP, CNT_LC, CNT_LCE, CNT_RR, CNT_DEP, CNT_ARR, CNT_N
};

struct Ctl {
  unsigned bar_count;
  unsigned bar_gen;
  int err;          // 0 ok, 1 barrier wait ran out, 2 index check failed
  int err_info;
  uint32_t n_act[2];
  uint32_t n_dep[2];
  uint32_t n_req, n_arr, n_chg, n_depwin;
  uint32_t free_count, n_slots;
  uint32_t due_pos, due_next;
  uint32_t pad[2];
  unsigned long long cnt[CNT_N];
};

struct Params {
  // network, read-only
  const EdgeMeta *em;
  const EdgeSig *es;
  const uint8_t *ntype;
  const uint32_t *esrc;        // tail node of each edge
  const uint32_t *lane_base;   // first global lane index of each edge
  const uint32_t *nin_off;     // in-lanes (global lane ids) of each node, (edge, lane) order
  const uint32_t *nin;
  const uint32_t *stop_nodes;
  const float *mtab;           // Eq. 2 probability by distance in cells
  // trips, read-only
  const uint32_t *route;       // edge | (lane mask toward the next route edge) << 24
  const uint32_t *route_off;
  const uint32_t *q_off;       // departure queue of each first edge
  const uint32_t *q_trip;
  const int32_t *due_step;     // trips in departure-step order
  const uint32_t *due_edge;
  // lane map
  uint8_t *atlas0, *atlas1;
  // vehicle SoA by slot
  float *x, *v;
  uint32_t *id, *rc, *rend, *e, *ld, *pcell;
  // lists
  uint32_t *act0, *act1, *freel, *chg, *req, *arr, *dep0, *dep1;
  float *req_x, *req_v;
  uint32_t *req_dw;
  // departure queues
  uint32_t *pending, *q_pos;
  unsigned long long *dep_key;
  // per-lane request and stop-line slots
  unsigned long long *req_key;
  uint32_t *req_tgt;
  uint32_t *slot_td, *slot_id;
  // per-node stop-sign state
  uint32_t *permit, *rr;
  // statistics
  uint32_t *entry, *exitc;
  unsigned long long *ssum;
  uint32_t *scnt;
  Ctl *ctl;
  // model constants
  float dt;
  int32_t L, H;
  float T[8], a[8], b[8], s0[8], v0f[8];
  int32_t s0c[8];
  float alpha_lo, alpha_hi, g_low, g_high, g_split, stop_eps;
  int32_t stop_dwell, win_steps, n_win, textbook;
  int64_t t0;
  uint64_t seed;
  uint32_t E, N, n_stop, n_trips, mtab_n;
  // launch
  int64_t k0;
  int32_t n_steps;
  uint64_t wait_limit_ns;
};
