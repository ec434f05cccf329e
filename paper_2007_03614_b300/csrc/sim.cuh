// sim.cuh -- device-side layout of a simulation (internal to libmanta).
//
// HBM layout (all device memory owned by one manta_sim):
//   lane map      two buffers; lane l of edge e is a 16-byte aligned row of
//                 C_e bytes at row0[e] + l * stride(C_e), stride = round_up(C_e, 16);
//                 padding bytes stay 0xFF.  One byte per 1 m cell: 0xFF empty,
//                 else the speed code of the vehicle whose front is there.
//   edge tables   EdgeMeta (16 B) and EdgeSig (8 B) per edge, read-only.
//   vehicles      structure of arrays indexed by active-list position, one
//                 set per list buffer (VehSet): (x, v); (id, route cursor,
//                 route end, edge); the lane word (lane, dwell, lane mask
//                 toward the next edge); the cell it left in the other map
//                 buffer (cleared next step); a copy of the current edge's
//                 record; the next route entry.  A warp working on consecutive
//                 list positions loads each array with one coalesced
//                 instruction.
//   lists         the active list (a vehicle keeps its position while on the
//                 network; arrivals leave holes, departures append, and a
//                 compaction pass moves the live vehicles into the other
//                 buffer's list and arrays when holes pass a quarter of the
//                 list), lane changers, crossing requesters, arrivals,
//                 departure edges (double buffered); appended with
//                 warp-aggregated atomics (the order of a list never changes a
//                 result).
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
  uint32_t dst;    // head node | MANTA_CLOSABLE if a lane of the edge has a closure window
};
#define MANTA_CLOSABLE 0x80000000u

struct EdgeSig {   // signal window of this in-edge at its head node
  int16_t cyc;     // 0: head node is not a signal
  int16_t off;     // offset mod cycle
  int16_t gs, gl;  // green window [gs, gs + gl) within the cycle
};

enum {
  CNT_UPD = 0, CNT_SCAN, CNT_CLAMP, CNT_LC, CNT_LCE, CNT_RR, CNT_DEP, CNT_ARR, CNT_LCS, CNT_N
};

// One vehicle in registers (and the 48-byte copy kept for lane-change
// candidates).  Its state carries a copy of its current edge's record so that
// no phase needs a dependent edge-table load before it can address the lane
// map.
struct __align__(16) Veh {
  float x;         // front position in cells from the start of the edge
  float v;         // speed, m/s
  uint32_t id;     // trip index
  uint32_t rc;     // index of the current edge in the route array
  uint32_t rend;   // one past the last route entry of the trip
  uint32_t e;      // current edge
  uint32_t ld;     // lane (bits 0-3) | next edge has a closure (bit 4) | dwell << 8 |
                   // lane-change target << 16 | lane mask toward the next edge << 24
  uint32_t pcell;  // its cell in the other map buffer (cleared next step), or none
  EdgeMeta em;     // record of edge e
};

// One vehicle-step of the event tape (calibration, Eq. 1 adjoint): the
// continuous state entering the step and the discrete events the adjoint
// holds fixed.  Written in P3 (and completed in P4 for crossing requests) at
// index (k - tape_k0) * n_trips + trip id; zero flags mean "not on the
// network at the start of step k".
struct TapeRec {
  float x, v;        // position (cells from the start of the edge) and speed entering the step
  float s, vL;       // gap to the leader or stop line (cells) and the leader's speed, when interacting
  float bnd;         // clamp bound (cell), when clamped
  float lim;         // speed limit of the edge (v0 = lim * v0f[class])
  uint32_t C;        // cells of the edge
  uint32_t flags;    // TF_* below
  uint32_t sample;   // statistics index (window * E + edge) of the speed sample after the step, or none
  uint32_t pad;
};
#define TF_PRESENT 0x1u
#define TF_KIND_SHIFT 1          // 0 free road, 1 interacting (Eq. 1 with gap s), 2 stopped in place
#define TF_BALLISTIC 0x8u        // v + acc dt >= 0 (else the vehicle stops within the step)
#define TF_CLAMP_SHIFT 4         // 0 none, 1 held at its old position, 2 set to the bound
#define TF_OUT_SHIFT 6           // 0 stays on its edge, 1 crossed, 2 held (old position kept),
                                 // 3 held at the stop line, 4 arrived, 5 crossing request pending
#define TF_CLASS_SHIFT 12
enum { TK_FREE = 0, TK_INTERACT = 1, TK_STOP = 2 };
enum { TO_STAY = 0, TO_CROSS = 1, TO_HELD_KEEP = 2, TO_HELD_LINE = 3, TO_ARRIVE = 4, TO_PENDING = 5 };

// Vehicle state by active-list position (structure of arrays).
struct VehSet {
  float2 *xv;      // front position (cells from the start of the edge), speed (m/s)
  uint4 *idr;      // trip id, route cursor, route end, current edge
  uint32_t *ld;    // lane word (as Veh::ld)
  uint32_t *pc;    // its cell in the other map buffer (cleared next step), or none
  uint4 *em;       // record of its current edge (as EdgeMeta)
  uint32_t *nx;    // the route entry after its current one (route[rc + 1]), or 0 on its last edge
};

// Link-speed statistic of one (window, edge): the sum of end-of-step speeds
// in 2^-20 m/s units and the number of vehicle-steps, in one 16-byte record
// so that a vehicle-step's two reductions touch one 32-byte sector.
struct __align__(16) LinkStat {
  unsigned long long sum;
  uint32_t cnt, pad;
};

struct Ctl {
  unsigned bar_count;
  unsigned bar_gen;
  int err;          // 0 ok, 1 barrier wait ran out, 2 index check failed
  int err_info;
  uint32_t n_act[2];      // active-list length (live slots and holes) at even / odd steps
  uint32_t act_sel[2];    // which buffer holds the active list at even / odd steps
  uint32_t n_holes[2];    // holes (arrived vehicles) in that list
  uint32_t n_compact;     // entries written by a compaction pass
  uint32_t next3;          // next chunk of the active list for phase P3
  uint32_t pad[2];
  long long k_next;        // step index the next launch starts from (each launch advances it)
  uint32_t n_dep[2];
  uint32_t n_req, n_arr, n_chg, pad2;
  uint32_t due_pos, due_hi;   // trips [due_pos, due_hi) of the due list join queues this step

  unsigned long long cnt[CNT_N];
  unsigned long long phase_ns[4];   // device time of phases P1..P4 as seen by block 0
};

// One lane change, written whole by its decision so that it applies in one
// round trip: active-list position (twice), old and new map cell; new lane
// word, first leader-scan batch, speed code.
struct LcMove {
  uint32_t slot, pos, from, to;
  uint32_t ld, p3a, code, pad;
};
static_assert(sizeof(LcMove) == 32, "two 16-byte loads per move");

struct Params {
  // network, read-only
  const EdgeMeta *em;
  const EdgeSig *es;
  const uint8_t *ntype;
  const uint32_t *esrc;        // tail node of each edge
  const uint2 *src_in;         // in-lane slot range [x, y) of each edge's tail node
  const uint32_t *lane_base;   // first global lane index of each edge
  const uint32_t *nin_off;     // each node's in-lane slots [nin_off[n], nin_off[n + 1]), (edge, lane) order
  const uint32_t *rslot;       // slot of lane 0 of each edge among its head node's in-lanes: the
                               // request and stop-line slots of lane l are rslot[e] + l
  const uint32_t *stop_nodes;
  const float *mtab;           // Eq. 2 probability by distance in cells
  const long long *clo_k0;     // closure window [k0, k1) of each lane (empty when k0 >= k1)
  const long long *clo_k1;
  const uint32_t *nclo;        // bit q: the edge after route entry q has a closure window
  // trips, read-only
  const uint32_t *route;       // edge | (lane mask toward the next route edge) << 24
  const uint32_t *route_off;
  const uint32_t *q_off;       // departure queue of each first edge
  const uint32_t *q_trip;
  const int32_t *due_step;     // trips in departure-step order
  const uint32_t *due_edge;
  // lane map
  uint8_t *atlas0, *atlas1;
  // vehicle state by active-list position: vs[0] with act0, vs[1] with act1
  VehSet vs[2];
  // lists (an active-list entry is its own position, or none for a hole)
  uint32_t *act0, *act1, *req, *arr, *dep0, *dep1;
  uint32_t *p3a;               // by active-list position: first lane-map batch of the leader scan
  LcMove *lcm;                 // lane changes decided in P1, applied in P2
  Veh *lcq;                    // lane-change candidates of the step by block region (record copies,
                               // list position in pcell)
  uint32_t *lcq_pos;           // their active-list positions
  float *req_x, *req_v;
  uint32_t *req_dw, *req_g, *req_t, *req_e2, *req_n;
  // departure queues
  uint32_t *pending, *q_pos;
  uint32_t *dep_info;          // per departure-list entry of the step: edge, head trip or none,
                               // competitors' slot range; the trip's first route entry, route end,
                               // lane word and next route entry (8 words, written in P3, read in P4)
  unsigned long long *dep_key;
  // per-lane request and stop-line slots
  unsigned long long *req_key;
  uint32_t *req_tgt;
  uint32_t *slot_td, *slot_id;
  // per-node stop-sign state
  uint32_t *permit, *rr;
  // statistics
  uint32_t *entry, *exitc;
  LinkStat *lstat;             // by window * E + edge
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
  float sigma_frac;            // per-driver speed limits (Section IV-B); 0: off
  uint32_t E, N, n_stop, n_trips, mtab_n;
  // launch
  int64_t k0;
  int32_t n_steps;
  int32_t k_from_ctl;          // take the first step index from ctl->k_next instead of k0
  // event tape (none when tape == nullptr)
  TapeRec *tape;
  int64_t tape_k0;
  int32_t tape_len;
  uint64_t wait_limit_ns;
  // capacities checked by the bounds-checked build (MANTA_CHECK_BOUNDS):
  // bytes of a lane-map buffer, vehicle slots, entries of the per-step lists,
  // entries of the lane-change candidate overflow list, per-lane slots
  uint64_t cap_map;
  uint32_t cap_slots, cap_list, cap_lcq, cap_lanes;
};
