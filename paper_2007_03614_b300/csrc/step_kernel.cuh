// step_kernel.cuh -- the persistent per-timestep update (sm_103a).
//
// One cooperative launch runs n_steps steps.  Per step k the grid goes
// through four phases separated by grid barriers with bounded waits:
//   P1  lane-change decisions on M_k (Section II-D, Eqs. 2-4); stop-sign
//       permits for this step; the departure-step range of the trips that
//       join queues at k + 1.  The step's record pass (clear last step's cells
//       in the spare map buffer, note the first lane-map batch of every
//       leader scan, list the lane-change candidates) ran in the previous
//       step's P4 phase, on the warps without merge items; it runs here at a
//       launch's first step and when the active list is compacted.
//   P2  lane-change apply in place, M_k -> M_k' (skipped when nobody changes)
//   P3  leader scan along the route on M_k', IDM (Eq. 1), ballistic update,
//       clamp; write M_{k+1} for vehicles that stay on their edge; crossing
//       requests; departure requests; arrivals
//   P4  merge resolution (lowest id wins per target lane), crossings,
//       departures, arrivals' cells, departure-queue bookkeeping; the record
//       pass of step k + 1 (P4 prepares the vehicles it finalises itself)
// Arithmetic is binary32 with the operation order of the definition; the
// library is compiled with -fmad=false -prec-div=true -prec-sqrt=true so
// every operation is one correctly rounded IEEE op.
//
// The path is latency-bound on dependent global loads (vehicle record ->
// lane-map row -> node data -> next row), so the code keeps many independent
// loads in flight: in P3 every lane runs its own vehicle through a state
// machine of one round trip per iteration and takes a new vehicle as soon as
// one is done; the vehicle record and its first row batch come back together;
// the main phase's walk batches (32 bytes first, then 64) land in a
// shared-memory slot per lane by asynchronous copies, holding no registers,
// while the lane-change scans load four 16-byte chunks per round trip into
// registers; and the next segment's node data comes with the batch that ends
// the current one.
#include <stdint.h>
#include "sim.cuh"
// 16-byte chunks per walk round trip and in the first batch (fetched with
// the vehicle's state).  32 and 64 bytes suit the congested states that
// dominate a morning (about 10 cells scanned per update) and cost nothing in
// free flow; test builds select other sizes.
#ifndef MANTA_WALK_CHUNKS
#define MANTA_WALK_CHUNKS 4
#endif
#ifndef MANTA_FIRST_CHUNKS
#define MANTA_FIRST_CHUNKS 2
#endif

// Threads per block of the helper kernels.  The step kernel is a template
// over its launch shape (threads per block, minimum blocks per SM), which
// sets its register budget; every shape computes the same results.
constexpr int kBlock = 256;
// fields of a finish-queue entry
enum { kFqX, kFqV, kFqId, kFqRc, kFqRend, kFqE, kFqLd, kFqRow0, kFqCnl, kFqLim, kFqDst, kFqS, kFqI, kFqCell,
       kFqKind, kFqCL, kFqVL, kFqE2, kFqE2cnl, kFqFields };
constexpr int kP3Words = 384 + kFqFields * 64;
// Row batches of the main phase's leader walk land in a shared-memory slot
// per lane (asynchronous copies, no registers held): the first batch, fetched
// with the vehicle record, has kFirstChunks 16-byte chunks; every later walk
// round trip up to kWalkChunks.  Slots are 16 bytes longer than a batch so
// that the lanes' 16-byte reads of the same chunk fall in different banks.
constexpr int kFirstChunks = MANTA_FIRST_CHUNKS;
constexpr int kWalkChunks = MANTA_WALK_CHUNKS;
constexpr int kSlotBytes = 16 * kWalkChunks + 16;
static_assert(kFirstChunks <= kWalkChunks, "the slot holds the first batch");
constexpr int kWarpWords = kP3Words + 32 * kSlotBytes / 4;
// lane-change candidates a block of `threads` keeps in its main-phase scratch
// (64 bytes each), and the entries of its overflow region in the global list
// when its record pass visits n_rec list entries with a stride of rstride
// threads (at least half the grid) and it runs its share of n_items
// merge-phase items (grid of gsz threads)
// (MANTA_LC_CAP, defined only in a test build, lowers the capacity so that
// the overflow region takes most candidates.)
__host__ __device__ constexpr uint32_t lc_cap_of(int threads) {
#ifdef MANTA_LC_CAP
  return (uint32_t)MANTA_LC_CAP < (uint32_t)(threads / 32) * kWarpWords * 4u / 64u
             ? (uint32_t)MANTA_LC_CAP
             : (uint32_t)(threads / 32) * kWarpWords * 4u / 64u;
#else
  return (uint32_t)(threads / 32) * kWarpWords * 4u / 64u;
#endif
}
__host__ __device__ constexpr uint32_t lc_bound(int threads, uint32_t rstride, uint32_t gsz, uint32_t n_rec,
                                                uint32_t n_items) {
  return (uint32_t)threads * ((n_rec + rstride - 1u) / rstride + (n_items + gsz - 1u) / gsz);
}
__host__ __device__ constexpr uint32_t lc_overflow(int threads, uint32_t rstride, uint32_t gsz, uint32_t n_rec,
                                                   uint32_t n_items) {
  return lc_bound(threads, rstride, gsz, n_rec, n_items) > lc_cap_of(threads)
             ? lc_bound(threads, rstride, gsz, n_rec, n_items) - lc_cap_of(threads)
             : 0u;
}
// dynamic shared memory of a step-kernel block of `threads` threads
constexpr size_t step_smem_bytes(int threads) { return (size_t)(threads / 32) * kWarpWords * 4; }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ldv(const uint32_t *p) { return *(const volatile uint32_t *)p; }
__device__ __forceinline__ int ldvi(const int *p) { return *(const volatile int *)p; }

// Grid barrier with a bounded wait.  The arrival counter only grows within a
// launch (the host zeroes it before every launch): barrier number b of the
// launch completes when the counter reaches b * gridDim.x, so arriving is one
// fire-and-forget release-add and waiting is an acquire-load spin by thread 0
// of each block.  A waiter that passes the wall-clock limit sets the sticky
// error word and adds kBarrierAbort to the counter, which releases every other
// waiter at once; all blocks then leave the kernel.
// The abort mark is one bit, set with an OR, so any number of blocks may set
// it (arrivals per launch stay far below 2^30).
constexpr unsigned kBarrierAbort = 1u << 30;

__device__ __noinline__ bool grid_sync(Ctl *ctl, unsigned &target, uint64_t limit_ns, int *s_ok) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
    unsigned c = ld_acquire(&ctl->bar_count);
#ifdef MANTA_CHECK_BOUNDS
    // a failed index check ends the launch: every block leaves at this
    // barrier (or, having passed it already, at the next one)
    if (ldvi(&ctl->err) != 0) {
      atomicOr(&ctl->bar_count, kBarrierAbort);
      c = kBarrierAbort;
    }
#endif
    if (c < target) {
      const uint64_t t0 = globaltimer();
      uint32_t spins = 0;
      while ((c = ld_acquire(&ctl->bar_count)) < target) {
        if ((++spins & 63u) == 0u && globaltimer() - t0 > limit_ns) {
          atomicCAS(&ctl->err, 0, 1);
          atomicOr(&ctl->bar_count, kBarrierAbort);
          c = kBarrierAbort;
          break;
        }
        if (spins > 32u) __nanosleep(128);
      }
    }
    *s_ok = c < kBarrierAbort;
  }
  __syncthreads();
  return *s_ok != 0;
}

// ------------------------------------------------------------ index checks
// A build with MANTA_CHECK_BOUNDS checks the index of every write the step
// kernel makes into the lane maps, vehicle records, lists, per-lane slots and
// statistics against the capacity of its array (Params cap_*).  A failing
// check skips the write and records the first failing site in the control
// block (err = 2, err_info = site); the next grid barrier ends the launch,
// and the host reports MANTA_E_DEVICE.  Other builds compile every check to
// `true`.
#ifdef MANTA_CHECK_BOUNDS
__device__ __noinline__ bool index_fail(Ctl *ctl, int site) {
  if (atomicCAS(&ctl->err, 0, 2) == 0) atomicExch(&ctl->err_info, site);
  return false;
}
#define IDX_OK(i, cap, site) ((uint64_t)(i) < (uint64_t)(cap) ? true : index_fail(p.ctl, (site)))
#else
#define IDX_OK(i, cap, site) true
#endif

// ------------------------------------------------------------ random numbers
// SplitMix64 (Steele, Lea, Flood 2014) of a key from (seed, id, step, stream).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint32_t draw24(uint64_t seed, uint32_t id, int64_t k, uint32_t stream) {
  const uint64_t key = seed ^ ((uint64_t)id * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)k * 0xC2B2AE3D27D4EB4Full) ^
                       (uint64_t)stream;
  return (uint32_t)(splitmix64(key) >> 40);
}
// uniform [0,1): 24 bits times 2^-24
__device__ __forceinline__ float uni(uint64_t seed, uint32_t id, int64_t k, uint32_t stream) {
  return __uint2float_rn(draw24(seed, id, k, stream)) * 5.9604644775390625e-8f;
}
// normal(0,1) approximated by the centred sum of twelve 24-bit uniforms
__device__ __forceinline__ float irwin_hall(uint64_t seed, uint32_t id, int64_t k, uint32_t s) {
  int32_t acc = 0;
#pragma unroll
  for (uint32_t j = 0; j < 12; ++j) acc += (int32_t)draw24(seed, id, k, 16u * s + j);
  return __int2float_rn(acc - 100663296) * 5.9604644775390625e-8f;
}

// A driver's own speed limit on the edge of route entry r (Section IV-B): the
// edge's limit s perturbed by 2 sigma_s z with sigma_s = sigma_frac x s and z
// the counter-based normal of (seed, trip id, r, stream 4), floored at s / 4.
// Drawn once when the vehicle enters the edge and kept in its record.
__device__ __forceinline__ float driver_limit(const Params &p, float s, uint32_t id, uint32_t r) {
  if (!(p.sigma_frac > 0.0f)) return s;
  const float z = irwin_hall(p.seed, id, (int64_t)r, 4);
  const float q = fmaxf(0.25f, 1.0f + (2.0f * p.sigma_frac) * z);
  return s * q;
}

// ---------------------------------------------------------------- records
__device__ __forceinline__ uint32_t cells_of(uint32_t cnl) { return cnl & 0xFFFFFFu; }
__device__ __forceinline__ int lanes_of(uint32_t cnl) { return (int)((cnl >> 24) & 0xFu); }
__device__ __forceinline__ int class_of(uint32_t cnl) { return (int)(cnl >> 28); }
__device__ __forceinline__ uint32_t stride_of(uint32_t cells) { return (cells + 15u) & ~15u; }
__device__ __forceinline__ uint8_t speed_code(float v) {
  const int c = (int)(v * 8.0f + 0.5f);
  return (uint8_t)(c > 254 ? 254 : c);
}
__device__ __forceinline__ float speed_decode(uint32_t c) { return __uint2float_rn(c) * 0.125f; }

__device__ __forceinline__ uint32_t node_of(const EdgeMeta &m) { return m.dst & ~MANTA_CLOSABLE; }
__device__ __forceinline__ bool closable(const EdgeMeta &m) { return (m.dst & MANTA_CLOSABLE) != 0u; }
// lane g (global lane index) is closed at step k
__device__ __forceinline__ bool lane_closed(const Params &p, uint32_t g, int64_t k) {
  return __ldg(p.clo_k0 + g) <= k && k < __ldg(p.clo_k1 + g);
}

__device__ __forceinline__ EdgeMeta load_em(const Params &p, uint32_t e) {
  const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p.em) + e);
  EdgeMeta m;
  m.row0 = q.x; m.cnl = q.y; m.lim = __uint_as_float(q.z); m.dst = q.w;
  return m;
}
__device__ __forceinline__ Veh load_veh_at(const Veh *r) {
  const uint4 *a = reinterpret_cast<const uint4 *>(r);
  const uint4 q0 = __ldcg(a), q1 = __ldcg(a + 1), q2 = __ldcg(a + 2);
  Veh w;
  w.x = __uint_as_float(q0.x); w.v = __uint_as_float(q0.y); w.id = q0.z; w.rc = q0.w;
  w.rend = q1.x; w.e = q1.y; w.ld = q1.z; w.pcell = q1.w;
  w.em.row0 = q2.x; w.em.cnl = q2.y; w.em.lim = __uint_as_float(q2.z); w.em.dst = q2.w;
  return w;
}
// The vehicle at active-list position i of a state set: five independent
// loads, each coalesced across a warp working on consecutive positions.
__device__ __forceinline__ Veh load_veh(const VehSet &R, uint32_t i) {
  const float2 a = __ldcg(R.xv + i);
  const uint4 b = __ldcg(R.idr + i);
  const uint32_t l = __ldcg(R.ld + i), c = __ldcg(R.pc + i);
  const uint4 m = __ldcg(R.em + i);
  Veh w;
  w.x = a.x; w.v = a.y; w.id = b.x; w.rc = b.y; w.rend = b.z; w.e = b.w; w.ld = l; w.pcell = c;
  w.em.row0 = m.x; w.em.cnl = m.y; w.em.lim = __uint_as_float(m.z); w.em.dst = m.w;
  return w;
}
// The main phase's view: everything but the previous cell, which it only writes.
__device__ __forceinline__ Veh load_veh_main(const VehSet &R, uint32_t i) {
  const float2 a = __ldcg(R.xv + i);
  const uint4 b = __ldcg(R.idr + i);
  const uint32_t l = __ldcg(R.ld + i);
  const uint4 m = __ldcg(R.em + i);
  Veh w;
  w.x = a.x; w.v = a.y; w.id = b.x; w.rc = b.y; w.rend = b.z; w.e = b.w; w.ld = l; w.pcell = MANTA_NONE;
  w.em.row0 = m.x; w.em.cnl = m.y; w.em.lim = __uint_as_float(m.z); w.em.dst = m.w;
  return w;
}
// position, speed, lane word, previous cell (edge and route cursor unchanged)
__device__ __forceinline__ void store_veh_state(const VehSet &R, uint32_t i, const Veh &w) {
  R.xv[i] = make_float2(w.x, w.v);
  R.ld[i] = w.ld;
  R.pc[i] = w.pcell;
}
__device__ __forceinline__ void store_veh(const VehSet &R, uint32_t i, const Veh &w) {
  store_veh_state(R, i, w);
  R.idr[i] = make_uint4(w.id, w.rc, w.rend, w.e);
  R.em[i] = make_uint4(w.em.row0, w.em.cnl, __float_as_uint(w.em.lim), w.em.dst);
}
// the state set that goes with list buffer `sel`
__device__ __forceinline__ VehSet veh_set(const Params &p, uint32_t sel) {
  VehSet r;
  r.xv = sel ? p.vs[1].xv : p.vs[0].xv;
  r.idr = sel ? p.vs[1].idr : p.vs[0].idr;
  r.ld = sel ? p.vs[1].ld : p.vs[0].ld;
  r.pc = sel ? p.vs[1].pc : p.vs[0].pc;
  r.em = sel ? p.vs[1].em : p.vs[0].em;
  r.nx = sel ? p.vs[1].nx : p.vs[0].nx;
  return r;
}

// lane word of a vehicle record
__device__ __forceinline__ int ld_lane(uint32_t ld) { return (int)(ld & 0xFu); }
__device__ __forceinline__ uint32_t ld_dwell(uint32_t ld) { return (ld >> 8) & 0xFFu; }
__device__ __forceinline__ uint32_t ld_mask(uint32_t ld) { return ld >> 24; }
__device__ __forceinline__ bool ld_nxclo(uint32_t ld) { return (ld >> 4) & 1u; }
// the bits fixed while the vehicle stays on its edge: mask toward the next edge, next-edge closure flag
constexpr uint32_t kLdEdgeBits = 0xFF000010u;
// lane word for a vehicle entering route entry r (mask from the route entry, closure flag from the bitset)
__device__ __forceinline__ uint32_t ld_for_entry(const Params &p, uint32_t r, uint32_t lane) {
  const uint32_t ent = __ldg(p.route + r);
  const uint32_t nx = (__ldg(p.nclo + (r >> 5)) >> (r & 31)) & 1u;
  return (ent & 0xFF000000u) | (nx << 4) | lane;
}

// ---------------------------------------------------------------- lane map
// bit 7 of each byte of the result is set iff that byte of w is not 0xFF
__device__ __forceinline__ uint32_t occupied_bits(uint32_t w) {
  const uint32_t t = ~w;
  return (t | ((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu)) & 0x80808080u;
}

// A run of four 16-byte chunks of a row, loaded in one round trip.
struct Batch {
  uint4 q[4];
};
__device__ __forceinline__ void load_batch(const uint8_t *row, int c, int hi, Batch &b) {
  const uint4 none = make_uint4(~0u, ~0u, ~0u, ~0u);
  b.q[0] = __ldcg(reinterpret_cast<const uint4 *>(row + c));
  b.q[1] = (c + 16 <= hi) ? __ldcg(reinterpret_cast<const uint4 *>(row + c + 16)) : none;
  b.q[2] = (c + 32 <= hi) ? __ldcg(reinterpret_cast<const uint4 *>(row + c + 32)) : none;
  b.q[3] = (c + 48 <= hi) ? __ldcg(reinterpret_cast<const uint4 *>(row + c + 48)) : none;
}
// First occupied cell in [lo, hi] within the batch starting at cell c, or -1.
// Cells below lo (only the first 16-byte chunk can hold them: lo lies in it for
// the first batch of a scan, below it for later batches) are made to look
// empty; empty chunks are recognised with three-input ANDs, and only the first
// non-empty chunk is searched byte by byte.  A first hit beyond hi means there
// is none in range.
__device__ __forceinline__ int check_batch(const Batch &b, int c, int lo, int hi, uint32_t &byte) {
  uint32_t w[16] = {b.q[0].x, b.q[0].y, b.q[0].z, b.q[0].w, b.q[1].x, b.q[1].y, b.q[1].z, b.q[1].w,
                    b.q[2].x, b.q[2].y, b.q[2].z, b.q[2].w, b.q[3].x, b.q[3].y, b.q[3].z, b.q[3].w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int d = lo - (c + 4 * k);
    w[k] |= d <= 0 ? 0u : (d >= 4 ? 0xFFFFFFFFu : ((1u << (8 * d)) - 1u));
  }
  const bool f0 = (w[0] & w[1] & w[2] & w[3]) != 0xFFFFFFFFu;
  const bool f1 = (w[4] & w[5] & w[6] & w[7]) != 0xFFFFFFFFu;
  const bool f2 = (w[8] & w[9] & w[10] & w[11]) != 0xFFFFFFFFu;
  const bool f3 = (w[12] & w[13] & w[14] & w[15]) != 0xFFFFFFFFu;
  if (!(f0 || f1 || f2 || f3)) return -1;
  const int j = f0 ? 0 : (f1 ? 1 : (f2 ? 2 : 3));
  const uint32_t a0 = f0 ? w[0] : (f1 ? w[4] : (f2 ? w[8] : w[12]));
  const uint32_t a1 = f0 ? w[1] : (f1 ? w[5] : (f2 ? w[9] : w[13]));
  const uint32_t a2 = f0 ? w[2] : (f1 ? w[6] : (f2 ? w[10] : w[14]));
  const uint32_t a3 = f0 ? w[3] : (f1 ? w[7] : (f2 ? w[11] : w[15]));
  const int t = a0 != 0xFFFFFFFFu ? 0 : (a1 != 0xFFFFFFFFu ? 1 : (a2 != 0xFFFFFFFFu ? 2 : 3));
  const uint32_t a = t == 0 ? a0 : (t == 1 ? a1 : (t == 2 ? a2 : a3));
  const int bpos = (__ffs(occupied_bits(a)) - 1) >> 3;
  const int first = c + 16 * j + 4 * t + bpos;
  byte = (a >> (8 * bpos)) & 0xFFu;          // the speed code, already in registers
  return first > hi ? -1 : first;
}
// 16-byte asynchronous copy from global memory (L2 only) into shared memory
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// n 16-byte chunks from g into the slot at shared address slot
__device__ __forceinline__ void slot_fetch(uint32_t slot, const uint8_t *g, int n) {
  for (int j = 0; j < n; ++j) cp_async16(slot + 16u * (uint32_t)j, g + 16 * j);
}
// First occupied cell in [lo, hi] among the n chunks of a slot whose chunk 0
// starts at row cell c (lo lies in chunk 0), or -1; the speed code in byte.
__device__ __forceinline__ int check_slot(const uint8_t *slot, int n, int c, int lo, int hi, uint32_t &byte) {
  // four chunks per pass, loaded together and tested branch-free
  const uint4 none = make_uint4(~0u, ~0u, ~0u, ~0u);
  const uint4 *q = reinterpret_cast<const uint4 *>(slot);
  for (int j = 0; j < n; j += 4) {
    Batch b;
    b.q[0] = q[j];
    b.q[1] = j + 1 < n ? q[j + 1] : none;
    b.q[2] = j + 2 < n ? q[j + 2] : none;
    b.q[3] = j + 3 < n ? q[j + 3] : none;
    const int r = check_batch(b, c + 16 * j, lo, hi, byte);
    if (r >= 0) return r;
  }
  return -1;
}
// First occupied cell of row[lo..hi] (inclusive), continuing from a batch
// already loaded at lo & ~15; -1 if none.  Rows are 16-byte aligned and padded.
__device__ __forceinline__ int scan_from(const uint8_t *row, int lo, int hi, Batch &b, uint32_t &byte) {
  int c = lo & ~15;
  for (;;) {
    const int r = check_batch(b, c, lo, hi, byte);
    if (r >= 0) return r;
    c += 64;
    if (c > hi) return -1;
    load_batch(row, c, hi, b);
  }
}
__device__ __forceinline__ int first_up(const uint8_t *row, int lo, int hi, uint32_t &byte) {
  if (lo > hi) return -1;
  Batch b;
  load_batch(row, lo & ~15, hi, b);
  return scan_from(row, lo, hi, b, byte);
}

// Last occupied cell in row[lo..hi] (scanning downward from hi) or -1;
// four 16-byte chunks per round trip, each block tested branch-free.
__device__ __forceinline__ int first_down(const uint8_t *row, int hi, int lo, uint32_t &byte) {
  if (lo > hi) return -1;
  const uint4 none = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (int c = hi & ~15; c + 15 >= lo; c -= 64) {
    uint4 q[4];
    q[0] = __ldcg(reinterpret_cast<const uint4 *>(row + c));
#pragma unroll
    for (int j = 1; j < 4; ++j)
      q[j] = (c - 16 * j >= 0 && c - 16 * j + 15 >= lo) ? __ldcg(reinterpret_cast<const uint4 *>(row + c - 16 * j)) : none;
    // word k covers cells c - 16 * (k / 4) + 4 * (k % 4) ...; keep the highest hit within [lo, hi]
    int best = -1;
#pragma unroll
    for (int j = 3; j >= 0; --j) {
      const uint32_t w[4] = {q[j].x, q[j].y, q[j].z, q[j].w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int base = c - 16 * j + 4 * t;
        uint32_t m = occupied_bits(w[t]);
        const int dl = lo - base, dh = base + 3 - hi;
        m = dl <= 0 ? m : (dl >= 4 ? 0u : (m & (0xFFFFFFFFu << (8 * dl))));
        m = dh <= 0 ? m : (dh >= 4 ? 0u : (m & (0xFFFFFFFFu >> (8 * dh))));
        const int bp = (31 - __clz(m)) >> 3;
        const int hit = base + bp;
        byte = (m && hit > best) ? ((w[t] >> (8 * bp)) & 0xFFu) : byte;
        best = m ? hit : best;
      }
    }
    if (best >= 0) return best;
    if (c < 64) break;
  }
  return -1;
}


__device__ __forceinline__ EdgeSig load_sig(const Params &p, uint32_t e) {
  const int2 w = __ldg(reinterpret_cast<const int2 *>(p.es) + e);
  EdgeSig s;
  s.cyc = (int16_t)(w.x & 0xFFFF); s.off = (int16_t)((uint32_t)w.x >> 16);
  s.gs = (int16_t)(w.y & 0xFFFF); s.gl = (int16_t)((uint32_t)w.y >> 16);
  return s;
}

__device__ __forceinline__ bool is_green(const EdgeSig &s, int64_t k) {
  if (s.cyc == 0) return true;
  const int64_t d = k - (int64_t)s.off;
  int64_t m;
  if ((uint64_t)d < (1ull << 32)) {
    m = (int64_t)((uint32_t)d % (uint32_t)s.cyc);   // the usual case, in 32 bits
  } else {
    m = d % (int64_t)s.cyc;
    if (m < 0) m += s.cyc;
  }
  return m >= s.gs && m < (int64_t)s.gs + s.gl;
}

// Warp-aggregated append: returns this lane's index in the list.
__device__ __forceinline__ uint32_t warp_append(uint32_t *counter, bool pred) {
  const unsigned am = __activemask();
  const unsigned bal = __ballot_sync(am, pred);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(am) - 1;
  uint32_t base = 0;
  if (lane == leader && bal) base = atomicAdd(counter, (uint32_t)__popc(bal));
  base = __shfl_sync(am, base, leader);
  return base + (uint32_t)__popc(bal & ((1u << lane) - 1u));
}

// ------------------------------------------------------------ lane change
// Target lane or -1 (Section II-D: mandatory vs discretionary; Eq. 2; Eqs. 3-4).
// The route entry (lane mask toward the next edge), the Eq. 2 probability and
// the first chunks of the own and target lane rows are fetched together.
// *lcs (the thread's counter in shared memory, so that no register holds it)
// receives the lane-map cells the rule's scans read, counted as separate scans
// in the rule's order (own-lane leader and target-lane lead of a discretionary
// change; the lateral-overlap window, the lead and the lag of the gap
// acceptance), each from its first cell to its hit or its end, although the
// scans here share their loads.
__device__ int lc_decide(const Params &p, const uint8_t *cur, int64_t k, const Veh &w, uint32_t &c_lce,
                         uint32_t *lcs) {
  const EdgeMeta &em = w.em;
  const int nl = lanes_of(em.cnl);
  const int lane = ld_lane(w.ld);
  const int dir = (k & 1) ? -1 : 1;
  const int lt = lane + dir;
  if (lt < 0 || lt >= nl) return -1;
  const int C = (int)cells_of(em.cnl), L = p.L, H = p.H;
  const int cell = (int)floorf(w.x);
  const float v = w.v;
  const bool has_next = w.rc + 1u < w.rend;
  const uint32_t stride = stride_of((uint32_t)C);
  const uint8_t *trow = cur + em.row0 + (uint32_t)lt * stride;
  const uint8_t *orow = cur + em.row0 + (uint32_t)lane * stride;
  const int hi = min(cell + H, C - 1);
  const int lo_t = max(0, cell - L + 1);     // target-lane cells from the lateral-overlap window on
  const bool next_clo = has_next && ld_nxclo(w.ld);
  const float mprob = __ldg(p.mtab + (C - 1 - cell));
  Batch bt, bo;
  load_batch(trow, lo_t & ~15, hi, bt);
  // a stopped vehicle cannot find a slower leader, so only a mandatory change
  // is possible: skip the own-lane fetch
  const bool own_scan = cell + 1 <= hi && v > 0.0f;
  if (own_scan) load_batch(orow, (cell + 1) & ~15, hi, bo);
  uint32_t mask = has_next ? ld_mask(w.ld) : 0xFFu;
  int obst = -1;
  bool closed_here = false;
  if (closable(em)) {
    const uint32_t lb = __ldg(p.lane_base + w.e);
    if (lane_closed(p, lb + (uint32_t)lt, k)) return -1;      // never into a closed lane
    obst = C / 2;
    closed_here = cell < obst && lane_closed(p, lb + (uint32_t)lane, k);
  }
  if (next_clo) {
    // lanes whose continuation on the next edge is closed are not allowed either
    const uint32_t e2 = __ldg(p.route + w.rc + 1u) & MANTA_EDGE_MASK;
    const int nl2 = lanes_of(load_em(p, e2).cnl);
    const uint32_t lb2 = __ldg(p.lane_base + e2);
    uint32_t open = 0;
    for (int q = 0; q < nl; ++q)
      if (!lane_closed(p, lb2 + (uint32_t)min(q, nl2 - 1), k)) open |= 1u << q;
    if (mask & open) mask &= open;
  }
  const bool ok_l = (mask >> lane) & 1u, ok_lt = (mask >> lt) & 1u;
  bool mandatory = false;
  if (closed_here) {
    mandatory = true;
  } else if (has_next && !ok_l) {
    int dp = 99, dm = 99;
    for (int q = lane + 1; q < nl; ++q)
      if ((mask >> q) & 1u) { dp = q - lane; break; }
    for (int q = lane - 1; q >= 0; --q)
      if ((mask >> q) & 1u) { dm = lane - q; break; }
    const bool toward = dir > 0 ? (dp < 99 && dp <= dm) : (dm < 99 && dm <= dp);
    if (!toward) return -1;
    mandatory = true;
  } else if (!ok_lt) {
    return -1;
  }
  int c1, ca;
  uint32_t bc1 = 0, bca = 0, bcb = 0;
  if (mandatory) {
    const float u1 = uni(p.seed, w.id, k, 0);
    // Eq. 2 at the distance to the end of the edge, or to the obstacle of a closed lane
    const float mp = closed_here ? __ldg(p.mtab + (obst - 1 - cell)) : mprob;
    if (!(u1 < mp)) return -1;
    c1 = scan_from(trow, lo_t, hi, bt, bc1);
    ca = c1;
    bca = bc1;
  } else {
    if (!own_scan) return -1;
    uint32_t bco;
    const int co = scan_from(orow, cell + 1, hi, bo, bco);
    if (co < 0) { *lcs += (uint32_t)(hi - cell); return -1; }         // own lane, cell + 1 .. hi
    if (!(speed_decode(bco) < v)) { *lcs += (uint32_t)(co - cell); return -1; }
    const int own_gap = co - L - cell;
    c1 = scan_from(trow, lo_t, hi, bt, bc1);
    if (c1 >= 0 && c1 <= cell + L - 1) ca = first_up(trow, cell + L, hi, bca);
    else { ca = c1; bca = bc1; }
    // the own lane (co - cell = own_gap + L cells) and the target lead, cell + L .. hi
    *lcs += (uint32_t)(own_gap + L + max(0, (ca >= 0 ? ca : hi) - (cell + L) + 1));
    if (ca >= 0 && !(ca - L - cell > own_gap)) return -1;
  }
  c_lce++;
  const bool overlap = c1 >= 0 && c1 <= cell + L - 1;
  // the lateral-overlap window lo_t .. min(cell + L - 1, C - 1)
  *lcs += (uint32_t)max(0, (overlap ? c1 : min(cell + L - 1, C - 1)) - lo_t + 1);
  if (overlap) return -1;
  *lcs += (uint32_t)max(0, (ca >= 0 ? ca : hi) - (cell + L) + 1);       // lead, cell + L .. hi
  const int cb = first_down(trow, cell - L, max(0, cell - H), bcb);
  *lcs += (uint32_t)max(0, (cell - L) - (cb >= 0 ? cb : max(0, cell - H)) + 1);  // lag, cell - L down
  const float g = v < p.g_split ? p.g_low : p.g_high;
  const float alpha = p.alpha_lo + (p.alpha_hi - p.alpha_lo) * uni(p.seed, w.id, 0, 3);
  if (ca >= 0) {
    const float va = speed_decode(bca);
    const float eps_a = irwin_hall(p.seed, w.id, k, 1);
    float t = g + alpha * v;          // Eq. 3, alpha_a = alpha_i
    t = t + alpha * (v - va);
    const float glead = fmaxf(g, t) + eps_a;
    if (!(__int2float_rn(ca - L - cell) >= glead)) return -1;
  }
  if (cb >= 0) {
    const float vb = speed_decode(bcb);
    const float eps_b = irwin_hall(p.seed, w.id, k, 2);
    float t = g + alpha * v;          // Eq. 4, alpha_b = alpha_i
    t = t + alpha * (v - vb);
    const float glag = fmaxf(g, t) + eps_b;
    if (!(__int2float_rn(cell - L - cb) >= glag)) return -1;
  }
  return lt;
}

// A vehicle joins step kk's lane-change candidates when the step's direction
// (+1 on even steps, -1 on odd) points at a lane of its edge, and either it
// moves (a discretionary change needs a slower leader) or a mandatory change
// is possible (lane not allowed for the next edge, closures here or next).
__device__ __forceinline__ bool lc_candidate(const Veh &w, int64_t kk) {
  const int nl = lanes_of(w.em.cnl), ln = ld_lane(w.ld);
  const int lt = ln + ((kk & 1) ? -1 : 1);
  return nl >= 2 && lt >= 0 && lt < nl &&
         (w.v > 0.0f || !((ld_mask(w.ld) >> ln) & 1u) || closable(w.em) || ld_nxclo(w.ld));
}
// A list entry of a vehicle that made a crossing request this step: its
// record is rewritten in P4, which prepares it for the next step itself.
constexpr uint32_t kReqMark = 0x80000000u;

// Key of lane l of edge e as a request target.
__device__ __forceinline__ uint32_t target_key(uint32_t e, uint32_t l) { return (e << 4) | l; }

// Lowest id among the other crossing requests for target lane key `tgt`
// posted this step (tag) by the in-lanes of a node, whose request slots are
// [o0, o1) (slots are numbered node by node), excluding slot `skip`;
// MANTA_NONE if there is none.  Eight in-lanes per round trip.
__device__ __forceinline__ uint32_t min_competitor(const Params &p, uint32_t o0, uint32_t o1, uint32_t skip,
                                                   uint32_t tgt, uint32_t tag) {
  uint32_t best = MANTA_NONE;
  for (uint32_t o = o0; o < o1; o += 8u) {
    unsigned long long key[8];
    uint32_t tg[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t g = o + (uint32_t)j;
      const bool use = g < o1 && g != skip;
      key[j] = use ? __ldcg(p.req_key + g) : 0ull;
      tg[j] = use ? __ldcg(p.req_tgt + g) : MANTA_NONE;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((uint32_t)(key[j] >> 32) == tag && tg[j] == tgt && (uint32_t)key[j] < best) best = (uint32_t)key[j];
  }
  return best;
}

// ------------------------------------------------------------ leader scan
enum { SC_FREE = 0, SC_LEADER = 1, SC_VIRTUAL = 2 };
struct Scan {
  int kind;
  int cL;            // route-relative front cell of the leader
  float vL;
  bool reached_own;  // the scan examined the vehicle's own head node
  bool stop_only;    // ... and only a stop sign (no permit) held it there
  uint32_t nt_own;   // type of the own head node, when reached
  uint32_t e2;       // next route edge, when reached
  uint32_t e2cnl;    // its cells | lanes | class word, when reached
};

// A leader scan in progress.  The walk goes along the route from the cell
// ahead, at most H cells, and stops at the first occupied byte or at a node
// that holds the vehicle (red signal; stop sign without the permit, or any
// stop sign beyond the own node).  A lane not allowed for the next edge does
// not hold the vehicle.  Each round trip fetches one batch of the current
// row; the batch that ends a segment also fetches the head node's type, the
// segment's signal window, the next edge's record and the route entry after
// it, so crossing a node costs no extra round trip.
struct Walk {
  int limit;         // last route-relative cell within the horizon
  int base;          // route-relative cell of the segment's first cell
  int pos;           // next route-relative cell to examine
  int sl;            // lane on the segment
  uint32_t r;        // route entry of the segment
  uint32_t se;       // its edge
  uint32_t nent;     // route entry r + 1 (for the vehicle's own edge from its state, then fetched one
                     // segment ahead)
  EdgeMeta sm;       // record of the segment's edge
  bool own;          // the segment is the vehicle's own edge
};
// What one walk round trip brings besides the row batch (which lands in the
// lane's shared-memory slot): the node data when the batch ends a segment.
struct Fetch {
  uint32_t nt;
  EdgeSig sig;
  EdgeMeta sm2;
  uint32_t nent2;
};

// Byte offset in a lane-map buffer of the first batch (kFirstChunks 16-byte
// chunks) a leader scan from `cell` reads on lane `lane` of edge record em
// (the batch holding cell + 1), or MANTA_NONE when the vehicle is at the last
// cell of its edge.  The buffers are padded so the batch may run past the row
// end.
__device__ __forceinline__ uint32_t first_batch(const EdgeMeta &em, int lane, int cell) {
  const uint32_t C = cells_of(em.cnl);
  return (uint32_t)cell + 1u < C ? em.row0 + (uint32_t)lane * stride_of(C) + (((uint32_t)cell + 1u) & ~15u) : MANTA_NONE;
}

// Sets up the walk of vehicle w from `cell`.  A closed own lane holds a
// stationary obstacle from mid-edge on (cell C / 2); when it lies within the
// horizon only the cells before it can hold the leader, and the scan is
// completed here (returns true).
__device__ __forceinline__ bool walk_start(const Params &p, const uint8_t *cur, int64_t k, const Veh &w, int cell,
                                           Walk &wk, Scan &s, uint32_t &c_scan) {
  s.kind = SC_FREE; s.cL = 0; s.vL = 0.0f; s.reached_own = false; s.stop_only = false;
  s.nt_own = 0u; s.e2 = MANTA_NONE; s.e2cnl = 0u;
  wk.limit = cell + p.H; wk.base = 0; wk.pos = cell + 1; wk.sl = ld_lane(w.ld);
  wk.r = w.rc; wk.se = w.e; wk.sm = w.em; wk.own = true;   // wk.nent: the next route entry, from the state
  const int C = (int)cells_of(w.em.cnl);
  if (closable(w.em)) {
    const int half = C / 2;
    if (cell < half && half <= wk.limit && lane_closed(p, __ldg(p.lane_base + w.e) + (uint32_t)wk.sl, k)) {
      const uint8_t *row = cur + w.em.row0 + (uint32_t)wk.sl * stride_of((uint32_t)C);
      uint32_t byte = 0;
      const int c = first_up(row, cell + 1, half - 1, byte);
      if (c >= 0) {
        s.kind = SC_LEADER; s.cL = c; s.vL = speed_decode(byte);
        c_scan += (uint32_t)(c - cell);
      } else {
        s.kind = SC_VIRTUAL; s.cL = half + p.L - 1; s.vL = 0.0f;
        c_scan += (uint32_t)(half - 1 - cell);
      }
      return true;
    }
  }
  return false;
}

// Consumes the first batch of the own row, fetched with the vehicle record:
// returns true when the scan is complete; otherwise the next round trip
// continues along the row or, when the batch reached the end of the scanned
// range, fetches the node data only.
__device__ __forceinline__ bool walk_first(const Params &p, const Veh &w, Walk &wk, const uint8_t *slot, int cell,
                                           Scan &s, uint32_t &c_scan) {
  const int segC = (int)cells_of(wk.sm.cnl);
  const int hi = min(wk.limit, segC - 1);
  const int lo = wk.pos;
  const int c0 = lo & ~15;
  uint32_t byte = 0;
  const int c = check_slot(slot, min(kFirstChunks, ((hi - c0) >> 4) + 1), c0, lo, hi, byte);
  if (c >= 0) {
    s.kind = SC_LEADER; s.cL = c; s.vL = speed_decode(byte);
    c_scan += (uint32_t)(c - cell);
    return true;
  }
  if (c0 + 16 * kFirstChunks <= hi) { wk.pos = c0 + 16 * kFirstChunks; return false; }
  if (segC > wk.limit) { c_scan += (uint32_t)p.H; return true; }
  if (wk.r + 1u >= w.rend) { c_scan += (uint32_t)(segC - 1 - cell); return true; }
  wk.pos = hi + 1;
  return false;
}

// Issues the loads of the walk's next round trip.
__device__ __forceinline__ void walk_issue(const Params &p, const uint8_t *cur, const Veh &w, const Walk &wk,
                                           uint32_t slot, Fetch &f) {
  const int segC = (int)cells_of(wk.sm.cnl);
  const int hi = min(wk.limit, wk.base + segC - 1) - wk.base;   // row-relative
  const int lo = wk.pos - wk.base;
  const int c0 = lo & ~15;
  if (lo <= hi)
    slot_fetch(slot, cur + wk.sm.row0 + (uint32_t)wk.sl * stride_of((uint32_t)segC) + c0,
               min(kWalkChunks, ((hi - c0) >> 4) + 1));
  const bool last = lo > hi || c0 + 16 * kWalkChunks > hi;
  if (last && wk.base + segC <= wk.limit && wk.r + 1u < w.rend) {
    f.nt = __ldg(p.ntype + node_of(wk.sm));
    f.sig = load_sig(p, wk.se);
    f.sm2 = load_em(p, wk.nent & MANTA_EDGE_MASK);
    f.nent2 = wk.r + 2u < w.rend ? __ldg(p.route + wk.r + 2u) : 0u;
  }
}

// Consumes the round trip issued by walk_issue: returns true when the scan
// is complete (result in s), otherwise advances the walk.
__device__ __forceinline__ bool walk_process(const Params &p, int64_t k, const Veh &w, int cell, Walk &wk,
                                             const Fetch &f, const uint8_t *slot, Scan &s, uint32_t &c_scan,
                                             uint32_t &c_rr) {
  const int segC = (int)cells_of(wk.sm.cnl);
  const int hi = min(wk.limit, wk.base + segC - 1) - wk.base;
  const int lo = wk.pos - wk.base;
  const int c0 = lo & ~15;
  const bool last = lo > hi || c0 + 16 * kWalkChunks > hi;
  if (lo <= hi) {
    uint32_t byte = 0;
    const int c = check_slot(slot, min(kWalkChunks, ((hi - c0) >> 4) + 1), c0, lo, hi, byte);
    if (c >= 0) {
      s.kind = SC_LEADER; s.cL = wk.base + c; s.vL = speed_decode(byte);
      c_scan += (uint32_t)(s.cL - cell);
      return true;
    }
    if (!last) { wk.pos = wk.base + c0 + 16 * kWalkChunks; return false; }
  }
  const int B = wk.base + segC;
  if (B > wk.limit) { c_scan += (uint32_t)p.H; return true; }
  if (wk.r + 1u >= w.rend) { c_scan += (uint32_t)(B - 1 - cell); return true; }
  c_rr++;
  const uint32_t n = node_of(wk.sm);
  const uint32_t e2 = wk.nent & MANTA_EDGE_MASK;
  bool blocked = false;
  if (f.nt == 2u && !is_green(f.sig, k)) blocked = true;
  if (closable(f.sm2) &&
      lane_closed(p, __ldg(p.lane_base + e2) + (uint32_t)min(wk.sl, lanes_of(f.sm2.cnl) - 1), k))
    blocked = true;                      // no entry into a closed lane
  if (wk.own) {
    const bool stop_np = (f.nt == 1u) && (ldv(p.permit + n) != w.id);
    s.reached_own = true;
    s.stop_only = stop_np;
    s.nt_own = f.nt;
    s.e2 = e2;
    s.e2cnl = f.sm2.cnl;
    if (stop_np) blocked = true;
  } else if (f.nt == 1u) {
    blocked = true;
  }
  if (blocked) {
    s.kind = SC_VIRTUAL; s.cL = B + p.L - 1; s.vL = 0.0f;
    c_scan += (uint32_t)(B - 1 - cell);
    return true;
  }
  wk.r = wk.r + 1u; wk.base = B; wk.pos = B; wk.se = e2;
  wk.sm = f.sm2;
  wk.sl = min(wk.sl, lanes_of(f.sm2.cnl) - 1);
  wk.own = false;
  wk.nent = f.nent2;
  return false;
}

// Appends the n crossing requests staged in buffer q (field-major, 32 per
// field) to the request list.  Called by the lanes in `am` (rank rk of cnt).
__device__ __forceinline__ void flush_requests(const Params &p, const uint32_t *q, int n, unsigned am, int rk,
                                               int cnt) {
  uint32_t g0 = 0;
  if (rk == 0) g0 = atomicAdd(&p.ctl->n_req, (uint32_t)n);
  g0 = __shfl_sync(am, g0, __ffs(am) - 1);
  for (int j = rk; j < n; j += cnt) {
    const uint32_t o = g0 + (uint32_t)j;
    if (!IDX_OK(o, p.cap_list, 22)) continue;
    p.req[o] = q[0 * 32 + j]; p.req_x[o] = __uint_as_float(q[1 * 32 + j]); p.req_v[o] = __uint_as_float(q[2 * 32 + j]);
    p.req_dw[o] = q[3 * 32 + j]; p.req_g[o] = q[4 * 32 + j]; p.req_t[o] = q[5 * 32 + j]; p.req_e2[o] = q[6 * 32 + j];
    p.req_n[o] = q[7 * 32 + j];
  }
  __syncwarp(am);
}

// ------------------------------------------------------------ the kernel
template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) manta_step_kernel(Params p) {
  __shared__ int s_ok;
  __shared__ unsigned long long s_cnt[CNT_N];
  __shared__ float s_sab2[8];                       // 2 sqrt(a b) per road class (Eq. 1)
  // Eq. 1 parameters per road class, read with the lane's own class: from
  // shared memory, a warp whose lanes hold vehicles of different classes
  // reads them in one access
  __shared__ float s_a[8], s_T[8], s_s0[8], s_v0f[8];
  __shared__ int s_s0c[8];
  // per-warp scratch of P3 (dynamic shared memory, kWarpWords words per
  // warp): the work pool (32 slots, list indices, first-batch offsets), 32
  // staged crossing requests (9 fields, field-major) and the finish queue
  // (kFqFields fields x 64 entries)
  extern __shared__ __align__(16) uint32_t s_wbuf[];
  __shared__ int s_rqn[BLOCK / 32];
  __shared__ uint32_t s_lcs[BLOCK];                 // per thread: cells read by lane-change scans
  __shared__ uint32_t s_lcn, s_lct;                 // lane-change candidates of the block; batches taken
  Ctl *ctl = p.ctl;
  if (threadIdx.x < CNT_N) s_cnt[threadIdx.x] = 0ull;
  if (threadIdx.x < 8) {
    s_sab2[threadIdx.x] = 2.0f * sqrtf(p.a[threadIdx.x] * p.b[threadIdx.x]);
    s_a[threadIdx.x] = p.a[threadIdx.x]; s_T[threadIdx.x] = p.T[threadIdx.x]; s_s0[threadIdx.x] = p.s0[threadIdx.x];
    s_v0f[threadIdx.x] = p.v0f[threadIdx.x]; s_s0c[threadIdx.x] = p.s0c[threadIdx.x];
  }
  if (threadIdx.x == 0) { s_lcn = 0u; s_lct = 0u; }
  s_lcs[threadIdx.x] = 0u;
  __syncthreads();
  // per-thread counters fit 32 bits over one launch (at most 2048 steps)
  uint32_t c_upd = 0, c_scan = 0, c_clamp = 0, c_lc = 0, c_lce = 0, c_rr = 0, c_dep = 0, c_arr = 0;
  __shared__ unsigned long long ph[4];
  if (threadIdx.x < 4) ph[threadIdx.x] = 0ull;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t gsz = gridDim.x * blockDim.x;
  // the same threads numbered so that consecutive warps of 32 lie in
  // different blocks: short item lists (lane changes, departures, merges)
  // spread over every SM instead of queueing on the first few SMs' load units
  const uint32_t gspr = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u + (threadIdx.x & 31u);
  const int L = p.L;
  bool alive = ldvi(&ctl->err) == 0;
  unsigned bar_target = 0;
  // first step of this launch: from the host, or from the control block when
  // the launch is replayed from a captured graph
  const int64_t kbase = p.k_from_ctl ? (int64_t)(*(const volatile long long *)&ctl->k_next) : p.k0;
  uint64_t tp = timer ? globaltimer() : 0;
  // The block's lane-change candidates: the first lc_cap in its (otherwise
  // idle) main-phase scratch, 64 bytes each; the rest in the block's region of
  // the global list.  A block lists at most one candidate per list entry its
  // record pass visits and one per merge-phase item it runs.
  constexpr uint32_t lc_cap = lc_cap_of(BLOCK);
  auto lc_region = [&](uint32_t rstride, uint32_t n_rec, uint32_t n_items) {
    return blockIdx.x * lc_overflow(BLOCK, rstride, gsz, n_rec, n_items);
  };
  auto lc_store = [&](uint32_t at, const Veh &w, uint32_t pos, uint32_t reg0) {
    if (at < lc_cap) {
      uint4 *e = reinterpret_cast<uint4 *>(s_wbuf) + 4u * at;
      e[0] = make_uint4(__float_as_uint(w.x), __float_as_uint(w.v), w.id, w.rc);
      e[1] = make_uint4(w.rend, w.e, w.ld, w.pcell);
      e[2] = make_uint4(w.em.row0, w.em.cnl, __float_as_uint(w.em.lim), w.em.dst);
      e[3].x = pos;
    } else if (IDX_OK(reg0 + (at - lc_cap), p.cap_lcq, 5)) {
      p.lcq[reg0 + (at - lc_cap)] = w;
      p.lcq_pos[reg0 + (at - lc_cap)] = pos;
    }
  };
  // The record pass that prepares step kk: over list positions [0, n) of ain
  // (vehicle state Rin), clear each vehicle's cell of M_{kk-1} in clr (the
  // buffer written during kk), note the first batch of its leader scan (p3a)
  // and list the block's lane-change candidates (a record copy with the list
  // position in pcell, and the list position).  With cmp the live vehicles
  // are compacted into aout and their state moved to Rout (else aout is ain
  // and Rout is Rin).  Entries marked kReqMark belong to the last step's
  // requesters, whose state P4 rewrote: the mark is removed, and when the
  // pass runs in that same merge phase (merged) P4 prepares them itself.
  // The pass runs on warps w0 .. w0 + nw - 1 of the spread numbering (gspr).
  auto rec = [&](int64_t kk, const uint32_t *ain, uint32_t *aout, const VehSet &Rin, const VehSet &Rout, uint32_t n,
                 bool cmp, uint8_t *clr, bool merged, uint32_t reg0, uint32_t w0, uint32_t nw) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = gspr >> 5;
    if (gw < w0) return;
    const uint32_t stride = 32u * nw;
    uint32_t base = 32u * (gw - w0);
    uint32_t s_nx = base + lane < n ? __ldcg(ain + base + lane) : MANTA_NONE;
    Veh w_nx;
    uint32_t r_nx = 0u;   // the next route entry, moved by a compaction
    if (base + lane < n) {
      w_nx = load_veh(Rin, base + lane);
      if (cmp) r_nx = __ldcg(Rin.nx + base + lane);
    }
    for (; base < n; base += stride) {
      const uint32_t i = base + (uint32_t)lane;
      uint32_t s = s_nx;
      Veh w = w_nx;
      const uint32_t rn = r_nx;
      // the warp's next entries and their state load while it works on
      // these (a hole's state is loaded and ignored)
      const uint32_t i2 = base + stride + (uint32_t)lane;
      s_nx = i2 < n ? __ldcg(ain + i2) : MANTA_NONE;
      if (i2 < n) {
        w_nx = load_veh(Rin, i2);
        if (cmp) r_nx = __ldcg(Rin.nx + i2);
      }
      bool skip = false;
      if (s != MANTA_NONE && (s & kReqMark) != 0u) {
        s &= ~kReqMark;
        if (!cmp && IDX_OK(i, p.cap_list, 1)) aout[i] = s;
        skip = merged;
      }
      uint32_t pos = i;
      if (cmp) {
        const uint32_t at = warp_append(&ctl->n_compact, s != MANTA_NONE);
        if (s != MANTA_NONE && IDX_OK(at, p.cap_list, 2)) aout[at] = at;
        pos = at;
      }
      bool cand = false;
      if (s != MANTA_NONE && !skip) {
        if (cmp && IDX_OK(pos, p.cap_slots, 39)) {
          store_veh(Rout, pos, w);
          Rout.nx[pos] = rn;
        }
        if (w.pcell != MANTA_NONE && IDX_OK(w.pcell, p.cap_map, 3)) clr[w.pcell] = (uint8_t)MANTA_EMPTY;
        if (IDX_OK(pos, p.cap_list, 4)) p.p3a[pos] = first_batch(w.em, ld_lane(w.ld), (int)floorf(w.x));
        cand = lc_candidate(w, kk);
        if (cand) w.pcell = pos;        // the candidate carries its list position in pcell
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, cand);
      uint32_t b = 0;
      if (lane == 0 && bal) b = atomicAdd(&s_lcn, (uint32_t)__popc(bal));
      b = __shfl_sync(0xFFFFFFFFu, b, 0);
      if (cand) lc_store(b + (uint32_t)__popc(bal & ((1u << lane) - 1u)), w, pos, reg0);
    }
  };
  // the record pass of the current step already ran in the last merge phase,
  // and the block's candidate list lives in region reg0_next
  bool rec_ready = false;
  uint32_t reg0_next = 0u;
  for (int it = 0; it < p.n_steps && alive; ++it) {
    const int64_t k = kbase + it;
    const int cb = (int)(k & 1);
    uint8_t *cur = cb ? p.atlas1 : p.atlas0;
    uint8_t *nxt = cb ? p.atlas0 : p.atlas1;
    const uint32_t sel = ldv(&ctl->act_sel[cb]);
    const uint32_t holes = ldv(&ctl->n_holes[cb]);
    uint32_t *dep = cb ? p.dep1 : p.dep0;
    uint32_t *dep_n = cb ? p.dep0 : p.dep1;
    uint32_t nact = ldv(&ctl->n_act[cb]);
    // compact the active list into the other buffer when holes pass a quarter
    // of it (only in a step whose record pass runs here)
    const bool compact = !rec_ready && holes > 0u && 4u * holes > nact;
    const uint32_t *act_in = sel ? p.act1 : p.act0;
    uint32_t *act = compact ? (sel ? p.act0 : p.act1) : (sel ? p.act1 : p.act0);
    const VehSet Rin = veh_set(p, sel);
    const VehSet R = veh_set(p, compact ? sel ^ 1u : sel);
    // ================================================================ P1
    if (gtid == 0) {
      ctl->next3 = 0u;
      ctl->n_req = 0u;
      ctl->n_arr = 0u;
      ctl->n_holes[cb ^ 1] = compact ? 0u : holes;
      ctl->act_sel[cb ^ 1] = compact ? (sel ^ 1u) : sel;
      ctl->n_dep[cb ^ 1] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
      // trips with departure step <= k + 1 not yet queued: [due_pos, due_hi)
      const uint32_t lo0 = ldv(&ctl->due_hi);
      uint32_t lo = lo0;
      for (;;) {
        const uint32_t i = lo + (threadIdx.x & 31);
        const bool le = i < p.n_trips && (int64_t)__ldg(p.due_step + i) <= k + 1;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, le);
        lo += (uint32_t)__popc(bal);
        if (bal != 0xFFFFFFFFu) break;
      }
      if (threadIdx.x == 0) { ctl->due_pos = lo0; ctl->due_hi = lo; }
    }
    {
      const int lane = threadIdx.x & 31;
      uint32_t reg0 = reg0_next;
      if (!rec_ready) {
        reg0 = lc_region(gsz, nact, 0u);
        rec(k, act_in, act, Rin, R, nact, compact, nxt, false, reg0, 0u, gsz / 32u);
      }
      // lane-change decisions on M_k, a full warp of candidates at a time
      __syncthreads();
      const uint32_t ncand = s_lcn;
      for (;;) {
        uint32_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&s_lct, 32u);
        b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
        if (b0 >= ncand) break;
        const uint32_t j = b0 + (uint32_t)lane;
        if (j < ncand) {
          Veh c;
          uint32_t cpos;
          if (j < lc_cap) {
            const uint4 *e = reinterpret_cast<const uint4 *>(s_wbuf) + 4u * j;
            const uint4 q0 = e[0], q1 = e[1], q2 = e[2];
            c.x = __uint_as_float(q0.x); c.v = __uint_as_float(q0.y); c.id = q0.z; c.rc = q0.w;
            c.rend = q1.x; c.e = q1.y; c.ld = q1.z; c.pcell = q1.w;
            c.em.row0 = q2.x; c.em.cnl = q2.y; c.em.lim = __uint_as_float(q2.z); c.em.dst = q2.w;
            cpos = e[3].x;
          } else {
            c = load_veh_at(p.lcq + reg0 + (j - lc_cap));
            cpos = __ldcg(p.lcq_pos + reg0 + (j - lc_cap));
          }
          const int tgt = lc_decide(p, cur, k, c, c_lce, &s_lcs[threadIdx.x]);
          const uint32_t at = warp_append(&ctl->n_chg, tgt >= 0);
          if (tgt >= 0 && IDX_OK(at, p.cap_list, 6)) {
            // the whole move, so that P2 applies it in one round trip; the
            // map byte at the vehicle's front cell is its own speed code
            const uint32_t stride = stride_of(cells_of(c.em.cnl));
            const int cell = (int)floorf(c.x);
            const uint32_t a = c.em.row0 + (uint32_t)ld_lane(c.ld) * stride + (uint32_t)cell;
            const uint32_t b = c.em.row0 + (uint32_t)tgt * stride + (uint32_t)cell;
            uint4 *m = reinterpret_cast<uint4 *>(p.lcm + at);
            m[0] = make_uint4(c.pcell, cpos, a, b);
            m[1] = make_uint4((c.ld & (kLdEdgeBits | 0x0000FF00u)) | (uint32_t)tgt, first_batch(c.em, tgt, cell),
                              speed_code(c.v), 0u);
          }
        }
      }
    }
    for (uint32_t j = gspr; j < p.n_stop; j += gsz) {
      const uint32_t n = __ldg(p.stop_nodes + j);
      if (ldv(p.permit + n) != MANTA_NONE) continue;
      const uint32_t o = __ldg(p.nin_off + n), m = __ldg(p.nin_off + n + 1) - o;
      const uint32_t r0 = ldv(p.rr + n);
      for (uint32_t t = 0; t < m; ++t) {
        const uint32_t idx = (r0 + t) % m;
        const uint32_t g = o + idx;      // the node's in-lane slots are consecutive
        const uint32_t td = ldv(p.slot_td + g);
        if ((td >> 8) == (uint32_t)(k & 0xFFFFFF) && (td & 0xFFu) >= (uint32_t)p.stop_dwell) {
          p.permit[n] = ldv(p.slot_id + g);
          p.rr[n] = (idx + 1u) % m;
          break;
        }
      }
    }
    if (!grid_sync(ctl, bar_target, p.wait_limit_ns, &s_ok)) { alive = false; break; }
    if (timer) { const uint64_t t = globaltimer(); ph[0] += t - tp; tp = t; }
    // ================================================================ P2
    const uint32_t nchg = ldv(&ctl->n_chg);
    if (nchg) {
      for (uint32_t i = gspr; i < nchg; i += gsz) {
        // (list position twice, old cell, new cell), (lane word, first scan
        // batch, speed code); the gap acceptance keeps every new cell free,
        // so no move's new cell is another's old one
        const uint4 *m = reinterpret_cast<const uint4 *>(p.lcm + i);
        const uint4 m0 = __ldcg(m), m1 = __ldcg(m + 1);
        if (IDX_OK(m0.w, p.cap_map, 7)) cur[m0.w] = (uint8_t)m1.z;
        if (IDX_OK(m0.z, p.cap_map, 8)) cur[m0.z] = (uint8_t)MANTA_EMPTY;
        if (IDX_OK(m0.y, p.cap_slots, 9)) R.ld[m0.y] = m1.x;
        if (IDX_OK(m0.y, p.cap_list, 10)) p.p3a[m0.y] = m1.y;
        c_lc++;
      }
      if (!grid_sync(ctl, bar_target, p.wait_limit_ns, &s_ok)) { alive = false; break; }
    }
    if (timer) { const uint64_t t = globaltimer(); ph[1] += t - tp; tp = t; }
    // ================================================================ P3
    if (compact) nact = ldv(&ctl->n_compact);
    if (gtid == 0) {
      ctl->n_chg = 0u;
      ctl->n_act[cb ^ 1] = nact;   // departures of this step append after it
    }
    const uint32_t tag = (uint32_t)(k + 1);
    // departure requests on M_k'
    const uint32_t ndep = ldv(&ctl->n_dep[cb]);
    for (uint32_t i = gspr; i < ndep; i += gsz) {
      const uint32_t e = __ldcg(dep + i);
      // the queue head (an edge on this list has a trip waiting) loads with
      // the edge record, and the head's trip id with the entry cells
      const EdgeMeta em = load_em(p, e);
      const uint32_t lb = __ldg(p.lane_base + e);
      const uint2 rg = __ldg(p.src_in + e);
      const uint32_t qh = __ldg(p.q_off + e) + __ldcg(p.q_pos + e);
      const uint32_t j = __ldg(p.q_trip + qh);
      const int C = (int)cells_of(em.cnl);
      const int need = min(C, L + s_s0c[class_of(em.cnl)]);
      bool req = !(closable(em) && lane_closed(p, lb, k));
      if (req) {
        uint32_t byte;
        req = first_up(cur + em.row0, 0, need - 1, byte) < 0;
      }
      if (req && IDX_OK(e, p.E, 11)) p.dep_key[e] = ((unsigned long long)tag << 32) | j;
      // what P4 needs of this departure in one entry: the edge, the queue
      // head's trip (none when it does not request entry), the slot range of
      // its competitors (the in-lanes of the edge's tail node), and the
      // trip's route bounds, lane word and next route entry, so that P4's
      // chain of dependent round trips starts at the competitors
      uint32_t rc = 0u, rend = 0u, ld0 = 0u, nx0 = 0u;
      if (req) {
        rc = __ldg(p.route_off + j);
        rend = __ldg(p.route_off + j + 1u);
        ld0 = ld_for_entry(p, rc, 0u);
        nx0 = rc + 1u < rend ? __ldg(p.route + rc + 1u) : 0u;
      }
      uint4 *di = reinterpret_cast<uint4 *>(p.dep_info) + 2u * i;
      di[0] = make_uint4(e, req ? j : MANTA_NONE, rg.x, rg.y);
      di[1] = make_uint4(rc, rend, ld0, nx0);
    }
    // vehicles
    const int64_t kr = k - p.t0;
    const int win = (kr >= 0 && kr / p.win_steps < p.n_win) ? (int)(kr / p.win_steps) : -1;
    // Each lane carries one vehicle through its record fetch and a leader
    // walk of one lane-map batch per round trip; every iteration first issues
    // the loads of all lanes and then consumes them, and a lane whose vehicle
    // is done takes the next one from the warp's pool at once, so lanes do
    // not wait for the longest walk of their warp.  The pool takes chunks of
    // list entries from a shared counter (holes dropped), the next chunk's
    // slots loading while the pool drains.  Chunks hold 32 entries while the
    // list is long and shrink as it runs out (guided self-scheduling), so
    // warps finish the phase close together.
    {
      const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5;
      const unsigned lt_mask = (1u << wl) - 1u;
      const uint32_t nwarps = gridDim.x * (BLOCK / 32);
      uint32_t *const wb = s_wbuf + wid * kWarpWords;
      uint32_t *pi = wb + 32, *pa = wb + 64;
      uint32_t *fq = wb + 384;   // finish queue: kFqFields fields x 64 entries
      // the lane's batch slot (shared-window address for the copies, pointer for the reads)
      const uint8_t *slot_p = reinterpret_cast<const uint8_t *>(wb + kP3Words) + wl * kSlotBytes;
      const uint32_t slot_s = (uint32_t)__cvta_generic_to_shared(slot_p);
      const uint32_t dyn0 = 32u * nwarps;   // every warp's first chunk is fixed
      uint32_t ch = gtid - (uint32_t)wl, csz = 32u;
      uint32_t cslot = ch + wl < nact ? __ldcg(act + ch + wl) : MANTA_NONE;
      uint32_t caddr = ch + wl < nact ? __ldcg(p.p3a + ch + wl) : MANTA_NONE;
      // the chunk after it: its counter value is taken one chunk ahead, so
      // installing a chunk never waits for the atomic (lane 0 holds it).  chn
      // is the raw counter; dyn0 is added only when the chunk is installed, as
      // an add inside lane 0's branch would wait there for the atomic's return
      // and hold the whole warp at the reconvergence point
      uint32_t chn = 0, cszn = 32u;
      if (wl == 0) chn = atomicAdd(&ctl->next3, 32u);
      uint32_t *rqb = wb + 96;
      if (wl == 0) s_rqn[wid] = 0;
      int pn = 0, pu = 0;         // pool size and entries taken (warp-uniform)
      int st = 0;                 // 0 idle, 1 record requested, 2 walking
      uint32_t s = 0, i = 0, a3 = MANTA_NONE;
      int cell = 0;
      // The update of the vehicle in finish-queue entry j (Eq. 1, ballistic
      // step, clamp, map write, requests, arrivals).
      auto finish = [&](int j) {
        Veh w;
        w.x = __uint_as_float(fq[kFqX * 64 + j]); w.v = __uint_as_float(fq[kFqV * 64 + j]);
        w.id = fq[kFqId * 64 + j]; w.rc = fq[kFqRc * 64 + j]; w.rend = fq[kFqRend * 64 + j];
        w.e = fq[kFqE * 64 + j]; w.ld = fq[kFqLd * 64 + j]; w.pcell = MANTA_NONE;
        w.em.row0 = fq[kFqRow0 * 64 + j]; w.em.cnl = fq[kFqCnl * 64 + j];
        w.em.lim = __uint_as_float(fq[kFqLim * 64 + j]); w.em.dst = fq[kFqDst * 64 + j];
        const uint32_t s = fq[kFqS * 64 + j], i = fq[kFqI * 64 + j];
        const int cell = (int)fq[kFqCell * 64 + j];
        Scan sc;
        const uint32_t kd = fq[kFqKind * 64 + j];
        sc.kind = (int)(kd & 3u); sc.reached_own = (kd >> 2) & 1u; sc.stop_only = (kd >> 3) & 1u; sc.nt_own = kd >> 4;
        sc.cL = (int)fq[kFqCL * 64 + j]; sc.vL = __uint_as_float(fq[kFqVL * 64 + j]);
        sc.e2 = fq[kFqE2 * 64 + j]; sc.e2cnl = fq[kFqE2cnl * 64 + j];
        const float x = w.x, v = w.v;
        const int lane = ld_lane(w.ld);
        const uint32_t dwell = ld_dwell(w.ld);
        const EdgeMeta em = w.em;
        const int C = (int)cells_of(em.cnl);
        const int cls = class_of(em.cnl);
        const uint32_t stride = stride_of((uint32_t)C);
        const uint32_t gcell = em.row0 + (uint32_t)lane * stride + (uint32_t)cell;
        const float a = s_a[cls], T = s_T[cls], s0 = s_s0[cls];
        const float v0 = em.lim * s_v0f[cls];
        const float r1 = v / v0, r2 = r1 * r1, r4 = r2 * r2;
        const bool has_next = w.rc + 1u < w.rend;
        float xn, vn;
        bool stop_in_place = false;
        float acc = 0.0f;
        float tsg = 0.0f, tbnd = 0.0f;
        uint32_t tflags = 0;     // event-tape flags of this step
        if (sc.kind == SC_FREE) {
          acc = a * (1.0f - r4);
        } else {
          const float sg = __int2float_rn(sc.cL - cell - L);
          tsg = sg;
          if (sg <= 0.0f) {
            stop_in_place = true;
          } else {
            const float dv = v - sc.vL;
            const float dyn = (v * dv) / s_sab2[cls];
            float ss;
            if (p.textbook) ss = s0 + fmaxf(0.0f, v * T + dyn);
            else ss = (s0 + v * T) + dyn;
            const float q = ss / sg;
            acc = a * ((1.0f - r4) - q * q);
          }
        }
        if (stop_in_place) {
          xn = x; vn = 0.0f;
          tflags = (uint32_t)TK_STOP << TF_KIND_SHIFT;
        } else {
          const float dt = p.dt;
          const float vt = v + acc * dt;
          float xt, vv;
          tflags = ((uint32_t)(sc.kind == SC_FREE ? TK_FREE : TK_INTERACT) << TF_KIND_SHIFT) |
                   (vt >= 0.0f ? TF_BALLISTIC : 0u);
          if (vt >= 0.0f) { xt = x + (v * dt + (0.5f * acc) * (dt * dt)); vv = vt; }
          else { xt = x - (v * v) / (2.0f * acc); vv = 0.0f; }
          bool has_bound = sc.kind != SC_FREE;
          int bnd = sc.cL - L;
          if (has_next && xt >= __int2float_rn(C)) {
            // at most one node per step: stay within the next edge
            const uint32_t cnl2 = sc.e2 != MANTA_NONE
                                      ? sc.e2cnl
                                      : load_em(p, __ldg(p.route + w.rc + 1u) & MANTA_EDGE_MASK).cnl;
            const int cap = C + (int)cells_of(cnl2) - 1;
            if (!has_bound || cap < bnd) { has_bound = true; bnd = cap; }
          }
          if (has_bound && xt > __int2float_rn(bnd)) {
            xn = fmaxf(x, __int2float_rn(bnd)); vn = 0.0f; c_clamp++;
            tbnd = __int2float_rn(bnd);
            tflags |= (x > tbnd ? 1u : 2u) << TF_CLAMP_SHIFT;
          } else { xn = xt; vn = vv; }
        }
        uint32_t dwn = 0;
        if (has_next && sc.reached_own && sc.stop_only) {
          const int zone = C - 1 - (s_s0c[cls] + 2);
          if ((int)floorf(xn) >= zone && vn < p.stop_eps) dwn = dwell < 255u ? dwell + 1u : 255u;
        }
        // request and stop-line slots of the vehicle's edge, loaded only where used
        if (has_next && sc.reached_own && sc.nt_own == 1u &&
            IDX_OK(__ldg(p.rslot + w.e) + (uint32_t)lane, p.cap_lanes, 12)) {
          const uint32_t g = __ldg(p.rslot + w.e) + (uint32_t)lane;
          p.slot_id[g] = w.id;
          p.slot_td[g] = ((uint32_t)(tag & 0xFFFFFF) << 8) | dwn;
        }
        c_upd++;
        const bool crossing = xn >= __int2float_rn(C);
        const bool arrive = crossing && !has_next;
        const bool request = crossing && has_next;
        if (arrive) {
          if (IDX_OK(w.e, p.E, 13)) atomicAdd(p.exitc + w.e, 1u);
          c_arr++;
        }
        uint32_t rq_g = 0, rq_t = 0, rq_e2 = 0;
        if (request) {
          rq_e2 = sc.e2 != MANTA_NONE ? sc.e2 : (__ldg(p.route + w.rc + 1u) & MANTA_EDGE_MASK);
          const uint32_t cnl2 = sc.e2 != MANTA_NONE ? sc.e2cnl : load_em(p, rq_e2).cnl;
          const int l2 = min(lane, lanes_of(cnl2) - 1);
          rq_g = __ldg(p.rslot + w.e) + (uint32_t)lane;
          rq_t = target_key(rq_e2, (uint32_t)l2);
          if (IDX_OK(rq_g, p.cap_lanes, 14)) {
            p.req_tgt[rq_g] = rq_t;
            p.req_key[rq_g] = ((unsigned long long)tag << 32) | w.id;
          }
        } else if (!arrive) {
          w.x = xn; w.v = vn;
          w.ld = (w.ld & kLdEdgeBits) | (uint32_t)lane | (dwn << 8);
          w.pcell = gcell;
          if (IDX_OK(s, p.cap_slots, 15)) store_veh_state(R, s, w);
          const uint32_t o_map = em.row0 + (uint32_t)lane * stride + (uint32_t)(int)floorf(xn);
          if (IDX_OK(o_map, p.cap_map, 16)) nxt[o_map] = speed_code(vn);
          if (win >= 0) {
            const size_t o = (size_t)win * p.E + w.e;
            if (IDX_OK(o, (uint64_t)p.n_win * p.E, 17)) {
              atomicAdd(&p.lstat[o].sum, (unsigned long long)(vn * 1048576.0f));
              atomicAdd(&p.lstat[o].cnt, 1u);
            }
          }
        }
        if (arrive) {
          if (IDX_OK(i, p.cap_list, 18)) act[i] = MANTA_NONE;
          const uint32_t ia = atomicAdd(&ctl->n_arr, 1u);
          if (IDX_OK(ia, p.cap_list, 19)) p.arr[ia] = gcell;
          atomicAdd(&ctl->n_holes[cb ^ 1], 1u);
        }
        if (request) {
          // staged in the warp's buffer; written out 32 at a time
          const unsigned am = __activemask();
          const int rk = __popc(am & lt_mask), cnt = __popc(am);
          int nb = s_rqn[wid];
          if (nb + cnt > 32) {
            flush_requests(p, rqb, nb, am, rk, cnt);
            nb = 0;
          }
          const int at = nb + rk;
          rqb[0 * 32 + at] = s; rqb[1 * 32 + at] = __float_as_uint(xn); rqb[2 * 32 + at] = __float_as_uint(vn);
          rqb[3 * 32 + at] = dwn; rqb[4 * 32 + at] = rq_g; rqb[5 * 32 + at] = rq_t; rqb[6 * 32 + at] = rq_e2;
          rqb[7 * 32 + at] = node_of(em);
          __syncwarp(am);
          if (rk == 0) s_rqn[wid] = nb + cnt;
          __syncwarp(am);
          // P4 rewrites this record: the next record pass leaves it to P4
          if (IDX_OK(i, p.cap_list, 21)) act[i] = s | kReqMark;
        }
        if (p.tape) {
          const int64_t tk = k - p.tape_k0;
          if (tk >= 0 && tk < p.tape_len) {
            const uint32_t out = arrive ? TO_ARRIVE : (request ? TO_PENDING : TO_STAY);
            TapeRec r;
            r.x = x; r.v = v; r.s = tsg; r.vL = sc.vL; r.bnd = tbnd; r.lim = em.lim; r.C = (uint32_t)C;
            r.flags = TF_PRESENT | tflags | (out << TF_OUT_SHIFT) | ((uint32_t)cls << TF_CLASS_SHIFT);
            r.sample = (out == TO_STAY && win >= 0) ? (uint32_t)((size_t)win * p.E + w.e) : MANTA_NONE;
            r.pad = 0u;
            p.tape[(size_t)tk * p.n_trips + w.id] = r;
          }
        }
      };
      int fqn = 0;                // finish-queue length (warp-uniform)
      Veh w;
      Walk wk;
      Scan sc;
      for (;;) {
        __syncwarp();
        unsigned need = __ballot_sync(0xFFFFFFFFu, st == 0);
        while (need != 0u) {
          if (pu == pn) {
            if (ch >= nact) break;
            // install the prefetched chunk, then prefetch the next one
            const bool valid = (uint32_t)wl < csz && cslot != MANTA_NONE;
            const unsigned vb = __ballot_sync(0xFFFFFFFFu, valid);
            __syncwarp();
            if (valid) {
              const int q = __popc(vb & lt_mask);
              pi[q] = ch + (uint32_t)wl;     // the list position is the vehicle's state index
              pa[q] = caddr;
            }
            pn = __popc(vb);
            pu = 0;
            ch = dyn0 + __shfl_sync(0xFFFFFFFFu, chn, 0);
            csz = __shfl_sync(0xFFFFFFFFu, cszn, 0);
            const bool inb = (uint32_t)wl < csz && ch + wl < nact;
            cslot = inb ? __ldcg(act + ch + wl) : MANTA_NONE;
            caddr = inb ? __ldcg(p.p3a + ch + wl) : MANTA_NONE;
            if (wl == 0) {
              const uint32_t rem = ch < nact ? nact - ch : 0u;
              cszn = min(32u, max(4u, rem / (2u * nwarps)));
              chn = atomicAdd(&ctl->next3, cszn);
            }
            __syncwarp();
            continue;
          }
          const int take = min(__popc(need), pn - pu);
          const int rank = __popc(need & lt_mask);
          if (st == 0 && rank < take) {
            i = pi[pu + rank];
            s = i;
            a3 = pa[pu + rank];
            st = 1;
          }
          pu += take;
          need = __ballot_sync(0xFFFFFFFFu, st == 0);
        }
        if (__ballot_sync(0xFFFFFFFFu, st != 0) == 0u) break;
        Fetch f;
        if (st == 1) {
          // the record and, in the same round trip, the first batch of its row
          w = load_veh_main(R, s);
          wk.nent = __ldcg(R.nx + s);
          if (a3 != MANTA_NONE) slot_fetch(slot_s, cur + a3, kFirstChunks);
        } else if (st == 2) {
          walk_issue(p, cur, w, wk, slot_s, f);
        }
        // while those loads are in flight, the whole warp updates 32 vehicles
        // of the finish queue (it holds at most 63 here: at most 31 left by
        // the last update and 32 added since)
        if (fqn >= 32) {
          __syncwarp();
          finish(fqn - 32 + wl);
          fqn -= 32;
          __syncwarp();
        }
        cp_async_wait_all();
        bool fin = false;
        if (st == 1) {
          cell = (int)floorf(w.x);
          fin = walk_start(p, cur, k, w, cell, wk, sc, c_scan);
          st = 2;
          if (!fin && a3 != MANTA_NONE) fin = walk_first(p, w, wk, slot_p, cell, sc, c_scan);
        } else if (st == 2) {
          fin = walk_process(p, k, w, cell, wk, f, slot_p, sc, c_scan, c_rr);
        }
        // completed vehicles join the warp's finish queue; the update itself
        // runs 32 at a time with the whole warp
        const unsigned fb = __ballot_sync(0xFFFFFFFFu, fin);
        if (fin) {
          st = 0;
          const int at = fqn + __popc(fb & lt_mask);
          fq[kFqX * 64 + at] = __float_as_uint(w.x); fq[kFqV * 64 + at] = __float_as_uint(w.v);
          fq[kFqId * 64 + at] = w.id; fq[kFqRc * 64 + at] = w.rc; fq[kFqRend * 64 + at] = w.rend;
          fq[kFqE * 64 + at] = w.e; fq[kFqLd * 64 + at] = w.ld; fq[kFqRow0 * 64 + at] = w.em.row0;
          fq[kFqCnl * 64 + at] = w.em.cnl; fq[kFqLim * 64 + at] = __float_as_uint(w.em.lim);
          fq[kFqDst * 64 + at] = w.em.dst; fq[kFqS * 64 + at] = s; fq[kFqI * 64 + at] = i;
          fq[kFqCell * 64 + at] = (uint32_t)cell;
          fq[kFqKind * 64 + at] = (uint32_t)sc.kind | ((uint32_t)sc.reached_own << 2) | ((uint32_t)sc.stop_only << 3) |
                                  (sc.nt_own << 4);
          fq[kFqCL * 64 + at] = (uint32_t)sc.cL; fq[kFqVL * 64 + at] = __float_as_uint(sc.vL);
          fq[kFqE2 * 64 + at] = sc.e2; fq[kFqE2cnl * 64 + at] = sc.e2cnl;
        }
        fqn += __popc(fb);
      }
      __syncwarp();
      if (wl < fqn) finish(wl);
      __syncwarp();
      if (fqn > 32 && wl < fqn - 32) finish(32 + wl);
      __syncwarp();
      const int nb = s_rqn[wid];
      if (nb > 0) flush_requests(p, rqb, nb, 0xFFFFFFFFu, wl, 32);
    }
    if (!grid_sync(ctl, bar_target, p.wait_limit_ns, &s_ok)) { alive = false; break; }
    if (timer) { const uint64_t t = globaltimer(); ph[2] += t - tp; tp = t; }
    // ================================================================ P4
    // Crossing requests, departures, arrivals' cells and the trips due at
    // k + 1 are independent of one another: they share one index space so
    // that their dependent loads overlap instead of running one after another.
    //  - crossing requests: the lowest id among requests for the same target
    //    lane wins
    //  - departures: the queue head wins unless a crossing with a lower id
    //    targets lane 0
    //  - arrivals leave the current map
    //  - trips due at step k + 1 join their edge's departure queue
    // Within each kind, loads that depend on the same earlier value go out
    // together, and independent counter updates overlap, so that the longest
    // chain of dependent round trips stays short.
    const uint32_t nreq = ldv(&ctl->n_req);
    const uint32_t narr = ldv(&ctl->n_arr);
    const uint32_t due_lo = ldv(&ctl->due_pos), due_hi = ldv(&ctl->due_hi);
    // This phase also runs the record pass of step k + 1 (the vehicles that
    // stayed on their edge in P3; P4's own vehicles are prepared where P4
    // finalises them), unless this is the launch's last step or k + 1 will
    // compact its list.  Every block takes the same decision.
    const uint32_t holes_n = ldv(&ctl->n_holes[cb ^ 1]);
    const bool ahead = it + 1 < p.n_steps && !(holes_n > 0u && 4u * holes_n > nact);
    // the pass runs on the warps that have no merge-phase item, when those are
    // at least half of all warps (items go to warps in gspr order)
    const uint32_t t_items = nreq + ndep + narr + (due_hi - due_lo);
    const uint32_t w_items = (t_items + 31u) / 32u, w_all = gsz / 32u;
    const uint32_t rw0 = 2u * w_items <= w_all ? w_items : 0u;
    const uint32_t reg0n = ahead ? lc_region(32u * (w_all - rw0), nact, nreq + ndep) : 0u;
    if (threadIdx.x == 0) { s_lcn = 0u; s_lct = 0u; }   // the block's lane-change list of step k + 1
    __syncthreads();
    auto lc_add1 = [&](Veh w, uint32_t pos, uint32_t slot) {
      w.pcell = slot;
      lc_store(atomicAdd(&s_lcn, 1u), w, pos, reg0n);
    };
    const uint32_t t_dep = nreq, t_arr = t_dep + ndep, t_due = t_arr + narr, t_end = t_due + (due_hi - due_lo);
    for (uint32_t t = gspr; t < t_end; t += gsz) {
      if (t < t_dep) {
        const uint32_t i = t;
        // round trip 1: the request (with its position and speed); 2: the
        // records it names and the node's slot range; 3: the competitors'
        // requests (the node's slots are consecutive) and the route entry
        // after the crossing
        const uint32_t s = __ldcg(p.req + i);
        const uint32_t gown = __ldcg(p.req_g + i), tgt = __ldcg(p.req_t + i);
        const uint32_t e2 = __ldcg(p.req_e2 + i), n = __ldcg(p.req_n + i);
        const float rx = __ldcg(p.req_x + i), rv = __ldcg(p.req_v + i);
        const uint32_t rpos = s;                // its list position
        const uint32_t o0 = __ldg(p.nin_off + n), o1 = __ldg(p.nin_off + n + 1);
        const unsigned long long dk = __ldcg(p.dep_key + e2);
        const EdgeMeta em2 = load_em(p, e2);
        Veh w = load_veh(R, s);
        const uint32_t ld2 = ld_for_entry(p, w.rc + 1u, tgt & 15u);   // with the competitors' slots
        const uint32_t nx2 = w.rc + 2u < w.rend ? __ldg(p.route + w.rc + 2u) : 0u;
        const int lane = ld_lane(w.ld);
        const EdgeMeta em = w.em;
        const uint32_t stride = stride_of(cells_of(em.cnl));
        bool win_it = min_competitor(p, o0, o1, gown, tgt, tag) > w.id;
        if (win_it && tgt == target_key(e2, 0u) && (uint32_t)(dk >> 32) == tag && (uint32_t)dk < w.id) win_it = false;
        const uint32_t cell = (uint32_t)(int)floorf(w.x);
        w.pcell = em.row0 + (uint32_t)lane * stride + cell;
        float xf, vf;
        uint32_t ef;
        if (win_it) {
          const int C = (int)cells_of(em.cnl);
          if (__ldg(p.ntype + n) == 1 && ldv(p.permit + n) == w.id) p.permit[n] = MANTA_NONE;
          if (IDX_OK(w.e, p.E, 23)) atomicAdd(p.exitc + w.e, 1u);
          if (IDX_OK(e2, p.E, 24)) atomicAdd(p.entry + e2, 1u);
          xf = rx - __int2float_rn(C);
          vf = rv;
          const uint32_t l2 = tgt & 15u;
          w.e = e2; w.rc = w.rc + 1u;
          w.ld = ld2;
          w.em = em2;
          w.em.lim = driver_limit(p, em2.lim, w.id, w.rc);
          const uint32_t o_map = em2.row0 + l2 * stride_of(cells_of(em2.cnl)) + (uint32_t)(int)floorf(xf);
          if (IDX_OK(o_map, p.cap_map, 25)) nxt[o_map] = speed_code(vf);
          ef = e2;
        } else {
          const int C = (int)cells_of(em.cnl);
          xf = fmaxf(w.x, __int2float_rn(C - 1));
          vf = 0.0f;
          w.ld = (w.ld & kLdEdgeBits) | (uint32_t)lane | (__ldcg(p.req_dw + i) << 8);
          const uint32_t o_map = em.row0 + (uint32_t)lane * stride + (uint32_t)(int)floorf(xf);
          if (IDX_OK(o_map, p.cap_map, 26)) nxt[o_map] = speed_code(vf);
          ef = w.e;
        }
        if (p.tape) {
          const int64_t tk = k - p.tape_k0;
          if (tk >= 0 && tk < p.tape_len) {
            TapeRec *r = p.tape + (size_t)tk * p.n_trips + w.id;
            // held: xf = max(old x, C - 1) keeps the old position or sets the stop line
            const uint32_t out = win_it ? TO_CROSS : (w.x == xf ? TO_HELD_KEEP : TO_HELD_LINE);
            r->flags = (r->flags & ~(7u << TF_OUT_SHIFT)) | (out << TF_OUT_SHIFT);
            r->sample = win >= 0 ? (uint32_t)((size_t)win * p.E + ef) : MANTA_NONE;
          }
        }
        w.x = xf; w.v = vf;
        if (IDX_OK(s, p.cap_slots, 27)) {
          store_veh(R, s, w);
          if (win_it) R.nx[s] = nx2;
        }
        if (win >= 0) {
          const size_t o = (size_t)win * p.E + ef;
          if (IDX_OK(o, (uint64_t)p.n_win * p.E, 28)) {
            atomicAdd(&p.lstat[o].sum, (unsigned long long)(vf * 1048576.0f));
            atomicAdd(&p.lstat[o].cnt, 1u);
          }
        }
        if (ahead) {
          // step k + 1's record pass for this vehicle: its M_k cell is in the
          // buffer written during k + 1
          if (IDX_OK(w.pcell, p.cap_map, 29)) cur[w.pcell] = (uint8_t)MANTA_EMPTY;
          if (IDX_OK(rpos, p.cap_list, 30)) p.p3a[rpos] = first_batch(w.em, ld_lane(w.ld), (int)floorf(w.x));
          if (lc_candidate(w, k + 1)) lc_add1(w, rpos, s);
        }
      } else if (t < t_arr) {
        const uint32_t i = t - t_dep;
        // round trip 1: the entry P3 wrote (edge, head trip, competitors'
        // slot range, the trip's route bounds, lane word and next route
        // entry); 2: the competitors' requests and the edge record; 3: the
        // winner's counter updates together
        const uint4 *dip = reinterpret_cast<const uint4 *>(p.dep_info) + 2u * i;
        const uint4 di = __ldcg(dip), dr = __ldcg(dip + 1);
        const uint32_t e = di.x, j = di.y;
        bool won = j != MANTA_NONE;
        const EdgeMeta em = load_em(p, e);
        const uint32_t qp = __ldcg(p.q_pos + e);
        const uint32_t rc = dr.x, rend = dr.y, ld0 = dr.z, nx0 = dr.w;
        if (won) won = min_competitor(p, di.z, di.w, MANTA_NONE, target_key(e, 0u), tag) > j;
        // the result of this atomic is first used after the list append
        // below, so the two round trips overlap; the new vehicle's state
        // goes to its list position
        uint32_t pend = 2u;
        if (won) pend = atomicSub(p.pending + e, 1u);
        const uint32_t ia = warp_append(&ctl->n_act[cb ^ 1], won);
        const uint32_t s = ia;
        const bool keep = pend > 1u;
        const uint32_t id2 = warp_append(&ctl->n_dep[cb ^ 1], keep);
        if (won) {
          Veh w;
          w.x = 0.0f; w.v = 0.0f; w.id = j; w.rc = rc; w.rend = rend;
          w.e = e; w.ld = ld0; w.pcell = MANTA_NONE; w.em = em;
          w.em.lim = driver_limit(p, em.lim, j, rc);
          if (IDX_OK(s, p.cap_slots, 31)) {
            store_veh(R, s, w);
            R.nx[s] = nx0;
          }
          if (IDX_OK(ia, p.cap_list, 32)) act[ia] = s;
          if (IDX_OK(em.row0, p.cap_map, 33)) nxt[em.row0] = speed_code(0.0f);
          atomicAdd(p.entry + e, 1u);
          c_dep++;
          p.q_pos[e] = qp + 1u;
          if (ahead && IDX_OK(ia, p.cap_list, 34)) {   // step k + 1's record pass for this vehicle
            p.p3a[ia] = first_batch(em, 0, 0);
            if (lc_candidate(w, k + 1)) lc_add1(w, ia, s);
          }
        }
        if (keep && IDX_OK(id2, p.E, 35)) dep_n[id2] = e;
      } else if (t < t_due) {
        const uint32_t o_map = __ldcg(p.arr + (t - t_arr));
        if (IDX_OK(o_map, p.cap_map, 36)) cur[o_map] = (uint8_t)MANTA_EMPTY;
      } else {
        const uint32_t i = due_lo + (t - t_due);
        const uint32_t e = __ldg(p.due_edge + i);
        const bool first = atomicAdd(p.pending + e, 1u) == 0u;
        const uint32_t id2 = warp_append(&ctl->n_dep[cb ^ 1], first);
        if (first && IDX_OK(id2, p.E, 37)) dep_n[id2] = e;
      }
    }
    // step k + 1's record pass over the vehicles that stayed on their edge
    if (ahead) rec(k + 1, act, act, R, R, nact, false, cur, true, reg0n, rw0, w_all - rw0);
    if (gtid == 0) ctl->n_compact = 0u;
    if (!grid_sync(ctl, bar_target, p.wait_limit_ns, &s_ok)) { alive = false; break; }
    if (timer) { const uint64_t t = globaltimer(); ph[3] += t - tp; tp = t; }
    rec_ready = ahead;
    reg0_next = reg0n;
  }
  // flush counters
  atomicAdd(&s_cnt[CNT_UPD], (unsigned long long)c_upd);
  atomicAdd(&s_cnt[CNT_SCAN], (unsigned long long)c_scan);
  atomicAdd(&s_cnt[CNT_CLAMP], (unsigned long long)c_clamp);
  atomicAdd(&s_cnt[CNT_LC], (unsigned long long)c_lc);
  atomicAdd(&s_cnt[CNT_LCE], (unsigned long long)c_lce);
  atomicAdd(&s_cnt[CNT_RR], (unsigned long long)c_rr);
  atomicAdd(&s_cnt[CNT_DEP], (unsigned long long)c_dep);
  atomicAdd(&s_cnt[CNT_ARR], (unsigned long long)c_arr);
  atomicAdd(&s_cnt[CNT_LCS], (unsigned long long)s_lcs[threadIdx.x]);
  __syncthreads();
  if (threadIdx.x < CNT_N && s_cnt[threadIdx.x]) atomicAdd(&ctl->cnt[threadIdx.x], s_cnt[threadIdx.x]);
  if (timer) {
    for (int q = 0; q < 4; ++q) ctl->phase_ns[q] += ph[q];
    if (alive) ctl->k_next = kbase + p.n_steps;
  }
}
