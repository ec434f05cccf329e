// adjoint.cuh -- reverse-mode derivatives of simulated link speeds with
// respect to the per-class IDM parameters (calibration, Section III).
//
// Along a recorded run every discrete event is held fixed (leader cell and
// speed code, lane, signal and stop state, merge winner, ballistic branch,
// clamp): the event tape written by the step kernel.  What remains is, per
// vehicle, the continuous map of one step,
//   acc  = a (1 - (v/v0)^4)                              on a free road
//   acc  = a (1 - (v/v0)^4 - (s*(v)/s)^2),
//   s*(v) = s0 + v T + v (v - vL) / (2 sqrt(a b))       behind a leader (Eq. 1, delta = 4)
//   (x, v) -> (x + v dt + acc dt^2 / 2, v + acc dt)      when v + acc dt >= 0,
//   (x, v) -> (x - v^2 / (2 acc), 0)                     otherwise (ballistic step),
// followed by the recorded clamp and node outcome, with v0 = limit * v0f.
// Vehicles interact only through the byte lane map, whose content is held
// fixed, so every vehicle's recurrence is independent: one thread carries a
// vehicle's adjoint backward through a tape segment.  Arithmetic is binary64.
//
// Both sweeps are reproducible bit for bit: no floating-point sum depends on
// the order in which threads run.  Parameter derivatives are summed per
// thread, then over each block in a fixed tree, then over the blocks in
// block order; replayed speeds are summed exactly, as 128-bit fixed-point
// numbers with 64 fractional bits, whose integer additions commute.
#pragma once
#include <stdint.h>
#include "sim.cuh"

// IDM parameters per road class, binary64.
struct IdmTheta {
  double v0f[8], T[8], a[8], b[8], s0[8];
};

// Acceleration of one interacting or free step and its derivatives with
// respect to v and to (v0f, T, a, b, s0) of the vehicle's class.
struct AccD {
  double acc, dv, dth[5];
};
__device__ __forceinline__ AccD idm_acc(const IdmTheta &th, int c, double lim, double v, bool interact, double s,
                                       double vL) {
  const double a = th.a[c], b = th.b[c], T = th.T[c], s0 = th.s0[c];
  const double v0 = lim * th.v0f[c];
  const double r = v / v0, r3 = r * r * r, r4 = r3 * r;
  AccD d;
  // free-road term a (1 - r^4)
  d.acc = a * (1.0 - r4);
  d.dv = -4.0 * a * r3 / v0;
  const double dacc_dv0 = 4.0 * a * r4 / v0;
  d.dth[0] = dacc_dv0 * lim;          // v0f
  d.dth[1] = 0.0;                     // T
  d.dth[2] = 1.0 - r4;                // a
  d.dth[3] = 0.0;                     // b
  d.dth[4] = 0.0;                     // s0
  if (interact) {
    const double D = 2.0 * sqrt(a * b);
    const double ss = s0 + v * T + v * (v - vL) / D;
    const double q = ss / s;
    d.acc -= a * q * q;
    // d(-a q^2) = -a 2 q dq
    const double k2 = -2.0 * a * q / s;          // times d(ss)
    d.dv += k2 * (T + (2.0 * v - vL) / D);
    d.dth[1] += k2 * v;                          // T
    const double w = v * (v - vL) / D;           // dynamic term; d/da = -w / (2a), d/db = -w / (2b)
    d.dth[2] += -q * q + k2 * (-w / (2.0 * a));  // a (the prefactor, then through D)
    d.dth[3] += k2 * (-w / (2.0 * b));           // b
    d.dth[4] += k2;                              // s0
  }
  return d;
}

// Continuous state after one recorded step (frozen events), binary64.
// Returns false when the vehicle leaves the network (arrival).
__device__ __forceinline__ bool replay_step(const IdmTheta &th, double dt, const TapeRec &r, double &x, double &v) {
  const uint32_t f = r.flags;
  const int kind = (int)((f >> TF_KIND_SHIFT) & 3u);
  const int clamp = (int)((f >> TF_CLAMP_SHIFT) & 3u);
  const int out = (int)((f >> TF_OUT_SHIFT) & 7u);
  const int c = (int)((f >> TF_CLASS_SHIFT) & 7u);
  const double x0 = x;
  double xp, vp;
  if (kind == TK_STOP) {
    xp = x; vp = 0.0;
  } else if (clamp == 1) {
    xp = x; vp = 0.0;
  } else if (clamp == 2) {
    xp = (double)r.bnd; vp = 0.0;
  } else {
    const AccD d = idm_acc(th, c, (double)r.lim, v, kind == TK_INTERACT, (double)r.s, (double)r.vL);
    if (f & TF_BALLISTIC) { xp = x + v * dt + 0.5 * d.acc * dt * dt; vp = v + d.acc * dt; }
    else { xp = x - v * v / (2.0 * d.acc); vp = 0.0; }
  }
  switch (out) {
    case TO_ARRIVE: return false;
    case TO_CROSS: x = xp - (double)r.C; v = vp; break;
    case TO_HELD_KEEP: x = x0; v = 0.0; break;
    case TO_HELD_LINE: x = (double)r.C - 1.0; v = 0.0; break;
    default: x = xp; v = vp; break;
  }
  return true;
}

// Exact accumulation of a binary64 value of magnitude below 2^62 into a
// 128-bit two's-complement fixed-point sum (acc[0]: 64 fractional bits,
// acc[1]: integer part): v = floor(v) + a fraction in [0, 1), both exact.
// The carry out of the low word is known from the value it held before the
// addition, so the final sum does not depend on the order of the additions.
__device__ __forceinline__ void fx128_add(unsigned long long *acc, double v) {
  const double ip = floor(v);
  const unsigned long long lo = __double2ull_rz((v - ip) * 18446744073709551616.0);   // x 2^64, exact
  const unsigned long long hi = (unsigned long long)__double2ll_rz(ip);
  const unsigned long long old = atomicAdd(acc, lo);
  const unsigned long long carry = old + lo < old ? 1ull : 0ull;
  if (hi + carry) atomicAdd(acc + 1, hi + carry);
}

// Forward replay of a tape segment of n_steps steps with parameters th:
// per trip, the state (x, v) carried in from the previous segment (present
// flag 1) or taken from the tape where the vehicle enters; the speed of every
// recorded sample is added to the fixed-point sum acc[2 * sample].  Used for
// finite differences on the frozen-event run.
__global__ void replay_kernel(const TapeRec *tape, int32_t n_steps, uint32_t n_trips, double dt, IdmTheta th,
                              double *xs, double *vs, uint8_t *present, unsigned long long *acc) {
  for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n_trips; id += gridDim.x * blockDim.x) {
    double x = xs[id], v = vs[id];
    bool prev = present[id] != 0;
    for (int32_t t = 0; t < n_steps; ++t) {
      const TapeRec r = tape[(size_t)t * n_trips + id];
      if (!(r.flags & TF_PRESENT)) { prev = false; continue; }
      if (!prev) { x = (double)r.x; v = (double)r.v; }
      const uint32_t out = (r.flags >> TF_OUT_SHIFT) & 7u;
      prev = replay_step(th, dt, r, x, v);
      if (r.sample != MANTA_NONE && (out == TO_STAY || out == TO_CROSS)) fx128_add(acc + 2 * (size_t)r.sample, v);
    }
    xs[id] = x; vs[id] = v; present[id] = prev ? 1 : 0;
  }
}

// sums[i] += the fixed-point sum acc[2 i], rounded once to binary64
__global__ void replay_sums_kernel(const unsigned long long *acc, size_t n, double *sums) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long lo = acc[2 * i], hi = acc[2 * i + 1];
    if (lo | hi) sums[i] += (double)(long long)hi + (double)lo * 5.421010862427522170037e-20;   // 2^-64
  }
}

// Reverse sweep of a tape segment: lam_x, lam_v hold, per trip, the adjoint
// of the state after the segment (in) and receive the adjoint of the state
// entering it (out).  seed[sample] = dLoss / d(sample speed).  Parameter
// derivatives of block b go to part[40 b + 5 * class + j], j over (v0f, T,
// a, b, s0); adjoint_grad_kernel adds the blocks' parts to grad in block
// order.  Launch with kAdjBlock threads per block.
constexpr int kAdjBlock = 256;
__global__ void __launch_bounds__(kAdjBlock) adjoint_kernel(const TapeRec *tape, int32_t n_steps, uint32_t n_trips,
                                                            double dt, IdmTheta th, const double *seed,
                                                            double *lam_x, double *lam_v, double *part) {
  __shared__ double red[kAdjBlock];
  double g[40];                          // this thread's derivatives, summed in its own order
#pragma unroll
  for (int q = 0; q < 40; ++q) g[q] = 0.0;
  for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n_trips; id += gridDim.x * blockDim.x) {
    double lx = lam_x[id], lv = lam_v[id];
    for (int32_t t = n_steps - 1; t >= 0; --t) {
      const TapeRec r = tape[(size_t)t * n_trips + id];
      const uint32_t f = r.flags;
      if (!(f & TF_PRESENT)) { lx = 0.0; lv = 0.0; continue; }
      const int out = (int)((f >> TF_OUT_SHIFT) & 7u);
      if (out == TO_ARRIVE) { lx = 0.0; lv = 0.0; continue; }
      // the speed sample taken after the step
      if (r.sample != MANTA_NONE && (out == TO_STAY || out == TO_CROSS)) lv += seed[r.sample];
      // through the node outcome: adjoint of the P3 result (xp, vp) and of the old x
      double lxp = 0.0, lvp = 0.0, lx0 = 0.0, lv0 = 0.0;
      if (out == TO_STAY || out == TO_CROSS) { lxp = lx; lvp = lv; }
      else if (out == TO_HELD_KEEP) lx0 = lx;
      // through the P3 update
      const int kind = (int)((f >> TF_KIND_SHIFT) & 3u);
      const int clamp = (int)((f >> TF_CLAMP_SHIFT) & 3u);
      const int c = (int)((f >> TF_CLASS_SHIFT) & 7u);
      if (kind == TK_STOP || clamp == 1) {
        lx0 += lxp;                       // xp = x, vp = 0
      } else if (clamp == 0) {
        const double v = (double)r.v;
        const AccD d = idm_acc(th, c, (double)r.lim, v, kind == TK_INTERACT, (double)r.s, (double)r.vL);
        double ga;                        // adjoint of acc
        lx0 += lxp;
        if (f & TF_BALLISTIC) {
          // xp = x + v dt + acc dt^2 / 2, vp = v + acc dt
          ga = lxp * 0.5 * dt * dt + lvp * dt;
          lv0 += lxp * dt + lvp;
        } else {
          // xp = x - v^2 / (2 acc), vp = 0
          ga = lxp * v * v / (2.0 * d.acc * d.acc);
          lv0 += lxp * (-v / d.acc);
        }
        lv0 += ga * d.dv;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q == c) {
#pragma unroll
            for (int j = 0; j < 5; ++j) g[5 * q + j] += ga * d.dth[j];
          }
      }
      // clamp == 2: xp = bound, vp = 0: nothing flows back
      lx = lx0; lv = lv0;
    }
    lam_x[id] = lx; lam_v[id] = lv;
  }
  // the block's sum of each derivative: a fixed binary tree over the threads
  for (int q = 0; q < 40; ++q) {
    red[threadIdx.x] = g[q];
    __syncthreads();
    for (int h = kAdjBlock / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[40 * (size_t)blockIdx.x + q] = red[0];
    __syncthreads();
  }
}

// grad[q] += the blocks' parts, summed in block order (one thread per q < nq)
__global__ void adjoint_grad_kernel(const double *part, int n_blocks, double *grad, int nq) {
  const int q = threadIdx.x;
  if (q >= nq) return;
  double s = 0.0;
  for (int b = 0; b < n_blocks; ++b) s += part[40 * (size_t)b + q];
  grad[q] += s;
}
