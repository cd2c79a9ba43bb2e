// Device helpers shared by the kernels: shape weights, Boris rotation,
// index wrapping.  Everything is templated on the real type R (float for the
// cell-relative FP32 path, double for the FP64 path).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic_internal.h"

namespace pic {

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Largest value below one (offsets live in [0, 1)).
template <class R> __device__ __forceinline__ R below_one();
template <> __device__ __forceinline__ float below_one<float>() { return 0.99999994f; }
template <> __device__ __forceinline__ double below_one<double>() { return 0.99999999999999989; }

// Quadratic B-spline (TSC) weights on the nodes nearest-1, nearest,
// nearest+1 for a particle at distance d = X - nearest, |d| <= 1/2.
template <class R> __device__ __forceinline__ void tsc3(R d, R w[3]) {
  const R a = R(0.5) - d, b = R(0.5) + d;
  w[0] = R(0.5) * a * a;
  w[1] = R(0.75) - d * d;
  w[2] = R(0.5) * b * b;
}

// Gather stencil along one axis for a particle at cell-relative offset f.
// Integer ("primal") positions m sit at m; half-integer ("dual") positions m
// sit at m + 1/2.  `rel` is the first node relative to the particle's cell.
// With `lower` (the energy-conserving gather) the half-integer weights use
// the shape one order lower: CIC instead of TSC, the nearest grid point (the
// half-integer node of the particle's own cell) instead of CIC.
template <class R, int ORDER> struct GatherAxis {
  static constexpr int NS = ORDER + 1;
  int relp, reld;
  R wp[NS], wd[NS];
  __device__ __forceinline__ void cic_dual(R f) {
    if (f >= R(0.5)) {
      reld = 0;
      wd[0] = R(1.5) - f;
      wd[1] = f - R(0.5);
    } else {
      reld = -1;
      wd[0] = R(0.5) - f;
      wd[1] = R(0.5) + f;
    }
  }
  __device__ __forceinline__ void set(R f, bool lower = false) {
    if (ORDER == 2) {
      const int h = f >= R(0.5);
      relp = h - 1;
      tsc3<R>(f - R(h), wp);
      if (lower) {
        cic_dual(f);
        wd[2] = R(0);
      } else {
        reld = -1;
        tsc3<R>(f - R(0.5), wd);
      }
    } else {
      relp = 0;
      wp[0] = R(1) - f;
      wp[1] = f;
      if (lower) {
        reld = 0;
        wd[0] = R(1);
        wd[1] = R(0);
      } else {
        cic_dual(f);
      }
    }
  }
};

// Deposit stencil along one axis (Esirkepov, compact form): the shapes
// before (S0, offset f in the old cell) and after (S1, offset fn in the cell
// shifted by s) a move, on NW = ORDER + 2 consecutive nodes starting at `rel`
// (relative to the old cell); DS = S1 - S0.
//
// DS is taken in factored form, never as the difference of the two shape
// values, so that it keeps the precision of the offsets however small the
// move (the difference would lose it: a particle moving 1e-4 cells changes
// its weights by 1e-4, and S1 - S0 in FP32 then carries a 1e-3 relative
// error).  With the nearest node N0 of the old position (TSC) and the
// offsets d0, d1 of the two positions from it:
//  - support unchanged: DS = (D (s - 1)/2, -D s, D (s + 1)/2) on N0-1..N0+1,
//    D = d1 - d0, s = d0 + d1 (differences of squares of the quadratic
//    pieces);
//  - nearest node moves up to N0 + 1: with g0, g1 the distances of the two
//    positions below and above the half-integer N0 + 1/2 they straddle,
//    DS = (-g0^2/2, -g1 (2 - g1)/2 - g0 (1 - g0), g1 (1 - g1) + g0 (2 - g0)/2,
//    g1^2/2) on N0-1..N0+2 (each piece of the shape changed from its value
//    at the half-integer, where the pieces meet);
//  - down to N0 - 1: the mirror image on N0-2..N0+1.
// CIC: DS = (-D, D) within a cell; across the face c+1 (down: c) with g0,
// g1 the distances to it, (-g0, g0 - g1, g1) (mirror: (g1, g0 - g1, -g0)).
// Each form equals S1 - S0 exactly in real arithmetic.
template <class R, int ORDER> struct DepositAxis {
  static constexpr int NW = ORDER + 2;
  int rel;
  R S0[NW], DS[NW];
  __device__ __forceinline__ void set(R f, int s, R fn) {
    if (ORDER == 2) {
      const int h0 = f >= R(0.5), h1 = fn >= R(0.5);
      const int k = s + h1 - h0;  // nearest node moves by k (|k| <= 1 under the Courant limit)
      const R d0 = f - R(h0);     // old position from N0, in [-1/2, 1/2)
      const R e1 = fn - R(h1);    // new position from its own nearest node
      R w0[3];
      tsc3<R>(d0, w0);
      if (k == 0) {
        rel = h0 - 1;
        const R dl = e1 - d0, sg = d0 + e1, hd = R(0.5) * dl;
        S0[0] = w0[0];
        S0[1] = w0[1];
        S0[2] = w0[2];
        DS[0] = hd * (sg - R(1));
        DS[1] = -dl * sg;
        DS[2] = hd * (sg + R(1));
        S0[NW - 1] = DS[NW - 1] = R(0);
      } else if (k > 0) {
        rel = h0 - 1;
        const R g0 = R(0.5) - d0, g1 = e1 + R(0.5);
        S0[0] = w0[0];
        S0[1] = w0[1];
        S0[2] = w0[2];
        S0[NW - 1] = R(0);
        DS[0] = R(-0.5) * g0 * g0;
        DS[1] = R(-0.5) * g1 * (R(2) - g1) - g0 * (R(1) - g0);
        DS[2] = g1 * (R(1) - g1) + R(0.5) * g0 * (R(2) - g0);
        DS[3] = R(0.5) * g1 * g1;
      } else {
        rel = h0 - 2;
        const R g0 = R(0.5) + d0, g1 = R(0.5) - e1;
        S0[0] = R(0);
        S0[1] = w0[0];
        S0[2] = w0[1];
        S0[3] = w0[2];
        DS[0] = R(0.5) * g1 * g1;
        DS[1] = g1 * (R(1) - g1) + R(0.5) * g0 * (R(2) - g0);
        DS[2] = R(-0.5) * g1 * (R(2) - g1) - g0 * (R(1) - g0);
        DS[3] = R(-0.5) * g0 * g0;
      }
    } else {
      if (s == 0) {
        rel = 0;
        const R dl = fn - f;
        S0[0] = R(1) - f;
        S0[1] = f;
        S0[2] = R(0);
        DS[0] = -dl;
        DS[1] = dl;
        DS[2] = R(0);
      } else if (s > 0) {
        rel = 0;
        const R g0 = R(1) - f, g1 = fn;
        S0[0] = g0;
        S0[1] = f;
        S0[2] = R(0);
        DS[0] = -g0;
        DS[1] = g0 - g1;
        DS[2] = g1;
      } else {
        rel = -1;
        const R g0 = f, g1 = R(1) - fn;
        S0[0] = R(0);
        S0[1] = R(1) - f;
        S0[2] = f;
        DS[0] = g1;
        DS[1] = g0 - g1;
        DS[2] = -g0;
      }
    }
  }
  __device__ __forceinline__ void zero() {
    rel = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      S0[k] = R(0);
      DS[k] = R(0);
    }
  }
};

// Boris rotation in the variable u = gamma v (ref [8] of the paper; §2 eq. 3):
// half electric kick, magnetic rotation, half electric kick.  h = q dt/(2m).
template <class R>
__device__ __forceinline__ void boris(R h, const R E[3], const R B[3], R u[3]) {
  const R umx = u[0] + h * E[0], umy = u[1] + h * E[1], umz = u[2] + h * E[2];
  const R ig = R(1) / sqrt(R(1) + umx * umx + umy * umy + umz * umz);
  const R tx = h * B[0] * ig, ty = h * B[1] * ig, tz = h * B[2] * ig;
  const R sf = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
  const R sx = sf * tx, sy = sf * ty, sz = sf * tz;
  const R upx = umx + (umy * tz - umz * ty);
  const R upy = umy + (umz * tx - umx * tz);
  const R upz = umz + (umx * ty - umy * tx);
  u[0] = umx + (upy * sz - upz * sy) + h * E[0];
  u[1] = umy + (upz * sx - upx * sz) + h * E[1];
  u[2] = umz + (upx * sy - upy * sx) + h * E[2];
}

// Block-wide sum of a double (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// Max of non-negative doubles through their bit patterns (order-preserving).
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace pic
