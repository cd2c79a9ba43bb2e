// Fused per-tile particle kernel: field gather -> Boris push -> leap-frog
// move -> Esirkepov current deposit (§2 eqs. 1-4 of the paper, Boris per its
// ref [8], the charge-conserving deposit for the continuity requirement it
// states in §2).
//
// One thread block owns one cell tile.  Particles are kept sorted by tile
// (then by cell), so the block's particles are a contiguous slot range.  The
// block stages E and B of the tile plus guard cells in shared memory,
// accumulates J of the tile plus guard in shared memory with shared atomics,
// then adds its J window to the global J with one atomic per non-zero value.
// A particle that has drifted further than `drift` cells outside its tile
// since the last sort takes the same arithmetic on global memory instead
// (gather from the global arrays, global atomics), so results never depend on
// the window size.
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

namespace {

template <class R> struct PushArgs {
  int n[3];
  int tile[3];
  int ntile[3];
  int drift;
  const R *E[3];
  const R *B[3];
  R *J[3];
  int32_t *cell;
  R *off[3];
  R *u[3];
  const R *w;
  const int64_t *tile_start;
  R qmh;      // q dt / (2 m)
  R dtdx[3];  // dt / dx_a
  R jfac[3];  // -q dx_a / dt  (Esirkepov running-sum scale, times w)
  R qz;       // q            (2D3V: Jz = q w vz S)
  Counters *ctr;
};

// margins of the E/B window and of the J window below / above a particle's cell
template <int ORDER> struct Margins {
  static constexpr int LOE = 1;
  static constexpr int HIE = ORDER == 2 ? 2 : 1;
  static constexpr int LOJ = ORDER == 2 ? 2 : 1;
  static constexpr int HIJ = ORDER == 2 ? 3 : 2;
};

// Weighted sum of one field component over the gather stencil.  ix/iy/iz are
// per-axis address offsets (already multiplied by the strides).
template <class R, int NS, int DIM>
__device__ __forceinline__ R gsum(const R *__restrict__ F, const int *ix, const R *wx, const int *iy, const R *wy,
                                  const int *iz, const R *wz) {
  R acc = R(0);
  if (DIM == 3) {
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      R accb = R(0);
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        const R *row = F + iz[c] + iy[b];
        R ra = R(0);
#pragma unroll
        for (int a = 0; a < NS; ++a) ra += row[ix[a]] * wx[a];
        accb += ra * wy[b];
      }
      acc += accb * wz[c];
    }
  } else {
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      const R *row = F + iy[b];
      R ra = R(0);
#pragma unroll
      for (int a = 0; a < NS; ++a) ra += row[ix[a]] * wx[a];
      acc += ra * wy[b];
    }
  }
  return acc;
}

// Gather E and B.  Each component uses its own Yee location: primal (p) or
// dual (d) stencil per axis.
template <class R, int ORDER, int DIM>
__device__ __forceinline__ void gather6(const R *const F[6], const GatherAxis<R, ORDER> ga[3], const int ixp[],
                                        const int ixd[], const int iyp[], const int iyd[], const int izp[],
                                        const int izd[], R E[3], R B[3]) {
  constexpr int NS = ORDER + 1;
  const GatherAxis<R, ORDER> &gx = ga[0], &gy = ga[1], &gz = ga[2];
  E[0] = gsum<R, NS, DIM>(F[0], ixd, gx.wd, iyp, gy.wp, izp, gz.wp);
  E[1] = gsum<R, NS, DIM>(F[1], ixp, gx.wp, iyd, gy.wd, izp, gz.wp);
  E[2] = gsum<R, NS, DIM>(F[2], ixp, gx.wp, iyp, gy.wp, izd, gz.wd);
  B[0] = gsum<R, NS, DIM>(F[3], ixp, gx.wp, iyd, gy.wd, izd, gz.wd);
  B[1] = gsum<R, NS, DIM>(F[4], ixd, gx.wd, iyp, gy.wp, izd, gz.wd);
  B[2] = gsum<R, NS, DIM>(F[5], ixd, gx.wd, iyd, gy.wd, izp, gz.wp);
}

// Esirkepov deposit of one move into J (shared window or global arrays).
// jx/jy/jz: per-axis address offsets of the NW stencil nodes.
template <class R, int ORDER, int DIM>
__device__ __forceinline__ void deposit(R *const J[3], const DepositAxis<R, ORDER> da[3], const int jx[],
                                        const int jy[], const int jz[], R cx, R cy, R cz, R qwvz) {
  constexpr int NW = ORDER + 2;
  const DepositAxis<R, ORDER> &X = da[0], &Y = da[1], &Z = da[2];
  // running sums of DS along each axis (the last one is zero)
  R Px[NW - 1], Py[NW - 1], Pz[NW - 1];
  {
    R a = R(0), b = R(0), c = R(0);
#pragma unroll
    for (int k = 0; k < NW - 1; ++k) {
      a += X.DS[k];
      b += Y.DS[k];
      c += Z.DS[k];
      Px[k] = cx * a;
      Py[k] = cy * b;
      Pz[k] = cz * c;
    }
  }
  if (DIM == 3) {
    // Jx(i+1/2, j, k): Px[i] * (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3)
#pragma unroll
    for (int c = 0; c < NW; ++c)
#pragma unroll
      for (int b = 0; b < NW; ++b) {
        const R br = Y.S0[b] * (Z.S0[c] + R(0.5) * Z.DS[c]) + Y.DS[b] * (R(0.5) * Z.S0[c] + Z.DS[c] * R(1.0 / 3.0));
        R *row = J[0] + jz[c] + jy[b];
#pragma unroll
        for (int a = 0; a < NW - 1; ++a) atomicAdd(row + jx[a], Px[a] * br);
      }
#pragma unroll
    for (int c = 0; c < NW; ++c)
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const R br = Z.S0[c] * (X.S0[a] + R(0.5) * X.DS[a]) + Z.DS[c] * (R(0.5) * X.S0[a] + X.DS[a] * R(1.0 / 3.0));
        R *col = J[1] + jz[c] + jx[a];
#pragma unroll
        for (int b = 0; b < NW - 1; ++b) atomicAdd(col + jy[b], Py[b] * br);
      }
#pragma unroll
    for (int b = 0; b < NW; ++b)
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const R br = X.S0[a] * (Y.S0[b] + R(0.5) * Y.DS[b]) + X.DS[a] * (R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0));
        R *col = J[2] + jy[b] + jx[a];
#pragma unroll
        for (int c = 0; c < NW - 1; ++c) atomicAdd(col + jz[c], Pz[c] * br);
      }
  } else {
    // 2D3V: Jx = Px (S0y + DSy/2), Jy = Py (S0x + DSx/2),
    //       Jz = q w vz (S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3)
#pragma unroll
    for (int b = 0; b < NW; ++b) {
      const R by = Y.S0[b] + R(0.5) * Y.DS[b];
      R *row = J[0] + jy[b];
#pragma unroll
      for (int a = 0; a < NW - 1; ++a) atomicAdd(row + jx[a], Px[a] * by);
    }
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      const R bx = X.S0[a] + R(0.5) * X.DS[a];
      R *col = J[1] + jx[a];
#pragma unroll
      for (int b = 0; b < NW - 1; ++b) atomicAdd(col + jy[b], Py[b] * bx);
    }
#pragma unroll
    for (int b = 0; b < NW; ++b) {
      const R s0 = Y.S0[b] + R(0.5) * Y.DS[b];
      const R s1 = R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0);
      R *row = J[2] + jy[b];
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const R v = qwvz * (X.S0[a] * s0 + X.DS[a] * s1);
        atomicAdd(row + jx[a], v);
      }
    }
  }
}

template <class R, int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_push(const PushArgs<R> a) {
  using M = Margins<ORDER>;
  constexpr int NS = ORDER + 1;
  constexpr int NW = ORDER + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sm = reinterpret_cast<R *>(smem_raw);
  __shared__ unsigned int s_esc, s_clamp;

  const int64_t t = blockIdx.x;
  const int64_t pb = a.tile_start[t], pe = a.tile_start[t + 1];
  if (pb >= pe) return;

  const int D = a.drift;
  int t0[3], ew[3], jw[3];
  {
    int tt = (int)t;
    const int tx = tt % a.ntile[0];
    tt /= a.ntile[0];
    const int ty = tt % a.ntile[1];
    const int tz = tt / a.ntile[1];
    t0[0] = tx * a.tile[0];
    t0[1] = ty * a.tile[1];
    t0[2] = tz * a.tile[2];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool act = d < DIM;
    ew[d] = act ? a.tile[d] + 2 * D + M::LOE + M::HIE : 1;
    jw[d] = act ? a.tile[d] + 2 * D + M::LOJ + M::HIJ : 1;
  }
  const int ebN = ew[0] * ew[1] * ew[2];
  const int jN = jw[0] * jw[1] * jw[2];
  R *sF[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) sF[c] = sm + c * ebN;
  R *sJ[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) sJ[c] = sm + 6 * ebN + c * jN;

  // stage E, B of the tile + guard (periodic wrap of global indices)
  for (int q = threadIdx.x; q < ebN; q += blockDim.x) {
    const int x = q % ew[0];
    const int r = q / ew[0];
    const int y = r % ew[1];
    const int z = r / ew[1];
    const int gi = wrapi(t0[0] - D - M::LOE + x, a.n[0]);
    const int gj = DIM >= 2 ? wrapi(t0[1] - D - M::LOE + y, a.n[1]) : 0;
    const int gk = DIM == 3 ? wrapi(t0[2] - D - M::LOE + z, a.n[2]) : 0;
    const int64_t g = gi + (int64_t)a.n[0] * (gj + (int64_t)a.n[1] * gk);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sF[c][q] = a.E[c][g];
      sF[3 + c][q] = a.B[c][g];
    }
  }
  for (int q = threadIdx.x; q < 3 * jN; q += blockDim.x) sJ[0][q] = R(0);
  if (threadIdx.x == 0) {
    s_esc = 0;
    s_clamp = 0;
  }
  __syncthreads();

  const R *F6s[6] = {sF[0], sF[1], sF[2], sF[3], sF[4], sF[5]};
  const R *F6g[6] = {a.E[0], a.E[1], a.E[2], a.B[0], a.B[1], a.B[2]};
  unsigned int my_esc = 0, my_clamp = 0;

  for (int64_t pi = pb + threadIdx.x; pi < pe; pi += blockDim.x) {
    const int c = a.cell[pi];
    if (c < 0) continue;
    int ci[3];
    ci[0] = c % a.n[0];
    {
      const int r = c / a.n[0];
      ci[1] = r % a.n[1];
      ci[2] = DIM == 3 ? r / a.n[1] : 0;
    }
    int l[3] = {0, 0, 0};
    bool inw = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      int dl = ci[d] - t0[d];
      if (dl > a.tile[d] - 1 + D) dl -= a.n[d];
      if (dl < -D) dl += a.n[d];
      l[d] = dl;
      inw = inw && dl >= -D && dl <= a.tile[d] - 1 + D;
    }
    R f[3], u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      f[d] = d < DIM ? a.off[d][pi] : R(0);
      u[d] = a.u[d][pi];
    }
    const R wq = a.w[pi];

    // ---- gather (§2: g-weighted average of the grid fields) ----
    GatherAxis<R, ORDER> ga[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ga[d].set(f[d]);
    R E[3], B[3];
    int ixp[NS], ixd[NS], iyp[NS], iyd[NS], izp[NS], izd[NS];
    if (inw) {
      const int o = D + M::LOE;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        ixp[k] = l[0] + ga[0].relp + k + o;
        ixd[k] = l[0] + ga[0].reld + k + o;
        iyp[k] = (l[1] + ga[1].relp + k + o) * ew[0];
        iyd[k] = (l[1] + ga[1].reld + k + o) * ew[0];
        izp[k] = DIM == 3 ? (l[2] + ga[2].relp + k + o) * ew[0] * ew[1] : 0;
        izd[k] = DIM == 3 ? (l[2] + ga[2].reld + k + o) * ew[0] * ew[1] : 0;
      }
      gather6<R, ORDER, DIM>(F6s, ga, ixp, ixd, iyp, iyd, izp, izd, E, B);
    } else {
      const int sy = a.n[0];
      const int sz = a.n[0] * a.n[1];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        ixp[k] = wrapi(ci[0] + ga[0].relp + k, a.n[0]);
        ixd[k] = wrapi(ci[0] + ga[0].reld + k, a.n[0]);
        iyp[k] = wrapi(ci[1] + ga[1].relp + k, a.n[1]) * sy;
        iyd[k] = wrapi(ci[1] + ga[1].reld + k, a.n[1]) * sy;
        izp[k] = DIM == 3 ? wrapi(ci[2] + ga[2].relp + k, a.n[2]) * sz : 0;
        izd[k] = DIM == 3 ? wrapi(ci[2] + ga[2].reld + k, a.n[2]) * sz : 0;
      }
      gather6<R, ORDER, DIM>(F6g, ga, ixp, ixd, iyp, iyd, izp, izd, E, B);
    }

    // ---- Boris push (§2 eq. 3) ----
    boris<R>(a.qmh, E, B, u);

    // ---- leap-frog move with integer cell carry ----
    const R ig = R(1) / sqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    R fn[3] = {R(0), R(0), R(0)};
    int s[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      R x = f[d] + a.dtdx[d] * u[d] * ig;
      const int sh = (x >= R(1)) ? 1 : ((x < R(0)) ? -1 : 0);
      x -= R(sh);
      if (x >= R(1)) {
        x = below_one<R>();
        ++my_clamp;
      }
      if (x < R(0)) {
        x = R(0);
        ++my_clamp;
      }
      fn[d] = x;
      s[d] = sh;
    }

    // ---- Esirkepov deposit (§2 eq. 4 + continuity) ----
    DepositAxis<R, ORDER> da[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d < DIM) {
        da[d].set(f[d], s[d], fn[d]);
      } else {
        // 2D: no z extent; a unit weight on the single layer keeps the 3D
        // formulas unused.
        da[d].rel = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
          da[d].S0[k] = R(0);
          da[d].DS[k] = R(0);
        }
      }
    }
    const R cx = a.jfac[0] * wq, cy = a.jfac[1] * wq, cz = a.jfac[2] * wq;
    const R qwvz = a.qz * wq * u[2] * ig;
    int jx[NW], jy[NW], jz[NW];
    if (inw) {
      const int o = D + M::LOJ;
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        jx[k] = l[0] + da[0].rel + k + o;
        jy[k] = (l[1] + da[1].rel + k + o) * jw[0];
        jz[k] = DIM == 3 ? (l[2] + da[2].rel + k + o) * jw[0] * jw[1] : 0;
      }
      deposit<R, ORDER, DIM>(sJ, da, jx, jy, jz, cx, cy, cz, qwvz);
    } else {
      ++my_esc;
      const int sy = a.n[0];
      const int sz = a.n[0] * a.n[1];
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        jx[k] = wrapi(ci[0] + da[0].rel + k, a.n[0]);
        jy[k] = wrapi(ci[1] + da[1].rel + k, a.n[1]) * sy;
        jz[k] = DIM == 3 ? wrapi(ci[2] + da[2].rel + k, a.n[2]) * sz : 0;
      }
      deposit<R, ORDER, DIM>(a.J, da, jx, jy, jz, cx, cy, cz, qwvz);
    }

    // ---- store the new state ----
    int nc[3] = {ci[0], ci[1], ci[2]};
#pragma unroll
    for (int d = 0; d < DIM; ++d) nc[d] = wrapi(ci[d] + s[d], a.n[d]);
    a.cell[pi] = nc[0] + a.n[0] * (nc[1] + a.n[1] * nc[2]);
#pragma unroll
    for (int d = 0; d < DIM; ++d) a.off[d][pi] = fn[d];
#pragma unroll
    for (int d = 0; d < 3; ++d) a.u[d][pi] = u[d];
  }

  if (my_esc) atomicAdd(&s_esc, my_esc);
  if (my_clamp) atomicAdd(&s_clamp, my_clamp);
  __syncthreads();

  // ---- flush the J window into global J ----
  for (int q = threadIdx.x; q < jN; q += blockDim.x) {
    const int x = q % jw[0];
    const int r = q / jw[0];
    const int y = r % jw[1];
    const int z = r / jw[1];
    const int gi = wrapi(t0[0] - D - M::LOJ + x, a.n[0]);
    const int gj = wrapi(t0[1] - D - M::LOJ + y, a.n[1]);
    const int gk = DIM == 3 ? wrapi(t0[2] - D - M::LOJ + z, a.n[2]) : 0;
    const int64_t g = gi + (int64_t)a.n[0] * (gj + (int64_t)a.n[1] * gk);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R v = sJ[c][q];
      if (v != R(0)) atomicAdd(a.J[c] + g, v);
    }
  }
  if (threadIdx.x == 0) {
    if (s_esc) atomicAdd(&a.ctr->escaped, (unsigned long long)s_esc);
    if (s_clamp) atomicAdd(&a.ctr->clamped, (unsigned long long)s_clamp);
  }
}

template <int ORDER> size_t window_bytes(const Grid &g, size_t rsize) {
  using M = Margins<ORDER>;
  size_t ebN = 1, jN = 1;
  for (int d = 0; d < g.dims; ++d) {
    ebN *= (size_t)(g.tile[d] + 2 * g.drift + M::LOE + M::HIE);
    jN *= (size_t)(g.tile[d] + 2 * g.drift + M::LOJ + M::HIJ);
  }
  return (6 * ebN + 3 * jN) * rsize;
}

template <class R, int DIM, int ORDER>
cudaError_t launch_t(const Grid &g, void *const E[3], void *const B[3], void *const J[3], const Particles &p,
                     const int64_t *tile_start, double q, double m, Counters *ctr, cudaStream_t st) {
  PushArgs<R> a;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.tile[d] = g.tile[d];
    a.ntile[d] = g.ntile[d];
    a.E[d] = static_cast<const R *>(E[d]);
    a.B[d] = static_cast<const R *>(B[d]);
    a.J[d] = static_cast<R *>(J[d]);
    a.off[d] = static_cast<R *>(p.off[d]);
    a.u[d] = static_cast<R *>(p.u[d]);
    a.dtdx[d] = (R)(g.dt / g.dx[d]);
    a.jfac[d] = (R)(-q * g.dx[d] / g.dt);
  }
  a.drift = g.drift;
  a.cell = p.cell;
  a.w = static_cast<const R *>(p.w);
  a.tile_start = tile_start;
  a.qmh = (R)(q * g.dt / (2.0 * m));
  a.qz = (R)q;
  a.ctr = ctr;
  const size_t smem = window_bytes<ORDER>(g, sizeof(R));
  auto fn = k_push<R, DIM, ORDER>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (g.ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  fn<<<(unsigned)g.ntiles, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t push_smem_bytes(const Grid &g) {
  const size_t rs = g.prec == 1 ? sizeof(double) : sizeof(float);
  return g.order == 2 ? window_bytes<2>(g, rs) : window_bytes<1>(g, rs);
}

cudaError_t launch_push(const Grid &g, void *const E[3], void *const B[3], void *const J[3], const Particles &p,
                        const int64_t *tile_start, double q, double m, Counters *ctr, cudaStream_t st) {
  const int key = (g.prec == 1 ? 100 : 0) + g.dims * 10 + g.order;
  switch (key) {
    case 21: return launch_t<float, 2, 1>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 22: return launch_t<float, 2, 2>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 31: return launch_t<float, 3, 1>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 32: return launch_t<float, 3, 2>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 121: return launch_t<double, 2, 1>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 122: return launch_t<double, 2, 2>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 131: return launch_t<double, 3, 1>(g, E, B, J, p, tile_start, q, m, ctr, st);
    case 132: return launch_t<double, 3, 2>(g, E, B, J, p, tile_start, q, m, ctr, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pic
