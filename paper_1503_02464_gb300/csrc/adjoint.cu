// Reverse-mode (adjoint) kernels of the PIC step, for gradients of an
// objective with respect to the laser amplitude and the particle weights
// (hence the initial density profile).
//
// Forward step n (what is being differentiated, §2 of the paper):
//   gather F = G(x^n; E^n, B^n) -> Boris u^{n+1/2} -> move x^{n+1}
//   -> Esirkepov J(x^n, x^{n+1}, w) -> B half / E (+ Mur walls, laser) / B half.
// Reverse step n, given the adjoints of the state after the step:
//   R5  adj_yee_b   lamE -= dt/2 C_B (M_B lamB)       (transpose of B half 2)
//   R4  adj_mur     transpose of the Mur wall update; dF/da0 accumulates
//   R3  adj_yee_e   lamJ = -dt M_E lamE; lamB += dt C_E (M_E lamE); + wall terms
//   R1  adj_yee_b   lamE -= dt/2 C_B (M_B lamB)       (transpose of B half 1)
//   P   adj_push    per particle: deposit^T, move^T, Boris^T, gather^T
// with C_B = C_E^T the Yee curls (curl B at E points, curl E at B points)
// and M_B, M_E masks of the rows the forward updated.  Particle adjoints are
// indexed by particle id; weight gradients accumulate in FP64.
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

namespace {

int nblocks(int64_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)nsm * 32;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

struct GridIdx {
  int n0, n1, n2;
  __device__ __forceinline__ void ijk(int64_t c, int &i, int &j, int &k) const {
    i = (int)(c % n0);
    const int64_t r = c / n0;
    j = (int)(r % n1);
    k = (int)(r / n1);
  }
};

// ---------------------------------------------------------------- fields
// lamE -= h * curl_at_E(M_B lamB): the transpose of "B -= h curl_at_B(E)"
// over the rows the forward updated (By, Bz of the last x cell are not
// updated when the x walls absorb).
//
// With `pend` (the second B half, R1), the Mur transpose's terms for the
// old time level (R4, kept in `pend` by k_adj_mur) are added to lamEy,
// lamEz at the wall nodes in the same pass: both updates only add to lamE.
template <class R, int DIM>
__global__ void __launch_bounds__(256)
    k_adj_yee_b(GridIdx g, int absorb, R rdx, R rdy, R rdz, R h, R *lE0, R *lE1, R *lE2, const R *lB0, const R *lB1,
                const R *lB2, const double *pend) {
  const int64_t ncell = (int64_t)g.n0 * g.n1 * g.n2;
  const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    g.ijk(c, i, j, k);
    const int64_t cxm = c - (i > 0 ? 1 : 1 - g.n0);
    const int64_t cym = c - (j > 0 ? sy : sy - sy * g.n1);
    const bool mx0 = absorb && i == g.n0 - 1;        // row (i) of By, Bz masked
    const bool mxm = absorb && (i == 0);             // row (i-1) wraps to the last x cell
    const R bx = lB0[c], by = mx0 ? R(0) : lB1[c], bz = mx0 ? R(0) : lB2[c];
    const R bzym = mx0 ? R(0) : lB2[cym];
    const R byxm = mxm ? R(0) : lB1[cxm], bzxm = mxm ? R(0) : lB2[cxm];
    const R bxym = lB0[cym];
    R cx = (bz - bzym) * rdy;
    R cy = -(bz - bzxm) * rdx;
    const R cz = (by - byxm) * rdx - (bx - bxym) * rdy;
    if (DIM == 3) {
      const int64_t czm = c - (k > 0 ? sz : sz - sz * g.n2);
      const R byzm = mx0 ? R(0) : lB1[czm];
      cx -= (by - byzm) * rdz;
      cy += (bx - lB0[czm]) * rdz;
    }
    R py = R(0), pz = R(0);
    if (pend && (i < 2 || i >= g.n0 - 2)) {
      // pend slots: nodes 0, 1, n0-2, n0-1 (for Ey, then for Ez), per row
      const int64_t nyz = (int64_t)g.n1 * g.n2, jk = c / g.n0;
      const int nodes[4] = {0, 1, g.n0 - 2, g.n0 - 1};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (nodes[q] == i) {
          py += (R)pend[q * nyz + jk];
          pz += (R)pend[(4 + q) * nyz + jk];
        }
    }
    lE0[c] -= h * cx;
    lE1[c] += py - h * cy;
    lE2[c] += pz - h * cz;
  }
}

// lamJ = -h M_E lamE ; lamB += h * curl_at_B(M_E lamE): the transpose of
// "E += h (curl_at_E(B) - J)" over the updated rows (with absorbing walls:
// Ex of the last x cell, Ey and Ez of the first and last x cells are not).
template <class R, int DIM>
__global__ void __launch_bounds__(256)
    k_adj_yee_e(GridIdx g, int absorb, R rdx, R rdy, R rdz, R h, const R *lE0, const R *lE1, const R *lE2, R *lB0,
                R *lB1, R *lB2, R *lJ0, R *lJ1, R *lJ2) {
  const int64_t ncell = (int64_t)g.n0 * g.n1 * g.n2;
  const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
  auto mex = [&](int i) { return absorb && i == g.n0 - 1; };
  auto meyz = [&](int i) { return absorb && (i == 0 || i == g.n0 - 1); };
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    g.ijk(c, i, j, k);
    const int ip = i + 1 < g.n0 ? i + 1 : 0;
    const int64_t cxp = c + (i + 1 < g.n0 ? 1 : 1 - g.n0);
    const int64_t cyp = c + (j + 1 < g.n1 ? sy : sy - sy * g.n1);
    const R ex = mex(i) ? R(0) : lE0[c], ey = meyz(i) ? R(0) : lE1[c], ez = meyz(i) ? R(0) : lE2[c];
    lJ0[c] = -h * ex;
    lJ1[c] = -h * ey;
    lJ2[c] = -h * ez;
    const R ezyp = meyz(i) ? R(0) : lE2[cyp];
    const R ezxp = meyz(ip) ? R(0) : lE2[cxp];
    const R eyxp = meyz(ip) ? R(0) : lE1[cxp];
    const R exyp = mex(i) ? R(0) : lE0[cyp];
    R cx = (ezyp - ez) * rdy;
    R cy = -(ezxp - ez) * rdx;
    const R cz = (eyxp - ey) * rdx - (exyp - ex) * rdy;
    if (DIM == 3) {
      const int64_t czp = c + (k + 1 < g.n2 ? sz : sz - sz * g.n2);
      const R eyzp = meyz(i) ? R(0) : lE1[czp];
      const R exzp = mex(i) ? R(0) : lE0[czp];
      cx -= (eyzp - ey) * rdz;
      cy += (exzp - ex) * rdz;
    }
    lB0[c] += h * cx;
    lB1[c] += h * cy;
    lB2[c] += h * cz;
  }
}

// Transpose of the Mur wall update (tangential components y, z):
//   E0' = L0n + S1o + k (S1n - S0o),  S = E - L     (left wall, laser)
//   Ez' = E(n0-2)o + k (E(n0-2)n - E(n0-1)o)      (right wall)
// g = lamE(wall) is consumed (the wall value was overwritten), k g goes to
// the neighbour at the new time, and g, -k g are kept in `pend` for the old
// time (added to lamE by the R1 pass of k_adj_yee_b).  dF/da0 += g dE0'/da0
// (the laser terms over a0).
template <class R>
__global__ void k_adj_mur(int n0, int n1, int n2, double dx, double dt, R *lEy, R *lEz, double *pend, LaserStep ls,
                          double *da0) {
  __shared__ double sh[32];
  const int64_t nyz = (int64_t)n1 * n2;
  const double kc = (dt - dx) / (dt + dx);
  double acc = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 2 * nyz; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / nyz);
    const int64_t jk = q % nyz;
    R *E = c == 0 ? lEy : lEz;
    double *pd = pend + (int64_t)c * 4 * nyz;  // slots: node 0, 1, n0-2, n0-1
    const int64_t row = (int64_t)n0 * jk;
    const double g0 = (double)E[row];
    E[row] = R(0);
    E[row + 1] += (R)(kc * g0);
    pd[0 * nyz + jk] = -kc * g0;
    pd[1 * nyz + jk] = g0;
    if (ls.pol == c + 1) {
      // unit-amplitude laser terms at the wall row: P(row) times the waveform
      const double p = ls.prof[jk];
      const double l0o = p * ls.amp[0], l1o = p * ls.amp[1], l0n = p * ls.amp[2], l1n = p * ls.amp[3];
      acc += g0 * (l0n - l1o - kc * l1n + kc * l0o);
    }
    const double gr = (double)E[row + n0 - 1];
    E[row + n0 - 1] = R(0);
    E[row + n0 - 2] += (R)(kc * gr);
    pd[2 * nyz + jk] = gr;
    pd[3 * nyz + jk] = -kc * gr;
  }
  const double v = block_sum(acc, sh);
  if (threadIdx.x == 0 && v != 0.0) atomicAdd(da0, v);
}

// ---------------------------------------------------------------- particles
// TSC weights and their derivatives w.r.t. the particle coordinate.
template <class R> __device__ __forceinline__ void tsc3d(R d, R w[3], R dw[3]) {
  const R a = R(0.5) - d, b = R(0.5) + d;
  w[0] = R(0.5) * a * a;
  w[1] = R(0.75) - d * d;
  w[2] = R(0.5) * b * b;
  dw[0] = -a;
  dw[1] = R(-2) * d;
  dw[2] = b;
}

// Gather stencil (TSC) with derivatives: primal nodes rel_p.., dual rel_d..
template <class R> struct GAxisD {
  int relp, reld;
  R wp[3], wd[3], dwp[3], dwd[3];
  __device__ __forceinline__ void set(R f) {
    const int h = f >= R(0.5);
    relp = h - 1;
    tsc3d<R>(f - R(h), wp, dwp);
    reld = -1;
    tsc3d<R>(f - R(0.5), wd, dwd);
  }
};

// Deposit stencil (TSC, 4 nodes) with derivatives of S0 w.r.t. f and of S1
// w.r.t. the new offset fn.
template <class R> struct DAxisD {
  int rel;
  R S0[4], S1[4], dS0[4], dS1[4];
  __device__ __forceinline__ void set(R f, int s, R fn) {
    R w0[3], w1[3], d0[3], d1[3];
    const int h0 = f >= R(0.5), h1 = fn >= R(0.5);
    tsc3d<R>(f - R(h0), w0, d0);
    tsc3d<R>(fn - R(h1), w1, d1);
    const int n0 = h0 - 1, n1 = s + h1 - 1;
    rel = n0 < n1 ? n0 : n1;
    // each support starts at node 0 or 1 of the window: a select between two
    // compile-time shifts (a run-time array index would put the weights in
    // local memory)
    const bool o0 = n0 != rel, o1 = n1 != rel;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ka = k < 3 ? k : 2, kb = k > 0 ? k - 1 : 0;
      const bool ina = k < 3, inb = k > 0;
      S0[k] = o0 ? (inb ? w0[kb] : R(0)) : (ina ? w0[ka] : R(0));
      dS0[k] = o0 ? (inb ? d0[kb] : R(0)) : (ina ? d0[ka] : R(0));
      S1[k] = o1 ? (inb ? w1[kb] : R(0)) : (ina ? w1[ka] : R(0));
      dS1[k] = o1 ? (inb ? d1[kb] : R(0)) : (ina ? d1[ka] : R(0));
    }
  }
};

template <class R> struct AdjPushArgs {
  int n[3];
  int absorb;
  // tape: particle state at the start of the step and the fields E^n, B^n
  const int32_t *cell;
  const R *off[3];
  const R *u[3];
  const R *w;
  const uint32_t *id;
  const int64_t *d_count;  // slots in use (device)
  const R *E[3];
  const R *B[3];
  // adjoints
  const R *lJ[3];
  R *lE[3];
  R *lB[3];
  R *lx[3];   // by id: adjoint of the position (cells)
  R *lu[3];   // by id: adjoint of u
  double *lw;  // by id: dF/dw accumulated
  int64_t id_cap;
  unsigned long long *err;
  R qmh, dtdx[3], cxu[3], q;
};

// The move's 1/gamma exactly as the forward push computes it.
template <class R> __device__ __forceinline__ R inv_sqrt_fwd(R x);
template <> __device__ __forceinline__ float inv_sqrt_fwd<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double inv_sqrt_fwd<double>(double x) { return 1.0 / sqrt(x); }

// The forward Boris step (the push's arithmetic) with its intermediates:
// u- = u0 + h E, t = h B / gamma-, s = 2 t / (1 + t^2), u' = u- + u- x t,
// u+ = u- + u' x s, uo = u+ + h E.
template <class R>
__device__ __forceinline__ void boris_fwd(R h, const R u0[3], const R F[6], R um[3], R t[3], R sv[3], R up[3],
                                          R uo[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) um[d] = u0[d] + h * F[d];
  const R gm = sqrt(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) t[d] = h * F[3 + d] / gm;
  const R den = R(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) sv[d] = R(2) * t[d] / den;
  up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  uo[0] = um[0] + (up[1] * sv[2] - up[2] * sv[1]) + h * F[0];
  uo[1] = um[1] + (up[2] * sv[0] - up[0] * sv[2]) + h * F[1];
  uo[2] = um[2] + (up[0] * sv[1] - up[1] * sv[0]) + h * F[2];
}

// Where one particle's stencils find their nodes: the node r cells along x
// and r' along y from the particle's cell has index x(r) + y(r') in the
// arrays it reads, F (E then B) and J (lamJ), and index sx(r) + sy(r') in the
// arrays it scatters into, L (lamE then lamB, in global memory: float
// atomics in shared memory would be compare-and-swap loops, and the lanes
// of a warp often share nodes).  GridNodes: the whole periodic grid in
// global memory.  WindowNodes: E, B and lamJ of a cell tile's window staged
// in shared memory (kAdjWin nodes per axis).
template <class R> struct GridNodes {
  int i0, j0, n0, n1;
  const R *const *F;  // [6]
  const R *const *J;  // [3]
  R *const *L;        // [6]
  __device__ __forceinline__ int x(int r) const { return wrapi(i0 + r, n0); }
  __device__ __forceinline__ int y(int r) const { return wrapi(j0 + r, n1) * n0; }
  __device__ __forceinline__ int sx(int r) const { return x(r); }
  __device__ __forceinline__ int sy(int r) const { return y(r); }
  __device__ __forceinline__ const R *f(int c) const { return F[c]; }
  __device__ __forceinline__ const R *j(int c) const { return J[c]; }
  __device__ __forceinline__ R *l(int c) const { return L[c]; }
};

constexpr int kAdjTile = 16;                           // largest tile edge of the windowed kernel
constexpr int kAdjDrift = 4;                           // cells a particle may have left its tile
constexpr int kAdjGuard = kAdjDrift + 2;               // window nodes below the tile (deposit reaches 2 below)
constexpr int kAdjWin = kAdjTile + 2 * kAdjGuard + 1;  // window nodes per axis (and 3 above)
constexpr int kAdjWinN = kAdjWin * kAdjWin;
constexpr int kAdjSub = 512;                           // slots of a work item one block takes

template <class R> struct WindowNodes {
  int wi, wj;  // the particle's cell in window coordinates
  const R *s;  // [9][kAdjWinN]: E, B, lamJ
  int i0, j0, n0, n1;
  R *const *L;  // [6]
  __device__ __forceinline__ int x(int r) const { return wi + r; }
  __device__ __forceinline__ int y(int r) const { return (wj + r) * kAdjWin; }
  __device__ __forceinline__ int sx(int r) const { return wrapi(i0 + r, n0); }
  __device__ __forceinline__ int sy(int r) const { return wrapi(j0 + r, n1) * n0; }
  __device__ __forceinline__ const R *f(int c) const { return s + c * kAdjWinN; }
  __device__ __forceinline__ const R *j(int c) const { return s + (6 + c) * kAdjWinN; }
  __device__ __forceinline__ R *l(int c) const { return L[c]; }
};

// Per-particle adjoint of gather -> Boris -> move -> Esirkepov (2D3V, TSC)
// for the particle in slot p (live, id pid), its nodes found through nd.
template <class R, class Nodes>
__device__ __forceinline__ void adj_particle(const AdjPushArgs<R> &a, const Nodes &nd, int64_t p, uint32_t pid) {
  {
    const R f[2] = {a.off[0][p], a.off[1][p]};
    const R u0[3] = {a.u[0][p], a.u[1][p], a.u[2][p]};
    const R wq = a.w[p];
    // ---- forward recomputation: gather (values only; the weight derivatives
    // and the field gradients at the particle are recomputed for gather^T at
    // the end, which keeps them out of the registers of the deposit^T)
    // component c: (dual x?, dual y?) for Ex Ey Ez Bx By Bz
    const bool dx_[6] = {true, false, false, false, true, true};
    const bool dy_[6] = {false, true, false, true, false, true};
    R F[6];
    {
      GatherAxis<R, 2> gx, gy;
      gx.set(f[0]);
      gy.set(f[1]);
      int ixp[3], ixd[3], iyp[3], iyd[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ixp[k] = nd.x(gx.relp + k);
        ixd[k] = nd.x(gx.reld + k);
        iyp[k] = nd.y(gy.relp + k);
        iyd[k] = nd.y(gy.reld + k);
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        const R *G = nd.f(cc);
        const int *ix = dx_[cc] ? ixd : ixp;
        const int *iy = dy_[cc] ? iyd : iyp;
        const R *wx = dx_[cc] ? gx.wd : gx.wp;
        const R *wy = dy_[cc] ? gy.wd : gy.wp;
        R s = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          R r = 0;
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) r += G[ix[aa] + iy[b]] * wx[aa];
          s += r * wy[b];
        }
        F[cc] = s;
      }
    }
    // Boris.  Its intermediate values are recomputed from u0 and F for the
    // transpose further down, rather than kept live through deposit^T.
    const R h = a.qmh;
    R uo[3];
    {
      R um[3], t[3], sv[3], up[3];
      boris_fwd<R>(h, u0, F, um, t, sv, up, uo);
    }
    // move
    const R ig = inv_sqrt_fwd<R>(R(1) + uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2]);
    R fn[2];
    int sh[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      R x = f[d] + a.dtdx[d] * uo[d] * ig;
      const int s = (x >= R(1)) ? 1 : ((x < R(0)) ? -1 : 0);
      x -= R(s);
      if (x >= R(1)) x = below_one<R>();
      if (x < R(0)) x = R(0);
      fn[d] = x;
      sh[d] = s;
    }
    const R vz = uo[2] * ig;
    DAxisD<R> X, Y;
    X.set(f[0], sh[0], fn[0]);
    Y.set(f[1], sh[1], fn[1]);

    // ---- deposit^T: gather lamJ on the deposit stencil
    int jx[4], jy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      jx[k] = nd.x(X.rel + k);
      jy[k] = nd.y(Y.rel + k);
    }
    const R cx = a.cxu[0] * wq, cy = a.cxu[1] * wq, qw = a.q * wq;
    R dS0x[4], dS1x[4], dS0y[4], dS1y[4];  // dL/dS
    R dLw;  // dL/dw of this step (contributions are linear in w); summed over steps in FP64
    // pass 1, Jx and Jy: Gx[a] = sum_b lamJx[a][b] Hy[b], Ky[b] = sum_a
    // lamJx[a][b] Px[a] (Px the prefix sums of S1 - S0, H the means of S0
    // and S1), and the same with x and y exchanged for Jy
    {
      R Px[3], Py[3];
      {
        R sx = 0, sy = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sx += X.S1[k] - X.S0[k];
          sy += Y.S1[k] - Y.S0[k];
          Px[k] = sx;
          Py[k] = sy;
        }
      }
      R Hx[4], Hy[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Hx[k] = R(0.5) * (X.S0[k] + X.S1[k]);
        Hy[k] = R(0.5) * (Y.S0[k] + Y.S1[k]);
      }
      R Gx[3] = {0, 0, 0}, Ky[4] = {0, 0, 0, 0};
      R Gy[3] = {0, 0, 0}, Kx[4] = {0, 0, 0, 0};
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
          const int node = jx[aa] + jy[b];
          if (aa < 3) {
            const R Ax = nd.j(0)[node];
            Gx[aa] += Ax * Hy[b];
            Ky[b] += Ax * Px[aa];
          }
          if (b < 3) {
            const R Ay = nd.j(1)[node];
            Gy[b] += Ay * Hx[aa];
            Kx[aa] += Ay * Py[b];
          }
        }
      // suffix sums R[k] = sum_{a>=k, a<3} G[a]
      R Rx[4], Ry[4];
      Rx[3] = 0;
      Ry[3] = 0;
#pragma unroll
      for (int k = 2; k >= 0; --k) {
        Rx[k] = Rx[k + 1] + Gx[k];
        Ry[k] = Ry[k + 1] + Gy[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        dS1x[k] = cx * Rx[k] + R(0.5) * cy * Kx[k];
        dS0x[k] = -cx * Rx[k] + R(0.5) * cy * Kx[k];
        dS1y[k] = cy * Ry[k] + R(0.5) * cx * Ky[k];
        dS0y[k] = -cy * Ry[k] + R(0.5) * cx * Ky[k];
      }
      R gxp = 0, gyp = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gxp += Gx[k] * Px[k];
        gyp += Gy[k] * Py[k];
      }
      dLw = a.cxu[0] * gxp + a.cxu[1] * gyp;
    }
    // pass 2, Jz: Zx0[a] = sum_b lamJz[a][b] SY0[b] (and with S1), Zy the
    // same over a
    R Tz = 0;
    {
      R Zx0[4] = {0, 0, 0, 0}, Zx1[4] = {0, 0, 0, 0}, Zy0[4] = {0, 0, 0, 0}, Zy1[4] = {0, 0, 0, 0};
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
          const R Az = nd.j(2)[jx[aa] + jy[b]];
          Zx0[aa] += Az * Y.S0[b];
          Zx1[aa] += Az * Y.S1[b];
          Zy0[b] += Az * X.S0[aa];
          Zy1[b] += Az * X.S1[aa];
        }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Tz += (X.S0[k] * Zx0[k] + X.S1[k] * Zx1[k]) * R(1.0 / 3.0) + (X.S0[k] * Zx1[k] + X.S1[k] * Zx0[k]) * R(1.0 / 6.0);
        dS1x[k] += qw * vz * (Zx1[k] * R(1.0 / 3.0) + Zx0[k] * R(1.0 / 6.0));
        dS0x[k] += qw * vz * (Zx0[k] * R(1.0 / 3.0) + Zx1[k] * R(1.0 / 6.0));
        dS1y[k] += qw * vz * (Zy1[k] * R(1.0 / 3.0) + Zy0[k] * R(1.0 / 6.0));
        dS0y[k] += qw * vz * (Zy0[k] * R(1.0 / 3.0) + Zy1[k] * R(1.0 / 6.0));
      }
    }
    dLw += a.q * vz * Tz;
    const R lvz = qw * Tz;  // dL/dvz
    R lf_old[2] = {0, 0}, lf_new[2] = {0, 0};
    {
      // shape derivatives, set up only now (X, Y are used for their values)
      DAxisD<R> Xd, Yd;
      Xd.set(f[0], sh[0], fn[0]);
      Yd.set(f[1], sh[1], fn[1]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        lf_old[0] += dS0x[k] * Xd.dS0[k];
        lf_new[0] += dS1x[k] * Xd.dS1[k];
        lf_old[1] += dS0y[k] * Yd.dS0[k];
        lf_new[1] += dS1y[k] * Yd.dS1[k];
      }
    }

    // ---- move^T: x' = x + D(u+), vz = u+_z / gamma
    R lX[2], lD[3];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const R lfut = a.lx[d][pid];
      lD[d] = (lfut + lf_new[d]) * a.dtdx[d];
      lX[d] = lfut + lf_new[d] + lf_old[d];
    }
    lD[2] = lvz;
    R lu[3];
    {
      const R ud = (uo[0] * lD[0] + uo[1] * lD[1] + uo[2] * lD[2]) * ig * ig;
#pragma unroll
      for (int d = 0; d < 3; ++d) lu[d] = a.lu[d][pid] + (lD[d] - uo[d] * ud) * ig;
    }

    // ---- Boris^T (the forward intermediates recomputed)
    R um[3], t[3], sv[3], up[3];
    {
      R uo_[3];
      boris_fwd<R>(h, u0, F, um, t, sv, up, uo_);
    }
    const R gm = sqrt(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    const R den = R(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    R lF[6];
#pragma unroll
    for (int d = 0; d < 3; ++d) lF[d] = h * lu[d];  // u_out = u+' + h E
    // u+' = um + up x sv
    R lum[3] = {lu[0], lu[1], lu[2]};
    R lup[3], lsv[3];
    // lambda_up = sv x lu ; lambda_sv = lu x up
    lup[0] = sv[1] * lu[2] - sv[2] * lu[1];
    lup[1] = sv[2] * lu[0] - sv[0] * lu[2];
    lup[2] = sv[0] * lu[1] - sv[1] * lu[0];
    lsv[0] = lu[1] * up[2] - lu[2] * up[1];
    lsv[1] = lu[2] * up[0] - lu[0] * up[2];
    lsv[2] = lu[0] * up[1] - lu[1] * up[0];
    // sv = 2 t / (1 + t^2)
    R lt[3];
    {
      const R tl = t[0] * lsv[0] + t[1] * lsv[1] + t[2] * lsv[2];
#pragma unroll
      for (int d = 0; d < 3; ++d) lt[d] = R(2) / den * lsv[d] - R(4) * t[d] * tl / (den * den);
    }
    // up = um + um x t: lambda_um += lup + t x lup ; lambda_t += lup x um
#pragma unroll
    for (int d = 0; d < 3; ++d) lum[d] += lup[d];
    lum[0] += t[1] * lup[2] - t[2] * lup[1];
    lum[1] += t[2] * lup[0] - t[0] * lup[2];
    lum[2] += t[0] * lup[1] - t[1] * lup[0];
    lt[0] += lup[1] * um[2] - lup[2] * um[1];
    lt[1] += lup[2] * um[0] - lup[0] * um[2];
    lt[2] += lup[0] * um[1] - lup[1] * um[0];
    // t = h B / gm
    R lgm = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lF[3 + d] = h / gm * lt[d];
      lgm -= h * F[3 + d] / (gm * gm) * lt[d];
    }
    // gm = sqrt(1 + um^2)
#pragma unroll
    for (int d = 0; d < 3; ++d) lum[d] += lgm * um[d] / gm;
    // um = u + h E
    R lu0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lu0[d] = lum[d];
      lF[d] += h * lum[d];
    }

    // ---- gather^T: scatter lamF into lamE, lamB; position derivative
    // (weights, their derivatives and the field values recomputed here)
    {
      GAxisD<R> gx, gy;
      gx.set(f[0]);
      gy.set(f[1]);
      int ixp[3], ixd[3], iyp[3], iyd[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ixp[k] = nd.x(gx.relp + k);
        ixd[k] = nd.x(gx.reld + k);
        iyp[k] = nd.y(gy.relp + k);
        iyd[k] = nd.y(gy.reld + k);
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        if (lF[cc] == R(0)) continue;
        const R *G = nd.f(cc);
        R *LG = nd.l(cc);
        const int *ix = dx_[cc] ? ixd : ixp;
        const int *iy = dy_[cc] ? iyd : iyp;
        const int rx = dx_[cc] ? gx.reld : gx.relp, ry = dy_[cc] ? gy.reld : gy.relp;
        const R *wx = dx_[cc] ? gx.wd : gx.wp, *dwx = dx_[cc] ? gx.dwd : gx.dwp;
        const R *wy = dy_[cc] ? gy.wd : gy.wp, *dwy = dy_[cc] ? gy.dwd : gy.dwp;
        R sx = 0, sy = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            const R v = G[ix[aa] + iy[b]];
            sx += v * dwx[aa] * wy[b];
            sy += v * wx[aa] * dwy[b];
            atomicAdd(LG + nd.sx(rx + aa) + nd.sy(ry + b), lF[cc] * wx[aa] * wy[b]);
          }
        lX[0] += lF[cc] * sx;
        lX[1] += lF[cc] * sy;
      }
    }

    // ---- new adjoint state (time n), weight gradient
    a.lx[0][pid] = lX[0];
    a.lx[1][pid] = lX[1];
#pragma unroll
    for (int d = 0; d < 3; ++d) a.lu[d][pid] = lu0[d];
    a.lw[pid] += (double)dLw;
  }
}

// The particle adjoint over all slots, nodes in global memory (particles
// not in tile order).  The kernel is latency-bound (scattered field and
// adjoint reads), so the register cap (3 blocks of 256 per SM for FP32, 2
// for FP64) trades spills for occupancy.
template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_adj_push2d(const AdjPushArgs<R> a) {
  const int n0 = a.n[0], n1 = a.n[1];
  const int64_t n = *a.d_count;
  const R *F[6] = {a.E[0], a.E[1], a.E[2], a.B[0], a.B[1], a.B[2]};
  R *L[6] = {a.lE[0], a.lE[1], a.lE[2], a.lB[0], a.lB[1], a.lB[2]};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = a.cell[p];
    if (c < 0) continue;
    const uint32_t pid = a.id[p];
    if ((int64_t)pid >= a.id_cap) {
      atomicOr(a.err, 1ull);  // id outside the adjoint arrays: skipped, reported
      continue;
    }
    const GridNodes<R> nd{c % n0, c / n0, n0, n1, F, a.lJ, L};
    adj_particle<R>(a, nd, p, pid);
  }
}

// Work items of a recorded particle buffer (the sort in effect when it was
// recorded): item i covers slots [work_pb[i], min(work_pb[i] + chunk,
// tile_start[t + 1])) of tile t = work_tile[i] (-1: none); nsub blocks share
// an item, kAdjSub slots each.
struct AdjWork {
  const int32_t *work_tile;
  const int64_t *work_pb;
  const int64_t *tile_start;
  int64_t chunk;
  int nsub;
  int nt0, t0, t1;
  unsigned long long *esc_total;  // running count of particles on the global path
};

// The particle adjoint over kAdjSub slots of one work item, one block: E, B
// and lamJ of the item's tile window are staged in shared memory (lamE and
// lamB are scattered to global memory).  A particle more than kAdjDrift
// cells outside its tile since the sort is set aside and done at the end of
// the block with all its nodes in global memory.
template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2)
    k_adj_push2d_win(const AdjPushArgs<R> a, const AdjWork w) {
  extern __shared__ __align__(16) unsigned char adj_smem[];
  R *s = reinterpret_cast<R *>(adj_smem);
  __shared__ int s_esc[kAdjSub];
  __shared__ int s_nesc;
  const int item = blockIdx.x / w.nsub;
  const int t = w.work_tile[item];
  if (t < 0) return;
  const int64_t te = w.tile_start[t + 1];
  const int64_t ib = w.work_pb[item];
  const int64_t ie = ib + w.chunk < te ? ib + w.chunk : te;
  const int64_t pb = ib + (int64_t)(blockIdx.x % w.nsub) * kAdjSub;
  if (pb >= ie) return;
  const int64_t pe = pb + kAdjSub < ie ? pb + kAdjSub : ie;
  const int n0 = a.n[0], n1 = a.n[1];
  const int tx = (t % w.nt0) * w.t0, ty = (t / w.nt0) * w.t1;  // the tile's first cell
  const int ox = tx - kAdjGuard, oy = ty - kAdjGuard;          // the window's first node
  const R *src[9] = {a.E[0], a.E[1], a.E[2], a.B[0], a.B[1], a.B[2], a.lJ[0], a.lJ[1], a.lJ[2]};
  R *L[6] = {a.lE[0], a.lE[1], a.lE[2], a.lB[0], a.lB[1], a.lB[2]};
  if (threadIdx.x == 0) s_nesc = 0;
  for (int k = threadIdx.x; k < kAdjWinN; k += blockDim.x) {
    const int g = wrapi(ox + k % kAdjWin, n0) + wrapi(oy + k / kAdjWin, n1) * n0;
#pragma unroll
    for (int c = 0; c < 9; ++c) s[c * kAdjWinN + k] = src[c][g];
  }
  __syncthreads();
  for (int64_t p = pb + threadIdx.x; p < pe; p += blockDim.x) {
    const int c = a.cell[p];
    if (c < 0) continue;
    const uint32_t pid = a.id[p];
    if ((int64_t)pid >= a.id_cap) {
      atomicOr(a.err, 1ull);  // id outside the adjoint arrays: skipped, reported
      continue;
    }
    // the cell relative to the tile, across the periodic seam if need be
    int il = c % n0 - tx, jl = c / n0 - ty;
    if (il >= w.t0 + kAdjDrift) il -= n0;
    else if (il < -kAdjDrift) il += n0;
    if (jl >= w.t1 + kAdjDrift) jl -= n1;
    else if (jl < -kAdjDrift) jl += n1;
    if (il < -kAdjDrift || il >= w.t0 + kAdjDrift || jl < -kAdjDrift || jl >= w.t1 + kAdjDrift) {
      s_esc[atomicAdd(&s_nesc, 1)] = (int)(p - pb);
      continue;
    }
    const WindowNodes<R> nd{il + kAdjGuard, jl + kAdjGuard, s, c % n0, c / n0, n0, n1, L};
    adj_particle<R>(a, nd, p, pid);
  }
  __syncthreads();
  // the particles set aside, nodes in global memory
  const int nesc = s_nesc;
  if (threadIdx.x == 0 && nesc > 0) atomicAdd(w.esc_total, (unsigned long long)nesc);
  const R *F[6] = {a.E[0], a.E[1], a.E[2], a.B[0], a.B[1], a.B[2]};
  for (int k = threadIdx.x; k < nesc; k += blockDim.x) {
    const int64_t p = pb + s_esc[k];
    const int c = a.cell[p];
    const GridNodes<R> nd{c % n0, c / n0, n0, n1, F, a.lJ, L};
    adj_particle<R>(a, nd, p, a.id[p]);
  }
}

// out[b] += sum of w[i] over the i < n with bin[i] == b (0 <= b < nbins):
// the lanes of a warp that share a bin are summed in lane order by their
// lowest lane, which adds the sum to out[b].
__global__ void k_sum_by_bin(const double *__restrict__ w, const int32_t *__restrict__ bin, int64_t n, int nbins,
                             double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count: every lane takes part in the warp operations
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t i = base + lane;
    int b = -1;
    double v = 0.0;
    if (i < n) {
      b = bin[i];
      v = w[i];
    }
    if (b < 0 || b >= nbins) b = -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    double sum = 0.0;
#pragma unroll 4
    for (int l = 0; l < 32; ++l) {
      const double t = __shfl_sync(0xffffffffu, v, l);
      if ((peers >> l) & 1u) sum += t;
    }
    if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(out + b, sum);
  }
}

// Objective F = sum over live particles with x column in [c_lo, c_hi) of
// w dV m (gamma - 1); seeds lam_u = w dV m u / gamma and dF/dw directly.
template <class R>
__global__ void k_adj_seed(int n0, const int32_t *cell, const R *u0, const R *u1, const R *u2, const R *w,
                           const uint32_t *id, const int64_t *d_count, int c_lo, int c_hi, double dVm, R *lu0, R *lu1,
                           R *lu2, double *lw, double *F, int64_t id_cap, unsigned long long *err) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int64_t nslots = *d_count;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nslots; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell[p];
    if (c < 0) continue;
    const int col = c % n0;
    if (col < c_lo || col >= c_hi) continue;
    const double ux = u0[p], uy = u1[p], uz = u2[p];
    const double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    const double ww = w[p];
    const uint32_t k = id[p];
    if ((int64_t)k >= id_cap) {
      atomicOr(err, 1ull);
      continue;
    }
    acc += ww * dVm * (g - 1.0);
    lw[k] += dVm * (g - 1.0);
    lu0[k] += (R)(ww * dVm * ux / g);
    lu1[k] += (R)(ww * dVm * uy / g);
    lu2[k] += (R)(ww * dVm * uz / g);
  }
  const double v = block_sum(acc, sh);
  if (threadIdx.x == 0 && v != 0.0) atomicAdd(F, v);
}

template <class R> GridIdx gidx(const Grid &g) { return GridIdx{g.n[0], g.n[1], g.n[2]}; }

}  // namespace

cudaError_t launch_adj_yee_b(const Grid &g, void *const lE[3], void *const lB[3], double h, const double *pend,
                             cudaStream_t st) {
  const int nb = nblocks(g.ncell);
  const int absorb = g.absorb_lo || g.absorb_hi;
  if (g.prec == 1) {
    auto E = [&](int c) { return static_cast<double *>(lE[c]); };
    auto B = [&](int c) { return static_cast<const double *>(lB[c]); };
    if (g.dims == 3)
      k_adj_yee_b<double, 3><<<nb, 256, 0, st>>>(gidx<double>(g), absorb, 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                                 h, E(0), E(1), E(2), B(0), B(1), B(2), pend);
    else
      k_adj_yee_b<double, 2><<<nb, 256, 0, st>>>(gidx<double>(g), absorb, 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                                 h, E(0), E(1), E(2), B(0), B(1), B(2), pend);
  } else {
    auto E = [&](int c) { return static_cast<float *>(lE[c]); };
    auto B = [&](int c) { return static_cast<const float *>(lB[c]); };
    if (g.dims == 3)
      k_adj_yee_b<float, 3><<<nb, 256, 0, st>>>(gidx<float>(g), absorb, (float)(1.0 / g.dx[0]), (float)(1.0 / g.dx[1]),
                                                (float)(1.0 / g.dx[2]), (float)h, E(0), E(1), E(2), B(0), B(1), B(2), pend);
    else
      k_adj_yee_b<float, 2><<<nb, 256, 0, st>>>(gidx<float>(g), absorb, (float)(1.0 / g.dx[0]), (float)(1.0 / g.dx[1]),
                                                (float)(1.0 / g.dx[2]), (float)h, E(0), E(1), E(2), B(0), B(1), B(2), pend);
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_yee_e(const Grid &g, void *const lE[3], void *const lB[3], void *const lJ[3], double h,
                             cudaStream_t st) {
  const int nb = nblocks(g.ncell);
  const int absorb = g.absorb_lo || g.absorb_hi;
  if (g.prec == 1) {
    auto E = [&](int c) { return static_cast<const double *>(lE[c]); };
    auto B = [&](int c) { return static_cast<double *>(lB[c]); };
    auto J = [&](int c) { return static_cast<double *>(lJ[c]); };
    if (g.dims == 3)
      k_adj_yee_e<double, 3><<<nb, 256, 0, st>>>(gidx<double>(g), absorb, 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                                 h, E(0), E(1), E(2), B(0), B(1), B(2), J(0), J(1), J(2));
    else
      k_adj_yee_e<double, 2><<<nb, 256, 0, st>>>(gidx<double>(g), absorb, 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                                 h, E(0), E(1), E(2), B(0), B(1), B(2), J(0), J(1), J(2));
  } else {
    auto E = [&](int c) { return static_cast<const float *>(lE[c]); };
    auto B = [&](int c) { return static_cast<float *>(lB[c]); };
    auto J = [&](int c) { return static_cast<float *>(lJ[c]); };
    const float r0 = (float)(1.0 / g.dx[0]), r1 = (float)(1.0 / g.dx[1]), r2 = (float)(1.0 / g.dx[2]);
    if (g.dims == 3)
      k_adj_yee_e<float, 3><<<nb, 256, 0, st>>>(gidx<float>(g), absorb, r0, r1, r2, (float)h, E(0), E(1), E(2), B(0),
                                                B(1), B(2), J(0), J(1), J(2));
    else
      k_adj_yee_e<float, 2><<<nb, 256, 0, st>>>(gidx<float>(g), absorb, r0, r1, r2, (float)h, E(0), E(1), E(2), B(0),
                                                B(1), B(2), J(0), J(1), J(2));
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_mur(const Grid &g, void *const lE[3], double *pend, const LaserStep &ls_unit, double *da0,
                           cudaStream_t st) {
  const int nb = nblocks(2LL * g.n[1] * g.n[2]);
  if (g.prec == 1)
    k_adj_mur<double><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], g.dx[0], g.dt, static_cast<double *>(lE[1]),
                                          static_cast<double *>(lE[2]), pend, ls_unit, da0);
  else
    k_adj_mur<float><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], g.dx[0], g.dt, static_cast<float *>(lE[1]),
                                         static_cast<float *>(lE[2]), pend, ls_unit, da0);
  return cudaGetLastError();
}

template <class R>
static cudaError_t adj_push_t(const Grid &g, const Particles &tp, const int64_t *d_count, int64_t nmax,
                              void *const E[3], void *const B[3], void *const lJ[3], void *const lE[3],
                              void *const lB[3], void *const lx[3], void *const lu[3], double *lw, int64_t id_cap,
                              unsigned long long *err, double q, double m, const AdjTiles *tt, cudaStream_t st,
                              int *nlaunch) {
  AdjPushArgs<R> a;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.off[d] = static_cast<const R *>(tp.off[d]);
    a.u[d] = static_cast<const R *>(tp.u[d]);
    a.E[d] = static_cast<const R *>(E[d]);
    a.B[d] = static_cast<const R *>(B[d]);
    a.lJ[d] = static_cast<const R *>(lJ[d]);
    a.lE[d] = static_cast<R *>(lE[d]);
    a.lB[d] = static_cast<R *>(lB[d]);
    a.lx[d] = static_cast<R *>(lx[d]);
    a.lu[d] = static_cast<R *>(lu[d]);
    a.dtdx[d] = (R)(g.dt / g.dx[d]);
    a.cxu[d] = (R)(-q * g.dx[d] / g.dt);
  }
  a.absorb = g.absorb_lo || g.absorb_hi;
  a.cell = tp.cell;
  a.w = static_cast<const R *>(tp.w);
  a.id = tp.id;
  a.d_count = d_count;
  a.lw = lw;
  a.id_cap = id_cap;
  a.err = err;
  a.qmh = (R)(q * g.dt / (2.0 * m));
  a.q = (R)q;
  const bool win = tt && tt->work_tile && tt->nwork > 0 && g.tile[0] <= kAdjTile && g.tile[1] <= kAdjTile;
  if (!win) {
    k_adj_push2d<R><<<nblocks(nmax), 256, 0, st>>>(a);
    if (nlaunch) *nlaunch = 1;
    return cudaGetLastError();
  }
  const size_t smem = (size_t)9 * kAdjWinN * sizeof(R);
  if (smem > 48 * 1024) {  // (set on every launch: the attribute belongs to the current device)
    cudaError_t e = cudaFuncSetAttribute(k_adj_push2d_win<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  AdjWork w;
  w.work_tile = tt->work_tile;
  w.work_pb = tt->work_pb;
  w.tile_start = tt->tile_start;
  w.chunk = tt->chunk;
  w.nsub = (int)((tt->chunk + kAdjSub - 1) / kAdjSub);
  w.nt0 = g.ntile[0];
  w.t0 = g.tile[0];
  w.t1 = g.tile[1];
  w.esc_total = tt->esc_total;
  const int64_t nblk = tt->nwork * w.nsub;
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_adj_push2d_win<R><<<(unsigned)nblk, 256, smem, st>>>(a, w);
  if (nlaunch) *nlaunch = 1;
  return cudaGetLastError();
}

cudaError_t launch_adj_push(const Grid &g, const Particles &tp, const int64_t *d_count, int64_t nmax,
                            void *const E[3], void *const B[3], void *const lJ[3], void *const lE[3],
                            void *const lB[3], void *const lx[3], void *const lu[3], double *lw, int64_t id_cap,
                            unsigned long long *err, double q, double m, const AdjTiles *tt, cudaStream_t st,
                            int *nlaunch) {
  if (nlaunch) *nlaunch = 0;
  if (g.dims != 2 || g.order != 2) return cudaErrorInvalidValue;
  if (nmax <= 0) return cudaSuccess;
  if (g.prec == 1)
    return adj_push_t<double>(g, tp, d_count, nmax, E, B, lJ, lE, lB, lx, lu, lw, id_cap, err, q, m, tt, st, nlaunch);
  return adj_push_t<float>(g, tp, d_count, nmax, E, B, lJ, lE, lB, lx, lu, lw, id_cap, err, q, m, tt, st, nlaunch);
}

cudaError_t launch_sum_by_bin(const double *w, const int32_t *bin, int64_t n, int nbins, double *out,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_sum_by_bin<<<nblocks(n), 256, 0, st>>>(w, bin, n, nbins, out);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, int c_lo,
                            int c_hi, double dVm, void *const lu[3], double *lw, double *F, int64_t id_cap,
                            unsigned long long *err, cudaStream_t st) {
  if (nmax <= 0) return cudaSuccess;
  const int nb = nblocks(nmax);
  if (g.prec == 1) {
    auto U = [&](int d) { return static_cast<const double *>(p.u[d]); };
    auto L = [&](int d) { return static_cast<double *>(lu[d]); };
    k_adj_seed<double><<<nb, 256, 0, st>>>(g.n[0], p.cell, U(0), U(1), U(2), static_cast<const double *>(p.w), p.id,
                                           d_count, c_lo, c_hi, dVm, L(0), L(1), L(2), lw, F, id_cap, err);
  } else {
    auto U = [&](int d) { return static_cast<const float *>(p.u[d]); };
    auto L = [&](int d) { return static_cast<float *>(lu[d]); };
    k_adj_seed<float><<<nb, 256, 0, st>>>(g.n[0], p.cell, U(0), U(1), U(2), static_cast<const float *>(p.w), p.id,
                                          d_count, c_lo, c_hi, dVm, L(0), L(1), L(2), lw, F, id_cap, err);
  }
  return cudaGetLastError();
}

}  // namespace pic
