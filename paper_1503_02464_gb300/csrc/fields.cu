// Grid kernels: Yee FDTD curl updates (§2 Maxwell curl equations, FDTD on
// the Yee lattice per ref [9] of the paper), particle load/unload between
// global FP64 coordinates and (cell, offset), and the FP64 diagnostics.
#include <cuda_runtime.h>
#include <math.h>

#include "pic_device.cuh"

namespace pic {

namespace {

int grid_blocks(int64_t n, int per_block) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + per_block - 1) / per_block;
  const int64_t cap = (int64_t)nsm * 32;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <class R> struct YeeArgs {
  int n[3];
  int absorb;  // x walls absorbing: wall nodes are left to the Mur kernels
  R rdx[3];  // 1/dx_a
  R h;       // time step of this update
  R *E[3];
  R *B[3];
  const R *J[3];
};

// B <- B - h curl E, curl E at the B locations.
template <class R, int DIM>
__global__ void __launch_bounds__(256) k_yee_b(YeeArgs<R> a) {
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const int64_t ncell = (int64_t)n0 * n1 * n2;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % n0);
    const int64_t r = c / n0;
    const int j = (int)(r % n1);
    const int k = (int)(r / n1);
    const int64_t cxp = c + (i + 1 < n0 ? 1 : 1 - n0);
    const int64_t cyp = c + (j + 1 < n1 ? sy : sy - sy * n1);
    const R ex = a.E[0][c], ey = a.E[1][c], ez = a.E[2][c];
    R cx = (a.E[2][cyp] - ez) * a.rdx[1];
    R cy = -(a.E[2][cxp] - ez) * a.rdx[0];
    const R cz = (a.E[1][cxp] - ey) * a.rdx[0] - (a.E[0][cyp] - ex) * a.rdx[1];
    if (DIM == 3) {
      const int64_t czp = c + (k + 1 < n2 ? sz : sz - sz * n2);
      cx -= (a.E[1][czp] - ey) * a.rdx[2];
      cy += (a.E[0][czp] - ex) * a.rdx[2];
    }
    a.B[0][c] -= a.h * cx;
    if (a.absorb && i == n0 - 1) continue;  // By, Bz half a cell beyond the last node
    a.B[1][c] -= a.h * cy;
    a.B[2][c] -= a.h * cz;
  }
}

// E <- E + h (curl B - J), curl B at the E locations.
template <class R, int DIM>
__global__ void __launch_bounds__(256) k_yee_e(YeeArgs<R> a) {
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const int64_t ncell = (int64_t)n0 * n1 * n2;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % n0);
    const int64_t r = c / n0;
    const int j = (int)(r % n1);
    const int k = (int)(r / n1);
    const int64_t cxm = c - (i > 0 ? 1 : 1 - n0);
    const int64_t cym = c - (j > 0 ? sy : sy - sy * n1);
    const R bx = a.B[0][c], by = a.B[1][c], bz = a.B[2][c];
    R cx = (bz - a.B[2][cym]) * a.rdx[1];
    R cy = -(bz - a.B[2][cxm]) * a.rdx[0];
    const R cz = (by - a.B[1][cxm]) * a.rdx[0] - (bx - a.B[0][cym]) * a.rdx[1];
    if (DIM == 3) {
      const int64_t czm = c - (k > 0 ? sz : sz - sz * n2);
      cx -= (by - a.B[1][czm]) * a.rdx[2];
      cy += (bx - a.B[0][czm]) * a.rdx[2];
    }
    if (a.absorb && i == n0 - 1) continue;  // wall node (Mur) and Ex beyond the last node
    a.E[0][c] += a.h * (cx - a.J[0][c]);
    if (a.absorb && i == 0) continue;       // wall node (Mur)
    a.E[1][c] += a.h * (cy - a.J[1][c]);
    a.E[2][c] += a.h * (cz - a.J[2][c]);
  }
}

// The same two updates with 16-byte vector accesses along x: a thread takes
// W = 16 / sizeof(R) consecutive cells of one row (four FP32 or two FP64
// values per component), on a 3D grid of (x groups, rows, planes), so there
// is no division per cell and every load and store of a warp is 512
// contiguous bytes.  The neighbour across the group's end in x is one extra
// scalar load (cached; the adjacent thread reads it too), with the periodic
// wrap at the ends of the row.  Used when the row length is a multiple of W
// (so every component array is 16-byte aligned); the scalar kernels above
// take the other grids.
template <class R> struct alignas(16) Pack {
  R v[16 / sizeof(R)];
};
template <class R> __device__ __forceinline__ Pack<R> ldp(const R *p) { return *reinterpret_cast<const Pack<R> *>(p); }
template <class R> __device__ __forceinline__ void stp(R *p, const Pack<R> &v) { *reinterpret_cast<Pack<R> *>(p) = v; }

template <class R, int DIM>
__global__ void __launch_bounds__(256) k_yee_b_vec(YeeArgs<R> a) {
  constexpr int W = 16 / sizeof(R);
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const int nq = n0 / W;
  const int iq = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (iq >= nq || j >= n1) return;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  const int64_t row = (int64_t)j * sy + (int64_t)k * sz;
  const int64_t c = row + (int64_t)iq * W;
  const int64_t cyp = j + 1 < n1 ? c + sy : c + sy - sy * n1;
  const int64_t cxn = iq + 1 < nq ? c + W : row;  // x + 1 of the group's last cell
  const Pack<R> ex = ldp(a.E[0] + c), ey = ldp(a.E[1] + c), ez = ldp(a.E[2] + c);
  const Pack<R> ex_yp = ldp(a.E[0] + cyp), ez_yp = ldp(a.E[2] + cyp);
  const R ey_xn = a.E[1][cxn], ez_xn = a.E[2][cxn];
  Pack<R> ex_zp, ey_zp;
  if (DIM == 3) {
    const int64_t czp = k + 1 < n2 ? c + sz : c + sz - sz * n2;
    ex_zp = ldp(a.E[0] + czp);
    ey_zp = ldp(a.E[1] + czp);
  }
  Pack<R> bx = ldp(a.B[0] + c), by = ldp(a.B[1] + c), bz = ldp(a.B[2] + c);
  // By, Bz half a cell beyond the last node stay as they are at absorbing walls
  const bool last = a.absorb && iq == nq - 1;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const R eyx = w + 1 < W ? ey.v[w + 1] : ey_xn, ezx = w + 1 < W ? ez.v[w + 1] : ez_xn;
    R cx = (ez_yp.v[w] - ez.v[w]) * a.rdx[1];
    R cy = -(ezx - ez.v[w]) * a.rdx[0];
    const R cz = (eyx - ey.v[w]) * a.rdx[0] - (ex_yp.v[w] - ex.v[w]) * a.rdx[1];
    if (DIM == 3) {
      cx -= (ey_zp.v[w] - ey.v[w]) * a.rdx[2];
      cy += (ex_zp.v[w] - ex.v[w]) * a.rdx[2];
    }
    bx.v[w] -= a.h * cx;
    if (!(last && w == W - 1)) {
      by.v[w] -= a.h * cy;
      bz.v[w] -= a.h * cz;
    }
  }
  stp(a.B[0] + c, bx);
  stp(a.B[1] + c, by);
  stp(a.B[2] + c, bz);
}

template <class R, int DIM>
__global__ void __launch_bounds__(256) k_yee_e_vec(YeeArgs<R> a) {
  constexpr int W = 16 / sizeof(R);
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const int nq = n0 / W;
  const int iq = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (iq >= nq || j >= n1) return;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  const int64_t row = (int64_t)j * sy + (int64_t)k * sz;
  const int64_t c = row + (int64_t)iq * W;
  const int64_t cym = j > 0 ? c - sy : c - sy + sy * n1;
  const int64_t cxp = iq > 0 ? c - 1 : row + n0 - 1;  // x - 1 of the group's first cell
  const Pack<R> bx = ldp(a.B[0] + c), by = ldp(a.B[1] + c), bz = ldp(a.B[2] + c);
  const Pack<R> bx_ym = ldp(a.B[0] + cym), bz_ym = ldp(a.B[2] + cym);
  const R by_xp = a.B[1][cxp], bz_xp = a.B[2][cxp];
  Pack<R> bx_zm, by_zm;
  if (DIM == 3) {
    const int64_t czm = k > 0 ? c - sz : c - sz + sz * n2;
    bx_zm = ldp(a.B[0] + czm);
    by_zm = ldp(a.B[1] + czm);
  }
  const Pack<R> jx = ldp(a.J[0] + c), jy = ldp(a.J[1] + c), jz = ldp(a.J[2] + c);
  Pack<R> ex = ldp(a.E[0] + c), ey = ldp(a.E[1] + c), ez = ldp(a.E[2] + c);
  // at absorbing walls the wall nodes belong to the Mur kernels, and Ex
  // half a cell beyond the last node is not updated
  const bool first = a.absorb && iq == 0, last = a.absorb && iq == nq - 1;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const R byx = w > 0 ? by.v[w - 1] : by_xp, bzx = w > 0 ? bz.v[w - 1] : bz_xp;
    R cx = (bz.v[w] - bz_ym.v[w]) * a.rdx[1];
    R cy = -(bz.v[w] - bzx) * a.rdx[0];
    const R cz = (by.v[w] - byx) * a.rdx[0] - (bx.v[w] - bx_ym.v[w]) * a.rdx[1];
    if (DIM == 3) {
      cx -= (by.v[w] - by_zm.v[w]) * a.rdx[2];
      cy += (bx.v[w] - bx_zm.v[w]) * a.rdx[2];
    }
    const bool wall_hi = last && w == W - 1, wall_lo = first && w == 0;
    if (!wall_hi) ex.v[w] += a.h * (cx - jx.v[w]);
    if (!wall_hi && !wall_lo) {
      ey.v[w] += a.h * (cy - jy.v[w]);
      ez.v[w] += a.h * (cz - jz.v[w]);
    }
  }
  stp(a.E[0] + c, ex);
  stp(a.E[1] + c, ey);
  stp(a.E[2] + c, ez);
}

// Vector path when the row length is a multiple of W and every array is
// 16-byte aligned; block (x groups, rows) with 256 threads.
template <class R> bool yee_vec_ok(const Grid &g, const YeeArgs<R> &a, bool with_j) {
  constexpr int W = 16 / sizeof(R);
  if (g.n[0] % W != 0 || g.n[2] > 65535) return false;
  for (int d = 0; d < 3; ++d) {
    if (reinterpret_cast<uintptr_t>(a.E[d]) % 16 || reinterpret_cast<uintptr_t>(a.B[d]) % 16) return false;
    if (with_j && reinterpret_cast<uintptr_t>(a.J[d]) % 16) return false;
  }
  return true;
}
template <class R> void yee_vec_shape(const Grid &g, dim3 &grid, dim3 &block) {
  constexpr int W = 16 / sizeof(R);
  const int nq = g.n[0] / W;
  const int bx = nq >= 64 ? 64 : 32;
  block = dim3(bx, 256 / bx, 1);
  grid = dim3((nq + bx - 1) / bx, (g.n[1] + block.y - 1) / block.y, g.n[2]);
}

template <class R>
__global__ void k_mur_save(int n0, int n1, int n2, const R *Ey, const R *Ez, double *buf) {
  const int64_t nyz = (int64_t)n1 * n2;
  const int nodes[4] = {0, 1, n0 - 2, n0 - 1};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 8 * nyz; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t jk = q % nyz;
    const int cq = (int)(q / nyz);  // component * 4 + node slot
    const R *E = cq < 4 ? Ey : Ez;
    buf[q] = (double)E[nodes[cq & 3] + (int64_t)n0 * jk];
  }
}

// E(0)^{n+1} = L(0)^{n+1} + S(1)^n + k (S(1)^{n+1} - S(0)^n), S = E - L the
// scattered field, k = (dt - dx)/(dt + dx); the same without L at x = n0-1.
// L = P(row) times the step's four waveform values (LaserStep).
template <class R>
__global__ void k_mur_apply(int n0, int n1, int n2, double dx, double dt, R *Ey, R *Ez, const double *buf,
                            LaserStep ls) {
  const int64_t nyz = (int64_t)n1 * n2;
  const double kc = (dt - dx) / (dt + dx);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 2 * nyz; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / nyz);  // 0: Ey, 1: Ez
    const int64_t jk = q % nyz;
    R *E = c == 0 ? Ey : Ez;
    const double *o = buf + (int64_t)c * 4 * nyz;
    double l0o = 0.0, l1o = 0.0, l0n = 0.0, l1n = 0.0;
    if (ls.pol == c + 1) {
      if (ls.oblique) {
        // the wall row's own delay and profile (Ey rows at (j + 1/2, k), Ez rows at (j, k + 1/2))
        const int j = (int)(jk % n1), k = (int)(jk / n1);
        const double y = (j + (c == 0 ? 0.5 : 0.0)) * ls.dy, z = (k + (c == 1 ? 0.5 : 0.0)) * ls.dz;
        l0o = laser_wave(ls, 0.0, y, z, ls.t_old);
        l1o = laser_wave(ls, ls.dx, y, z, ls.t_old);
        l0n = laser_wave(ls, 0.0, y, z, ls.t_new);
        l1n = laser_wave(ls, ls.dx, y, z, ls.t_new);
      } else {
        const double p = ls.prof[jk];
        l0o = p * ls.amp[0];
        l1o = p * ls.amp[1];
        l0n = p * ls.amp[2];
        l1n = p * ls.amp[3];
      }
    }
    const int64_t row = (int64_t)n0 * jk;
    const double s0o = o[0 * nyz + jk] - l0o;
    const double s1o = o[1 * nyz + jk] - l1o;
    const double s1n = (double)E[row + 1] - l1n;
    E[row] = (R)(l0n + s1o + kc * (s1n - s0o));
    const double r1o = o[2 * nyz + jk], r0o = o[3 * nyz + jk];
    const double r1n = (double)E[row + n0 - 2];
    E[row + n0 - 1] = (R)(r1o + kc * (r1n - r0o));
  }
}

template <class R>
YeeArgs<R> yee_args(const Grid &g, void *const E[3], void *const B[3], void *const J[3], double h) {
  YeeArgs<R> a;
  a.absorb = g.absorb_lo || g.absorb_hi;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.rdx[d] = (R)(1.0 / g.dx[d]);
    a.E[d] = static_cast<R *>(E[d]);
    a.B[d] = static_cast<R *>(B[d]);
    a.J[d] = J ? static_cast<const R *>(J[d]) : nullptr;
  }
  a.h = (R)h;
  return a;
}

// ---- particle load: global (x, y, z) -> (cell, offset) ----
template <class R>
__global__ void k_load(int dims, int n0, int n1, int n2, double rdx0, double rdx1, double rdx2, int absorb, Particles p,
                       int64_t offset, int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, const double *__restrict__ ux, const double *__restrict__ uy,
                       const double *__restrict__ uz, const double *__restrict__ w, const uint32_t *__restrict__ id,
                       uint32_t id_base, unsigned long long *bad) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double pos[3] = {x[q] * rdx0, y[q] * rdx1, dims == 3 ? z[q] * rdx2 : 0.0};
    const int nn[3] = {n0, n1, n2};
    int ci[3] = {0, 0, 0};
    R off[3] = {R(0), R(0), R(0)};
    // non-finite positions, momenta or weights are not loaded (marked dead)
    bool ok = isfinite(ux[q]) && isfinite(uy[q]) && isfinite(uz[q]) && isfinite(w[q]);
    for (int d = 0; d < dims; ++d) {
      if (!isfinite(pos[d])) {
        ok = false;
        continue;
      }
      const double fl = floor(pos[d]);
      double f = pos[d] - fl;
      long long i = (long long)fl;
      R fr = (R)f;
      if (fr >= R(1)) {  // rounding of the narrowing conversion
        fr = R(0);
        i += 1;
      }
      if (d == 0 && absorb && (pos[0] < kWallLo || pos[0] >= nn[0] - kWallHiMargin)) ok = false;
      i %= nn[d];
      if (i < 0) i += nn[d];
      ci[d] = (int)i;
      off[d] = fr;
    }
    const int64_t s = offset + q;
    if (!ok) {
      atomicAdd(bad, 1ull);
      p.cell[s] = -1;
    } else {
      p.cell[s] = ci[0] + n0 * (ci[1] + n1 * ci[2]);
    }
    for (int d = 0; d < 3; ++d) {
      if (d < dims) static_cast<R *>(p.off[d])[s] = off[d];
    }
    static_cast<R *>(p.u[0])[s] = (R)ux[q];
    static_cast<R *>(p.u[1])[s] = (R)uy[q];
    static_cast<R *>(p.u[2])[s] = (R)uz[q];
    static_cast<R *>(p.w)[s] = (R)w[q];
    p.id[s] = id ? id[q] : id_base + (uint32_t)q;  // no tags given: running index
  }
}

// ---- validation of particle storage copied in from outside (state resume) ----
// A slot below n is valid when it is dead (cell -1) or when its cell lies in
// the grid (and, with absorbing x walls, its position between them), its
// offsets on the grid's axes are in [0, 1) and its momenta and weight are
// finite.  Invalid slots are counted in *bad.
template <class R>
__global__ void k_check_particles(int dims, int n0, int64_t ncell, int absorb, Particles p, int64_t n,
                                  unsigned long long *bad) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = p.cell[q];
    if (c == -1) continue;
    bool ok = c >= 0 && (int64_t)c < ncell;
    for (int d = 0; d < dims; ++d) {
      const R f = static_cast<const R *>(p.off[d])[q];
      ok = ok && f >= R(0) && f < R(1);  // false for NaN
    }
    for (int d = 0; d < 3; ++d) ok = ok && isfinite(static_cast<const R *>(p.u[d])[q]);
    ok = ok && isfinite(static_cast<const R *>(p.w)[q]);
    if (ok && absorb) {
      const double X = (double)(c % n0) + (double)static_cast<const R *>(p.off[0])[q];
      ok = X >= kWallLo && X < n0 - kWallHiMargin;
    }
    if (!ok) atomicAdd(bad, 1ull);
  }
}

// ---- particle unload: (cell, offset) -> global FP64 ----
template <class R>
__global__ void k_unload(int dims, int n0, int n1, double dx0, double dx1, double dx2, Particles p,
                         const int64_t *__restrict__ d_count, double *x, double *y, double *z, double *ux, double *uy,
                         double *uz, double *w, uint32_t *id, int32_t *alive) {
  const int64_t n = *d_count;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = p.cell[q];
    const int i = c < 0 ? 0 : c % n0;
    const int r = c < 0 ? 0 : c / n0;
    const int j = r % n1;
    const int k = r / n1;
    if (x) x[q] = ((double)i + (double)static_cast<const R *>(p.off[0])[q]) * dx0;
    if (y) y[q] = ((double)j + (double)static_cast<const R *>(p.off[1])[q]) * dx1;
    if (z) z[q] = dims == 3 ? ((double)k + (double)static_cast<const R *>(p.off[2])[q]) * dx2 : 0.0;
    if (ux) ux[q] = (double)static_cast<const R *>(p.u[0])[q];
    if (uy) uy[q] = (double)static_cast<const R *>(p.u[1])[q];
    if (uz) uz[q] = (double)static_cast<const R *>(p.u[2])[q];
    if (w) w[q] = (double)static_cast<const R *>(p.w)[q];
    if (id) id[q] = p.id[q];
    if (alive) alive[q] = c >= 0 ? 1 : 0;
  }
}

template <class Rs, class Rd>
__global__ void k_convert(const Rs *__restrict__ s, Rd *__restrict__ d, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    d[q] = (Rd)s[q];
}

// ---- charge density at the nodes: rho += q w S(X-i) S(Y-j) S(Z-k) ----
template <class R>
__global__ void k_rho(int dims, int order, int n0, int n1, int n2, double q, Particles p,
                      const int64_t *__restrict__ d_count, double *rho) {
  const int64_t n = *d_count;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int c = p.cell[s];
    if (c < 0) continue;
    const int ci[3] = {c % n0, (c / n0) % n1, dims == 3 ? c / (n0 * n1) : 0};
    const int nn[3] = {n0, n1, n2};
    int base[3] = {0, 0, 0};
    double wt[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}};
    int ns[3] = {1, 1, 1};
    for (int d = 0; d < dims; ++d) {
      const double f = (double)static_cast<const R *>(p.off[d])[s];
      if (order == 2) {
        const int h = f >= 0.5;
        const double dd = f - h;
        const double a = 0.5 - dd, b = 0.5 + dd;
        wt[d][0] = 0.5 * a * a;
        wt[d][1] = 0.75 - dd * dd;
        wt[d][2] = 0.5 * b * b;
        base[d] = ci[d] + h - 1;
        ns[d] = 3;
      } else {
        wt[d][0] = 1.0 - f;
        wt[d][1] = f;
        base[d] = ci[d];
        ns[d] = 2;
      }
    }
    const double qw = q * (double)static_cast<const R *>(p.w)[s];
    for (int kz = 0; kz < ns[2]; ++kz)
      for (int ky = 0; ky < ns[1]; ++ky)
        for (int kx = 0; kx < ns[0]; ++kx) {
          const int gi = wrapi(base[0] + kx, nn[0]);
          const int gj = wrapi(base[1] + ky, nn[1]);
          const int gk = dims == 3 ? wrapi(base[2] + kz, nn[2]) : 0;
          atomicAdd(rho + gi + (int64_t)n0 * (gj + (int64_t)n1 * gk), qw * wt[0][kx] * wt[1][ky] * wt[2][kz]);
        }
  }
}

template <class R>
__global__ void __launch_bounds__(256)
    k_field_diag(int dims, int n0, int n1, int n2, double rdx0, double rdx1, double rdx2, double rdt, const R *Ex,
                 const R *Ey, const R *Ez, const R *Bx, const R *By, const R *Bz, const R *Jx, const R *Jy,
                 const R *Jz, const double *rho, const double *rho_prev, double *out) {
  __shared__ double sh[32];
  double se = 0, sb = 0, sq = 0, gm = 0, cm = 0, nf = 0;
  // one x row per block and pass (no per-cell index division)
  const int64_t nrows = (int64_t)n1 * n2;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int j = (int)(r % n1), k = (int)(r / n1);
    const int64_t dy = j > 0 ? n0 : (int64_t)n0 - (int64_t)n0 * n1;  // to the y - 1 row, periodic
    const int64_t dz = k > 0 ? (int64_t)n0 * n1 : (int64_t)n0 * n1 - (int64_t)n0 * n1 * n2;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      const int64_t c = r * n0 + i;
      const double ex = Ex[c], ey = Ey[c], ez = Ez[c], bx = Bx[c], by = By[c], bz = Bz[c];
      se += ex * ex + ey * ey + ez * ez;
      sb += bx * bx + by * by + bz * bz;
      if (!isfinite(ex) || !isfinite(ey) || !isfinite(ez) || !isfinite(bx) || !isfinite(by) || !isfinite(bz)) nf += 1;
      const int64_t cxm = c - (i > 0 ? 1 : 1 - n0);
      const int64_t cym = c - dy;
      const int64_t czm = c - dz;
      double div = ((double)Ex[c] - (double)Ex[cxm]) * rdx0 + ((double)Ey[c] - (double)Ey[cym]) * rdx1;
      double dj = ((double)Jx[c] - (double)Jx[cxm]) * rdx0 + ((double)Jy[c] - (double)Jy[cym]) * rdx1;
      if (dims == 3) {
        div += ((double)Ez[c] - (double)Ez[czm]) * rdx2;
        dj += ((double)Jz[c] - (double)Jz[czm]) * rdx2;
      }
      sq += rho[c];
      gm = fmax(gm, fabs(div - rho[c]));
      if (rho_prev) cm = fmax(cm, fabs((rho[c] - rho_prev[c]) * rdt + dj));
    }
  }
  double v;
  v = block_sum(se, sh);
  if (threadIdx.x == 0) atomicAdd(out + 0, v);
  v = block_sum(sb, sh);
  if (threadIdx.x == 0) atomicAdd(out + 1, v);
  v = block_sum(sq, sh);
  if (threadIdx.x == 0) atomicAdd(out + 2, v);
  v = block_max(gm, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(out + 3, v);
  v = block_max(cm, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(out + 4, v);
  v = block_sum(nf, sh);
  if (threadIdx.x == 0) atomicAdd(out + 5, v);
}

// A thread's running sum of per-element terms computed in R.  FP64 runs add
// in FP64.  FP32 runs keep a compensated FP32 sum (Neumaier's variant of
// Kahan summation), which stays off the slow FP64 pipe and is exact to a few
// FP32 ulps of the summed magnitudes; block and grid sums are FP64.
template <class R> struct ThreadSum;
template <> struct ThreadSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct ThreadSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;  // the rounding error of s + x, exactly
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// sum E^2, sum B^2 (squares in the storage precision)
template <class R>
__global__ void __launch_bounds__(256)
    k_field_energy(int64_t ncell, const R *Ex, const R *Ey, const R *Ez, const R *Bx, const R *By, const R *Bz,
                   double *out) {
  __shared__ double sh[32];
  ThreadSum<R> se, sb;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const R ex = Ex[c], ey = Ey[c], ez = Ez[c], bx = Bx[c], by = By[c], bz = Bz[c];
    se.add(ex * ex + ey * ey + ez * ez);
    sb.add(bx * bx + by * by + bz * bz);
  }
  double v = block_sum(se.value(), sh);
  if (threadIdx.x == 0) atomicAdd(out + 0, v);
  v = block_sum(sb.value(), sh);
  if (threadIdx.x == 0) atomicAdd(out + 1, v);
}

template <class R>
__global__ void __launch_bounds__(256)
    k_particle_diag(Particles p, const int64_t *__restrict__ d_count, double m, double *out) {
  __shared__ double sh[32];
  const int64_t n = *d_count;
  const int32_t *__restrict__ cell = p.cell;
  const R *__restrict__ u0 = static_cast<const R *>(p.u[0]);
  const R *__restrict__ u1 = static_cast<const R *>(p.u[1]);
  const R *__restrict__ u2p = static_cast<const R *>(p.u[2]);
  const R *__restrict__ w = static_cast<const R *>(p.w);
  ThreadSum<R> ek;
  int64_t cnt = 0, nf = 0;
  // four slots per thread and pass, every load issued before any is used
  // (a dead slot's momenta are read and dropped rather than skipped, so
  // the loads do not wait for the cell index)
  constexpr int kU = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s0 < n; s0 += kU * stride) {
    int c[kU];
    R ux[kU], uy[kU], uz[kU], wq[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int64_t s = s0 + k * stride;
      const bool in = s < n;
      c[k] = in ? cell[s] : -1;
      ux[k] = in ? u0[s] : R(0);
      uy[k] = in ? u1[s] : R(0);
      uz[k] = in ? u2p[s] : R(0);
      wq[k] = in ? w[s] : R(0);
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      if (c[k] < 0) continue;
      // per-particle terms in the storage precision
      const R u2 = ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k];
      // gamma - 1 = u^2 / (sqrt(1 + u^2) + 1), free of cancellation
      ek.add(wq[k] * (u2 / (sqrt(R(1) + u2) + R(1))));
      ++cnt;
      nf += !isfinite(u2);
    }
  }
  double v = block_sum(ek.value(), sh);
  if (threadIdx.x == 0) atomicAdd(out + 0, m * v);
  v = block_sum((double)cnt, sh);
  if (threadIdx.x == 0) atomicAdd(out + 1, v);
  v = block_sum((double)nf, sh);
  if (threadIdx.x == 0) atomicAdd(out + 2, v);
}

// One smoothing pass along `axis`: out = alpha in + side (in[-1] + in[+1]),
// periodic (side = (1 - alpha)/2).  A Fourier mode exp(i k x) is multiplied
// by alpha + (1 - alpha) cos(k dx).
template <class R>
__global__ void __launch_bounds__(256)
    k_smooth_axis(const R *__restrict__ in, R *__restrict__ out, int n0, int n1, int n2, int axis, R alpha, R side) {
  const int64_t ncell = (int64_t)n0 * n1 * n2;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo, hi;
    if (axis == 0) {
      const int i = (int)(c % n0);
      lo = c + (i > 0 ? -1 : n0 - 1);
      hi = c + (i + 1 < n0 ? 1 : 1 - n0);
    } else if (axis == 1) {
      const int j = (int)((c / n0) % n1);
      lo = c + (j > 0 ? -sy : sy * (n1 - 1));
      hi = c + (j + 1 < n1 ? sy : sy - sy * n1);
    } else {
      const int k = (int)(c / sz);
      lo = c + (k > 0 ? -sz : sz * (n2 - 1));
      hi = c + (k + 1 < n2 ? sz : sz - sz * n2);
    }
    out[c] = alpha * in[c] + side * (in[lo] + in[hi]);
  }
}

template <class R>
cudaError_t smooth_t(const Grid &g, R *f, R *tmp, int passes, int compensate, cudaStream_t st, int *nlaunch) {
  const int nb = grid_blocks(g.ncell, 256);
  R *src = f, *dst = tmp;
  int nl = 0;
  auto pass = [&](int axis, double alpha) {
    k_smooth_axis<R><<<nb, 256, 0, st>>>(src, dst, g.n[0], g.n[1], g.n[2], axis, (R)alpha, (R)(0.5 * (1.0 - alpha)));
    R *t = src;
    src = dst;
    dst = t;
    ++nl;
  };
  for (int p = 0; p < passes; ++p)
    for (int a = 0; a < g.dims; ++a) pass(a, 0.5);
  if (compensate && passes > 0)
    for (int a = 0; a < g.dims; ++a) pass(a, 1.0 + 0.5 * passes);
  if (nlaunch) *nlaunch = nl;
  if (src != f) {
    const cudaError_t e = cudaMemcpyAsync(f, src, sizeof(R) * (size_t)g.ncell, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_smooth(const Grid &g, void *f, bool f64, void *tmp, int passes, int compensate, cudaStream_t st,
                          int *nlaunch) {
  if (f64 || g.prec == 1)
    return smooth_t<double>(g, static_cast<double *>(f), static_cast<double *>(tmp), passes, compensate, st, nlaunch);
  return smooth_t<float>(g, static_cast<float *>(f), static_cast<float *>(tmp), passes, compensate, st, nlaunch);
}

template <class R> void yee_b_t(const Grid &g, void *const E[3], void *const B[3], double h, cudaStream_t st) {
  auto a = yee_args<R>(g, E, B, nullptr, h);
  if (yee_vec_ok<R>(g, a, false)) {
    dim3 grid, block;
    yee_vec_shape<R>(g, grid, block);
    if (g.dims == 3) k_yee_b_vec<R, 3><<<grid, block, 0, st>>>(a);
    else k_yee_b_vec<R, 2><<<grid, block, 0, st>>>(a);
  } else {
    const int nb = grid_blocks(g.ncell, 256);
    if (g.dims == 3) k_yee_b<R, 3><<<nb, 256, 0, st>>>(a);
    else k_yee_b<R, 2><<<nb, 256, 0, st>>>(a);
  }
}

template <class R>
void yee_e_t(const Grid &g, void *const E[3], void *const B[3], void *const J[3], double h, cudaStream_t st) {
  auto a = yee_args<R>(g, E, B, J, h);
  if (yee_vec_ok<R>(g, a, true)) {
    dim3 grid, block;
    yee_vec_shape<R>(g, grid, block);
    if (g.dims == 3) k_yee_e_vec<R, 3><<<grid, block, 0, st>>>(a);
    else k_yee_e_vec<R, 2><<<grid, block, 0, st>>>(a);
  } else {
    const int nb = grid_blocks(g.ncell, 256);
    if (g.dims == 3) k_yee_e<R, 3><<<nb, 256, 0, st>>>(a);
    else k_yee_e<R, 2><<<nb, 256, 0, st>>>(a);
  }
}

cudaError_t launch_yee_b(const Grid &g, void *const E[3], void *const B[3], double h, cudaStream_t st) {
  if (g.prec == 1) yee_b_t<double>(g, E, B, h, st);
  else yee_b_t<float>(g, E, B, h, st);
  return cudaGetLastError();
}

cudaError_t launch_yee_e(const Grid &g, void *const E[3], void *const B[3], void *const J[3], double h,
                         cudaStream_t st) {
  if (g.prec == 1) yee_e_t<double>(g, E, B, J, h, st);
  else yee_e_t<float>(g, E, B, J, h, st);
  return cudaGetLastError();
}

cudaError_t launch_mur_save(const Grid &g, void *const E[3], double *buf, cudaStream_t st) {
  const int nb = grid_blocks(8LL * g.n[1] * g.n[2], 256);
  if (g.prec == 1)
    k_mur_save<double><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], static_cast<const double *>(E[1]),
                                           static_cast<const double *>(E[2]), buf);
  else
    k_mur_save<float><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], static_cast<const float *>(E[1]),
                                          static_cast<const float *>(E[2]), buf);
  return cudaGetLastError();
}

double laser_waveform(const Laser &L, double tau) {
  if (tau <= 0.0 || tau >= L.duration) return 0.0;
  const double env = sin(3.14159265358979323846 * tau / L.duration);
  return env * env * sin(tau);
}

LaserStep laser_step(const Laser &L, const double *prof, double amplitude, const Grid &g, double t_old, double t_new) {
  LaserStep ls{};
  const double dx = g.dx[0];
  ls.pol = L.enabled ? L.pol : 0;
  ls.prof = prof;
  ls.amp[0] = amplitude * laser_waveform(L, t_old);
  ls.amp[1] = amplitude * laser_waveform(L, t_old - dx);
  ls.amp[2] = amplitude * laser_waveform(L, t_new);
  ls.amp[3] = amplitude * laser_waveform(L, t_new - dx);
  ls.oblique = L.enabled && L.angle != 0.0;
  if (ls.oblique) {
    ls.dims = g.dims;
    ls.cos_t = cos(L.angle);
    ls.sin_t = sin(L.angle);
    // E in the x-y plane: its y component is cos(angle) of the amplitude
    ls.a = amplitude * (L.pol == 1 ? ls.cos_t : 1.0);
    ls.y0 = L.angle > 0.0 ? 0.0 : g.n[1] * g.dx[1];  // the wall edge the tilted fronts reach first
    ls.yc = L.yc;
    ls.zc = L.zc;
    ls.inv_w2 = 1.0 / (L.waist * L.waist);
    ls.duration = L.duration;
    ls.t_old = t_old;
    ls.t_new = t_new;
    ls.dx = dx;
    ls.dy = g.dx[1];
    ls.dz = g.dx[2];
  }
  return ls;
}

cudaError_t launch_mur_apply(const Grid &g, void *const E[3], const double *buf, const LaserStep &ls,
                             cudaStream_t st) {
  const int nb = grid_blocks(2LL * g.n[1] * g.n[2], 256);
  if (g.prec == 1)
    k_mur_apply<double><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], g.dx[0], g.dt, static_cast<double *>(E[1]),
                                            static_cast<double *>(E[2]), buf, ls);
  else
    k_mur_apply<float><<<nb, 256, 0, st>>>(g.n[0], g.n[1], g.n[2], g.dx[0], g.dt, static_cast<float *>(E[1]),
                                           static_cast<float *>(E[2]), buf, ls);
  return cudaGetLastError();
}

cudaError_t launch_load(const Grid &g, const Particles &p, int64_t offset, int64_t n, const double *x,
                        const double *y, const double *z, const double *ux, const double *uy, const double *uz,
                        const double *w, const uint32_t *id, uint32_t id_base, unsigned long long *bad,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = grid_blocks(n, 256);
  const int absorb = g.absorb_lo || g.absorb_hi;
  if (g.prec == 1)
    k_load<double><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.n[2], 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                       absorb, p, offset, n, x, y, z, ux, uy, uz, w, id, id_base, bad);
  else
    k_load<float><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.n[2], 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
                                      absorb, p, offset, n, x, y, z, ux, uy, uz, w, id, id_base, bad);
  return cudaGetLastError();
}

cudaError_t launch_check_particles(const Grid &g, const Particles &p, int64_t n, unsigned long long *bad,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = grid_blocks(n, 256);
  const int absorb = g.absorb_lo || g.absorb_hi;
  if (g.prec == 1)
    k_check_particles<double><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.ncell, absorb, p, n, bad);
  else
    k_check_particles<float><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.ncell, absorb, p, n, bad);
  return cudaGetLastError();
}

cudaError_t launch_unload(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double *x,
                          double *y, double *z, double *ux, double *uy, double *uz, double *w, uint32_t *id,
                          int32_t *alive, cudaStream_t st) {
  const int nb = grid_blocks(nmax, 256);
  if (g.prec == 1)
    k_unload<double><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.dx[0], g.dx[1], g.dx[2], p, d_count, x, y, z, ux,
                                         uy, uz, w, id, alive);
  else
    k_unload<float><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.dx[0], g.dx[1], g.dx[2], p, d_count, x, y, z, ux,
                                        uy, uz, w, id, alive);
  return cudaGetLastError();
}

cudaError_t launch_field_to_f64(const Grid &g, const void *src, double *dst, cudaStream_t st) {
  const int nb = grid_blocks(g.ncell, 256);
  if (g.prec == 1)
    return cudaMemcpyAsync(dst, src, sizeof(double) * g.ncell, cudaMemcpyDeviceToDevice, st);
  k_convert<float, double><<<nb, 256, 0, st>>>(static_cast<const float *>(src), dst, g.ncell);
  return cudaGetLastError();
}

cudaError_t launch_field_from_f64(const Grid &g, const double *src, void *dst, cudaStream_t st) {
  const int nb = grid_blocks(g.ncell, 256);
  if (g.prec == 1)
    return cudaMemcpyAsync(dst, src, sizeof(double) * g.ncell, cudaMemcpyDeviceToDevice, st);
  k_convert<double, float><<<nb, 256, 0, st>>>(src, static_cast<float *>(dst), g.ncell);
  return cudaGetLastError();
}

cudaError_t launch_to_f64(int prec, const void *src, double *dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec == 1) return cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  k_convert<float, double><<<grid_blocks(n, 256), 256, 0, st>>>(static_cast<const float *>(src), dst, n);
  return cudaGetLastError();
}

cudaError_t launch_from_f64(int prec, const double *src, void *dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec == 1) return cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  k_convert<double, float><<<grid_blocks(n, 256), 256, 0, st>>>(src, static_cast<float *>(dst), n);
  return cudaGetLastError();
}

cudaError_t launch_rho(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double q,
                       double *rho, cudaStream_t st) {
  const int nb = grid_blocks(nmax, 256);
  if (g.prec == 1)
    k_rho<double><<<nb, 256, 0, st>>>(g.dims, g.order, g.n[0], g.n[1], g.n[2], q, p, d_count, rho);
  else
    k_rho<float><<<nb, 256, 0, st>>>(g.dims, g.order, g.n[0], g.n[1], g.n[2], q, p, d_count, rho);
  return cudaGetLastError();
}

cudaError_t launch_field_diag(const Grid &g, void *const E[3], void *const B[3], void *const J[3],
                              const double *rho, const double *rho_prev, double *out, cudaStream_t st) {
  const int nb = grid_blocks(g.ncell, 256);
  const double r0 = 1.0 / g.dx[0], r1 = 1.0 / g.dx[1], r2 = 1.0 / g.dx[2], rdt = 1.0 / g.dt;
  if (g.prec == 1) {
    auto c = [](void *v) { return static_cast<const double *>(v); };
    k_field_diag<double><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.n[2], r0, r1, r2, rdt, c(E[0]), c(E[1]),
                                             c(E[2]), c(B[0]), c(B[1]), c(B[2]), c(J[0]), c(J[1]), c(J[2]), rho,
                                             rho_prev, out);
  } else {
    auto c = [](void *v) { return static_cast<const float *>(v); };
    k_field_diag<float><<<nb, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.n[2], r0, r1, r2, rdt, c(E[0]), c(E[1]),
                                            c(E[2]), c(B[0]), c(B[1]), c(B[2]), c(J[0]), c(J[1]), c(J[2]), rho,
                                            rho_prev, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_field_energy(const Grid &g, void *const E[3], void *const B[3], double *out, cudaStream_t st) {
  const int nb = grid_blocks(g.ncell, 256);
  if (g.prec == 1) {
    auto c = [](void *v) { return static_cast<const double *>(v); };
    k_field_energy<double><<<nb, 256, 0, st>>>(g.ncell, c(E[0]), c(E[1]), c(E[2]), c(B[0]), c(B[1]), c(B[2]), out);
  } else {
    auto c = [](void *v) { return static_cast<const float *>(v); };
    k_field_energy<float><<<nb, 256, 0, st>>>(g.ncell, c(E[0]), c(E[1]), c(E[2]), c(B[0]), c(B[1]), c(B[2]), out);
  }
  return cudaGetLastError();
}

cudaError_t launch_particle_diag(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double m,
                                 double *out, cudaStream_t st) {
  const int nb = grid_blocks(nmax, 256);
  if (g.prec == 1) k_particle_diag<double><<<nb, 256, 0, st>>>(p, d_count, m, out);
  else k_particle_diag<float><<<nb, 256, 0, st>>>(p, d_count, m, out);
  return cudaGetLastError();
}

}  // namespace pic
