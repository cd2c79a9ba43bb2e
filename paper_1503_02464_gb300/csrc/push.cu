// Fused per-tile particle kernel: field gather -> Boris push -> leap-frog
// move -> Esirkepov current deposit (§2 eqs. 1-4 of the paper, Boris per its
// ref [8], the charge-conserving deposit for the continuity requirement it
// states in §2).
//
// Cell tiles are 8x8x4 in 3D, 16x16 in 2D.  The sort keeps each tile's
// particles in one contiguous, 4-aligned slot range and cuts that range into
// work items of bounded size; one thread block takes one work item.  The
// block stages E and B of the tile plus guard cells in shared memory and
// accumulates J of the tile plus guard with shared-memory atomics (fixed
// point in FP32 runs), then adds its J window to the global J (one atomic per
// non-zero value).
//
// Particles stream through a 256-slot shared staging chunk, loaded with
// coalesced accesses in slot order.  The deposit runs in a permuted order that
// gives the 32 lanes of a warp particles eight slots apart: slots are
// cell-sorted, so lanes then sit in different cells and their shared atomics
// hit different addresses and banks.  FP32 3D runs gather and push in slot
// order first (lanes of a warp in a few cells read the same field nodes),
// write the new state to global memory and leave a deposit job for the
// permuted phase after a block barrier (see k_push).
//
// A particle that has drifted more than D = 1 cell outside its tile since the
// last sort is not handled here: its slot is appended to an escape list and
// k_push_escaped applies the same arithmetic on global memory afterwards.
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

namespace {

constexpr int kThreads = 256;

// i mod n for i within a few periods of [0, n) (window coordinates)
__device__ __forceinline__ int wrap_near(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}
constexpr int32_t kEscFlag = 0x40000000;  // set in `cell` while a particle waits for the escape kernel

// Compile-time tile and window geometry.
template <int DIM, int ORDER> struct Geo {
  static constexpr int TX = DIM == 3 ? 8 : 16;
  static constexpr int TY = DIM == 3 ? 8 : 16;
  static constexpr int TZ = DIM == 3 ? 4 : 1;
  static constexpr int D = 1;  // drift allowance (cells)
  static constexpr int LOE = 1, HIE = ORDER == 2 ? 2 : 1;  // gather reach below / above the cell
  static constexpr int LOJ = ORDER == 2 ? 2 : 1, HIJ = ORDER == 2 ? 3 : 2;  // deposit reach
  static constexpr int EX = TX + 2 * D + LOE + HIE;
  static constexpr int EY = TY + 2 * D + LOE + HIE;
  static constexpr int EZ = DIM == 3 ? TZ + 2 * D + LOE + HIE : 1;
  static constexpr int JX = TX + 2 * D + LOJ + HIJ;
  static constexpr int JY = TY + 2 * D + LOJ + HIJ;
  static constexpr int JZ = DIM == 3 ? TZ + 2 * D + LOJ + HIJ : 1;
  static constexpr int EN = EX * EY * EZ;
  // J window plane stride.  For 3D TSC it is padded from 15 x 15 = 225 to 231
  // nodes: the deposit's atomics come from 32 lanes in 32 neighbouring cells,
  // each offset by its particle's stencil start, and with 231 those addresses
  // fall on fewer shared banks twice (a count over thermal-plasma tiles: 2.6
  // -> 2.2 wavefronts per atomic instruction).  The padding nodes stay zero.
  static constexpr int JP = (DIM == 3 && ORDER == 2) ? JX * JY + 6 : JX * JY;
  static constexpr int JN = JP * JZ;
  static constexpr int JS = JN + (ORDER == 2 ? 32 : 0);  // word-array stride of the shared J window (TSC: + 32 scratch words)
  static constexpr int NS = ORDER + 1;  // gather stencil width
  static constexpr int NW = ORDER + 2;  // deposit stencil width
};

// Division by a runtime constant (Granlund-Montgomery): q = (umulhi(n,m) + n) >> l.
struct FastDiv {
  uint32_t m, l;
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> l);
  }
};

FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.l = l;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  return f;
}

template <class R> struct PushArgs {
  int n[3];
  int ntile[2];
  FastDiv dn0, dn1;
  const R *E[3];
  const R *B[3];
  R *J[3];
  int32_t *cell;
  R *off[3];
  R *u[3];
  const R *w;
  const int64_t *tile_start;
  double qabs;                      // |q|
  const int32_t *work_tile;         // work item -> tile (-1: none)
  const int64_t *work_pb;           // work item -> first slot
  int64_t chunk;                    // slots per work item at most
  float *tq;                        // per item: [2i] sum |w|, [2i+1] sum |w| min(1, |u|) (FP32 runs)
  int fresh;                        // tile contents changed (sorted) since tq was written
  int32_t *esc_list;                // slots deferred to k_push_escaped
  unsigned long long *esc_count;
  unsigned long long *q_jobs;       // deferred deposit jobs of this launch (counted at each drain)
  R qmh;      // q dt / (2 m)
  R dtdx[3];  // dt / dx_a
  R jfac[3];  // -q dx_a / dt  (Esirkepov running-sum scale, times w)
  R qz;       // q            (2D3V: Jz = q w vz S)
  int absorb;  // absorbing x walls: remove particles leaving [kWallLo, n0 - kWallHiMargin)
  int ec;      // energy-conserving gather
  Counters *ctr;
};

// True when a particle at cell index i0 with offset f has left the region
// allowed between absorbing x walls.
template <class R> __device__ __forceinline__ bool outside_walls(int absorb, int i0, R f, int n0) {
  if (!absorb) return false;
  const R X = (R)i0 + f;
  return X < (R)kWallLo || X >= (R)(n0 - kWallHiMargin);
}

template <class R> __device__ __forceinline__ R inv_sqrt(R x);
template <> __device__ __forceinline__ float inv_sqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double inv_sqrt<double>(double x) { return 1.0 / sqrt(x); }

// Weighted sum of one field component over the gather stencil; the stencil
// offsets are compile-time (row stride SY, plane stride SZ).
template <class R, int NS, int DIM, int SY, int SZ>
__device__ __forceinline__ R gsum(const R *__restrict__ F, const R *wx, const R *wy, const R *wz) {
  R acc = R(0);
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? NS : 1); ++c) {
    R accb = R(0);
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      const R *row = F + c * SZ + b * SY;
      R ra = row[0] * wx[0];
#pragma unroll
      for (int a = 1; a < NS; ++a) ra += row[a] * wx[a];
      accb += ra * wy[b];
    }
    acc += DIM == 3 ? accb * wz[c] : accb;
  }
  return acc;
}

// Shared-memory J window.  FP32 runs accumulate in fixed point: FP32 shared
// atomics are compare-and-swap loops costing several shared-memory
// wavefronts each, integer shared atomics are single native operations, and
// integer sums are exact and independent of order.  A contribution v becomes
// the integer X = rint(v * 2^K), K chosen per tile from a bound on |J| at any
// node: each Esirkepov contribution of a particle satisfies |v| <= |q w| |v_p|
// and Boris raises |u| by at most |q/m| dt |E|, so
//   |J_node| <= Q = sum over the tile's particles of |q w| min(1, |u| + |q/m| dt Emax)
// with Emax bounding |E| over the tile's field window; 2^K keeps Q 2^K below
// 2^kLimitLog2.  X is kept as two signed 32-bit words, X = hi * 2^16 + lo
// with |lo| <= 2^15, both found with FP32 FMAs and adds only (adding
// 1.5 * 2^(23 + s) rounds a float of magnitude below 2^(22 + s) to a multiple
// of 2^s held in the low mantissa bits), because float-to-64-bit conversions
// run on the slow FP64 pipe.  With
// |X| < 2^37 the hi sums cannot overflow, and the lo sums cannot overflow for
// fewer than 65,536 contributions per node.  FP64 runs use plain double
// shared atomics, keeping FP64 rounding.
template <class R> struct WinAcc;
template <> struct WinAcc<float> {
  int *w;       // [3][2][jn]: per component lo words, then hi words
  int jn;       // word stride: the window's nodes (then, for TSC, 32 scratch words)
  int dummy;    // TSC: this lane's scratch word (past the nodes, bank = lane)
  float scale;  // 2^K
  float unit;   // 2^-K
  static constexpr int kLimitLog2 = 37;
  static constexpr float kMagic = 12582912.0f;        // 1.5 * 2^23: ulp 1
  static constexpr float kMagicHi = 824633720832.0f;  // 1.5 * 2^39: ulp 2^16
  // Add the contribution p q (already in units of 2^-K): X = p q is split
  // into hi 2^16 + lo without the FP64 pipe.  The first FMA rounds X to a
  // multiple of 2^16 (|X| < 2^37, so the sum stays in [2^39, 2^40), where
  // the float spacing is 2^16) and its bit pattern minus the magic's is hi;
  // the second FMA gives X - hi 2^16 with one rounding, |.| <= 2^15, and a
  // round-to-nearest conversion gives the integer lo (one instruction where
  // adding and removing the 1.5 * 2^23 magic took two).
  template <bool kScratch>
  __device__ __forceinline__ void add(int comp, int idx, float p, float q) const {
    const float y = fmaf(p, q, kMagicHi);
    const float r = y - kMagicHi;  // hi 2^16, exact
    const float lf = fmaf(p, q, -r);
    const int hi = __float_as_int(y) - __float_as_int(kMagicHi);
    const int lo = __float2int_rn(lf);  // round to nearest even, as the 2^23 magic would
    // Both words are added unconditionally: a branch around the pair (or a
    // predicate on it) cost more than the adds.  With kScratch (TSC) a zero
    // contribution goes to the lane's own scratch word instead of the node,
    // so that it does not collide with the other lanes' nodes in their
    // banks (for CIC's smaller stencils the select costs more than it
    // saves).  Warps whose particles all deposit nothing skip the whole
    // stencil instead (deposit_particle).
    const int at = (!kScratch || (hi | lo)) ? idx : dummy;
    const unsigned s = (unsigned)__cvta_generic_to_shared(w + comp * 2 * jn + at);
    asm volatile("red.shared.add.s32 [%0], %1;\n\tred.shared.add.s32 [%2], %3;" ::"r"(s), "r"(lo),
                 "r"(s + 4u * (unsigned)jn), "r"(hi));
  }
  __device__ __forceinline__ float get(int comp, int idx) const {
    const int *b = w + comp * 2 * jn + idx;
    return fmaf((float)b[jn], 65536.0f * unit, (float)b[0] * unit);
  }
};
template <> struct WinAcc<double> {
  double *w;  // [3][jn], plain double sums (the FP64 path keeps FP64 rounding)
  int jn;
  int dummy;  // (unused)
  double scale;  // 1: contributions are passed unscaled
  double unit;
  template <bool kScratch>
  __device__ __forceinline__ void add(int comp, int idx, double p, double q) const {
    const double x = p * q;
    if (x != 0.0) atomicAdd(w + comp * jn + idx, x);
  }
  __device__ __forceinline__ double get(int comp, int idx) const { return w[comp * jn + idx]; }
};

// Esirkepov deposit into the shared J window (compile-time strides).
// base: window index of the stencil's first node.  The last running sum of
// each axis is -DS[last] (the running sum over the whole stencil vanishes),
// so it is exactly zero for a particle that keeps its nearest node on that
// axis.  lx, ly, lz: some active lane of the warp uses the last stencil node
// of that axis (warp-uniform); otherwise every contribution on that outer
// shell is zero and is skipped with a uniform branch.
template <class R, int ORDER, int DIM, int SY, int SZ>
__device__ __forceinline__ void deposit_win(const WinAcc<R> &acc, int base, const DepositAxis<R, ORDER> &X,
                                            const DepositAxis<R, ORDER> &Y, const DepositAxis<R, ORDER> &Z, R cx,
                                            R cy, R cz, R qwvz, bool lx, bool ly, bool lz) {
  constexpr int NW = ORDER + 2;
  constexpr int M = NW - 1;
  R Px[M], Py[M], Pz[M];
  {
    R a = R(0), b = R(0), c = R(0);
#pragma unroll
    for (int k = 0; k < M - 1; ++k) {
      a += X.DS[k];
      b += Y.DS[k];
      c += Z.DS[k];
      Px[k] = cx * a;
      Py[k] = cy * b;
      Pz[k] = cz * c;
    }
    Px[M - 1] = -cx * X.DS[NW - 1];
    Py[M - 1] = -cy * Y.DS[NW - 1];
    Pz[M - 1] = -cz * Z.DS[NW - 1];
  }
  if (DIM == 3) {
    // Jx(i+1/2,j,k) += Px[i] (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3), cyclic for y, z
    R hz[NW], tz[NW], hx[NW], tx[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      hz[k] = Z.S0[k] + R(0.5) * Z.DS[k];
      tz[k] = R(0.5) * Z.S0[k] + Z.DS[k] * R(1.0 / 3.0);
      hx[k] = X.S0[k] + R(0.5) * X.DS[k];
      tx[k] = R(0.5) * X.S0[k] + X.DS[k] * R(1.0 / 3.0);
    }
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      if (c == NW - 1 && !lz) continue;
#pragma unroll
      for (int b = 0; b < NW; ++b) {
        if (b == NW - 1 && !ly) continue;
        const R br = Y.S0[b] * hz[c] + Y.DS[b] * tz[c];
#pragma unroll
        for (int a = 0; a < M; ++a) {
          if (a == M - 1 && !lx) continue;
          acc.template add<ORDER == 2>(0, base + c * SZ + b * SY + a, Px[a], br);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      if (c == NW - 1 && !lz) continue;
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        if (a == NW - 1 && !lx) continue;
        const R br = Z.S0[c] * hx[a] + Z.DS[c] * tx[a];
#pragma unroll
        for (int b = 0; b < M; ++b) {
          if (b == M - 1 && !ly) continue;
          acc.template add<ORDER == 2>(1, base + c * SZ + b * SY + a, Py[b], br);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < NW; ++b) {
      if (b == NW - 1 && !ly) continue;
      const R hy = Y.S0[b] + R(0.5) * Y.DS[b];
      const R ty = R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0);
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        if (a == NW - 1 && !lx) continue;
        const R br = X.S0[a] * hy + X.DS[a] * ty;
#pragma unroll
        for (int c = 0; c < M; ++c) {
          if (c == M - 1 && !lz) continue;
          acc.template add<ORDER == 2>(2, base + c * SZ + b * SY + a, Pz[c], br);
        }
      }
    }
  } else {
    // 2D3V: Jx = Px (S0y + DSy/2), Jy = Py (S0x + DSx/2),
    //       Jz = q w vz (S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3)
#pragma unroll
    for (int b = 0; b < NW; ++b) {
      if (b == NW - 1 && !ly) continue;
      const R hy = Y.S0[b] + R(0.5) * Y.DS[b];
      const R ty = R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0);
#pragma unroll
      for (int a = 0; a < M; ++a) {
        if (a == M - 1 && !lx) continue;
        acc.template add<ORDER == 2>(0, base + b * SY + a, Px[a], hy);
      }
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        if (a == NW - 1 && !lx) continue;
        acc.template add<ORDER == 2>(2, base + b * SY + a, qwvz, X.S0[a] * hy + X.DS[a] * ty);
      }
    }
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      if (a == NW - 1 && !lx) continue;
      const R hx = X.S0[a] + R(0.5) * X.DS[a];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        if (b == M - 1 && !ly) continue;
        acc.template add<ORDER == 2>(1, base + b * SY + a, Py[b], hx);
      }
    }
  }
}

// A deposit job: the particle's cell relative to the tile (l in [-1, 16] on
// every axis) and its cell shift (s in {-1, 0, 1}), 5 + 2 bits per axis, and
// bit 30 set so that a job is never 0.
__device__ __forceinline__ int pack_job(const int l[3], const int s[3]) {
  return (1 << 30) | (l[0] + 1) | ((l[1] + 1) << 5) | ((l[2] + 1) << 10) | ((s[0] + 1) << 15) |
         ((s[1] + 1) << 17) | ((s[2] + 1) << 19);
}
__device__ __forceinline__ void unpack_job(int j, int l[3], int s[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    l[d] = ((j >> (5 * d)) & 31) - 1;
    s[d] = ((j >> (15 + 2 * d)) & 3) - 1;
  }
}

// ---- settled deposit ----------------------------------------------------
// Most particles keep their shape support over a step: for TSC the nearest
// node does not change, for CIC the cell does not.  For them the Esirkepov
// stencil shrinks from ORDER + 2 to ORDER + 1 nodes per axis (3D TSC: 54
// contributions instead of up to 144).  The shape change DS = S1 - S0 is
// taken in the factored form of DepositAxis (TSC, offsets d0, d1 of the two
// positions from their common nearest node, D = d1 - d0, sg = d0 + d1:
//   DS = (D (sg - 1) / 2, -D sg, D (sg + 1) / 2);  CIC: DS = (-D, D)),
// which keeps FP32's relative precision however small the move, where the
// difference of the two shapes would lose it.  The factored values equal
// S1 - S0 in exact arithmetic, so the current still satisfies the discrete
// continuity equation with rho = sum q w S (to FP32 round-off of S).
template <class R, int ORDER> struct SettledAxis {
  static constexpr int NS = ORDER + 1;
  int rel;    // first support node relative to the old cell
  R S0[NS], DS[NS];
  R dl;       // displacement in cells
  // false when the support changes (then nothing is set)
  __device__ __forceinline__ bool set(R f0, int s, R f1) {
    if (ORDER == 2) {
      const int h0 = f0 >= R(0.5), h1 = f1 >= R(0.5);
      if (s + h1 != h0) return false;
      rel = h0 - 1;
      const R d0 = f0 - R(h0), d1 = f1 - R(h1);  // both from the same node
      dl = d1 - d0;
      const R sg = d0 + d1;
      tsc3<R>(d0, S0);
      const R hd = R(0.5) * dl;
      DS[0] = hd * (sg - R(1));
      DS[1] = -dl * sg;
      DS[2] = hd * (sg + R(1));
    } else {
      if (s != 0) return false;
      rel = 0;
      S0[0] = R(1) - f0;
      S0[1] = f0;
      dl = f1 - f0;
      DS[0] = -dl;
      DS[NS - 1] = dl;
    }
    return true;
  }
  __device__ __forceinline__ void zero() {
    rel = 0;
    dl = R(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) S0[k] = DS[k] = R(0);
    S0[0] = R(1);
  }
};

// Add the contribution p q (window units) at the shared byte address sa of
// its low word; the high word lies JS words further.  Same split as
// WinAcc<float>::add, without the scratch-word select, so that the address
// is one base register plus a compile-time offset for the whole stencil.
template <int JS> __device__ __forceinline__ void fx_add(unsigned sa, float p, float q) {
  const float y = fmaf(p, q, WinAcc<float>::kMagicHi);
  const float r = y - WinAcc<float>::kMagicHi;
  const float lf = fmaf(p, q, -r);
  const int hi = __float_as_int(y) - __float_as_int(WinAcc<float>::kMagicHi);
  const int lo = __float2int_rn(lf);
  asm volatile("red.shared.add.s32 [%0], %1;\n\tred.shared.add.s32 [%2], %3;" ::"r"(sa), "r"(lo),
               "r"(sa + 4u * (unsigned)JS), "r"(hi));
}

// One contribution p q to component comp at node offset off (compile-time)
// from the stencil's first node.  FP32: fixed point at the byte address
// base + ...; FP64: a double shared atomic at the node (zero skipped), as in
// WinAcc<double>.
template <class R, int JS> struct SettledSink;
template <int JS> struct SettledSink<float, JS> {
  unsigned sb;  // byte address of the Jx low word of the stencil's first node
  __device__ __forceinline__ void add(int comp, int off, float p, float q) const {
    fx_add<JS>(sb + 8u * (unsigned)JS * (unsigned)comp + 4u * (unsigned)off, p, q);
  }
};
template <int JS> struct SettledSink<double, JS> {
  double *w;  // Jx value of the stencil's first node (components JS doubles apart)
  __device__ __forceinline__ void add(int comp, int off, double p, double q) const {
    const double x = p * q;
    if (x != 0.0) atomicAdd(w + comp * JS + off, x);
  }
};

// Esirkepov deposit of a settled particle on its ORDER + 1 support nodes per
// axis (compile-time strides SY, SZ in nodes).  Same brackets as deposit_win:
// Jx gets Px (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3), cyclic; in 2D3V
// Jz = q w vz (S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3).  The running
// sums of DS along an axis end at -DS[last] (the whole sum vanishes).
template <class R, int ORDER, int DIM, int SY, int SZ, int JS>
__device__ __forceinline__ void deposit_settled_win(const SettledSink<R, JS> &out, const SettledAxis<R, ORDER> &X,
                                                    const SettledAxis<R, ORDER> &Y, const SettledAxis<R, ORDER> &Z,
                                                    R cx, R cy, R cz, R qwvz) {
  constexpr int NS = ORDER + 1, M = ORDER;
  R Px[M], Py[M], Pz[M];
  {
    R ra = R(0), rb = R(0), rc = R(0);
#pragma unroll
    for (int k = 0; k < M - 1; ++k) {
      ra += X.DS[k];
      rb += Y.DS[k];
      rc += Z.DS[k];
      Px[k] = cx * ra;
      Py[k] = cy * rb;
      Pz[k] = cz * rc;
    }
    Px[M - 1] = -cx * X.DS[NS - 1];
    Py[M - 1] = -cy * Y.DS[NS - 1];
    Pz[M - 1] = -cz * Z.DS[NS - 1];
  }
  if (DIM == 3) {
    R hz[NS], tz[NS], hx[NS], tx[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      hz[k] = Z.S0[k] + R(0.5) * Z.DS[k];
      tz[k] = R(0.5) * Z.S0[k] + Z.DS[k] * R(1.0 / 3.0);
      hx[k] = X.S0[k] + R(0.5) * X.DS[k];
      tx[k] = R(0.5) * X.S0[k] + X.DS[k] * R(1.0 / 3.0);
    }
#pragma unroll
    for (int c = 0; c < NS; ++c)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        const R br = Y.S0[b] * hz[c] + Y.DS[b] * tz[c];
#pragma unroll
        for (int a = 0; a < M; ++a) out.add(0, c * SZ + b * SY + a, Px[a], br);
      }
#pragma unroll
    for (int c = 0; c < NS; ++c)
#pragma unroll
      for (int a = 0; a < NS; ++a) {
        const R br = Z.S0[c] * hx[a] + Z.DS[c] * tx[a];
#pragma unroll
        for (int b = 0; b < M; ++b) out.add(1, c * SZ + b * SY + a, Py[b], br);
      }
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      const R hy = Y.S0[b] + R(0.5) * Y.DS[b];
      const R ty = R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0);
#pragma unroll
      for (int a = 0; a < NS; ++a) {
        const R br = X.S0[a] * hy + X.DS[a] * ty;
#pragma unroll
        for (int c = 0; c < M; ++c) out.add(2, c * SZ + b * SY + a, Pz[c], br);
      }
    }
  } else {
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      const R hy = Y.S0[b] + R(0.5) * Y.DS[b];
      const R ty = R(0.5) * Y.S0[b] + Y.DS[b] * R(1.0 / 3.0);
#pragma unroll
      for (int a = 0; a < M; ++a) out.add(0, b * SY + a, Px[a], hy);
#pragma unroll
      for (int a = 0; a < NS; ++a) out.add(2, b * SY + a, qwvz, X.S0[a] * hy + X.DS[a] * ty);
    }
#pragma unroll
    for (int a = 0; a < NS; ++a) {
      const R hx = X.S0[a] + R(0.5) * X.DS[a];
#pragma unroll
      for (int b = 0; b < M; ++b) out.add(1, b * SY + a, Py[b], hx);
    }
  }
}

// Deposit of a particle whose support did not change.  Returns false,
// depositing nothing, when the support changes on some axis: such a particle
// takes the general ORDER + 2 node stencil (deposit_particle), through the
// block's queue of deferred jobs.
template <class R, int DIM, int ORDER>
__device__ __forceinline__ bool deposit_settled(const PushArgs<R> &a, const WinAcc<R> &acc, const int l[3],
                                                const int s[3], const R f[3], const R fn[3], R w, R vz) {
  using G = Geo<DIM, ORDER>;
  SettledAxis<R, ORDER> X, Y, Z;
  bool ok = X.set(f[0], s[0], fn[0]);
  ok = Y.set(f[1], s[1], fn[1]) && ok;
  if (DIM == 3) ok = Z.set(f[2], s[2], fn[2]) && ok;
  else Z.zero();
  if (!ok) return false;
  // a warp whose settled particles neither move nor (2D3V) carry vz deposits nothing
  const bool moves = w != R(0) && (X.dl != R(0) || Y.dl != R(0) || (DIM == 3 ? Z.dl != R(0) : vz != R(0)));
  if (!__any_sync(__activemask(), moves)) return true;
  constexpr int oJ = G::D + G::LOJ;
#ifdef PIC_CHECKED
  {
    const int rel[3] = {X.rel, Y.rel, Z.rel};
    constexpr int JW[3] = {G::JX, G::JY, G::JZ};
    bool in = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) in = in && l[d] + rel[d] + oJ >= 0 && l[d] + rel[d] + oJ + ORDER < JW[d];
    if (!PIC_CHECK(in, a.ctr)) return true;
  }
#endif
  const int jb = (l[0] + X.rel + oJ) + (l[1] + Y.rel + oJ) * G::JX + (DIM == 3 ? (l[2] + Z.rel + oJ) * G::JP : 0);
  SettledSink<R, G::JS> out;
  if constexpr (sizeof(R) == 4) out.sb = (unsigned)__cvta_generic_to_shared(acc.w) + 4u * (unsigned)jb;
  else out.w = acc.w + jb;
  const R ws = w * acc.scale;
  deposit_settled_win<R, ORDER, DIM, G::JX, G::JP, G::JS>(out, X, Y, Z, a.jfac[0] * ws, a.jfac[1] * ws,
                                                           a.jfac[2] * ws, a.qz * ws * vz);
  return true;
}

// Deferred deposit jobs of particles whose support changes: up to kQCap
// entries in shared memory, appended by warps through a shared counter and
// deposited once, at the end of the work item, by all threads together
// (dq_drain), so that the general stencil runs on full warps instead of on
// the few lanes of every warp that hold such a particle.  A job that finds
// the queue full is deposited on the spot.
constexpr int kQCap = kPushQueueCap;
// A chunk after which the queue could not take another chunk's worth of jobs
// (1.5 times what the last chunk added) drains it, the whole block taking
// one job per thread, so that plasmas whose particles change support often
// (fast beams) do not overflow it and deposit in divergent lanes.  A plasma
// with few such particles drains once, at the end of the work item: every
// drain costs a partly idle block-wide pass.
template <class R> struct DepQueue {
  int *job;  // [kQCap] packed cell and shift (pack_job) | axes whose support changes << 22
  R *f;      // [7][kQCap]: old offsets x y z, new offsets x y z, weight (2D3V: vz in the old z slot)
  int *tail;  // shared counter of appended jobs
};

// Append this lane's job; false when the queue is full.
template <class R>
__device__ __forceinline__ bool dq_push(const DepQueue<R> &q, int job, const R f[3], const R fn[3], R w, R vz,
                                        bool twod) {
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(q.tail, __popc(act));
  base = __shfl_sync(act, base, leader);
  const int at = base + __popc(act & ((1u << lane) - 1u));
  if (at >= kQCap) return false;
  q.job[at] = job;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    q.f[d * kQCap + at] = (twod && d == 2) ? vz : f[d];
    q.f[(3 + d) * kQCap + at] = fn[d];
  }
  q.f[6 * kQCap + at] = w;
  return true;
}

// The axes (bit d) on which a particle's shape support changes over a move.
template <class R, int ORDER>
__device__ __forceinline__ int support_change(const R f[3], const int s[3], const R fn[3]) {
  int m = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool ch = ORDER == 2 ? (s[d] + (fn[d] >= R(0.5)) != (f[d] >= R(0.5))) : s[d] != 0;
    m |= ch ? 1 << d : 0;
  }
  return m;
}

// The per-particle physics shared by the tile kernel and the escape kernel:
// given gathered E, B, advance u, move, and build the deposit stencils.
template <class R, int ORDER, int DIM>
__device__ __forceinline__ void push_move(const PushArgs<R> &a, R u[3], const R E[3], const R B[3], const R f[3],
                                          R fn[3], int s[3], R &ig, unsigned &clamp) {
  boris<R>(a.qmh, E, B, u);
  ig = inv_sqrt<R>(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fn[d] = R(0);
    s[d] = 0;
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R x = f[d] + a.dtdx[d] * u[d] * ig;
    const int sh = (x >= R(1)) ? 1 : ((x < R(0)) ? -1 : 0);
    x -= R(sh);
    if (x >= R(1)) {
      x = below_one<R>();
      ++clamp;
    }
    if (x < R(0)) {
      x = R(0);
      ++clamp;
    }
    fn[d] = x;
    s[d] = sh;
  }
}

// Esirkepov deposit of one particle's move into the J window (§2 eq. 4 and
// the continuity equation): l is its cell relative to the tile, s its cell
// shift, f -> fn its offsets before and after the move, w its weight, vz its
// velocity along z (the 2D3V Jz term).  Returns false when the checked build
// finds the stencil outside the window (nothing deposited).
template <class R, int DIM, int ORDER>
__device__ __forceinline__ bool deposit_particle(const PushArgs<R> &a, const WinAcc<R> &acc, const int l[3],
                                                 const int s[3], const R f[3], const R fn[3], R w, R vz) {
  using G = Geo<DIM, ORDER>;
  // A particle that keeps its place (and, in 2D3V, has vz = 0) or has no
  // weight deposits nothing; a warp of such particles (a cold target before
  // the pulse reaches it) skips the stencil with a uniform branch.
  const unsigned act = __activemask();
  const bool moves = w != R(0) && ((s[0] | s[1] | s[2]) != 0 || f[0] != fn[0] || f[1] != fn[1] ||
                                   (DIM == 3 ? f[2] != fn[2] : vz != R(0)));
  if (!__any_sync(act, moves)) return true;
  DepositAxis<R, ORDER> dx, dy, dz;
  dx.set(f[0], s[0], fn[0]);
  dy.set(f[1], s[1], fn[1]);
  if (DIM == 3) dz.set(f[2], s[2], fn[2]);
  else dz.zero();
  constexpr int oJ = G::D + G::LOJ;
#ifdef PIC_CHECKED
  {
    // every deposit stencil inside the J window (checked builds)
    const int rel[3] = {dx.rel, dy.rel, dz.rel};
    constexpr int JW[3] = {G::JX, G::JY, G::JZ};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) ok = ok && l[d] + rel[d] + oJ >= 0 && l[d] + rel[d] + oJ + G::NW - 1 < JW[d];
    if (!PIC_CHECK(ok, a.ctr)) return false;
  }
#endif
  const int jb = (l[0] + dx.rel + oJ) + (l[1] + dy.rel + oJ) * G::JX +
                 (DIM == 3 ? (l[2] + dz.rel + oJ) * G::JP : 0);
  const R ws = w * acc.scale;  // fixed-point units folded into the factors
  // does some lane of this warp use the last stencil node of an axis?
  const bool lx = __any_sync(act, dx.S0[G::NW - 1] != R(0) || dx.DS[G::NW - 1] != R(0));
  const bool ly = __any_sync(act, dy.S0[G::NW - 1] != R(0) || dy.DS[G::NW - 1] != R(0));
  const bool lz = DIM == 3 && __any_sync(act, dz.S0[G::NW - 1] != R(0) || dz.DS[G::NW - 1] != R(0));
  deposit_win<R, ORDER, DIM, G::JX, G::JP>(acc, jb, dx, dy, dz, a.jfac[0] * ws, a.jfac[1] * ws,
                                                    a.jfac[2] * ws, a.qz * ws * vz, lx, ly, lz);
  return true;
}

// Deposit the n <= kQCap queued jobs on the general stencil, one per thread
// (with `reset`, the queue is emptied for the jobs of the next chunks).
// The jobs are first ordered by the axes on which their support changes
// (a counting sort into `order`, kQCap ints of shared memory), so that the
// lanes of a warp mostly share that set and the warp-uniform skip of the
// outer stencil shell in deposit_particle drops the axes that did not
// change.  Block-wide: every thread of the block calls it.
template <class R, int DIM, int ORDER>
__device__ __forceinline__ void dq_drain(const PushArgs<R> &a, const WinAcc<R> &acc, const DepQueue<R> &q, int n,
                                         int *order, bool reset) {
  __shared__ int s_cls[8];
  const int i = threadIdx.x;
  if (i < 8) s_cls[i] = 0;
  __syncthreads();
  // every thread has read the count: the queue may start over (appends
  // resume only after the next chunk's barriers)
  if (reset && i == 0) *q.tail = 0;
  int cls = 0, rank = 0;
  if (i < n) {
    cls = (q.job[i] >> 22) & 7;
    rank = atomicAdd(&s_cls[cls], 1);
  }
  __syncthreads();
  if (i < n) {
    int start = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) start += c < cls ? s_cls[c] : 0;
    order[start + rank] = i;
  }
  __syncthreads();
  if (i >= n) return;
  const int at = order[i];
  int l[3], sh[3];
  unpack_job(q.job[at] & ((1 << 22) - 1), l, sh);
  R f[3], fn[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d] = (DIM == 2 && d == 2) ? R(0) : q.f[d * kQCap + at];
    fn[d] = q.f[(3 + d) * kQCap + at];
  }
  const R vz = DIM == 2 ? q.f[2 * kQCap + at] : R(0);
  deposit_particle<R, DIM, ORDER>(a, acc, l, sh, f, fn, q.f[6 * kQCap + at], vz);
}

// MID: drain the queue between chunks when it fills (for plasmas whose
// particles change support often; see the launcher).
template <class R, int DIM, int ORDER, bool MID>
// Blocks per SM the register allocation is held to: FP32 3D TSC windows
// fill half the shared memory (two blocks); the 3D CIC windows leave room for
// three, which fit at 72 registers (1.27x faster than two); FP32 2D windows
// are small, and at 64 registers four blocks fit (1.46x faster on a 2D slab
// than two); none of these spill.  FP64 runs are bound by the FP64 pipe
// whatever their occupancy.
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? (DIM == 2 ? 4 : (ORDER == 1 ? 3 : 2)) : 1)
    k_push(const PushArgs<R> a) {
  using G = Geo<DIM, ORDER>;
  constexpr int NS = G::NS;
  static_assert(G::TX + G::D < 31 && G::TY + G::D < 31 && G::TZ + G::D < 31, "deposit job packing");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sF = reinterpret_cast<R *>(smem_raw);    // 6 * EN: Ex Ey Ez Bx By Bz
  // J window: 24 bytes per node (3 components x 8 bytes of fixed point)
  unsigned char *sJraw = smem_raw + 6 * G::EN * sizeof(R);
  R *sOff = reinterpret_cast<R *>(sJraw + 24 * G::JS);  // DIM x 256
  R *sU = sOff + DIM * kThreads;              // 3 x 256
  R *sW = sU + 3 * kThreads;                  // 256
  int32_t *sCell = reinterpret_cast<int32_t *>(sW + kThreads);  // 256
  int32_t *sJob = sCell + kThreads;  // FP32 3D: 256 deposit jobs
  // queue of deferred deposit jobs (after the jobs in 3D FP32, after the cells otherwise)
  constexpr bool kSplitLayout = DIM == 3 && sizeof(R) == 4;
  // the settled stencils and the queue: all but FP64 2D, whose kernel is
  // bound by the FP64 pipe in its gather and lost occupancy to the extra
  // registers and shared memory (measured 2.22 -> 1.91 G particle-steps/s
  // on the 2D laser slab)
  constexpr bool kSettled = !(sizeof(R) == 8 && DIM == 2);
  constexpr int kQJobBytes = 4 * kQCap;  // a multiple of 8: the R array that follows stays aligned
  DepQueue<R> dq;
  dq.job = sCell + (kSplitLayout ? 2 : 1) * kThreads;
  dq.f = reinterpret_cast<R *>(reinterpret_cast<char *>(dq.job) + kQJobBytes);
  __shared__ int s_qtail;
  dq.tail = &s_qtail;
  int q_prev = 0;  // jobs queued at the end of the previous chunk (the same in every thread)
  __shared__ unsigned int s_clamp;
  __shared__ double s_scale;
  __shared__ unsigned int s_emax[3];
  __shared__ float s_qsum, s_wsum, s_q1;
  float emax[3] = {0.f, 0.f, 0.f};

  const int wi = blockIdx.x;  // work item
  const int t = a.work_tile[wi];
  if (t < 0) return;
  const int64_t pb = a.work_pb[wi];
  const int64_t pe = pb + a.chunk < a.tile_start[t + 1] ? pb + a.chunk : a.tile_start[t + 1];
  if (pb >= pe) return;
  const int tid = threadIdx.x;
  int t0[3];
  {
    const int tx = t % a.ntile[0];
    const int r = t / a.ntile[0];
    t0[0] = tx * G::TX;
    t0[1] = (r % a.ntile[1]) * G::TY;
    t0[2] = (r / a.ntile[1]) * G::TZ;
  }

  // ---- stage E, B of the tile + guard (periodic wrap of global indices) ----
  for (int q = tid; q < G::EN; q += kThreads) {
    const int x = q % G::EX;
    const int y = (q / G::EX) % G::EY;
    const int z = q / (G::EX * G::EY);
    const int gi = wrap_near(t0[0] - G::D - G::LOE + x, a.n[0]);
    const int gj = wrap_near(t0[1] - G::D - G::LOE + y, a.n[1]);
    const int gk = DIM == 3 ? wrap_near(t0[2] - G::D - G::LOE + z, a.n[2]) : 0;
    const int64_t g = gi + (int64_t)a.n[0] * (gj + (int64_t)a.n[1] * gk);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R ev = a.E[c][g];
      sF[c * G::EN + q] = ev;
      sF[(3 + c) * G::EN + q] = a.B[c][g];
      emax[c] = fmax(emax[c], fabs((float)ev));
    }
  }
  for (int q = tid; q < 6 * G::JS; q += kThreads) reinterpret_cast<int *>(sJraw)[q] = 0;  // 24 B per node
  if (tid == 0) {
    s_clamp = 0;
    s_qtail = 0;
    s_emax[0] = s_emax[1] = s_emax[2] = 0u;
    s_qsum = 0.f;
    s_wsum = 0.f;
    s_q1 = 0.f;
  }
  __syncthreads();
  if (sizeof(R) == 4) {
    // fixed-point scale: bound Q on |J| at any node of the window (see WinAcc)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (emax[c] > 0.f) atomicMax(&s_emax[c], __float_as_uint(emax[c]));
    __syncthreads();
    const float ex = __uint_as_float(s_emax[0]), ey = __uint_as_float(s_emax[1]), ez = __uint_as_float(s_emax[2]);
    const float kick = (float)(2.0 * fabs((double)a.qmh)) * sqrtf(ex * ex + ey * ey + ez * ez);
    if (a.fresh) {
      // tile contents are new (sorted): bound from the particles themselves
      float qs = 0.f, w0 = 0.f;
      for (int64_t p = pb + tid; p < pe; p += kThreads) {
        if (a.cell[p] < 0) continue;
        const float ux = (float)a.u[0][p], uy = (float)a.u[1][p], uz = (float)a.u[2][p];
        const float aw = fabsf((float)a.w[p]);
        qs += aw * fminf(1.f, sqrtf(ux * ux + uy * uy + uz * uz) + kick);
        w0 += aw;
      }
      for (int o = 16; o > 0; o >>= 1) {
        qs += __shfl_down_sync(0xffffffffu, qs, o);
        w0 += __shfl_down_sync(0xffffffffu, w0, o);
      }
      if ((tid & 31) == 0) {
        if (qs > 0.f) atomicAdd(&s_qsum, qs);
        if (w0 > 0.f) atomicAdd(&s_wsum, w0);
      }
    } else if (tid == 0) {
      // |u| min'ed at 1 from the previous push, plus the kick of this step:
      // sum |w| min(1, |u| + kick) <= sum |w| min(1, |u|) + kick sum |w|
      s_wsum = a.tq[2 * wi];
      s_qsum = a.tq[2 * wi + 1] + kick * s_wsum;
    }
    __syncthreads();
    if (tid == 0) {
      // 1.01: room for the FP32 rounding of the sums above
      const double Q = 1.01 * a.qabs * (double)s_qsum;
      int e2 = 0;
      if (Q > 0.0) frexp(Q, &e2);  // Q < 2^e2
      int K = Q > 0.0 ? WinAcc<float>::kLimitLog2 - e2 : 100;
      K = K > 100 ? 100 : (K < -100 ? -100 : K);
      s_scale = ldexp(1.0, K);
    }
  } else if (tid == 0) {
    s_scale = 1.0;
  }
  __syncthreads();
  WinAcc<R> acc;
  acc.w = reinterpret_cast<decltype(acc.w)>(sJraw);
  acc.jn = G::JS;
  acc.dummy = G::JN + (tid & 31);
  acc.scale = (R)s_scale;
  acc.unit = (R)(1.0 / s_scale);

  // Slot assignment.  The deposit runs on the lane-spreading permutation e
  // (bijective; lane l of warp w takes slot 8l + ((w + l/4) mod 8)): the
  // slots are cell-sorted, so a warp's lanes sit about one cell apart and
  // their atomics hit different nodes.  In 3D the gather and push run first
  // on slot tid instead, where a warp's lanes sit in a few neighbouring cells
  // and mostly read the same field nodes (shared-memory broadcasts instead of
  // bank conflicts on the 162-node TSC gather); each pushed particle then
  // writes its new state to global memory and leaves a deposit job behind
  // (old offsets in sU, new ones in sOff, tile cell and cell shift packed in
  // sJob) for the deposit phase after a block barrier.  In 2D the gather is a third of that, and FP64 runs are bound by
  // the FP64 pipe: there the extra barrier and staging traffic cost more than
  // they save, so one thread pushes and deposits slot e.
  constexpr bool kSplit = DIM == 3 && sizeof(R) == 4;
  const int lane = tid & 31, warp = tid >> 5;
  const int e = 8 * lane + ((warp + (lane >> 2)) & 7);
  const int ep = kSplit ? tid : e;  // slot gathered and pushed by this thread
  unsigned my_clamp = 0, my_absorbed = 0;
  float my_q1 = 0.f;

  for (int64_t c0 = pb; c0 < pe; c0 += kThreads) {
    const int cn = (int)(pe - c0 < kThreads ? pe - c0 : kThreads);
    // coalesced load of the chunk, slot order
    if (tid < cn) {
      const int64_t p = c0 + tid;
      sCell[tid] = a.cell[p];
#pragma unroll
      for (int d = 0; d < DIM; ++d) sOff[d * kThreads + tid] = a.off[d][p];
#pragma unroll
      for (int d = 0; d < 3; ++d) sU[d * kThreads + tid] = a.u[d][p];
      sW[tid] = a.w[p];
    }
    __syncthreads();
    // ---- gather, Boris, move (and, in 2D, deposit) of slot ep ----
    if (ep < cn) {
      int job = 0;
      const int c = sCell[ep];
      if (c >= 0) {
        // decode the cell and its position relative to the tile
        const uint32_t r0 = a.dn0.div((uint32_t)c);
        int ci[3];
        ci[0] = c - (int)r0 * a.n[0];
        if (DIM == 3) {
          const uint32_t r1 = a.dn1.div(r0);
          ci[1] = (int)r0 - (int)r1 * a.n[1];
          ci[2] = (int)r1;
        } else {
          ci[1] = (int)r0;
          ci[2] = 0;
        }
        int l[3] = {0, 0, 0};
        bool inw = true;
        constexpr int TT[3] = {G::TX, G::TY, G::TZ};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          int dl = ci[d] - t0[d];
          if (dl > TT[d] - 1 + G::D) dl -= a.n[d];
          if (dl < -G::D) dl += a.n[d];
          l[d] = dl;
          inw = inw && dl >= -G::D && dl <= TT[d] - 1 + G::D;
        }
        if (!inw) {
          // defer to k_push_escaped (state left untouched)
          if (kSplit) a.cell[c0 + ep] = c | kEscFlag;
          else sCell[ep] = c | kEscFlag;
          const unsigned long long slot = atomicAdd(a.esc_count, 1ull);
          a.esc_list[slot] = (int32_t)(c0 + ep);
          my_q1 += fabsf((float)sW[ep]);  // its new |u| is not known here: bound by 1
        } else do {  // (a single pass: the checked build leaves it early on a bad index)
          R f[3], u[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            f[d] = d < DIM ? sOff[d * kThreads + ep] : R(0);
            u[d] = sU[d * kThreads + ep];
          }
          // ---- gather (§2: g-weighted average of the grid fields) ----
          GatherAxis<R, ORDER> gx, gy, gz;
          gx.set(f[0], a.ec);
          gy.set(f[1], a.ec);
          gz.set(f[2], a.ec);
          constexpr int oE = G::D + G::LOE;
#ifdef PIC_CHECKED
          {
            // every gather stencil inside the E/B window (checked builds)
            const GatherAxis<R, ORDER> *ga[3] = {&gx, &gy, &gz};
            constexpr int EW[3] = {G::EX, G::EY, G::EZ};
            bool ok = true;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              const int lo = l[d] + (ga[d]->relp < ga[d]->reld ? ga[d]->relp : ga[d]->reld) + oE;
              const int hi = l[d] + (ga[d]->relp > ga[d]->reld ? ga[d]->relp : ga[d]->reld) + oE + NS - 1;
              ok = ok && lo >= 0 && hi < EW[d];
            }
            if (!PIC_CHECK(ok, a.ctr)) break;  // leaves the particle as it was
          }
#endif
          const int xp = l[0] + gx.relp + oE, xd = l[0] + gx.reld + oE;
          const int yp = (l[1] + gy.relp + oE) * G::EX, yd = (l[1] + gy.reld + oE) * G::EX;
          const int zp = DIM == 3 ? (l[2] + gz.relp + oE) * G::EX * G::EY : 0;
          const int zd = DIM == 3 ? (l[2] + gz.reld + oE) * G::EX * G::EY : 0;
          constexpr int SY = G::EX, SZ = G::EX * G::EY;
          R E[3], B[3];
          E[0] = gsum<R, NS, DIM, SY, SZ>(sF + 0 * G::EN + xd + yp + zp, gx.wd, gy.wp, gz.wp);
          E[1] = gsum<R, NS, DIM, SY, SZ>(sF + 1 * G::EN + xp + yd + zp, gx.wp, gy.wd, gz.wp);
          E[2] = gsum<R, NS, DIM, SY, SZ>(sF + 2 * G::EN + xp + yp + zd, gx.wp, gy.wp, gz.wd);
          B[0] = gsum<R, NS, DIM, SY, SZ>(sF + 3 * G::EN + xp + yd + zd, gx.wp, gy.wd, gz.wd);
          B[1] = gsum<R, NS, DIM, SY, SZ>(sF + 4 * G::EN + xd + yp + zd, gx.wd, gy.wp, gz.wd);
          B[2] = gsum<R, NS, DIM, SY, SZ>(sF + 5 * G::EN + xd + yd + zp, gx.wd, gy.wd, gz.wp);

          // ---- Boris push (§2 eq. 3) and leap-frog move ----
          R fn[3], ig;
          int s[3];
          push_move<R, ORDER, DIM>(a, u, E, B, f, fn, s, ig, my_clamp);
          if (sizeof(R) == 4)
            my_q1 += fabsf((float)sW[ep]) * fminf(1.f, sqrtf((float)(u[0] * u[0] + u[1] * u[1] + u[2] * u[2])));

          if (!kSplit) {
            bool done = false;
            if constexpr (kSettled) {
              const R vz = u[2] * ig;
              done = deposit_settled<R, DIM, ORDER>(a, acc, l, s, f, fn, sW[ep], vz) ||
                     dq_push<R>(dq, pack_job(l, s) | support_change<R, ORDER>(f, s, fn) << 22, f, fn, sW[ep], vz,
                                DIM == 2);
            }
            if (!done && !deposit_particle<R, DIM, ORDER>(a, acc, l, s, f, fn, sW[ep], u[2] * ig))
              break;  // (checked build) leaves the particle as it was
          }

          // ---- the new state ----
          int nc = -1;  // removed at an absorbing wall after depositing its move
          if (outside_walls<R>(a.absorb, ci[0] + s[0], fn[0], a.n[0])) {
            ++my_absorbed;
          } else {
            nc = c;
            const int i0 = ci[0] + s[0];
            nc += s[0] + (i0 < 0 ? a.n[0] : (i0 >= a.n[0] ? -a.n[0] : 0));
            const int i1 = ci[1] + s[1];
            nc += (s[1] + (i1 < 0 ? a.n[1] : (i1 >= a.n[1] ? -a.n[1] : 0))) * a.n[0];
            if (DIM == 3) {
              const int i2 = ci[2] + s[2];
              nc += (s[2] + (i2 < 0 ? a.n[2] : (i2 >= a.n[2] ? -a.n[2] : 0))) * a.n[0] * a.n[1];
            }
          }
          if (kSplit) {
            // Slot ep is this thread's own index: the state goes straight to
            // global memory (coalesced).  The deposit job keeps the old
            // offsets in sU (u is no longer needed there) and the new ones
            // in sOff.
            const int64_t p = c0 + ep;
            a.cell[p] = nc;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              a.off[d][p] = fn[d];
              sU[d * kThreads + ep] = f[d];
              sOff[d * kThreads + ep] = fn[d];
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) a.u[d][p] = u[d];
            job = pack_job(l, s);
          } else {
            // back into the staging slot, stored after the chunk
#pragma unroll
            for (int d = 0; d < DIM; ++d) sOff[d * kThreads + ep] = fn[d];
#pragma unroll
            for (int d = 0; d < 3; ++d) sU[d * kThreads + ep] = u[d];
            sCell[ep] = nc;
          }
        } while (0);
      }
      if (kSplit) sJob[ep] = job;
    }
    if (kSplit) {
      __syncthreads();
      // ---- Esirkepov deposit of slot e (3D) ----
      if (e < cn) {
        const int job = sJob[e];
        if (job) {
          int l[3], s[3];
          unpack_job(job, l, s);
          R f[3], fn[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            f[d] = sU[d * kThreads + e];
            fn[d] = sOff[d * kThreads + e];
          }
          bool done = false;
          if constexpr (kSettled)
            done = deposit_settled<R, DIM, ORDER>(a, acc, l, s, f, fn, sW[e], R(0)) ||
                   dq_push<R>(dq, job | support_change<R, ORDER>(f, s, fn) << 22, f, fn, sW[e], R(0), false);
          if (!done) deposit_particle<R, DIM, ORDER>(a, acc, l, s, f, fn, sW[e], R(0));
        }
      }
    }
    __syncthreads();
    // coalesced store of the chunk (w is unchanged; 3D FP32 stored its state in phase 1)
    if (!kSplit && tid < cn) {
      const int64_t p = c0 + tid;
      a.cell[p] = sCell[tid];
#pragma unroll
      for (int d = 0; d < DIM; ++d) a.off[d][p] = sOff[d * kThreads + tid];
#pragma unroll
      for (int d = 0; d < 3; ++d) a.u[d][p] = sU[d * kThreads + tid];
    }
    if constexpr (kSettled && MID) {
      const int nq = *(volatile int *)dq.tail;  // read by every thread after the barrier above
      const int inc = nq - q_prev;
      if (nq + inc + inc / 2 > kQCap) {
        if (tid == 0) atomicAdd(a.q_jobs, (unsigned long long)nq);
        dq_drain<R, DIM, ORDER>(a, acc, dq, nq > kQCap ? kQCap : nq, sCell, true);
        q_prev = 0;
      } else {
        q_prev = nq;
      }
    }
  }
  if constexpr (kSettled) {
    // the deferred jobs still queued (the chunk loop ended on a barrier)
    const int nq = *(volatile int *)dq.tail;
    if (tid == 0 && nq > 0) atomicAdd(a.q_jobs, (unsigned long long)nq);
    dq_drain<R, DIM, ORDER>(a, acc, dq, nq > kQCap ? kQCap : nq, sCell, false);
  }

  if (my_clamp) atomicAdd(&s_clamp, my_clamp);
  if (my_absorbed) atomicAdd(&a.ctr->absorbed, (unsigned long long)my_absorbed);
  if (sizeof(R) == 4) {
    for (int o = 16; o > 0; o >>= 1) my_q1 += __shfl_down_sync(0xffffffffu, my_q1, o);
    if ((tid & 31) == 0 && my_q1 > 0.f) atomicAdd(&s_q1, my_q1);
  }
  __syncthreads();
  if (sizeof(R) == 4 && tid == 0) {
    // bound inputs for the next step (the item keeps its slots until the next sort)
    a.tq[2 * wi] = s_wsum;
    a.tq[2 * wi + 1] = s_q1 * 1.0001f;
  }

  // ---- flush the J window into global J ----
  if (sizeof(R) == 4 && (a.n[0] & 3) == 0) {
    // FP32 with rows of a multiple of four cells: runs of four nodes along x
    // aligned in global memory, one vector reduction each (every element
    // added atomically); a run reaching past the window's x ends adds zeros
    // there.  A run never straddles the periodic seam.
    const int xs = t0[0] - G::D - G::LOJ;          // the window's first node, global x (unwrapped)
    const int a0 = xs - (((xs % 4) + 4) & 3);      // the multiple of 4 at or below it
    constexpr int NG = (G::JX + 6) / 4;            // runs per window row (the last may start past it)
    for (int q = tid; q < NG * G::JY * G::JZ; q += kThreads) {
      const int m = q % NG, row = q / NG;
      const int y = row % G::JY, z = row / G::JY;
      const int wx0 = a0 + 4 * m - xs;  // window x of the run's first node
      if (wx0 >= G::JX) continue;
      const int gi = wrap_near(a0 + 4 * m, a.n[0]);
      const int gj = wrap_near(t0[1] - G::D - G::LOJ + y, a.n[1]);
      const int gk = DIM == 3 ? wrap_near(t0[2] - G::D - G::LOJ + z, a.n[2]) : 0;
      const int64_t g = gi + (int64_t)a.n[0] * (gj + (int64_t)a.n[1] * gk);
      const int wrow = z * G::JP + y * G::JX;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int wx = wx0 + e;
          v[e] = (wx >= 0 && wx < G::JX) ? (float)acc.get(c, wrow + wx) : 0.f;
        }
        if (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a.J[c] + g), "f"(v[0]), "f"(v[1]),
                       "f"(v[2]), "f"(v[3])
                       : "memory");
      }
    }
  } else {
    for (int q = tid; q < G::JN; q += kThreads) {
      const int z = q / G::JP;
      const int x = (q - z * G::JP) % G::JX;
      const int y = (q - z * G::JP) / G::JX;
      if (y >= G::JY) continue;  // plane padding
      const int gi = wrap_near(t0[0] - G::D - G::LOJ + x, a.n[0]);
      const int gj = wrap_near(t0[1] - G::D - G::LOJ + y, a.n[1]);
      const int gk = DIM == 3 ? wrap_near(t0[2] - G::D - G::LOJ + z, a.n[2]) : 0;
      const int64_t g = gi + (int64_t)a.n[0] * (gj + (int64_t)a.n[1] * gk);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R v = acc.get(c, q);
        if (v != R(0)) atomicAdd(a.J[c] + g, v);
      }
    }
  }
  if (tid == 0 && s_clamp) atomicAdd(&a.ctr->clamped, (unsigned long long)s_clamp);
}

// Particles deferred by the tile kernel: the same gather / Boris / move /
// Esirkepov arithmetic, reading E, B from and adding J to global memory with
// periodic index wrapping.
template <class R, int DIM, int ORDER>
__global__ void __launch_bounds__(kThreads) k_push_escaped(const PushArgs<R> a) {
  constexpr int NS = ORDER + 1;
  constexpr int NW = ORDER + 2;
  const unsigned long long nesc = *a.esc_count;
  unsigned my_clamp = 0;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < nesc;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t p = a.esc_list[q];
    const int c = a.cell[p] & ~kEscFlag;
    int ci[3];
    ci[0] = c % a.n[0];
    ci[1] = (c / a.n[0]) % a.n[1];
    ci[2] = DIM == 3 ? c / (a.n[0] * a.n[1]) : 0;
    R f[3], u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      f[d] = d < DIM ? a.off[d][p] : R(0);
      u[d] = a.u[d][p];
    }
    GatherAxis<R, ORDER> ga[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ga[d].set(f[d], a.ec);
    const int64_t sy = a.n[0], sz = (int64_t)a.n[0] * a.n[1];
    auto fetch = [&](const R *F, const bool dual[3]) {
      R acc = R(0);
      for (int cz = 0; cz < (DIM == 3 ? NS : 1); ++cz) {
        const int kz = DIM == 3 ? wrapi(ci[2] + (dual[2] ? ga[2].reld : ga[2].relp) + cz, a.n[2]) : 0;
        const R wz = DIM == 3 ? (dual[2] ? ga[2].wd[cz] : ga[2].wp[cz]) : R(1);
        for (int by = 0; by < NS; ++by) {
          const int ky = wrapi(ci[1] + (dual[1] ? ga[1].reld : ga[1].relp) + by, a.n[1]);
          const R wy = dual[1] ? ga[1].wd[by] : ga[1].wp[by];
          for (int ax = 0; ax < NS; ++ax) {
            const int kx = wrapi(ci[0] + (dual[0] ? ga[0].reld : ga[0].relp) + ax, a.n[0]);
            const R wx = dual[0] ? ga[0].wd[ax] : ga[0].wp[ax];
            acc += F[kx + sy * ky + sz * kz] * (wx * wy * wz);
          }
        }
      }
      return acc;
    };
    const bool sE[3][3] = {{true, false, false}, {false, true, false}, {false, false, true}};
    const bool sB[3][3] = {{false, true, true}, {true, false, true}, {true, true, false}};
    R E[3], B[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      E[k] = fetch(a.E[k], sE[k]);
      B[k] = fetch(a.B[k], sB[k]);
    }
    R fn[3], ig;
    int s[3];
    push_move<R, ORDER, DIM>(a, u, E, B, f, fn, s, ig, my_clamp);
    DepositAxis<R, ORDER> da[3];
    da[0].set(f[0], s[0], fn[0]);
    da[1].set(f[1], s[1], fn[1]);
    if (DIM == 3) da[2].set(f[2], s[2], fn[2]);
    else da[2].zero();
    const R wq = a.w[p];
    // global Esirkepov with wrapped node indices
    R P[3][NW - 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R run = R(0);
      for (int k = 0; k < NW - 2; ++k) {
        run += da[d].DS[k];
        P[d][k] = a.jfac[d] * wq * run;
      }
      P[d][NW - 2] = -a.jfac[d] * wq * da[d].DS[NW - 1];  // the full running sum vanishes
    }
    int gx[NW], gy[NW], gz[NW];
    for (int k = 0; k < NW; ++k) {
      gx[k] = wrapi(ci[0] + da[0].rel + k, a.n[0]);
      gy[k] = wrapi(ci[1] + da[1].rel + k, a.n[1]);
      gz[k] = DIM == 3 ? wrapi(ci[2] + da[2].rel + k, a.n[2]) : 0;
    }
    const DepositAxis<R, ORDER> &X = da[0], &Y = da[1], &Z = da[2];
    if (DIM == 3) {
      for (int cz = 0; cz < NW; ++cz)
        for (int by = 0; by < NW; ++by)
          for (int ax = 0; ax < NW; ++ax) {
            const int64_t g = gx[ax] + sy * gy[by] + sz * gz[cz];
            const R bx = Y.S0[by] * (Z.S0[cz] + R(0.5) * Z.DS[cz]) + Y.DS[by] * (R(0.5) * Z.S0[cz] + Z.DS[cz] * R(1.0 / 3.0));
            const R byy = Z.S0[cz] * (X.S0[ax] + R(0.5) * X.DS[ax]) + Z.DS[cz] * (R(0.5) * X.S0[ax] + X.DS[ax] * R(1.0 / 3.0));
            const R bz = X.S0[ax] * (Y.S0[by] + R(0.5) * Y.DS[by]) + X.DS[ax] * (R(0.5) * Y.S0[by] + Y.DS[by] * R(1.0 / 3.0));
            if (ax < NW - 1) atomicAdd(a.J[0] + g, P[0][ax] * bx);
            if (by < NW - 1) atomicAdd(a.J[1] + g, P[1][by] * byy);
            if (cz < NW - 1) atomicAdd(a.J[2] + g, P[2][cz] * bz);
          }
    } else {
      const R qwvz = a.qz * wq * u[2] * ig;
      for (int by = 0; by < NW; ++by)
        for (int ax = 0; ax < NW; ++ax) {
          const int64_t g = gx[ax] + sy * gy[by];
          const R hy = Y.S0[by] + R(0.5) * Y.DS[by];
          const R ty = R(0.5) * Y.S0[by] + Y.DS[by] * R(1.0 / 3.0);
          const R hx = X.S0[ax] + R(0.5) * X.DS[ax];
          if (ax < NW - 1) atomicAdd(a.J[0] + g, P[0][ax] * hy);
          if (by < NW - 1) atomicAdd(a.J[1] + g, P[1][by] * hx);
          atomicAdd(a.J[2] + g, qwvz * (X.S0[ax] * hy + X.DS[ax] * ty));
        }
    }
    if (outside_walls<R>(a.absorb, ci[0] + s[0], fn[0], a.n[0])) {
      a.cell[p] = -1;  // removed at an absorbing wall after depositing its move
      atomicAdd(&a.ctr->absorbed, 1ull);
      continue;
    }
    int nc[3] = {ci[0], ci[1], ci[2]};
#pragma unroll
    for (int d = 0; d < DIM; ++d) nc[d] = wrapi(ci[d] + s[d], a.n[d]);
    a.cell[p] = nc[0] + a.n[0] * (nc[1] + a.n[1] * nc[2]);
#pragma unroll
    for (int d = 0; d < DIM; ++d) a.off[d][p] = fn[d];
#pragma unroll
    for (int d = 0; d < 3; ++d) a.u[d][p] = u[d];
  }
  if (my_clamp) atomicAdd(&a.ctr->clamped, (unsigned long long)my_clamp);
  // escaped particle-steps are counted by the host-visible counter
  if (blockIdx.x == 0 && threadIdx.x == 0 && nesc) atomicAdd(&a.ctr->escaped, nesc);
}

template <class R, int DIM, int ORDER> constexpr size_t smem_bytes() {
  using G = Geo<DIM, ORDER>;
  // E, B window; J window; staging of cell, offsets, u, w; for FP32 3D the
  // deposit jobs (a packed int per slot)
  constexpr bool split = DIM == 3 && sizeof(R) == 4;
  return (size_t)(6 * G::EN + (DIM + 4) * kThreads) * sizeof(R) + 24 * (size_t)G::JS +
         (split ? 2 : 1) * kThreads * sizeof(int32_t) +
         (sizeof(R) == 8 && DIM == 2 ? 0 : kQCap * (sizeof(int32_t) + 7 * sizeof(R)));
}

template <class R, int DIM, int ORDER>
cudaError_t launch_t(const Grid &g, void *const E[3], void *const B[3], void *const J[3], const Particles &p,
                     const int64_t *tile_start, const WorkSplit &ws, float *tq, int fresh, int32_t *esc_list,
                     unsigned long long *esc_count, double q, double m, Counters *ctr, cudaStream_t st,
                     int *nlaunch, bool mid_drain) {
  PushArgs<R> a;
  a.work_tile = ws.work_tile;
  a.work_pb = ws.work_pb;
  a.chunk = ws.chunk;
  a.tq = tq;
  a.fresh = fresh;
  a.qabs = q < 0 ? -q : q;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.E[d] = static_cast<const R *>(E[d]);
    a.B[d] = static_cast<const R *>(B[d]);
    a.J[d] = static_cast<R *>(J[d]);
    a.off[d] = static_cast<R *>(p.off[d]);
    a.u[d] = static_cast<R *>(p.u[d]);
    a.dtdx[d] = (R)(g.dt / g.dx[d]);
    a.jfac[d] = (R)(-q * g.dx[d] / g.dt);
  }
  a.ntile[0] = g.ntile[0];
  a.ntile[1] = g.ntile[1];
  a.dn0 = make_fastdiv((uint32_t)g.n[0]);
  a.dn1 = make_fastdiv((uint32_t)g.n[1]);
  a.cell = p.cell;
  a.w = static_cast<const R *>(p.w);
  a.tile_start = tile_start;
  a.esc_list = esc_list;
  a.esc_count = esc_count;
  a.q_jobs = esc_count + 1;
  a.qmh = (R)(q * g.dt / (2.0 * m));
  a.qz = (R)q;
  a.absorb = g.absorb_lo || g.absorb_hi;
  a.ec = g.gather_ec;
  a.ctr = ctr;
  constexpr size_t smem = smem_bytes<R, DIM, ORDER>();
  // the variant that drains between chunks only where it can matter (3D;
  // 2D targets queue few jobs)
  auto fn = (DIM == 3 && mid_drain) ? k_push<R, DIM, ORDER, DIM == 3> : k_push<R, DIM, ORDER, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ws.nwork > 0x7fffffff) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(esc_count, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)ws.nwork, kThreads, smem, st>>>(a);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  k_push_escaped<R, DIM, ORDER><<<nsm, kThreads, 0, st>>>(a);
  if (nlaunch) *nlaunch = 2;
  return cudaGetLastError();
}

// Charge density at the nodes for the diagnostics, rho += q w S(X-i)S(Y-j)S(Z-k),
// one block per tile like k_push, particles taken in the same lane-spread
// order (a warp's lanes about one cell apart, so that their atomics hit
// different nodes).  The block's window sums are exact fixed point, scaled
// from a bound on the tile's charge (|rho_node| <= sum |q w|), so the window
// does not depend on the order of the additions; each node then receives
// one FP64 add per tile that reaches it.  Particles more than one cell
// outside their tile add to the global array directly.
//  FP32 runs: weights and products in FP32 (their positions carry FP32
//   rounding anyway), the tile's bound scaled to 2^37 and each product split
//   into int32 words hi 2^16 + lo by FP32 FMAs, as in the push's current
//   window; each particle's contributions sum exactly to its charge (the
//   last node takes the remainder), so the total charge is conserved; a
//   tile of more than kMaxWindowSlots particles is flushed in pieces so that
//   the lo sums cannot overflow.
//  FP64 runs: weights in FP64, the bound scaled to 2^61, one 64-bit word per
//   node.
template <class R, int DIM, int ORDER>
__global__ void __launch_bounds__(kThreads)
    k_rho_tile(int n0, int n1, int n2, int ntile0, int ntile1, FastDiv dn0, FastDiv dn1, const int32_t *__restrict__ cell,
               const R *__restrict__ off0, const R *__restrict__ off1, const R *__restrict__ off2,
               const R *__restrict__ w, const int64_t *__restrict__ tile_start, double q, double *rho,
               Counters *ctr) {
  using G = Geo<DIM, ORDER>;
  constexpr int NS = ORDER + 1;
  constexpr int RX = G::EX, RY = G::EY, RZ = G::EZ;  // window: cell-1 .. cell+2 around the tile (+ drift)
  constexpr int RN = RX * RY * RZ;
  constexpr bool kF32 = sizeof(R) == 4;
  __shared__ unsigned long long win[RN];  // FP32: int32 lo words [0, RN), hi words [RN, 2 RN)
  int *wlo = reinterpret_cast<int *>(win);
  __shared__ double s_sum;
  const int t = blockIdx.x;
  const int64_t pb = tile_start[t], pe = tile_start[t + 1];
  if (pb >= pe) return;
  const int tid = threadIdx.x;
  int t0[3];
  t0[0] = (t % ntile0) * G::TX;
  t0[1] = ((t / ntile0) % ntile1) * G::TY;
  t0[2] = (t / ntile0 / ntile1) * G::TZ;
  if (tid == 0) s_sum = 0.0;
  __syncthreads();
  {
    R part = R(0);
    for (int64_t p = pb + tid; p < pe; p += kThreads)
      if (cell[p] >= 0) part += fabs(w[p]);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0 && part > R(0)) atomicAdd(&s_sum, (double)part);
  }
  __syncthreads();
  // 1.01: room for the rounding of the sum above
  const double Q = fabs(q) * s_sum * 1.01;
  int e2 = 0;
  if (Q > 0.0) frexp(Q, &e2);  // Q < 2^e2
  int K = Q > 0.0 ? (kF32 ? WinAcc<float>::kLimitLog2 : 61) - e2 : 0;
  K = K > 100 ? 100 : (K < -100 ? -100 : K);
  const double scale = ldexp(1.0, K);
  const R *offs[3] = {off0, off1, off2};
  const int nn[3] = {n0, n1, n2};
  constexpr int TT[3] = {G::TX, G::TY, G::TZ};
  const int lane = tid & 31, warp = tid >> 5;
  const int e = 8 * lane + ((warp + (lane >> 2)) & 7);  // lane-spread slot of a 256-slot chunk
  for (int64_t s0 = pb; s0 < pe; s0 += kMaxWindowSlots) {
    const int64_t se = pe - s0 < kMaxWindowSlots ? pe : s0 + kMaxWindowSlots;
    for (int i = tid; i < (kF32 ? 2 * RN : RN); i += kThreads) {
      if (kF32) wlo[i] = 0;
      else win[i] = 0ull;
    }
    __syncthreads();
    for (int64_t c0 = s0; c0 < se; c0 += kThreads) {
      const int64_t p = c0 + e;
      if (p >= se) continue;
      const int c = cell[p];
      if (c < 0) continue;
      const uint32_t r0 = dn0.div((uint32_t)c);
      const int ci[3] = {c - (int)r0 * n0, DIM == 3 ? (int)(r0 - dn1.div(r0) * n1) : (int)r0,
                         DIM == 3 ? (int)dn1.div(r0) : 0};
      int l[3] = {0, 0, 0};
      bool inw = true;
      int base[3] = {0, 0, 0};
      R wt[3][NS];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (d >= DIM) {
          wt[d][0] = R(1);
          for (int k = 1; k < NS; ++k) wt[d][k] = R(0);
          continue;
        }
        int dl = ci[d] - t0[d];
        if (dl > TT[d] - 1 + G::D) dl -= nn[d];
        if (dl < -G::D) dl += nn[d];
        l[d] = dl;
        inw = inw && dl >= -G::D && dl <= TT[d] - 1 + G::D;
        const R f = offs[d][p];
        if (ORDER == 2) {
          const int h = f >= R(0.5);
          const R dd = f - R(h), a = R(0.5) - dd, b = R(0.5) + dd;
          wt[d][0] = R(0.5) * a * a;
          wt[d][1] = R(0.75) - dd * dd;
          wt[d][NS - 1] = R(0.5) * b * b;
          base[d] = h - 1;
        } else {
          wt[d][0] = R(1) - f;
          wt[d][NS - 1] = f;
          base[d] = 0;
        }
      }
      // q w S_x, in window units (2^K) for particles in the window
      const R qw = inw ? (R)(q * scale) * w[p] : (R)q * w[p];
      R qwx[NS];
#pragma unroll
      for (int kx = 0; kx < NS; ++kx) qwx[kx] = qw * wt[0][kx];
      // FP32 runs: the particle's last node takes its whole charge minus what
      // the other nodes received, so that its integer contributions sum to
      // the integer q w 2^K exactly (and a particle outside the window adds
      // q w minus the other FP64 products): the FP32 weights need not sum to
      // one exactly for the total charge to be conserved.
      int hi_t = 0, lo_t = 0;
      double v_t = 0.0;
      if (kF32) {
        if (inw) {
          const float y = qw + WinAcc<float>::kMagicHi;  // |q w 2^K| < 2^37: hi 2^16 + lo as below
          hi_t = __float_as_int(y) - __float_as_int(WinAcc<float>::kMagicHi);
          lo_t = __float_as_int((qw - (y - WinAcc<float>::kMagicHi)) + WinAcc<float>::kMagic) -
                 __float_as_int(WinAcc<float>::kMagic);
        } else {
          v_t = (double)qw;
        }
      }
#pragma unroll
      for (int kz = 0; kz < (DIM == 3 ? NS : 1); ++kz)
#pragma unroll
        for (int ky = 0; ky < NS; ++ky) {
          const R wyz = wt[1][ky] * wt[2][kz];
#pragma unroll
          for (int kx = 0; kx < NS; ++kx) {
            const bool last = kF32 && kx == NS - 1 && ky == NS - 1 && kz == (DIM == 3 ? NS - 1 : 0);
            if (inw) {
              const int ix = l[0] + base[0] + kx + G::D + G::LOE;
              const int iy = l[1] + base[1] + ky + G::D + G::LOE;
              const int iz = DIM == 3 ? l[2] + base[2] + kz + G::D + G::LOE : 0;
              if (!PIC_CHECK(ix >= 0 && ix < RX && iy >= 0 && iy < RY && iz >= 0 && iz < RZ, ctr)) continue;
              const int at = ix + RX * (iy + RY * iz);
              if constexpr (kF32) {
                // X = qwx wyz 2^K < 2^37 as hi 2^16 + lo, the push's split
                int hi, lo;
                if (last) {
                  hi = hi_t;
                  lo = lo_t;
                  const int carry = (lo + 32768) >> 16;  // back to |lo| <= 2^15
                  hi += carry;
                  lo -= carry * 65536;
                } else {
                  const float y = fmaf(qwx[kx], wyz, WinAcc<float>::kMagicHi);
                  const float r = y - WinAcc<float>::kMagicHi;
                  const float lf = fmaf(qwx[kx], wyz, -r);
                  hi = __float_as_int(y) - __float_as_int(WinAcc<float>::kMagicHi);
                  lo = __float_as_int(lf + WinAcc<float>::kMagic) - __float_as_int(WinAcc<float>::kMagic);
                  hi_t -= hi;
                  lo_t -= lo;
                }
                atomicAdd(wlo + at, lo);
                atomicAdd(wlo + RN + at, hi);
              } else {
                atomicAdd(&win[at], (unsigned long long)__double2ll_rn(qwx[kx] * wyz));
              }
            } else {
              double v = (double)qwx[kx] * (double)wyz;
              if (last) v = v_t;
              else v_t -= v;
              const int gi = wrapi(ci[0] + base[0] + kx, n0), gj = wrapi(ci[1] + base[1] + ky, n1);
              const int gk = DIM == 3 ? wrapi(ci[2] + base[2] + kz, n2) : 0;
              atomicAdd(rho + gi + (int64_t)n0 * (gj + (int64_t)n1 * gk), v);
            }
          }
        }
    }
    __syncthreads();
    for (int i = tid; i < RN; i += kThreads) {
      const long long X = kF32 ? (long long)wlo[RN + i] * 65536 + wlo[i] : (long long)win[i];
      if (X == 0) continue;
      const int x = i % RX, y = (i / RX) % RY, z = i / (RX * RY);
      const int gi = wrap_near(t0[0] - G::D - G::LOE + x, n0);
      const int gj = wrap_near(t0[1] - G::D - G::LOE + y, n1);
      const int gk = DIM == 3 ? wrap_near(t0[2] - G::D - G::LOE + z, n2) : 0;
      atomicAdd(rho + gi + (int64_t)n0 * (gj + (int64_t)n1 * gk), (double)X / scale);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_rho_tiled(const Grid &g, const Particles &p, const int64_t *tile_start, double q, double *rho,
                             Counters *ctr, cudaStream_t st) {
  if (g.ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  const FastDiv d0 = make_fastdiv((uint32_t)g.n[0]), d1 = make_fastdiv((uint32_t)g.n[1]);
  const unsigned nb = (unsigned)g.ntiles;
#define PIC_RHO_CASE(K, R, D, O)                                                                                 \
  case K:                                                                                                        \
    k_rho_tile<R, D, O><<<nb, kThreads, 0, st>>>(g.n[0], g.n[1], g.n[2], g.ntile[0], g.ntile[1], d0, d1, p.cell, \
                                                  static_cast<const R *>(p.off[0]), static_cast<const R *>(p.off[1]), \
                                                  static_cast<const R *>(p.off[2]), static_cast<const R *>(p.w),  \
                                                  tile_start, q, rho, ctr);                                      \
    break;
  switch ((g.prec == 1 ? 100 : 0) + g.dims * 10 + g.order) {
    PIC_RHO_CASE(21, float, 2, 1)
    PIC_RHO_CASE(22, float, 2, 2)
    PIC_RHO_CASE(31, float, 3, 1)
    PIC_RHO_CASE(32, float, 3, 2)
    PIC_RHO_CASE(121, double, 2, 1)
    PIC_RHO_CASE(122, double, 2, 2)
    PIC_RHO_CASE(131, double, 3, 1)
    PIC_RHO_CASE(132, double, 3, 2)
    default: return cudaErrorInvalidValue;
  }
#undef PIC_RHO_CASE
  return cudaGetLastError();
}

// Tile shape compiled into the push kernel for a given dimensionality.
void push_tile_shape(int dims, int tile[3]) {
  tile[0] = dims == 3 ? Geo<3, 2>::TX : Geo<2, 2>::TX;
  tile[1] = dims == 3 ? Geo<3, 2>::TY : Geo<2, 2>::TY;
  tile[2] = dims == 3 ? Geo<3, 2>::TZ : 1;
}

size_t push_smem_bytes(const Grid &g) {
  const int key = (g.prec == 1 ? 100 : 0) + g.dims * 10 + g.order;
  switch (key) {
    case 21: return smem_bytes<float, 2, 1>();
    case 22: return smem_bytes<float, 2, 2>();
    case 31: return smem_bytes<float, 3, 1>();
    case 32: return smem_bytes<float, 3, 2>();
    case 121: return smem_bytes<double, 2, 1>();
    case 122: return smem_bytes<double, 2, 2>();
    case 131: return smem_bytes<double, 3, 1>();
    case 132: return smem_bytes<double, 3, 2>();
    default: return 0;
  }
}

cudaError_t launch_push(const Grid &g, void *const E[3], void *const B[3], void *const J[3], const Particles &p,
                        const int64_t *tile_start, const WorkSplit &ws, float *tq, int fresh, int32_t *esc_list,
                        unsigned long long *esc_count, double q, double m, Counters *ctr, cudaStream_t st,
                        int *nlaunch, int mid_drain) {
  const int key = (g.prec == 1 ? 100 : 0) + g.dims * 10 + g.order;
#define PIC_PUSH_CASE(K, R, D, O)                                                                        \
  case K:                                                                                                \
    return launch_t<R, D, O>(g, E, B, J, p, tile_start, ws, tq, fresh, esc_list, esc_count, q, m, ctr, st, \
                             nlaunch, mid_drain != 0);
  switch (key) {
    PIC_PUSH_CASE(21, float, 2, 1)
    PIC_PUSH_CASE(22, float, 2, 2)
    PIC_PUSH_CASE(31, float, 3, 1)
    PIC_PUSH_CASE(32, float, 3, 2)
    PIC_PUSH_CASE(121, double, 2, 1)
    PIC_PUSH_CASE(122, double, 2, 2)
    PIC_PUSH_CASE(131, double, 3, 1)
    PIC_PUSH_CASE(132, double, 3, 2)
    default: return cudaErrorInvalidValue;
  }
#undef PIC_PUSH_CASE
}

}  // namespace pic
