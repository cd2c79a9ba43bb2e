// Output capture kernels: the device side of the output manager (§3.1 of
// the paper: reduced-dimension outputs -- a plane of a 3D run, a line of a
// multidimensional one -- and sub-domain outputs, restricted in time to a
// window and a frequency).  A capture copies one field on a box of grid
// positions, or the particles of one species inside a box of cells, into a
// frame of a device buffer owned by the request.
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

namespace {

int out_blocks(int64_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)nsm * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// Field box [lo, hi) -> FP64 frame, x fastest.
template <class R>
__global__ void __launch_bounds__(256) k_out_field(const R *__restrict__ f, int n0, int n1, OutBox b,
                                                   double *__restrict__ out) {
  const int bx = b.hi[0] - b.lo[0], by = b.hi[1] - b.lo[1], bz = b.hi[2] - b.lo[2];
  const int64_t nb = (int64_t)bx * by * bz;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % bx);
    const int64_t r = q / bx;
    const int j = (int)(r % by);
    const int k = (int)(r / by);
    const int64_t c = (int64_t)(b.lo[0] + i) + (int64_t)n0 * ((b.lo[1] + j) + (int64_t)n1 * (b.lo[2] + k));
    out[q] = (double)f[c];
  }
}

// Particles whose cell lies in the box -> records of 8 doubles (x, y, z,
// ux, uy, uz, w, id) in global units.  The slot of a record comes from a
// warp-aggregated atomic counter, so the record order is not defined; the
// counter keeps counting past `cap` (records beyond it are not written).
template <class R>
__global__ void __launch_bounds__(256)
    k_out_particles(int dims, int n0, int n1, double dx0, double dx1, double dx2, Particles p,
                    const int64_t *__restrict__ d_count, OutBox b, double *__restrict__ out,
                    unsigned long long *__restrict__ count, int64_t cap) {
  const int64_t n = *d_count;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;  // whole warps take part in the vote
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nround; q += stride) {
    bool in = false;
    int i = 0, j = 0, k = 0;
    if (q < n) {
      const int c = p.cell[q];
      if (c >= 0) {
        i = c % n0;
        const int r = c / n0;
        j = r % n1;
        k = r / n1;
        in = i >= b.lo[0] && i < b.hi[0] && j >= b.lo[1] && j < b.hi[1] && k >= b.lo[2] && k < b.hi[2];
      }
    }
    const unsigned vote = __ballot_sync(0xffffffffu, in);
    if (!vote) continue;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(vote) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(vote));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!in) continue;
    const unsigned long long slot = base + __popc(vote & ((1u << lane) - 1u));
    if ((int64_t)slot >= cap) continue;
    double *rec = out + 8 * slot;
    rec[0] = ((double)i + (double)static_cast<const R *>(p.off[0])[q]) * dx0;
    rec[1] = ((double)j + (double)static_cast<const R *>(p.off[1])[q]) * dx1;
    rec[2] = dims == 3 ? ((double)k + (double)static_cast<const R *>(p.off[2])[q]) * dx2 : 0.0;
    rec[3] = (double)static_cast<const R *>(p.u[0])[q];
    rec[4] = (double)static_cast<const R *>(p.u[1])[q];
    rec[5] = (double)static_cast<const R *>(p.u[2])[q];
    rec[6] = (double)static_cast<const R *>(p.w)[q];
    rec[7] = (double)p.id[q];
  }
}

}  // namespace

cudaError_t launch_out_field(const Grid &g, const void *f, bool f64, const OutBox &b, double *out, cudaStream_t st) {
  const int64_t nb = (int64_t)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
  const int nbk = out_blocks(nb);
  if (f64 || g.prec == 1)
    k_out_field<double><<<nbk, 256, 0, st>>>(static_cast<const double *>(f), g.n[0], g.n[1], b, out);
  else
    k_out_field<float><<<nbk, 256, 0, st>>>(static_cast<const float *>(f), g.n[0], g.n[1], b, out);
  return cudaGetLastError();
}

cudaError_t launch_out_particles(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax,
                                 const OutBox &b, double *out, unsigned long long *count, int64_t cap,
                                 cudaStream_t st) {
  const int nbk = out_blocks(nmax);
  if (g.prec == 1)
    k_out_particles<double><<<nbk, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.dx[0], g.dx[1], g.dx[2], p, d_count, b,
                                                 out, count, cap);
  else
    k_out_particles<float><<<nbk, 256, 0, st>>>(g.dims, g.n[0], g.n[1], g.dx[0], g.dx[1], g.dx[2], p, d_count, b,
                                                out, count, cap);
  return cudaGetLastError();
}

}  // namespace pic
