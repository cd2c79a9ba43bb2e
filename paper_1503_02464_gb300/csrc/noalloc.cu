// pic_field_energy_noalloc: the FP64 field-energy reduction of pic_diag,
// for callers that must not allocate device memory.
//
// The paper has no counterpart; this is a library service.  cudaMalloc and
// cudaFree can synchronise the whole device and enter the driver's allocator,
// which some callers cannot afford: code running inside an application whose
// device memory is owned by its own pool or fixed budget, code called from a
// host callback or a latency-critical thread, or code that must leave an
// enclosing framework's allocator untouched.  This entry point therefore uses
// only caller-owned inputs/outputs and the file-scope scratch array below.
//
// Scratch: g_energy_scratch holds 2 doubles per reduction block (at most
// kMaxPartials blocks of kChunk cells, so at most kMaxCells cells per call)
// plus 2 result slots.  Every GPU that loads the library keeps these
// 2 * (kMaxPartials + 1) doubles (32 KB) until the process exits.  Each call
// overwrites exactly the slots it later reads, so nothing needs zeroing; all
// calls share the array, so calls that overlap on the GPU (different streams,
// or different host threads on one device) race and must be serialised by
// the caller.
//
// In host code `g_energy_scratch` names a host-side stand-in, not device
// memory; its device address is looked up once per device with
// cudaGetSymbolAddress (first call on that device, with it current), so the
// first call on each device should come before any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "pic.h"
#include "pic_device.cuh"
#include "pic_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 16384;       // cells per reduction block
constexpr int kMaxPartials = 2048;      // reduction blocks per call
constexpr int64_t kMaxCells = kChunk * kMaxPartials;  // 33,554,432 cells
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[2 * kMaxPartials + 2];

std::mutex g_mu;
double *g_scratch_dev[kMaxDevices] = {};

template <class R>
__global__ void __launch_bounds__(kThreads)
    k_energy_partials(const R *__restrict__ e0, const R *__restrict__ e1, const R *__restrict__ e2,
                      const R *__restrict__ b0, const R *__restrict__ b1, const R *__restrict__ b2, int64_t ncell,
                      double *__restrict__ partials) {
  __shared__ double sh[32];
  const int64_t beg = blockIdx.x * kChunk;
  const int64_t end = beg + kChunk < ncell ? beg + kChunk : ncell;
  double se = 0.0, sb = 0.0;
  for (int64_t c = beg + threadIdx.x; c < end; c += kThreads) {
    const double ex = e0[c], ey = e1[c], ez = e2[c];
    const double bx = b0[c], by = b1[c], bz = b2[c];
    se += ex * ex + ey * ey + ez * ez;
    sb += bx * bx + by * by + bz * bz;
  }
  const double te = pic::block_sum(se, sh);
  const double tb = pic::block_sum(sb, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = te;
    partials[2 * blockIdx.x + 1] = tb;
  }
}

// One block: fixed-order sum of the partials -> out[0..1].
__global__ void __launch_bounds__(kThreads)
    k_energy_final(const double *__restrict__ partials, int nblocks, double half_dv, double *__restrict__ out) {
  __shared__ double sh[32];
  double se = 0.0, sb = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    se += partials[2 * b];
    sb += partials[2 * b + 1];
  }
  const double te = pic::block_sum(se, sh);
  const double tb = pic::block_sum(sb, sh);
  if (threadIdx.x == 0) {
    out[0] = half_dv * te;
    out[1] = half_dv * tb;
  }
}

int scratch_for_current_device(double **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    pic::set_global_error(std::string("pic_field_energy_noalloc: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    pic::set_global_error("pic_field_energy_noalloc: device ordinal above 63");
    return PIC_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || !p) {
      pic::set_global_error(std::string("pic_field_energy_noalloc: cudaGetSymbolAddress failed: ") +
                            cudaGetErrorString(e));
      return PIC_ECUDA;
    }
    g_scratch_dev[dev] = static_cast<double *>(p);
  }
  *ptr = g_scratch_dev[dev];
  return PIC_OK;
}

}  // namespace

extern "C" int pic_field_energy_noalloc(int precision, const void *const E[3], const void *const B[3], int64_t ncell,
                                        double cell_volume, double *out, int mem_kind, void *stream) {
  if (precision != PIC_FP32 && precision != PIC_FP64) {
    pic::set_global_error("pic_field_energy_noalloc: precision must be PIC_FP32 or PIC_FP64");
    return PIC_EINVAL;
  }
  if (!E || !B || !out || !E[0] || !E[1] || !E[2] || !B[0] || !B[1] || !B[2]) {
    pic::set_global_error("pic_field_energy_noalloc: NULL array");
    return PIC_EINVAL;
  }
  if (ncell < 1 || ncell > kMaxCells) {
    pic::set_global_error("pic_field_energy_noalloc: ncell must be in [1, 33554432] (the size of its static "
                          "scratch); use pic_diag for larger grids");
    return PIC_EINVAL;
  }
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) {
    pic::set_global_error("pic_field_energy_noalloc: bad mem_kind");
    return PIC_EINVAL;
  }
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != PIC_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nblocks = (int)((ncell + kChunk - 1) / kChunk);
  if (precision == PIC_FP64) {
    auto c = [](const void *v) { return static_cast<const double *>(v); };
    k_energy_partials<double><<<nblocks, kThreads, 0, st>>>(c(E[0]), c(E[1]), c(E[2]), c(B[0]), c(B[1]), c(B[2]),
                                                             ncell, scratch);
  } else {
    auto c = [](const void *v) { return static_cast<const float *>(v); };
    k_energy_partials<float><<<nblocks, kThreads, 0, st>>>(c(E[0]), c(E[1]), c(E[2]), c(B[0]), c(B[1]), c(B[2]),
                                                            ncell, scratch);
  }
  double *result = mem_kind == PIC_MEM_DEVICE ? out : scratch + 2 * kMaxPartials;
  k_energy_final<<<1, kThreads, 0, st>>>(scratch, nblocks, 0.5 * cell_volume, result);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mem_kind == PIC_MEM_HOST) {
    e = cudaMemcpyAsync(out, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    pic::set_global_error(std::string("pic_field_energy_noalloc: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  return PIC_OK;
}
