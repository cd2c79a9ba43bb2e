// Host runtime and C ABI of libpic.so (declared in include/pic.h).
//
// Owns the device state of one simulation (fields, per-species particle
// buffers, sort scratch, counters), orders the kernels of a PIC step on the
// caller's stream, and converts between the caller's FP64 global view and the
// library's (cell, offset) particle storage.
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "pic.h"
#include "pic_internal.h"

using pic::Counters;
using pic::Grid;
using pic::Particles;

namespace {

constexpr int kMaxSpecies = 8;

struct Species {
  double q = 0, m = 1;
  int64_t capacity = 0;         // particles the caller may load
  int64_t slots = 0;            // allocated slots: capacity + tile padding
  Particles buf[2] = {};
  int cur = 0;
  int64_t *d_count = nullptr;   // slots in use (device)
  int64_t h_count = 0;          // host mirror, valid while !stepped_since_count
  int32_t *rank = nullptr;
  int64_t *tile_start = nullptr;
  pic::WorkSplit work;          // push work items (tile pieces of at most work.chunk slots)
  float *tq = nullptr;          // per-item deposit bound carried between pushes
  // escapes of the last push, read back without blocking (adaptive sort)
  unsigned long long *esc_host = nullptr;  // page-locked: [0] escapes, [1] deferred deposit jobs
  cudaEvent_t esc_ev = nullptr;
  bool esc_pending = false;
  bool mid_drain = false;       // push variant draining its job queue between chunks
  bool fast = false;            // the last escape count read was above 1/8 of the early-sort threshold
  int count_age = 0;            // steps since an escape count was last read
  int64_t esc_step = -1;        // step of the push whose escape count is being read back
  bool fresh = true;            // sorted since the last push
  bool need_sort = true;
  int64_t sorted_at = -1;  // step count at the last sort
  int64_t sorts = 0;       // sorts so far (names the slot order in effect)
};

struct TimerRec {
  int cls;
  cudaEvent_t a, b;
};

// Device copy of one species' particle state (and its slot count).
struct PCopy {
  Particles p{};
  int64_t *count = nullptr;
  // Tape entries: the work items of the sort in effect (tiled = false when
  // the species was unsorted at the copy).  meta is this copy's own buffer;
  // work_pb, tile_start, work_tile point to it or, when the previous tape
  // entry was recorded under the same sort, to that entry's arrays.
  void *meta = nullptr;
  const int32_t *work_tile = nullptr;
  const int64_t *work_pb = nullptr;
  const int64_t *tile_start = nullptr;
  int64_t nwork = 0, chunk = 0, sorts = -1;
  bool tiled = false;
};

// Full simulation state at a step boundary (checkpoint) or at the start of a
// recorded step after its sort (tape entry).
struct Snapshot {
  void *mem = nullptr;  // the one allocation holding everything below
  PCopy sp[kMaxSpecies];
  void *E[3] = {}, *B[3] = {};
  int64_t step = -1;
  int nsp = 0;  // species the buffers were sized for
  bool allocated = false;
};

// Adjoint arrays of one species, indexed by particle id.
struct SpeciesAdjoint {
  void *lx[3] = {}, *lu[3] = {};
  double *lw = nullptr;
};

// One output request (§3.1 output manager) and the frames it holds.
struct OutputReq {
  pic_output_t req{};
  bool active = false;
  double *buf = nullptr;                  // max_frames * frame_doubles
  unsigned long long *found = nullptr;    // particles found per frame (device)
  int64_t frame_doubles = 0;
  std::vector<int64_t> steps;             // completed steps at each frame
  int64_t dropped = 0;
};

std::string g_create_error;

}  // namespace

struct pic_handle {
  pic_config cfg;
  Grid g;
  cudaStream_t st = nullptr;
  size_t rsize = 4;
  void *E[3] = {}, *B[3] = {}, *J[3] = {};
  double *rho_bg = nullptr, *rho = nullptr, *rho_prev = nullptr, *f64 = nullptr, *red = nullptr;
  int64_t rho_prev_step = -2;
  int32_t *keys = nullptr;
  int64_t *tile_tmp = nullptr;
  double *mur = nullptr;  // Mur wall planes (8 * n1 * n2)
  double *laser_prof = nullptr;  // laser profile P at the wall rows of the polarised component (n1 * n2)
  pic::Laser laser{};
  unsigned long long *esc_count = nullptr;
  Counters *ctr = nullptr;
  unsigned long long *bad = nullptr;
  Species sp[kMaxSpecies];
  int nsp = 0;
  int64_t step = 0;
  int64_t launches = 0;
  int64_t adaptive_sorts = 0;  // sorts triggered by escapes rather than by the cadence
  int64_t mid_drain_pushes = 0;  // species pushes launched with the between-chunk drain variant
  std::string err;
  bool profiling = false;
  std::vector<TimerRec> timers;
  std::vector<cudaEvent_t> event_pool;
  // differentiable runs
  std::vector<Snapshot> ckpt;
  // Two tape buffers: the reverse sweep of one segment (on st_adj) runs
  // while the next segment is recomputed and recorded into the other (on st).
  std::vector<Snapshot> tapes[2];
  int tape_buf = 1;  // the buffer last begun (recorded, then reversed)
  int tape_len = 0;
  bool taping = false;
  cudaStream_t st_adj = nullptr;  // the adjoint kernels' stream
  cudaEvent_t tape_free[2] = {};  // on st_adj: the last reversal of each tape buffer has run
  cudaEvent_t ev_main = nullptr;  // on st: what an adjoint step must wait for
  cudaEvent_t ev_adj = nullptr;   // on st_adj: what work on st touching the adjoint state must wait for
  bool adj_ready = false;
  int64_t id_cap = 0;
  void *lE[3] = {}, *lB[3] = {}, *lJ[3] = {};
  double *pend = nullptr, *da0 = nullptr, *objF = nullptr;
  double *adj_stage = nullptr;  // FP64 staging of id-indexed adjoint arrays (id_cap doubles)
  unsigned long long *adj_err = nullptr;
  unsigned long long *adj_esc = nullptr;  // particle adjoints on the global-memory path since pic_adjoint_begin
  SpeciesAdjoint adj[kMaxSpecies];
  // output manager
  std::vector<OutputReq> outputs;
};

namespace {

int fail(pic_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(pic_handle *h, cudaError_t e, const char *where) {
  return fail(h, PIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call, where)                         \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

cudaEvent_t take_event(pic_handle *h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// NVTX range names of the kernel classes (seen by a timeline profiler; the
// calls cost nothing when none is attached).
const char *const kClassNames[pic::KC_N] = {"sort",   "zero_j",    "push",     "yee_b", "yee_e",
                                            "boundary", "filter", "adj_field", "adj_push", "tape"};

// Scope of one kernel class within a step: an NVTX range, and CUDA events
// on the simulation stream while profiling is on (pic_profile).
struct Timed {
  pic_handle *h;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Timed(pic_handle *h_, int c, cudaStream_t s = nullptr) : h(h_), cls(c), st(s ? s : h_->st) {
    nvtxRangePushA(kClassNames[c]);
    if (h->profiling) {
      a = take_event(h);
      cudaEventRecord(a, st);
    }
  }
  ~Timed() {
    if (h->profiling) {
      cudaEvent_t b = take_event(h);
      cudaEventRecord(b, st);
      h->timers.push_back({cls, a, b});
    }
    nvtxRangePop();
  }
};

// The tape buffer being recorded or reversed.
std::vector<Snapshot> &cur_tape(pic_handle *h) { return h->tapes[h->tape_buf]; }

// Work about to be enqueued on st that reads or writes the adjoint state
// waits for the adjoint kernels enqueued so far on st_adj.
cudaError_t join_adj(pic_handle *h) {
  if (!h->st_adj) return cudaSuccess;
  cudaError_t e = cudaEventRecord(h->ev_adj, h->st_adj);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, h->ev_adj, 0);
  return e;
}

// The ordering events (created once).
cudaError_t make_tape_events(pic_handle *h) {
  cudaError_t e = cudaSuccess;
  for (auto &ev : h->tape_free)
    if (!ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (!h->ev_main && e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming);
  if (!h->ev_adj && e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_adj, cudaEventDisableTiming);
  return e;
}

// A particle buffer is one allocation holding the SoA arrays back to back
// (cell, off[0..dims), u[0..3), w, id, each 256-byte aligned), so that a
// checkpoint or tape copy is one memcpy.  `cell` is the allocation's base.
size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t particles_bytes(int64_t cap, size_t rs, int dims) {
  const size_t n = (size_t)(cap > 0 ? cap : 1);
  return align256(n * sizeof(int32_t)) + (size_t)(dims + 4) * align256(n * rs) + align256(n * sizeof(uint32_t));
}

// A sort's outputs in one allocation: work_pb[nwork], tile_start[ntiles + 1],
// work_tile[nwork].
size_t sort_meta_bytes(int64_t nwork, int64_t ntiles) {
  return sizeof(int64_t) * (size_t)(nwork + ntiles + 1) + sizeof(int32_t) * (size_t)nwork;
}

void set_sort_meta(void *base, int64_t nwork, int64_t ntiles, int64_t *&work_pb, int64_t *&tile_start,
                   int32_t *&work_tile) {
  work_pb = static_cast<int64_t *>(base);
  tile_start = work_pb + nwork;
  work_tile = reinterpret_cast<int32_t *>(tile_start + ntiles + 1);
}

void free_particles(Particles &p) {
  cudaFree(p.cell);
  p = Particles{};
}

// The SoA arrays of `cap` slots laid out from base (particles_bytes).
void carve_particles(Particles &p, char *base, int64_t cap, size_t rs, int dims) {
  const size_t n = (size_t)(cap > 0 ? cap : 1);
  p = Particles{};
  p.cell = reinterpret_cast<int32_t *>(base);
  char *q = base + align256(n * sizeof(int32_t));
  for (int d = 0; d < dims; ++d, q += align256(n * rs)) p.off[d] = q;
  for (int d = 0; d < 3; ++d, q += align256(n * rs)) p.u[d] = q;
  p.w = q;
  q += align256(n * rs);
  p.id = reinterpret_cast<uint32_t *>(q);
}

// Stream-ordered allocations (snapshots, load staging) that are freed stay
// in the device's default memory pool, up to a quarter of the device's
// memory, for reuse by later ones of this process (a process-wide pool
// attribute, set once).
void keep_pooled_memory(int dev) {
  static bool done = false;
  if (done) return;
  done = true;
  cudaMemPool_t pool;
  size_t free_b = 0, total_b = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  uint64_t keep = total_b / 4;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  cudaGetLastError();
}

// cudaMalloc that, when the device is full, first returns the memory kept
// in the default pool and tries once more.
cudaError_t dev_malloc(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaErrorMemoryAllocation) return e;
  cudaGetLastError();
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return e;
  cudaDeviceSynchronize();
  cudaMemPoolTrimTo(pool, 0);
  return cudaMalloc(p, bytes);
}

cudaError_t alloc_particles(Particles &p, int64_t cap, size_t rs, int dims) {
  char *base = nullptr;
  const cudaError_t e = dev_malloc(reinterpret_cast<void **>(&base), particles_bytes(cap, rs, dims));
  if (e != cudaSuccess) return e;
  carve_particles(p, base, cap, rs, dims);
  return cudaSuccess;
}

int check_device_errors(pic_handle *h) {
  Counters c;
  CK(h, cudaMemcpyAsync(&c, h->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st), "read counters");
  CK(h, cudaStreamSynchronize(h->st), "stream sync");
  if (c.error & pic::kErrBounds) return fail(h, PIC_EOVERFLOW, "an index outside its buffer was caught (checked build)");
  if (c.error) return fail(h, PIC_EOVERFLOW, "device-side error flags set");
  return PIC_OK;
}

// Copy a device buffer to caller memory (host or device).
int copy_out(pic_handle *h, void *dst, const void *src, size_t bytes, int mem_kind) {
  CK(h,
     cudaMemcpyAsync(dst, src, bytes, mem_kind == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     h->st),
     "copy out");
  return PIC_OK;
}

int sort_species(pic_handle *h, Species &s) {
  int nl = 0;
  Timed tm(h, pic::KC_SORT);
  CK(h,
     pic::launch_sort(h->g, s.buf[s.cur], s.buf[1 - s.cur], s.d_count, s.slots, h->keys, s.rank, s.tile_start,
                      h->tile_tmp, s.work, h->ctr, h->st, &nl),
     "sort");
  h->launches += nl;
  s.cur = 1 - s.cur;
  s.need_sort = false;
  s.sorted_at = h->step;
  s.sorts++;
  s.fresh = true;
  return PIC_OK;
}

int compute_rho(pic_handle *h, double *rho) {
  CK(h, cudaMemcpyAsync(rho, h->rho_bg, sizeof(double) * h->g.ncell, cudaMemcpyDeviceToDevice, h->st), "rho init");
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    if (s.need_sort)  // slots not grouped by tile yet (just loaded)
      CK(h, pic::launch_rho(h->g, s.buf[s.cur], s.d_count, s.slots, s.q, rho, h->st), "rho deposit");
    else
      CK(h, pic::launch_rho_tiled(h->g, s.buf[s.cur], s.tile_start, s.q, rho, h->ctr, h->st), "rho deposit");
    h->launches++;
  }
  return PIC_OK;
}

int64_t read_count(pic_handle *h, Species &s) {
  int64_t n = 0;
  cudaMemcpyAsync(&n, s.d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, h->st);
  cudaStreamSynchronize(h->st);
  s.h_count = n;
  return n;
}

void free_snapshot(Snapshot &sn, cudaStream_t st);

// One stream-ordered allocation per snapshot: E and B back to back (like
// the live fields, one copy), then per species its particle buffer, slot
// count and sort work items.  Freed snapshots return to the device's
// memory pool (kept for reuse, see pic_create), so that recording many
// steps again in a later run costs no fresh allocation.
cudaError_t alloc_snapshot(pic_handle *h, Snapshot &sn) {
  if (sn.allocated && sn.nsp == h->nsp) return cudaSuccess;
  if (sn.allocated) free_snapshot(sn, h->st);
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  size_t total = align256(6 * fb);
  for (int i = 0; i < h->nsp; ++i)
    total += particles_bytes(h->sp[i].slots, h->rsize, h->g.dims) + 256 +
             align256(sort_meta_bytes(h->sp[i].work.nwork, h->g.ntiles));
  char *base = nullptr;
  const cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), total, h->st);
  if (e != cudaSuccess) return e;
  sn.mem = base;
  sn.E[0] = base;
  for (int d = 0; d < 3; ++d) {
    sn.E[d] = base + d * fb;
    sn.B[d] = base + (3 + d) * fb;
  }
  char *q = base + align256(6 * fb);
  for (int i = 0; i < h->nsp; ++i) {
    PCopy &c = sn.sp[i];
    carve_particles(c.p, q, h->sp[i].slots, h->rsize, h->g.dims);
    q += particles_bytes(h->sp[i].slots, h->rsize, h->g.dims);
    c.count = reinterpret_cast<int64_t *>(q);
    q += 256;
    c.meta = q;
    q += align256(sort_meta_bytes(h->sp[i].work.nwork, h->g.ntiles));
  }
  sn.allocated = true;
  sn.nsp = h->nsp;
  return cudaSuccess;
}

void free_snapshot(Snapshot &sn, cudaStream_t st) {
  if (sn.mem) cudaFreeAsync(sn.mem, st);
  sn = Snapshot{};
}

// Both buffers were made by alloc_particles with `slots` slots.
cudaError_t copy_particles(pic_handle *h, const Particles &dst, int64_t *dcount, const Particles &src,
                           const int64_t *scount, int64_t slots) {
  cudaError_t e = cudaMemcpyAsync(dst.cell, src.cell, particles_bytes(slots, h->rsize, h->g.dims),
                                  cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcount, scount, sizeof(int64_t), cudaMemcpyDeviceToDevice, h->st);
  return e;
}

// Copy the live state (current particle buffers, E, B, step) into sn.  A
// tape entry (prev: the entry recorded before it, or null) also keeps the
// work items of the sort in effect, copied unless prev already holds them.
cudaError_t save_snapshot(pic_handle *h, Snapshot &sn, bool tape = false, const Snapshot *prev = nullptr) {
  cudaError_t e = alloc_snapshot(h, sn);
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  if (e == cudaSuccess) e = cudaMemcpyAsync(sn.E[0], h->E[0], 6 * fb, cudaMemcpyDeviceToDevice, h->st);
  for (int i = 0; i < h->nsp && e == cudaSuccess; ++i) {
    Species &s = h->sp[i];
    PCopy &c = sn.sp[i];
    e = copy_particles(h, c.p, c.count, s.buf[s.cur], s.d_count, s.slots);
    // the slot order is that of the last sort unless a sort is pending
    c.tiled = tape && !s.need_sort && s.work.nwork > 0;
    c.nwork = s.work.nwork;
    c.chunk = s.work.chunk;
    c.sorts = s.sorts;
    if (!c.tiled || e != cudaSuccess) continue;
    const PCopy *q = prev ? &prev->sp[i] : nullptr;
    if (q && q->tiled && q->sorts == s.sorts) {
      c.work_pb = q->work_pb;
      c.tile_start = q->tile_start;
      c.work_tile = q->work_tile;
    } else {
      e = cudaMemcpyAsync(c.meta, s.work.work_pb, sort_meta_bytes(s.work.nwork, h->g.ntiles), cudaMemcpyDeviceToDevice,
                          h->st);
      int64_t *pb = nullptr, *ts = nullptr;
      int32_t *wt = nullptr;
      set_sort_meta(c.meta, s.work.nwork, h->g.ntiles, pb, ts, wt);
      c.work_pb = pb;
      c.tile_start = ts;
      c.work_tile = wt;
    }
  }
  sn.step = h->step;
  return e;
}

void free_adjoint(pic_handle *h) {
  for (int d = 0; d < 3; ++d) {
    cudaFree(h->lE[d]);
    cudaFree(h->lB[d]);
    cudaFree(h->lJ[d]);
    h->lE[d] = h->lB[d] = h->lJ[d] = nullptr;
  }
  cudaFree(h->pend);
  cudaFree(h->da0);
  cudaFree(h->objF);
  cudaFree(h->adj_err);
  cudaFree(h->adj_stage);
  cudaFree(h->adj_esc);
  h->pend = h->da0 = h->objF = h->adj_stage = nullptr;
  h->adj_err = nullptr;
  h->adj_esc = nullptr;
  for (int i = 0; i < kMaxSpecies; ++i) {
    for (int d = 0; d < 3; ++d) {
      cudaFree(h->adj[i].lx[d]);
      cudaFree(h->adj[i].lu[d]);
    }
    cudaFree(h->adj[i].lw);
    h->adj[i] = SpeciesAdjoint{};
  }
  h->adj_ready = false;
  h->id_cap = 0;
}

}  // namespace

namespace pic {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace pic

extern "C" {

int pic_create(const pic_config *cfg, pic_handle **out) {
  if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, PIC_EINVAL, "cfg is NULL");
  const pic_config &c = *cfg;
  if (c.dims != 2 && c.dims != 3) return fail(nullptr, PIC_EINVAL, "dims must be 2 or 3");
  if (c.shape_order != 1 && c.shape_order != 2) return fail(nullptr, PIC_EINVAL, "shape_order must be 1 or 2");
  if (c.precision != PIC_FP32 && c.precision != PIC_FP64) return fail(nullptr, PIC_EINVAL, "bad precision");
  for (int d = 0; d < c.dims; ++d) {
    if (c.n[d] < 1 || !(c.dx[d] > 0)) return fail(nullptr, PIC_EINVAL, "n and dx must be positive");
    if (c.bc_lo[d] != PIC_BC_PERIODIC || c.bc_hi[d] != PIC_BC_PERIODIC) {
      if (d != 0) return fail(nullptr, PIC_EINVAL, "only x walls may be absorbing");
    }
  }
  for (int d = 0; d < 3; ++d)
    if ((c.bc_lo[d] != PIC_BC_PERIODIC && c.bc_lo[d] != PIC_BC_ABSORBING) ||
        (c.bc_hi[d] != PIC_BC_PERIODIC && c.bc_hi[d] != PIC_BC_ABSORBING))
      return fail(nullptr, PIC_EINVAL, "unknown boundary kind");
  const bool absorb = c.bc_lo[0] == PIC_BC_ABSORBING || c.bc_hi[0] == PIC_BC_ABSORBING;
  if (absorb && (c.bc_lo[0] != PIC_BC_ABSORBING || c.bc_hi[0] != PIC_BC_ABSORBING))
    return fail(nullptr, PIC_EINVAL, "absorbing x walls come in pairs (bc_lo[0] = bc_hi[0])");
  if (absorb && c.n[0] < 16) return fail(nullptr, PIC_EINVAL, "absorbing x walls need n[0] >= 16");
  if (c.laser.enabled) {
    if (!absorb) return fail(nullptr, PIC_EINVAL, "the laser enters through an absorbing x = 0 wall");
    if (!(c.laser.duration > 0) || !(c.laser.waist > 0) || (c.laser.polarization != 1 && c.laser.polarization != 2) ||
        !(fabs(c.laser.angle) < 0.5 * 3.14159265358979323846))
      return fail(nullptr, PIC_EINVAL, "bad laser parameters (duration, waist > 0; polarization 1 or 2; |angle| < pi/2)");
  }
  if (c.dims == 2 && c.n[2] != 1 && c.n[2] != 0) return fail(nullptr, PIC_EINVAL, "2D needs n[2] = 1");
  if (c.filter_passes < 0 || c.filter_passes > 8 || (c.filter_compensate != 0 && c.filter_compensate != 1))
    return fail(nullptr, PIC_EINVAL, "filter_passes must be 0..8 and filter_compensate 0 or 1");
  if (c.gather != PIC_GATHER_MOMENTUM && c.gather != PIC_GATHER_ENERGY)
    return fail(nullptr, PIC_EINVAL, "gather must be PIC_GATHER_MOMENTUM or PIC_GATHER_ENERGY");
  if (!(c.dt > 0)) return fail(nullptr, PIC_EINVAL, "dt must be positive");
  double s = 0;
  for (int d = 0; d < c.dims; ++d) s += 1.0 / (c.dx[d] * c.dx[d]);
  const double lim = 1.0 / sqrt(s);
  if (c.dt > lim) {
    char b[160];
    snprintf(b, sizeof b, "dt = %.6g exceeds the Yee limit (sum dx^-2)^(-1/2) = %.6g", c.dt, lim);
    return fail(nullptr, PIC_ECOURANT, b);
  }
  const int64_t ncell = (int64_t)c.n[0] * c.n[1] * (c.dims == 3 ? c.n[2] : 1);
  if (ncell >= (1LL << 30)) return fail(nullptr, PIC_EINVAL, "2^30 cells or more");
  int ctile[3];
  pic::push_tile_shape(c.dims, ctile);
  for (int d = 0; d < c.dims; ++d)
    if (c.tile[d] != 0 && c.tile[d] != ctile[d])
      return fail(nullptr, PIC_EINVAL, "tile must be 0 (default) or the compiled tile shape (8x8x4 in 3D, 16x16 in 2D)");
  if (c.drift_guard != 0 && c.drift_guard != 1)
    return fail(nullptr, PIC_EINVAL, "drift_guard must be 0 or 1 (the compiled drift allowance)");

  pic_handle *h = new pic_handle();
  h->cfg = c;
  Grid &g = h->g;
  g.dims = c.dims;
  g.order = c.shape_order;
  g.prec = c.precision;
  g.n[0] = c.n[0];
  g.n[1] = c.n[1];
  g.n[2] = c.dims == 3 ? c.n[2] : 1;
  g.dx[0] = c.dx[0];
  g.dx[1] = c.dx[1];
  g.dx[2] = c.dims == 3 ? c.dx[2] : 1.0;
  g.dt = c.dt;
  g.ncell = ncell;
  g.drift = 1;
  g.absorb_lo = c.bc_lo[0] == PIC_BC_ABSORBING;
  g.gather_ec = c.gather == PIC_GATHER_ENERGY;
  g.absorb_hi = c.bc_hi[0] == PIC_BC_ABSORBING;
  g.ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    const int t = ctile[d];
    g.tile[d] = t;
    g.ntile[d] = (g.n[d] + t - 1) / t;
    g.ntiles *= g.ntile[d];
  }
  h->rsize = g.prec == PIC_FP64 ? sizeof(double) : sizeof(float);
  h->laser.enabled = c.laser.enabled;
  h->laser.a0 = c.laser.a0;
  h->laser.waist = c.laser.waist;
  h->laser.duration = c.laser.duration;
  h->laser.yc = c.laser.y_center;
  h->laser.zc = c.laser.z_center;
  h->laser.pol = c.laser.polarization;
  h->laser.angle = c.laser.enabled ? c.laser.angle : 0.0;
  h->st = static_cast<cudaStream_t>(c.stream);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int maxsm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, PIC_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  keep_pooled_memory(dev);
  if (pic::push_smem_bytes(g) > (size_t)maxsm) {
    delete h;
    return fail(nullptr, PIC_EINVAL, "tile + guard window does not fit in shared memory; use a smaller tile");
  }
  const size_t fb = (size_t)ncell * h->rsize;
  // E, B in one block (a checkpoint copies them with one memcpy) and the
  // three J components in another (one memset clears J)
  bool ok = cudaMalloc(&h->E[0], 6 * fb) == cudaSuccess && cudaMalloc(&h->J[0], 3 * fb) == cudaSuccess;
  if (ok)
    for (int d = 0; d < 3; ++d) {
      h->E[d] = static_cast<char *>(h->E[0]) + d * fb;
      h->B[d] = static_cast<char *>(h->E[0]) + (3 + d) * fb;
      h->J[d] = static_cast<char *>(h->J[0]) + d * fb;
    }
  const size_t db = (size_t)ncell * sizeof(double);
  const int64_t nkeys = g.ntiles * g.tile[0] * g.tile[1] * g.tile[2];
  ok = ok && cudaMalloc(&h->rho_bg, db) == cudaSuccess && cudaMalloc(&h->rho, db) == cudaSuccess &&
       cudaMalloc(&h->rho_prev, db) == cudaSuccess && cudaMalloc(&h->f64, db) == cudaSuccess &&
       cudaMalloc(&h->red, 16 * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&h->keys, (size_t)nkeys * sizeof(int32_t)) == cudaSuccess &&
       cudaMalloc(&h->tile_tmp, (size_t)(g.ntiles + 1) * sizeof(int64_t)) == cudaSuccess &&
       cudaMalloc(&h->ctr, sizeof(Counters)) == cudaSuccess && cudaMalloc(&h->bad, sizeof(unsigned long long)) == cudaSuccess &&
       cudaMalloc(&h->esc_count, 2 * sizeof(unsigned long long)) == cudaSuccess &&
       cudaMalloc(&h->mur, 8 * sizeof(double) * (size_t)g.n[1] * g.n[2]) == cudaSuccess;
  if (!ok) {
    pic_destroy(h);
    return fail(nullptr, PIC_ENOMEM, "device allocation failed in pic_create");
  }
  cudaMemsetAsync(h->E[0], 0, 6 * fb, h->st);
  cudaMemsetAsync(h->J[0], 0, 3 * fb, h->st);
  cudaMemsetAsync(h->rho_bg, 0, db, h->st);
  cudaMemsetAsync(h->ctr, 0, sizeof(Counters), h->st);
  // laser profile P = exp(-r^2/waist^2) at the wall rows of the polarised
  // component (Ey at (j + 1/2, k), Ez at (j, k + 1/2)), once for the run
  const int64_t nyz = (int64_t)g.n[1] * g.n[2];
  std::vector<double> prof((size_t)nyz, 0.0);
  if (h->laser.enabled) {
    const bool ey = h->laser.pol == 1;
    for (int64_t jk = 0; jk < nyz; ++jk) {
      const int j = (int)(jk % g.n[1]), k = (int)(jk / g.n[1]);
      const double y = (j + (ey ? 0.5 : 0.0)) * g.dx[1], z = (k + (ey ? 0.0 : 0.5)) * g.dx[2];
      double r2 = (y - h->laser.yc) * (y - h->laser.yc);
      if (g.dims == 3) r2 += (z - h->laser.zc) * (z - h->laser.zc);
      prof[(size_t)jk] = exp(-r2 / (h->laser.waist * h->laser.waist));
    }
  }
  e = cudaMalloc(&h->laser_prof, sizeof(double) * (size_t)nyz);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->laser_prof, prof.data(), sizeof(double) * (size_t)nyz, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    pic_destroy(h);
    return fail(nullptr, PIC_ECUDA, std::string("pic_create: ") + cudaGetErrorString(e));
  }
  *out = h;
  return PIC_OK;
}

int pic_destroy(pic_handle *h) {
  if (!h) return PIC_OK;
  cudaStreamSynchronize(h->st);
  cudaFree(h->E[0]);  // E and B share one block
  cudaFree(h->J[0]);  // so do the three J components
  cudaFree(h->rho_bg);
  cudaFree(h->rho);
  cudaFree(h->rho_prev);
  cudaFree(h->f64);
  cudaFree(h->red);
  cudaFree(h->keys);
  cudaFree(h->tile_tmp);
  cudaFree(h->ctr);
  cudaFree(h->bad);
  cudaFree(h->esc_count);
  cudaFree(h->mur);
  cudaFree(h->laser_prof);
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    free_particles(s.buf[0]);
    free_particles(s.buf[1]);
    cudaFree(s.d_count);
    cudaFree(s.rank);
    cudaFree(s.work.work_pb);  // with tile_start and work_tile
    cudaFree(s.tq);
    cudaFreeHost(s.esc_host);
    if (s.esc_ev) cudaEventDestroy(s.esc_ev);
  }
  for (auto &o : h->outputs) {
    cudaFree(o.buf);
    cudaFree(o.found);
  }
  for (auto &t : h->timers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  for (auto &sn : h->ckpt) free_snapshot(sn, h->st);
  join_adj(h);
  for (auto &tb : h->tapes)
    for (auto &sn : tb) free_snapshot(sn, h->st);
  cudaStreamSynchronize(h->st);
  free_adjoint(h);
  if (h->st_adj) cudaStreamDestroy(h->st_adj);
  for (cudaEvent_t ev : h->tape_free)
    if (ev) cudaEventDestroy(ev);
  if (h->ev_main) cudaEventDestroy(h->ev_main);
  if (h->ev_adj) cudaEventDestroy(h->ev_adj);
  delete h;
  return PIC_OK;
}

const char *pic_last_error(const pic_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int pic_add_species(pic_handle *h, double q, double m, int64_t capacity, int *species) {
  if (!h || !species) return fail(h, PIC_EINVAL, "NULL argument");
  if (h->nsp >= kMaxSpecies) return fail(h, PIC_EINVAL, "too many species");
  if (!(m > 0) || capacity < 0 || capacity > 0x7fffffffLL) return fail(h, PIC_EINVAL, "bad mass or capacity");
  Species &s = h->sp[h->nsp];
  s = Species{};
  s.q = q;
  s.m = m;
  s.capacity = capacity;
  s.slots = capacity + (pic::kTilePad - 1) * h->g.ntiles;
  if (s.slots > 0x7fffffffLL) return fail(h, PIC_EINVAL, "capacity plus tile padding exceeds 2^31 slots");
  cudaError_t e = alloc_particles(s.buf[0], s.slots, h->rsize, h->g.dims);
  if (e == cudaSuccess) e = alloc_particles(s.buf[1], s.slots, h->rsize, h->g.dims);
  if (e == cudaSuccess) e = cudaMalloc(&s.d_count, sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&s.rank, (size_t)(s.slots > 0 ? s.slots : 1) * sizeof(int32_t));
  // Work items: pieces of at most `chunk` slots per tile, chunk sized so that
  // a species spread over few tiles (a thin slab, a small grid) still gives
  // about 16 blocks per SM, never below 512 slots and never above the
  // fixed-point window's limit (kMaxWindowSlots).
  {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t chunk = s.slots / (16 * (int64_t)(nsm > 0 ? nsm : 1));
    chunk = (chunk + 255) / 256 * 256;
    chunk = chunk < 512 ? 512 : chunk;
    s.work.chunk = chunk > pic::kMaxWindowSlots ? pic::kMaxWindowSlots : chunk;
    s.work.nwork = s.slots / s.work.chunk + 1 + h->g.ntiles;
  }
  if (e == cudaSuccess) e = cudaMalloc(&s.tq, (size_t)2 * s.work.nwork * sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost(&s.esc_host, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.esc_ev, cudaEventDisableTiming);
  // the sort's outputs in one allocation (one copy for a tape entry):
  // work_pb[nwork], tile_start[ntiles + 1], work_tile[nwork]
  if (e == cudaSuccess) {
    void *meta = nullptr;
    e = cudaMalloc(&meta, sort_meta_bytes(s.work.nwork, h->g.ntiles));
    if (e == cudaSuccess) set_sort_meta(meta, s.work.nwork, h->g.ntiles, s.work.work_pb, s.tile_start, s.work.work_tile);
  }
  if (e != cudaSuccess) {
    free_particles(s.buf[0]);
    free_particles(s.buf[1]);
    cudaFree(s.d_count);
    cudaFree(s.rank);
    cudaFree(s.work.work_pb);  // with tile_start and work_tile
    cudaFree(s.tq);
    cudaFreeHost(s.esc_host);
    if (s.esc_ev) cudaEventDestroy(s.esc_ev);
    s = Species{};
    cudaGetLastError();
    return fail(h, PIC_ENOMEM, "device allocation failed in pic_add_species");
  }
  cudaMemsetAsync(s.d_count, 0, sizeof(int64_t), h->st);
  cudaMemsetAsync(s.tile_start, 0, (size_t)(h->g.ntiles + 1) * sizeof(int64_t), h->st);
  *species = h->nsp++;
  return PIC_OK;
}

namespace {
// Particles per chunk of a host load (two staging buffers of 60 B each).
constexpr int64_t kLoadChunk = int64_t(1) << 22;

// The copy stream, events and staging buffers of a chunked host load.  On
// every exit the copies in flight finish before the buffers are released
// (stream-ordered on the simulation stream, after the kernels that read them).
struct LoadPipe {
  cudaStream_t st = nullptr, cs = nullptr;
  cudaEvent_t ev[5] = {};  // copied[2], converted[2], allocated
  void *stage[2] = {};
  ~LoadPipe() {
    if (cs) cudaStreamSynchronize(cs);
    for (void *p : stage)
      if (p) cudaFreeAsync(p, st);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
  }
};
}  // namespace

int pic_load_particles(pic_handle *h, int species, int64_t n, const double *x, const double *y, const double *z,
                       const double *ux, const double *uy, const double *uz, const double *w, const uint32_t *id,
                       int mem_kind) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  if (n < 0) return fail(h, PIC_EINVAL, "negative count");
  if (n == 0) return PIC_OK;
  if (!x || !y || (h->g.dims == 3 && !z) || !ux || !uy || !uz || !w)
    return fail(h, PIC_EINVAL, "NULL particle array");
  Species &s = h->sp[species];
  const int64_t cur = read_count(h, s);
  if (cur + n > s.capacity) return fail(h, PIC_ENOMEM, "species capacity exceeded");
  const double *src[7] = {x, y, z, ux, uy, uz, w};
  CK(h, cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), h->st), "memset");
  if (mem_kind == PIC_MEM_HOST) {
    // Host arrays travel in chunks through two device staging buffers: the
    // copy engine fills one (cudaMemcpyAsync on a copy stream) while the
    // load kernel converts the other on the simulation stream.  From
    // page-locked memory this runs at the host link's DMA rate (about three
    // times what the load kernel reaches reading mapped host memory in place).
    LoadPipe lp;
    lp.st = h->st;
    const int64_t chunk = n < kLoadChunk ? n : kLoadChunk;
    const size_t stride = (size_t)chunk * sizeof(double);  // one array of a chunk
    const size_t bytes = 7 * stride + (size_t)chunk * sizeof(uint32_t);
    const int nbuf = n > chunk ? 2 : 1;
    CK(h, cudaStreamCreateWithFlags(&lp.cs, cudaStreamNonBlocking), "copy stream");
    for (auto &e : lp.ev) CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    for (int b = 0; b < nbuf; ++b) CK(h, cudaMallocAsync(&lp.stage[b], bytes, h->st), "load staging alloc");
    CK(h, cudaEventRecord(lp.ev[4], h->st), "event");
    CK(h, cudaStreamWaitEvent(lp.cs, lp.ev[4], 0), "event wait");  // staging allocated
    for (int64_t c0 = 0, k = 0; c0 < n; c0 += chunk, ++k) {
      const int b = (int)(k & 1);
      const int64_t m = n - c0 < chunk ? n - c0 : chunk;
      unsigned char *d = static_cast<unsigned char *>(lp.stage[b]);
      if (k >= 2) CK(h, cudaStreamWaitEvent(lp.cs, lp.ev[2 + b], 0), "event wait");  // buffer converted
      const double *ds[7] = {};
      for (int a = 0; a < 7; ++a) {
        if (!src[a]) continue;
        CK(h, cudaMemcpyAsync(d + a * stride, src[a] + c0, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, lp.cs),
           "load H2D");
        ds[a] = reinterpret_cast<const double *>(d + a * stride);
      }
      const uint32_t *did = nullptr;
      if (id) {
        CK(h, cudaMemcpyAsync(d + 7 * stride, id + c0, (size_t)m * sizeof(uint32_t), cudaMemcpyHostToDevice, lp.cs),
           "load H2D");
        did = reinterpret_cast<const uint32_t *>(d + 7 * stride);
      }
      CK(h, cudaEventRecord(lp.ev[b], lp.cs), "event");
      CK(h, cudaStreamWaitEvent(h->st, lp.ev[b], 0), "event wait");  // chunk arrived
      CK(h,
         pic::launch_load(h->g, s.buf[s.cur], cur + c0, m, ds[0], ds[1], ds[2], ds[3], ds[4], ds[5], ds[6], did,
                          (uint32_t)(cur + c0), h->bad, h->st),
         "load kernel");
      h->launches++;
      CK(h, cudaEventRecord(lp.ev[2 + b], h->st), "event");
    }
  } else {
    CK(h,
       pic::launch_load(h->g, s.buf[s.cur], cur, n, src[0], src[1], src[2], src[3], src[4], src[5], src[6], id,
                        (uint32_t)cur, h->bad, h->st),
       "load kernel");
    h->launches++;
  }
  const int64_t nn = cur + n;
  CK(h, cudaMemcpyAsync(s.d_count, &nn, sizeof(int64_t), cudaMemcpyHostToDevice, h->st), "count");
  unsigned long long bad = 0;
  CK(h, cudaMemcpyAsync(&bad, h->bad, sizeof(bad), cudaMemcpyDeviceToHost, h->st), "bad count");
  CK(h, cudaStreamSynchronize(h->st), "load sync");
  s.h_count = nn;
  s.need_sort = true;
  if (bad)
    return fail(h, PIC_EINVAL, "particles outside an absorbing wall or with non-finite values were marked dead");
  return PIC_OK;
}

int pic_neutralize(pic_handle *h) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  // rho_bg = -rho of the particles: deposit them with the opposite charge.
  // Freshly loaded species are sorted first (the next step would sort them
  // anyway), so that the tiled fixed-point deposit serves: input in cell
  // order sends a warp's global atomics to the same nodes.
  CK(h, cudaMemsetAsync(h->rho_bg, 0, sizeof(double) * h->g.ncell, h->st), "memset");
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    if (s.need_sort) {
      const int r = sort_species(h, s);
      if (r) return r;
    }
    CK(h, pic::launch_rho_tiled(h->g, s.buf[s.cur], s.tile_start, -s.q, h->rho_bg, h->ctr, h->st), "rho deposit");
    h->launches++;
  }
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_set_background(pic_handle *h, const double *rho_bg, int mem_kind) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (!rho_bg) return fail(h, PIC_EINVAL, "NULL background");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  const size_t nb = sizeof(double) * (size_t)h->g.ncell;
  std::vector<double> tmp((size_t)h->g.ncell);
  if (mem_kind == PIC_MEM_HOST) {
    memcpy(tmp.data(), rho_bg, nb);
  } else {
    CK(h, cudaMemcpyAsync(tmp.data(), rho_bg, nb, cudaMemcpyDeviceToHost, h->st), "D2H");
    CK(h, cudaStreamSynchronize(h->st), "sync");
  }
  for (double v : tmp)
    if (!std::isfinite(v)) return fail(h, PIC_EINVAL, "non-finite background");
  CK(h, cudaMemcpyAsync(h->rho_bg, tmp.data(), nb, cudaMemcpyHostToDevice, h->st), "H2D");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

namespace {

// Take one frame of an output request at the current state (or count it as
// dropped when its buffer is full).
int output_capture(pic_handle *h, OutputReq &o) {
  if ((int64_t)o.steps.size() >= o.req.max_frames) {
    o.dropped++;
    return PIC_OK;
  }
  const int64_t f = (int64_t)o.steps.size();
  double *dst = o.buf + f * o.frame_doubles;
  pic::OutBox b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = o.req.lo[a];
    b.hi[a] = o.req.hi[a];
  }
  if (o.req.kind == PIC_OUT_FIELD) {
    const int w = o.req.which;
    if (w == PIC_RHO) {
      const int r = compute_rho(h, h->rho);
      if (r) return r;
      CK(h, pic::launch_out_field(h->g, h->rho, true, b, dst, h->st), "output field");
    } else {
      const void *src = w < 3 ? h->E[w] : w < 6 ? h->B[w - 3] : h->J[w - 6];
      CK(h, pic::launch_out_field(h->g, src, false, b, dst, h->st), "output field");
    }
  } else {
    Species &s = h->sp[o.req.which];
    CK(h,
       pic::launch_out_particles(h->g, s.buf[s.cur], s.d_count, s.slots, b, dst, o.found + f, o.req.max_particles,
                                 h->st),
       "output particles");
  }
  h->launches++;
  o.steps.push_back(h->step);
  return PIC_OK;
}

OutputReq *output_get(pic_handle *h, int id) {
  if (!h || id < 0 || id >= (int)h->outputs.size() || !h->outputs[id].active) return nullptr;
  return &h->outputs[id];
}

}  // namespace

// ---- state blob: header, then E B | J | rho_bg | per species particle block
namespace {

struct StateHeader {
  char magic[8];
  int32_t version, dims, n[3], order, prec, nsp, bc_lo0, bc_hi0, laser_on, filter_passes, filter_comp, gather, pad;
  double dx[3], dt, laser_a0, laser_waist, laser_duration, laser_angle;
  int64_t step, ncell;
  int64_t slots[kMaxSpecies], count[kMaxSpecies];
  double q[kMaxSpecies], m[kMaxSpecies];
  Counters ctr;
};
constexpr char kStateMagic[8] = {'P', 'I', 'C', 'S', 'T', 'A', 'T', 'E'};

StateHeader state_header(pic_handle *h) {
  StateHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kStateMagic, 8);
  hd.version = 2;
  hd.dims = h->g.dims;
  for (int d = 0; d < 3; ++d) {
    hd.n[d] = h->g.n[d];
    hd.dx[d] = h->g.dx[d];
  }
  hd.order = h->g.order;
  hd.prec = h->g.prec;
  hd.nsp = h->nsp;
  hd.bc_lo0 = h->g.absorb_lo;
  hd.bc_hi0 = h->g.absorb_hi;
  hd.laser_on = h->laser.enabled;
  hd.filter_passes = h->cfg.filter_passes;
  hd.filter_comp = h->cfg.filter_compensate;
  hd.gather = h->cfg.gather;
  hd.dt = h->g.dt;
  hd.laser_a0 = h->laser.enabled ? h->laser.a0 : 0.0;
  hd.laser_waist = h->laser.enabled ? h->laser.waist : 0.0;
  hd.laser_duration = h->laser.enabled ? h->laser.duration : 0.0;
  hd.laser_angle = h->laser.enabled ? h->laser.angle : 0.0;
  hd.step = h->step;
  hd.ncell = h->g.ncell;
  for (int i = 0; i < h->nsp; ++i) {
    hd.slots[i] = h->sp[i].slots;
    hd.q[i] = h->sp[i].q;
    hd.m[i] = h->sp[i].m;
  }
  return hd;
}

int64_t state_bytes(pic_handle *h) {
  const int64_t fb = h->g.ncell * (int64_t)h->rsize;
  int64_t b = (int64_t)sizeof(StateHeader) + 9 * fb + h->g.ncell * (int64_t)sizeof(double);
  for (int i = 0; i < h->nsp; ++i) b += (int64_t)particles_bytes(h->sp[i].slots, h->rsize, h->g.dims);
  return b;
}

}  // namespace

int pic_state_size(pic_handle *h, int64_t *bytes) {
  if (!h || !bytes) return fail(h, PIC_EINVAL, "NULL argument");
  *bytes = state_bytes(h);
  return PIC_OK;
}

int pic_state_save(pic_handle *h, void *buf, int64_t bytes, int mem_kind) {
  if (!h || !buf) return fail(h, PIC_EINVAL, "NULL argument");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  if (bytes < state_bytes(h)) return fail(h, PIC_EINVAL, "state buffer too small");
  StateHeader hd = state_header(h);
  for (int i = 0; i < h->nsp; ++i) hd.count[i] = read_count(h, h->sp[i]);
  CK(h, cudaMemcpyAsync(&hd.ctr, h->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  const cudaMemcpyKind to = mem_kind == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  char *p = static_cast<char *>(buf);
  CK(h, cudaMemcpyAsync(p, &hd, sizeof hd, mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice,
                        h->st),
     "state header");
  p += sizeof hd;
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  CK(h, cudaMemcpyAsync(p, h->E[0], 6 * fb, to, h->st), "state fields");
  p += 6 * fb;
  CK(h, cudaMemcpyAsync(p, h->J[0], 3 * fb, to, h->st), "state J");
  p += 3 * fb;
  CK(h, cudaMemcpyAsync(p, h->rho_bg, sizeof(double) * (size_t)h->g.ncell, to, h->st), "state background");
  p += sizeof(double) * (size_t)h->g.ncell;
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    const size_t pb = particles_bytes(s.slots, h->rsize, h->g.dims);
    CK(h, cudaMemcpyAsync(p, s.buf[s.cur].cell, pb, to, h->st), "state particles");
    p += pb;
  }
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return check_device_errors(h);
}

int pic_state_load(pic_handle *h, const void *buf, int64_t bytes, int mem_kind) {
  if (!h || !buf) return fail(h, PIC_EINVAL, "NULL argument");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  if (bytes < (int64_t)sizeof(StateHeader)) return fail(h, PIC_EINVAL, "state blob too small");
  StateHeader hd;
  CK(h,
     cudaMemcpyAsync(&hd, buf, sizeof hd, mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost,
                     h->st),
     "state header");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  // the blob must come from a handle of the same configuration and species
  StateHeader me = state_header(h);
  bool same = memcmp(hd.magic, kStateMagic, 8) == 0 && hd.version == me.version && hd.dims == me.dims &&
              hd.order == me.order && hd.prec == me.prec && hd.nsp == me.nsp && hd.bc_lo0 == me.bc_lo0 &&
              hd.bc_hi0 == me.bc_hi0 && hd.laser_on == me.laser_on && hd.filter_passes == me.filter_passes &&
              hd.filter_comp == me.filter_comp && hd.gather == me.gather && hd.dt == me.dt &&
              hd.laser_a0 == me.laser_a0 && hd.laser_waist == me.laser_waist &&
              hd.laser_duration == me.laser_duration && hd.laser_angle == me.laser_angle && hd.ncell == me.ncell;
  for (int d = 0; d < 3; ++d) same = same && hd.n[d] == me.n[d] && hd.dx[d] == me.dx[d];
  for (int i = 0; i < me.nsp && same; ++i)
    same = hd.slots[i] == me.slots[i] && hd.q[i] == me.q[i] && hd.m[i] == me.m[i] && hd.count[i] >= 0 &&
           hd.count[i] <= me.slots[i];
  if (!same) return fail(h, PIC_EINVAL, "state blob does not match this simulation's configuration and species");
  if (bytes < state_bytes(h)) return fail(h, PIC_EINVAL, "state blob too small");
  const cudaMemcpyKind from = mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const char *p = static_cast<const char *>(buf) + sizeof hd;
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  const char *pf = p;  // fields, J and background
  p += 9 * fb + sizeof(double) * (size_t)h->g.ncell;
  // Particles go first into each species' spare sort buffer and are
  // validated there on the device (cells inside the grid, offsets in [0, 1),
  // finite momenta and weights), so that a corrupt blob is refused before it
  // replaces anything: the next sort indexes its counters by cell.
  CK(h, cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), h->st), "memset");
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    const size_t pb = particles_bytes(s.slots, h->rsize, h->g.dims);
    CK(h, cudaMemcpyAsync(s.buf[1 - s.cur].cell, p, pb, from, h->st), "state particles");
    p += pb;
    CK(h, pic::launch_check_particles(h->g, s.buf[1 - s.cur], hd.count[i], h->bad, h->st), "state check");
  }
  unsigned long long bad = 0;
  CK(h, cudaMemcpyAsync(&bad, h->bad, sizeof(bad), cudaMemcpyDeviceToHost, h->st), "bad count");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  if (bad)
    return fail(h, PIC_EINVAL,
                "state blob holds " + std::to_string(bad) +
                    " invalid particle slot(s) (cell outside the grid, offset outside [0, 1), non-finite momentum "
                    "or weight, or beyond an absorbing wall); nothing was loaded");
  CK(h, cudaMemcpyAsync(h->E[0], pf, 6 * fb, from, h->st), "state fields");
  pf += 6 * fb;
  CK(h, cudaMemcpyAsync(h->J[0], pf, 3 * fb, from, h->st), "state J");
  pf += 3 * fb;
  CK(h, cudaMemcpyAsync(h->rho_bg, pf, sizeof(double) * (size_t)h->g.ncell, from, h->st), "state background");
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    s.cur = 1 - s.cur;
    CK(h, cudaMemcpyAsync(s.d_count, &hd.count[i], sizeof(int64_t), cudaMemcpyHostToDevice, h->st), "count");
    s.h_count = hd.count[i];
    s.need_sort = true;
  }
  CK(h, cudaMemcpyAsync(h->ctr, &hd.ctr, sizeof(Counters), cudaMemcpyHostToDevice, h->st), "counters");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  h->step = hd.step;
  h->rho_prev_step = -2;
  return PIC_OK;
}

int pic_output_due(const pic_output_t *req, int64_t step) {
  if (!req || req->every < 1) return 0;
  return step >= req->first && step <= req->last && (step - req->first) % req->every == 0;
}

int pic_output_add(pic_handle *h, const pic_output_t *req, int *id) {
  if (!h || !req || !id) return fail(h, PIC_EINVAL, "NULL argument");
  const pic_output_t &q = *req;
  if (q.kind == PIC_OUT_FIELD) {
    if (q.which < PIC_EX || q.which > PIC_RHO) return fail(h, PIC_EINVAL, "bad field id");
  } else if (q.kind == PIC_OUT_PARTICLES) {
    if (q.which < 0 || q.which >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
    if (q.max_particles < 1) return fail(h, PIC_EINVAL, "max_particles must be >= 1");
  } else {
    return fail(h, PIC_EINVAL, "kind must be PIC_OUT_FIELD or PIC_OUT_PARTICLES");
  }
  int64_t box = 1;
  for (int a = 0; a < 3; ++a) {
    if (q.lo[a] < 0 || q.hi[a] > h->g.n[a] || q.lo[a] >= q.hi[a]) return fail(h, PIC_EINVAL, "bad output box");
    box *= q.hi[a] - q.lo[a];
  }
  if (q.first < 0 || q.last < q.first || q.every < 1 || q.max_frames < 1)
    return fail(h, PIC_EINVAL, "bad output schedule (0 <= first <= last, every >= 1, max_frames >= 1)");
  OutputReq o;
  o.req = q;
  o.frame_doubles = q.kind == PIC_OUT_FIELD ? box : 8 * q.max_particles;
  if (q.max_frames > (int64_t)1 << 40 || o.frame_doubles > ((int64_t)1 << 40) / q.max_frames)
    return fail(h, PIC_ENOMEM, "output buffer too large");
  if (cudaMalloc(&o.buf, sizeof(double) * (size_t)(o.frame_doubles * q.max_frames)) != cudaSuccess ||
      cudaMalloc(&o.found, sizeof(unsigned long long) * (size_t)q.max_frames) != cudaSuccess) {
    cudaFree(o.buf);
    cudaFree(o.found);
    cudaGetLastError();
    return fail(h, PIC_ENOMEM, "device allocation failed in pic_output_add");
  }
  CK(h, cudaMemsetAsync(o.found, 0, sizeof(unsigned long long) * (size_t)q.max_frames, h->st), "memset");
  o.active = true;
  h->outputs.push_back(std::move(o));
  *id = (int)h->outputs.size() - 1;
  return PIC_OK;
}

int pic_output_capture(pic_handle *h, int id) {
  OutputReq *o = output_get(h, id);
  if (!o) return fail(h, PIC_EINVAL, "no such output request");
  return output_capture(h, *o);
}

int pic_output_count(pic_handle *h, int id, int64_t *nframes, int64_t *dropped) {
  OutputReq *o = output_get(h, id);
  if (!o || !nframes) return fail(h, PIC_EINVAL, "no such output request or NULL argument");
  *nframes = (int64_t)o->steps.size();
  if (dropped) *dropped = o->dropped;
  return check_device_errors(h);
}

int pic_output_read(pic_handle *h, int id, int64_t frame, double *out, int64_t *count, int64_t *step,
                    int mem_kind) {
  OutputReq *o = output_get(h, id);
  if (!o || !out || !count) return fail(h, PIC_EINVAL, "no such output request or NULL argument");
  if (frame < 0 || frame >= (int64_t)o->steps.size()) return fail(h, PIC_EINVAL, "no such frame");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  const double *src = o->buf + frame * o->frame_doubles;
  int64_t n = o->frame_doubles, found = o->frame_doubles;
  if (o->req.kind == PIC_OUT_PARTICLES) {
    unsigned long long f = 0;
    CK(h, cudaMemcpyAsync(&f, o->found + frame, sizeof(f), cudaMemcpyDeviceToHost, h->st), "D2H");
    CK(h, cudaStreamSynchronize(h->st), "sync");
    found = (int64_t)f;
    n = 8 * (found < o->req.max_particles ? found : o->req.max_particles);
  }
  if (n > 0)
    CK(h,
       cudaMemcpyAsync(out, src, sizeof(double) * (size_t)n,
                       mem_kind == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st),
       "output copy");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  *count = found;
  if (step) *step = o->steps[(size_t)frame];
  if (o->req.kind == PIC_OUT_PARTICLES && found > o->req.max_particles)
    return fail(h, PIC_EOVERFLOW, "more particles in the box than max_particles");
  return check_device_errors(h);
}

int pic_output_remove(pic_handle *h, int id) {
  OutputReq *o = output_get(h, id);
  if (!o) return fail(h, PIC_EINVAL, "no such output request");
  cudaStreamSynchronize(h->st);
  cudaFree(o->buf);
  cudaFree(o->found);
  o->buf = nullptr;
  o->found = nullptr;
  o->steps.clear();
  o->active = false;
  return PIC_OK;
}

int pic_step(pic_handle *h, int nsteps) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(h, PIC_EINVAL, "negative step count");
  const int every = h->cfg.sort_every > 0 ? h->cfg.sort_every : 20;
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  for (int t = 0; t < nsteps; ++t) {
    struct StepRange {
      StepRange() { nvtxRangePushA("pic_step"); }
      ~StepRange() { nvtxRangePop(); }
    } step_range;
    for (int i = 0; i < h->nsp; ++i) {
      Species &s = h->sp[i];
      // Sort on the cadence, or early when the last push sent more than
      // 0.5 % of the particles down the escape path (they drifted beyond
      // their tile's guard cells).  The escape count of a push is read back
      // asynchronously.  A species whose last count was above 1/8 of that
      // threshold waits for the count of its previous push; the others wait
      // once four steps have passed without a count, so that a long
      // pic_step call, whose host loop runs ahead of the device, still
      // learns how the particles drift.  (On large grids a wait costs no
      // device time: the last step's field updates are still queued behind
      // the push when it ends.)
      bool many_escapes = false;
      if (s.esc_pending) {
        cudaError_t q;
        if (s.fast || s.count_age >= 4) {
          CK(h, cudaEventSynchronize(s.esc_ev), "escape count");
          q = cudaSuccess;
        } else {
          q = cudaEventQuery(s.esc_ev);
        }
        if (q == cudaSuccess) {
          s.esc_pending = false;
          s.count_age = 0;
          const unsigned long long lim = (unsigned long long)(s.h_count / 200 > 1024 ? s.h_count / 200 : 1024);
          // (a count from before the last sort says nothing about the order now)
          many_escapes = s.esc_step >= s.sorted_at && s.esc_host[0] > lim;
          s.fast = s.esc_host[0] > lim / 8;
          // many particles changing shape support per step (fast beams): the
          // push variant that drains its deferred-job queue between chunks
          s.mid_drain = s.esc_host[1] > (unsigned long long)pic::kPushQueueMidDrain * (unsigned long long)s.work.nwork;
        } else {
          cudaGetLastError();  // not ready: not an error
          s.count_age++;
        }
      }
      // (a species sorted since the last push, e.g. by pic_neutralize, is not sorted again)
      if (s.need_sort || (h->step % every == 0 && s.sorted_at != h->step) || many_escapes) {
        if (many_escapes) h->adaptive_sorts++;
        int r = sort_species(h, s);
        if (r) return r;
      }
    }
    if (h->taping) {
      std::vector<Snapshot> &tape = cur_tape(h);
      if (h->tape_len < (int)tape.size()) {
        Timed tm(h, pic::KC_TAPE);
        CK(h, save_snapshot(h, tape[h->tape_len], true, h->tape_len > 0 ? &tape[h->tape_len - 1] : nullptr),
           "tape record");
        h->tape_len++;
      }
      if (h->tape_len >= (int)tape.size()) h->taping = false;
    }
    {
      Timed tm(h, pic::KC_ZEROJ);
      CK(h, cudaMemsetAsync(h->J[0], 0, 3 * fb, h->st), "zero J");
    }
    for (int i = 0; i < h->nsp; ++i) {
      Species &s = h->sp[i];
      Timed tm(h, pic::KC_PUSH);
      int nl = 0;
      CK(h,
         pic::launch_push(h->g, h->E, h->B, h->J, s.buf[s.cur], s.tile_start, s.work, s.tq, s.fresh ? 1 : 0,
                          s.rank, h->esc_count, s.q, s.m, h->ctr, h->st, &nl, s.mid_drain ? 1 : 0),
         "push");
      s.fresh = false;
      h->launches += nl;
      if (s.mid_drain) h->mid_drain_pushes++;
      if (s.esc_host && !s.esc_pending) {
        CK(h, cudaMemcpyAsync(s.esc_host, h->esc_count, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                              h->st),
           "escape count");
        CK(h, cudaEventRecord(s.esc_ev, h->st), "escape event");
        s.esc_pending = true;
        s.esc_step = h->step;
      }
    }
    if (h->cfg.filter_passes > 0) {
      Timed tm(h, pic::KC_FILTER);
      for (int d = 0; d < 3; ++d) {
        int nl = 0;
        CK(h,
           pic::launch_smooth(h->g, h->J[d], false, h->f64, h->cfg.filter_passes, h->cfg.filter_compensate, h->st,
                              &nl),
           "smooth J");
        h->launches += nl;
      }
    }
    {
      Timed tm(h, pic::KC_YEE_B);
      CK(h, pic::launch_yee_b(h->g, h->E, h->B, 0.5 * h->g.dt, h->st), "yee B");
    }
    const bool walls = h->g.absorb_lo || h->g.absorb_hi;
    if (walls) {
      Timed tm(h, pic::KC_BOUNDARY);
      CK(h, pic::launch_mur_save(h->g, h->E, h->mur, h->st), "mur save");
      h->launches++;
    }
    {
      Timed tm(h, pic::KC_YEE_E);
      CK(h, pic::launch_yee_e(h->g, h->E, h->B, h->J, h->g.dt, h->st), "yee E");
    }
    if (walls) {
      Timed tm(h, pic::KC_BOUNDARY);
      CK(h,
         pic::launch_mur_apply(h->g, h->E, h->mur,
                               pic::laser_step(h->laser, h->laser_prof, h->laser.a0, h->g, h->step * h->g.dt,
                                               (h->step + 1) * h->g.dt),
                               h->st),
         "mur apply");
      h->launches++;
    }
    {
      Timed tm(h, pic::KC_YEE_B);
      CK(h, pic::launch_yee_b(h->g, h->E, h->B, 0.5 * h->g.dt, h->st), "yee B");
    }
    h->launches += 3;
    h->step++;
    for (auto &o : h->outputs)
      if (o.active && pic_output_due(&o.req, h->step)) {
        const int r = output_capture(h, o);
        if (r) return r;
      }
  }
  return PIC_OK;
}

int pic_fields(pic_handle *h, int which, double *out, int mem_kind) {
  if (!h || !out) return fail(h, PIC_EINVAL, "NULL argument");
  if (which < PIC_EX || which > PIC_RHO) return fail(h, PIC_EINVAL, "bad field selector");
  const size_t db = sizeof(double) * h->g.ncell;
  if (which == PIC_RHO) {
    int r = compute_rho(h, h->rho);
    if (r) return r;
    r = copy_out(h, out, h->rho, db, mem_kind);
    if (r) return r;
  } else {
    void *src = which < 3 ? h->E[which] : which < 6 ? h->B[which - 3] : h->J[which - 6];
    CK(h, pic::launch_field_to_f64(h->g, src, h->f64, h->st), "convert");
    int r = copy_out(h, out, h->f64, db, mem_kind);
    if (r) return r;
  }
  return check_device_errors(h);
}

int pic_set_field(pic_handle *h, int which, const double *in, int mem_kind) {
  if (!h || !in) return fail(h, PIC_EINVAL, "NULL argument");
  if (which < PIC_EX || which > PIC_JZ) return fail(h, PIC_EINVAL, "bad field selector");
  const size_t db = sizeof(double) * h->g.ncell;
  CK(h, cudaMemcpyAsync(h->f64, in, db, mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                        h->st),
     "set field copy");
  void *dst = which < 3 ? h->E[which] : which < 6 ? h->B[which - 3] : h->J[which - 6];
  CK(h, pic::launch_field_from_f64(h->g, h->f64, dst, h->st), "convert");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_num_particles(pic_handle *h, int species, int64_t *n) {
  if (!h || !n) return fail(h, PIC_EINVAL, "NULL argument");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  *n = read_count(h, h->sp[species]);
  return PIC_OK;
}

int pic_particles(pic_handle *h, int species, double *x, double *y, double *z, double *ux, double *uy, double *uz,
                  double *w, uint32_t *id, int32_t *alive, int mem_kind) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  Species &s = h->sp[species];
  const int64_t n = read_count(h, s);
  if (n == 0) return PIC_OK;
  double *outs[7] = {x, y, z, ux, uy, uz, w};
  double *dev[7] = {};
  uint32_t *did = nullptr;
  int32_t *dal = nullptr;
  std::vector<void *> tmp;
  auto dalloc = [&](size_t b) -> void * {
    void *p = nullptr;
    if (cudaMallocAsync(&p, b, h->st) != cudaSuccess) return nullptr;
    tmp.push_back(p);
    return p;
  };
  const bool host = mem_kind == PIC_MEM_HOST;
  for (int a = 0; a < 7; ++a)
    if (outs[a]) dev[a] = host ? static_cast<double *>(dalloc((size_t)n * sizeof(double))) : outs[a];
  if (id) did = host ? static_cast<uint32_t *>(dalloc((size_t)n * sizeof(uint32_t))) : id;
  if (alive) dal = host ? static_cast<int32_t *>(dalloc((size_t)n * sizeof(int32_t))) : alive;
  for (int a = 0; a < 7; ++a)
    if (outs[a] && !dev[a]) return fail(h, PIC_ENOMEM, "staging allocation failed");
  CK(h,
     pic::launch_unload(h->g, s.buf[s.cur], s.d_count, n, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], dev[6],
                        did, dal, h->st),
     "unload");
  h->launches++;
  if (host) {
    for (int a = 0; a < 7; ++a)
      if (outs[a]) CK(h, cudaMemcpyAsync(outs[a], dev[a], (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->st), "D2H");
    if (id) CK(h, cudaMemcpyAsync(id, did, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->st), "D2H");
    if (alive) CK(h, cudaMemcpyAsync(alive, dal, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st), "D2H");
  }
  for (void *p : tmp) cudaFreeAsync(p, h->st);
  return check_device_errors(h);
}

int pic_diag(pic_handle *h, pic_diag_t *out) {
  if (!h || !out) return fail(h, PIC_EINVAL, "NULL argument");
  memset(out, 0, sizeof(*out));
  int r = compute_rho(h, h->rho);
  if (r) return r;
  if (h->cfg.filter_passes > 0) {
    // Gauss's law and continuity hold for the equally smoothed charge
    int nl = 0;
    CK(h, pic::launch_smooth(h->g, h->rho, true, h->f64, h->cfg.filter_passes, h->cfg.filter_compensate, h->st, &nl),
       "smooth rho");
    h->launches += nl;
  }
  CK(h, cudaMemsetAsync(h->red, 0, 16 * sizeof(double), h->st), "memset");
  const bool have_prev = h->rho_prev_step == h->step - 1;
  CK(h, pic::launch_field_diag(h->g, h->E, h->B, h->J, h->rho, have_prev ? h->rho_prev : nullptr, h->red, h->st),
     "field diag");
  h->launches++;
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    CK(h, pic::launch_particle_diag(h->g, s.buf[s.cur], s.d_count, s.slots, s.m, h->red + 8, h->st), "part diag");
    h->launches++;
  }
  double red[16];
  Counters c;
  CK(h, cudaMemcpyAsync(red, h->red, sizeof red, cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaMemcpyAsync(&c, h->ctr, sizeof c, cudaMemcpyDeviceToHost, h->st), "D2H");
  unsigned long long adj_esc = 0;
  if (h->adj_esc) {
    CK(h, join_adj(h), "adjoint join");  // the count is kept by the adjoint stream
    CK(h, cudaMemcpyAsync(&adj_esc, h->adj_esc, sizeof adj_esc, cudaMemcpyDeviceToHost, h->st), "D2H");
  }
  CK(h, cudaMemcpyAsync(h->rho_prev, h->rho, sizeof(double) * h->g.ncell, cudaMemcpyDeviceToDevice, h->st), "copy");
  CK(h, cudaStreamSynchronize(h->st), "diag sync");
  h->rho_prev_step = h->step;
  const double dV = h->g.dx[0] * h->g.dx[1] * h->g.dx[2];
  out->energy_e = 0.5 * red[0] * dV;
  out->energy_b = 0.5 * red[1] * dV;
  out->energy_field = out->energy_e + out->energy_b;
  out->charge = red[2] * dV;
  out->gauss_max = red[3];
  out->continuity_max = have_prev ? red[4] : -1.0;
  out->energy_kinetic = red[8] * dV;
  out->n_alive = (int64_t)red[9];
  out->n_escaped = (int64_t)c.escaped;
  out->n_clamped = (int64_t)c.clamped;
  out->n_absorbed = (int64_t)c.absorbed;
  out->n_sorts_adaptive = h->adaptive_sorts;
  out->n_push_mid_drain = h->mid_drain_pushes;
  out->n_adj_escaped = (int64_t)adj_esc;
  out->step = h->step;
  if (c.error & pic::kErrBounds) return fail(h, PIC_EOVERFLOW, "an index outside its buffer was caught (checked build)");
  if (c.error) return fail(h, PIC_EOVERFLOW, "device-side error flags set");
  if (red[5] > 0 || red[10] > 0) return fail(h, PIC_ENAN, "non-finite field or momentum values");
  return PIC_OK;
}

int pic_energy(pic_handle *h, pic_energy_t *out) {
  if (!h || !out) return fail(h, PIC_EINVAL, "NULL argument");
  CK(h, cudaMemsetAsync(h->red, 0, 16 * sizeof(double), h->st), "memset");
  CK(h, pic::launch_field_energy(h->g, h->E, h->B, h->red, h->st), "field energy");
  h->launches++;
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    CK(h, pic::launch_particle_diag(h->g, s.buf[s.cur], s.d_count, s.slots, s.m, h->red + 8, h->st), "part diag");
    h->launches++;
  }
  double red[16];
  CK(h, cudaMemcpyAsync(red, h->red, sizeof red, cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaStreamSynchronize(h->st), "energy sync");
  const double dV = h->g.dx[0] * h->g.dx[1] * h->g.dx[2];
  out->energy_e = 0.5 * red[0] * dV;
  out->energy_b = 0.5 * red[1] * dV;
  out->energy_kinetic = red[8] * dV;
  out->n_alive = (int64_t)red[9];
  out->step = h->step;
  if (red[10] > 0) return fail(h, PIC_ENAN, "non-finite momenta");
  return PIC_OK;
}

int pic_sync(pic_handle *h) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  CK(h, join_adj(h), "adjoint join");
  return check_device_errors(h);
}

int pic_profile(pic_handle *h, int enable) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  join_adj(h);
  cudaStreamSynchronize(h->st);
  for (auto &t : h->timers) {
    h->event_pool.push_back(t.a);
    h->event_pool.push_back(t.b);
  }
  h->timers.clear();
  h->profiling = enable != 0;
  return PIC_OK;
}

int pic_timings(pic_handle *h, double *ms, int64_t *launches, int nmax, int *ncls) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  CK(h, join_adj(h), "adjoint join");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  double acc[pic::KC_N] = {};
  int64_t cnt[pic::KC_N] = {};
  for (auto &t : h->timers) {
    float v = 0.f;
    CK(h, cudaEventElapsedTime(&v, t.a, t.b), "event time");
    acc[t.cls] += v;
    cnt[t.cls] += 1;
  }
  const int n = nmax < pic::KC_N ? nmax : pic::KC_N;
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = cnt[i];
  }
  if (ncls) *ncls = n;
  return PIC_OK;
}

int pic_checkpoint(pic_handle *h, int slot) {
  if (!h || slot < 0 || slot > 4096) return fail(h, PIC_EINVAL, "bad checkpoint slot");
  if ((int)h->ckpt.size() <= slot) h->ckpt.resize(slot + 1);
  Timed tm(h, pic::KC_TAPE);
  cudaError_t e = save_snapshot(h, h->ckpt[slot]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(h, PIC_ENOMEM, "checkpoint allocation failed")
                                          : cuda_fail(h, e, "checkpoint");
  }
  return PIC_OK;
}

int pic_restore(pic_handle *h, int slot) {
  if (!h || slot < 0 || slot >= (int)h->ckpt.size() || !h->ckpt[slot].allocated)
    return fail(h, PIC_EINVAL, "no such checkpoint");
  Snapshot &sn = h->ckpt[slot];
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  Timed tm(h, pic::KC_TAPE);
  CK(h, cudaMemcpyAsync(h->E[0], sn.E[0], 6 * fb, cudaMemcpyDeviceToDevice, h->st), "restore");
  for (int i = 0; i < h->nsp; ++i) {
    Species &s = h->sp[i];
    CK(h, copy_particles(h, s.buf[s.cur], s.d_count, sn.sp[i].p, sn.sp[i].count, s.slots), "restore");
    s.need_sort = true;
  }
  h->step = sn.step;
  return PIC_OK;
}

int pic_tape_begin(pic_handle *h, int nsteps) {
  if (!h || nsteps < 0 || nsteps > 100000) return fail(h, PIC_EINVAL, "bad tape length");
  CK(h, make_tape_events(h), "events");
  // the other buffer, once its last reversal (on st_adj) has run
  h->tape_buf ^= 1;
  CK(h, cudaStreamWaitEvent(h->st, h->tape_free[h->tape_buf], 0), "tape buffer wait");
  std::vector<Snapshot> &tape = cur_tape(h);
  while ((int)tape.size() > nsteps) {
    free_snapshot(tape.back(), h->st);
    tape.pop_back();
  }
  tape.resize(nsteps);
  for (int k = 0; k < nsteps; ++k) {
    cudaError_t e = alloc_snapshot(h, tape[k]);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, PIC_ENOMEM, "tape allocation failed");
    }
  }
  h->tape_len = 0;
  h->taping = nsteps > 0;
  return PIC_OK;
}

int pic_tape_record(pic_handle *h) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  std::vector<Snapshot> &tape = cur_tape(h);
  if (!h->taping || h->tape_len >= (int)tape.size())
    return fail(h, PIC_EINVAL, "no tape entry left to record (pic_tape_begin)");
  {
    Timed tm(h, pic::KC_TAPE);
    CK(h, save_snapshot(h, tape[h->tape_len], true, h->tape_len > 0 ? &tape[h->tape_len - 1] : nullptr),
       "tape record");
  }
  h->tape_len++;
  if (h->tape_len >= (int)tape.size()) h->taping = false;
  return PIC_OK;
}

int pic_adjoint_begin(pic_handle *h, int64_t id_capacity) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  CK(h, make_tape_events(h), "events");
  if (!h->st_adj) CK(h, cudaStreamCreateWithFlags(&h->st_adj, cudaStreamNonBlocking), "adjoint stream");
  CK(h, join_adj(h), "adjoint join");
  if (h->g.dims != 2 || h->g.order != 2)
    return fail(h, PIC_EINVAL, "adjoint kernels exist for 2D3V with the TSC shape only");
  if (h->cfg.filter_passes > 0 || h->cfg.gather != PIC_GATHER_MOMENTUM)
    return fail(h, PIC_EINVAL, "adjoint kernels cover the unfiltered momentum-conserving cycle only");
  if (h->laser.enabled && h->laser.angle != 0.0)
    return fail(h, PIC_EINVAL, "adjoint kernels cover a laser at normal incidence only");
  if (id_capacity <= 0 || id_capacity > 0x7fffffffLL) return fail(h, PIC_EINVAL, "bad id capacity");
  if (!h->adj_ready || h->id_cap != id_capacity) {
    free_adjoint(h);
    const size_t fb = (size_t)h->g.ncell * h->rsize;
    const size_t ib = (size_t)id_capacity * h->rsize;
    bool ok = true;
    for (int d = 0; d < 3 && ok; ++d)
      ok = cudaMalloc(&h->lE[d], fb) == cudaSuccess && cudaMalloc(&h->lB[d], fb) == cudaSuccess &&
           cudaMalloc(&h->lJ[d], fb) == cudaSuccess;
    ok = ok && cudaMalloc(&h->pend, 8 * sizeof(double) * (size_t)h->g.n[1] * h->g.n[2]) == cudaSuccess &&
         cudaMalloc(&h->da0, sizeof(double)) == cudaSuccess && cudaMalloc(&h->objF, sizeof(double)) == cudaSuccess &&
         cudaMalloc(&h->adj_err, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc(&h->adj_esc, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc(&h->adj_stage, (size_t)id_capacity * sizeof(double)) == cudaSuccess;
    for (int i = 0; i < h->nsp && ok; ++i) {
      for (int d = 0; d < 3 && ok; ++d)
        ok = cudaMalloc(&h->adj[i].lx[d], ib) == cudaSuccess && cudaMalloc(&h->adj[i].lu[d], ib) == cudaSuccess;
      ok = ok && cudaMalloc(&h->adj[i].lw, (size_t)id_capacity * sizeof(double)) == cudaSuccess;
    }
    if (!ok) {
      free_adjoint(h);
      cudaGetLastError();
      return fail(h, PIC_ENOMEM, "adjoint allocation failed");
    }
    h->id_cap = id_capacity;
    h->adj_ready = true;
  }
  CK(h, cudaMemsetAsync(h->adj_esc, 0, sizeof(unsigned long long), h->st), "zero");
  const size_t fb = (size_t)h->g.ncell * h->rsize;
  const size_t ib = (size_t)h->id_cap * h->rsize;
  for (int d = 0; d < 3; ++d) {
    CK(h, cudaMemsetAsync(h->lE[d], 0, fb, h->st), "zero");
    CK(h, cudaMemsetAsync(h->lB[d], 0, fb, h->st), "zero");
    CK(h, cudaMemsetAsync(h->lJ[d], 0, fb, h->st), "zero");
  }
  for (int i = 0; i < h->nsp; ++i) {
    for (int d = 0; d < 3; ++d) {
      CK(h, cudaMemsetAsync(h->adj[i].lx[d], 0, ib, h->st), "zero");
      CK(h, cudaMemsetAsync(h->adj[i].lu[d], 0, ib, h->st), "zero");
    }
    CK(h, cudaMemsetAsync(h->adj[i].lw, 0, (size_t)h->id_cap * sizeof(double), h->st), "zero");
  }
  CK(h, cudaMemsetAsync(h->da0, 0, sizeof(double), h->st), "zero");
  CK(h, cudaMemsetAsync(h->objF, 0, sizeof(double), h->st), "zero");
  CK(h, cudaMemsetAsync(h->adj_err, 0, sizeof(unsigned long long), h->st), "zero");
  return PIC_OK;
}

int pic_adjoint_seed_kinetic(pic_handle *h, int species, int col_lo, int col_hi, double *F) {
  if (!h || !h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  if (col_lo < 0 || col_hi > h->g.n[0] || col_lo >= col_hi) return fail(h, PIC_EINVAL, "bad column range");
  Species &s = h->sp[species];
  const double dVm = h->g.dx[0] * h->g.dx[1] * h->g.dx[2] * s.m;
  CK(h, join_adj(h), "adjoint join");
  CK(h, cudaMemsetAsync(h->objF, 0, sizeof(double), h->st), "zero");
  CK(h,
     pic::launch_adj_seed(h->g, s.buf[s.cur], s.d_count, s.slots, col_lo, col_hi, dVm, h->adj[species].lu,
                          h->adj[species].lw, h->objF, h->id_cap, h->adj_err, h->st),
     "adjoint seed");
  h->launches++;
  double v = 0;
  unsigned long long err = 0;
  CK(h, cudaMemcpyAsync(&v, h->objF, sizeof(double), cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaMemcpyAsync(&err, h->adj_err, sizeof(err), cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  if (err) return fail(h, PIC_EINVAL, "a particle id is not below the adjoint id capacity");
  if (F) *F = v;
  return PIC_OK;
}

int pic_adjoint_step(pic_handle *h, int nsteps) {
  if (!h || !h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (nsteps < 0 || nsteps > h->tape_len) return fail(h, PIC_EINVAL, "more adjoint steps than recorded steps");
  const bool walls = h->g.absorb_lo || h->g.absorb_hi;
  // The reversal runs on st_adj after everything enqueued on st so far (the
  // tape's recording, seeds, adjoint writes), so that st can go on with the
  // next segment's recomputation meanwhile.
  cudaStream_t sa = h->st_adj;
  CK(h, cudaEventRecord(h->ev_main, h->st), "event");
  CK(h, cudaStreamWaitEvent(sa, h->ev_main, 0), "event wait");
  std::vector<Snapshot> &tape = cur_tape(h);
  for (int t = 0; t < nsteps; ++t) {
    Snapshot &en = tape[h->tape_len - 1];
    const double t_old = en.step * h->g.dt, t_new = (en.step + 1) * h->g.dt;
    {
      Timed tm(h, pic::KC_ADJ_FIELD, sa);
      CK(h, pic::launch_adj_yee_b(h->g, h->lE, h->lB, 0.5 * h->g.dt, nullptr, sa), "adjoint B half");
      if (walls)
        CK(h,
           pic::launch_adj_mur(h->g, h->lE, h->pend,
                               pic::laser_step(h->laser, h->laser_prof, 1.0, h->g, t_old, t_new), h->da0, sa),
           "adjoint Mur");
      CK(h, pic::launch_adj_yee_e(h->g, h->lE, h->lB, h->lJ, h->g.dt, sa), "adjoint E");
      // the second B half also adds the Mur transpose's old-time terms
      CK(h, pic::launch_adj_yee_b(h->g, h->lE, h->lB, 0.5 * h->g.dt, walls ? h->pend : nullptr, sa),
         "adjoint B half");
    }
    h->launches += walls ? 4 : 3;
    for (int i = 0; i < h->nsp; ++i) {
      Species &s = h->sp[i];
      Timed tm(h, pic::KC_ADJ_PUSH, sa);
      const PCopy &c = en.sp[i];
      pic::AdjTiles tt;
      tt.work_tile = c.work_tile;
      tt.work_pb = c.work_pb;
      tt.tile_start = c.tile_start;
      tt.nwork = c.nwork;
      tt.chunk = c.chunk;
      tt.esc_total = h->adj_esc;
      int nl = 0;
      CK(h,
         pic::launch_adj_push(h->g, c.p, c.count, s.slots, en.E, en.B, h->lJ, h->lE, h->lB, h->adj[i].lx,
                              h->adj[i].lu, h->adj[i].lw, h->id_cap, h->adj_err, s.q, s.m, c.tiled ? &tt : nullptr,
                              sa, &nl),
         "adjoint push");
      h->launches += nl;
    }
    h->tape_len--;
  }
  // the tape buffer may be recorded into again once this has run
  CK(h, cudaEventRecord(h->tape_free[h->tape_buf], sa), "event");
  return PIC_OK;
}

int pic_grad(pic_handle *h, double *d_a0, int species, double *d_w, int mem_kind) {
  if (!h || !h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (d_w && (species < 0 || species >= h->nsp)) return fail(h, PIC_EINVAL, "bad species index");
  CK(h, join_adj(h), "adjoint join");
  const cudaMemcpyKind kind = mem_kind == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (d_a0) CK(h, cudaMemcpyAsync(d_a0, h->da0, sizeof(double), kind, h->st), "grad copy");
  if (d_w) CK(h, cudaMemcpyAsync(d_w, h->adj[species].lw, (size_t)h->id_cap * sizeof(double), kind, h->st), "grad copy");
  unsigned long long err = 0;
  CK(h, cudaMemcpyAsync(&err, h->adj_err, sizeof(err), cudaMemcpyDeviceToHost, h->st), "D2H");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  if (err) return fail(h, PIC_EINVAL, "a particle id is not below the adjoint id capacity");
  return PIC_OK;
}

int pic_grad_binned(pic_handle *h, int species, const int32_t *bin_of_id, int64_t n_ids, int nbins, double *out,
                    int mem_kind) {
  if (!h || !bin_of_id || !out) return fail(h, PIC_EINVAL, "NULL argument");
  if (!h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  if (n_ids < 0 || n_ids > h->id_cap) return fail(h, PIC_EINVAL, "n_ids outside [0, id capacity]");
  if (nbins < 1) return fail(h, PIC_EINVAL, "nbins < 1");
  CK(h, join_adj(h), "adjoint join");
  const bool host = mem_kind == PIC_MEM_HOST;
  int32_t *dbin = nullptr;
  double *dout = nullptr;
  bool ok = cudaMallocAsync(&dout, sizeof(double) * (size_t)nbins, h->st) == cudaSuccess;
  if (ok && host && n_ids > 0) ok = cudaMallocAsync(&dbin, sizeof(int32_t) * (size_t)n_ids, h->st) == cudaSuccess;
  int r = PIC_OK;
  if (!ok) {
    cudaGetLastError();
    r = fail(h, PIC_ENOMEM, "gradient bins allocation failed");
  }
  cudaError_t e = cudaSuccess;
  if (!r) e = cudaMemsetAsync(dout, 0, sizeof(double) * (size_t)nbins, h->st);
  if (!r && e == cudaSuccess && dbin)
    e = cudaMemcpyAsync(dbin, bin_of_id, sizeof(int32_t) * (size_t)n_ids, cudaMemcpyHostToDevice, h->st);
  if (!r && e == cudaSuccess)
    e = pic::launch_sum_by_bin(h->adj[species].lw, host ? dbin : bin_of_id, n_ids, nbins, dout, h->st);
  if (!r && e == cudaSuccess) {
    h->launches++;
    e = cudaMemcpyAsync(out, dout, sizeof(double) * (size_t)nbins,
                        host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st);
  }
  unsigned long long err = 0;
  if (!r && e == cudaSuccess) e = cudaMemcpyAsync(&err, h->adj_err, sizeof(err), cudaMemcpyDeviceToHost, h->st);
  if (dbin) cudaFreeAsync(dbin, h->st);
  if (dout) cudaFreeAsync(dout, h->st);
  if (!r && e != cudaSuccess) r = cuda_fail(h, e, "gradient bins");
  if (r) return r;
  CK(h, cudaStreamSynchronize(h->st), "sync");
  if (err) return fail(h, PIC_EINVAL, "a particle id is not below the adjoint id capacity");
  return PIC_OK;
}

int pic_adjoint_field(pic_handle *h, int which, double *out, int mem_kind) {
  if (!h || !out) return fail(h, PIC_EINVAL, "NULL argument");
  if (!h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (which < PIC_EX || which > PIC_JZ) return fail(h, PIC_EINVAL, "bad field selector (PIC_EX .. PIC_JZ)");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  CK(h, join_adj(h), "adjoint join");
  const void *src = which < 3 ? h->lE[which] : which < 6 ? h->lB[which - 3] : h->lJ[which - 6];
  CK(h, pic::launch_field_to_f64(h->g, src, h->f64, h->st), "convert");
  int r = copy_out(h, out, h->f64, sizeof(double) * h->g.ncell, mem_kind);
  if (r) return r;
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_adjoint_set_field(pic_handle *h, int which, const double *in, int mem_kind) {
  if (!h || !in) return fail(h, PIC_EINVAL, "NULL argument");
  if (!h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (which < PIC_EX || which > PIC_BZ) return fail(h, PIC_EINVAL, "bad field selector (PIC_EX .. PIC_BZ)");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  CK(h, join_adj(h), "adjoint join");
  CK(h,
     cudaMemcpyAsync(h->f64, in, sizeof(double) * h->g.ncell,
                     mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st),
     "copy in");
  void *dst = which < 3 ? h->lE[which] : h->lB[which - 3];
  CK(h, pic::launch_field_from_f64(h->g, h->f64, dst, h->st), "convert");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_adjoint_momenta(pic_handle *h, int species, double *lux, double *luy, double *luz, int mem_kind) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (!h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  CK(h, join_adj(h), "adjoint join");
  double *outs[3] = {lux, luy, luz};
  for (int d = 0; d < 3; ++d) {
    if (!outs[d]) continue;
    CK(h, pic::launch_to_f64(h->g.prec, h->adj[species].lu[d], h->adj_stage, h->id_cap, h->st), "convert");
    int r = copy_out(h, outs[d], h->adj_stage, sizeof(double) * (size_t)h->id_cap, mem_kind);
    if (r) return r;
  }
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_adjoint_set_momenta(pic_handle *h, int species, const double *lux, const double *luy, const double *luz,
                            int mem_kind) {
  if (!h) return fail(h, PIC_EINVAL, "NULL handle");
  if (!h->adj_ready) return fail(h, PIC_EINVAL, "call pic_adjoint_begin first");
  if (species < 0 || species >= h->nsp) return fail(h, PIC_EINVAL, "bad species index");
  if (mem_kind != PIC_MEM_HOST && mem_kind != PIC_MEM_DEVICE) return fail(h, PIC_EINVAL, "bad memory kind");
  CK(h, join_adj(h), "adjoint join");
  const double *ins[3] = {lux, luy, luz};
  for (int d = 0; d < 3; ++d) {
    if (!ins[d]) continue;
    CK(h,
       cudaMemcpyAsync(h->adj_stage, ins[d], sizeof(double) * (size_t)h->id_cap,
                       mem_kind == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st),
       "copy in");
    CK(h, pic::launch_from_f64(h->g.prec, h->adj_stage, h->adj[species].lu[d], h->id_cap, h->st), "convert");
  }
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return PIC_OK;
}

int pic_launch_count(pic_handle *h, int64_t *count) {
  if (!h || !count) return fail(h, PIC_EINVAL, "NULL argument");
  *count = h->launches;
  return PIC_OK;
}

}  // extern "C"
