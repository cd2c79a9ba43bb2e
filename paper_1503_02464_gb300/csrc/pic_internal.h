// Internal interface between the host runtime (api.cu) and the kernel
// translation units.  Not part of the public ABI (include/pic.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace pic {

// Geometry of the grid and of the push kernel's cell tiles.
struct Grid {
  int dims;        // 2 or 3
  int order;       // 1 CIC, 2 TSC
  int prec;        // PIC_FP32 / PIC_FP64
  int n[3];        // cells per axis (n[2] = 1 in 2D)
  double dx[3];    // cell sizes
  double dt;
  int tile[3];     // tile shape (tile[2] = 1 in 2D)
  int ntile[3];    // tiles per axis (ceil)
  int64_t ntiles;  // product
  int drift;       // cells a particle may leave its tile and still use the window
  int64_t ncell;
  int absorb_lo, absorb_hi;  // x walls absorbing
  int gather_ec;             // energy-conserving gather (lower order at half-integer positions)
};

// Laser entering through the x = 0 wall (copied from pic_config).  At normal
// incidence its polarised field is a0 P(y, z) T(t - x): the transverse
// profile P = exp(-r^2 / waist^2), r measured from the spot centre (yc, zc),
// times the waveform T(tau) = sin^2(pi tau / duration) sin(tau) on
// 0 < tau < duration (carrier frequency 1), 0 elsewhere.  A tilt `angle` in
// the x-y plane delays the wall rows along y and tilts the profile with the
// beam axis (laser_wave).
struct Laser {
  int enabled;
  double a0, waist, duration, yc, zc;
  int pol;       // 1: E in the x-y plane (Ey at the wall), 2: E along z
  double angle;  // propagation direction (cos, sin, 0) in the x-y plane
};

// The waveform T(tau) (host).
double laser_waveform(const Laser &L, double tau);

// What the Mur kernels need of the laser for one step from t_old to t_new.
// Normal incidence: amp = {T(t_old), T(t_old - dx), T(t_new), T(t_new - dx)}
// times the amplitude (a0 for the forward update, 1 for the adjoint's
// dF/da0), and prof = P at the wall rows of the polarised component (n1 * n2
// doubles: Ey rows at (j + 1/2, k), Ez rows at (j, k + 1/2)); pol = 0: no
// laser.  Oblique incidence (oblique = 1): the wave's delay and profile vary
// along the wall, so the kernel evaluates it per row from the parameters
// below (laser_wave).
struct LaserStep {
  int pol;
  double amp[4];
  const double *prof;
  int oblique, dims;
  double a, cos_t, sin_t, y0, yc, zc, inv_w2, duration, t_old, t_new, dx, dy, dz;
};
LaserStep laser_step(const Laser &L, const double *prof, double amplitude, const Grid &g, double t_old, double t_new);

// The incoming oblique wave's polarised component at (x, y, z, t) (device).
__host__ __device__ inline double laser_wave(const LaserStep &ls, double x, double y, double z, double t) {
  const double tau = t - x * ls.cos_t - (y - ls.y0) * ls.sin_t;
  if (tau <= 0.0 || tau >= ls.duration) return 0.0;
  const double env = sin(3.14159265358979323846 * tau / ls.duration);
  const double rp = (y - ls.yc) * ls.cos_t - x * ls.sin_t;  // distance from the beam axis in the x-y plane
  const double r2 = rp * rp + (ls.dims == 3 ? (z - ls.zc) * (z - ls.zc) : 0.0);
  return ls.a * exp(-r2 * ls.inv_w2) * env * env * sin(tau);
}

// Particles whose new position leaves [kWallLo, n0 - kWallHiMargin) cells in
// x are removed at absorbing walls (after depositing their move).
constexpr double kWallLo = 3.0;
constexpr double kWallHiMargin = 4.0;

// One buffer of a species' structure-of-arrays particle storage.  Real
// arrays are float (FP32 path) or double (FP64 path).
struct Particles {
  int32_t *cell;   // linear cell index i + n0*(j + n1*k); -1 = dead slot
  void *off[3];    // in-cell offset in [0,1) per axis
  void *u[3];      // momentum u = gamma v
  void *w;         // weight
  uint32_t *id;    // tag (permuted only by the sort)
};

// Device-side counters, one block per simulation.
struct Counters {
  unsigned long long escaped;   // particle-steps taken on the global-memory path
  unsigned long long clamped;   // FP32/FP64 offsets clamped after a carry
  unsigned long long absorbed;  // particles removed at absorbing walls
  unsigned long long error;     // bit flags of device-side errors
};

// Device-side error bits of Counters::error.
constexpr unsigned long long kErrBounds = 2ull;  // an index outside its buffer (checked builds)

// Index checks of the checked build (PIC_CHECKED): a failed check sets
// kErrBounds in *ctr and evaluates to false, so the caller skips the access;
// release builds compile the check away (always true).
#ifdef PIC_CHECKED
#define PIC_CHECK(cond, ctr) ((cond) || (atomicOr(&(ctr)->error, ::pic::kErrBounds), false))
#else
#define PIC_CHECK(cond, ctr) true
#endif

// Error text reported by pic_last_error(NULL) (entry points without a handle).
void set_global_error(const std::string &msg);

constexpr int kTilePad = 4;

// Most particle slots one block accumulates into a shared window: FP32 runs
// keep each node's fixed-point sum as a pair of int32 words, and the low word
// (at most 2^15 in magnitude per contribution, one contribution per particle
// and node) cannot overflow below 65,536 contributions.
constexpr int64_t kMaxWindowSlots = 65280;

enum KernelClass {
  KC_SORT = 0, KC_ZEROJ = 1, KC_PUSH = 2, KC_YEE_B = 3, KC_YEE_E = 4, KC_BOUNDARY = 5, KC_FILTER = 6,
  KC_ADJ_FIELD = 7, KC_ADJ_PUSH = 8, KC_TAPE = 9, KC_N = 10
};

// ---- push (push.cu) ----
// Tile shape compiled into the push kernel (8x8x4 in 3D, 16x16 in 2D); the
// drift allowance is one cell.
void push_tile_shape(int dims, int tile[3]);
size_t push_smem_bytes(const Grid &g);
// Work items of the push kernel: each tile's slot run is cut into pieces of
// at most `chunk` slots; item i covers slots [work_pb[i], min(work_pb[i] +
// chunk, tile_start[t + 1])) of tile t = work_tile[i] (-1: no work).  nwork
// bounds the item count (slots / chunk + 1 + ntiles).
struct WorkSplit {
  int64_t chunk = 0;
  int64_t nwork = 0;
  int32_t *work_tile = nullptr;
  int64_t *work_pb = nullptr;
};

// Tile kernel (one block per work item) + escape kernel.  tq (2 floats per
// work item) carries the bound of the FP32 fixed-point deposit from one step
// to the next; fresh = 1 on the first push after a sort (tq is recomputed
// from the particles).
// esc_list (one int per slot) is scratch for particles deferred to the
// escape kernel; esc_count (two counters) receives their number and the
// number of deferred deposit jobs (particles whose shape support changed)
// of the launch.  mid_drain selects the kernel variant that deposits those
// jobs between chunks when its queue fills (3D): the caller turns it on for
// a species whose last push averaged more than kPushQueueMidDrain jobs per
// work item.
constexpr int kPushQueueCap = 224;      // deferred deposit jobs a work item queues at a time
constexpr int kPushQueueMidDrain = 168;  // 3/4 of the queue
cudaError_t launch_push(const Grid &g, void *const E[3], void *const B[3], void *const J[3], const Particles &p,
                        const int64_t *tile_start, const WorkSplit &ws, float *tq, int fresh, int32_t *esc_list,
                        unsigned long long *esc_count, double q, double m, Counters *ctr, cudaStream_t st,
                        int *nlaunch, int mid_drain);

// Diagnostics charge density of particles sorted by tile (exact 64-bit
// fixed-point window sums; adds into rho).
cudaError_t launch_rho_tiled(const Grid &g, const Particles &p, const int64_t *tile_start, double q, double *rho,
                             Counters *ctr, cudaStream_t st);

// ---- sort (sort.cu) ----
// Counting sort of the slots [0, *d_count) of `src` by (tile, cell-in-tile),
// dead slots dropped; result in `dst`, *d_count updated, tile_start[ntiles+1]
// written.  Each tile's run is padded with dead slots to a multiple of
// kTilePad.  `keys` has ntiles*tile_cells ints, `rank` one int per slot.

cudaError_t launch_sort(const Grid &g, const Particles &src, const Particles &dst, int64_t *d_count,
                        int64_t capacity, int32_t *keys, int32_t *rank, int64_t *tile_start, int64_t *tile_tmp,
                        const WorkSplit &ws, Counters *ctr, cudaStream_t st, int *nlaunch);

// ---- fields and particle conversion (fields.cu) ----
cudaError_t launch_yee_b(const Grid &g, void *const E[3], void *const B[3], double h, cudaStream_t st);
cudaError_t launch_yee_e(const Grid &g, void *const E[3], void *const B[3], void *const J[3], double h,
                         cudaStream_t st);
// First-order Mur walls: save E^n (y, z) of the nodes 0, 1, n0-2, n0-1 into
// `buf` (8 * n1 * n2 values) before the E update; apply afterwards, with the
// incoming laser wave at x = 0 (times t_old = n dt, t_new = (n+1) dt).
cudaError_t launch_mur_save(const Grid &g, void *const E[3], double *buf, cudaStream_t st);
cudaError_t launch_mur_apply(const Grid &g, void *const E[3], const double *buf, const LaserStep &ls,
                             cudaStream_t st);
// Load n particles into slots [offset, offset+n).
cudaError_t launch_load(const Grid &g, const Particles &p, int64_t offset, int64_t n, const double *x,
                        const double *y, const double *z, const double *ux, const double *uy, const double *uz,
                        const double *w, const uint32_t *id, uint32_t id_base, unsigned long long *bad,
                        cudaStream_t st);
// Count (into *bad) the slots below n of p that are neither dead nor a valid
// particle of the grid: cell outside it, offsets outside [0, 1), non-finite
// momenta or weight, or a position beyond absorbing walls.
cudaError_t launch_check_particles(const Grid &g, const Particles &p, int64_t n, unsigned long long *bad,
                                  cudaStream_t st);
cudaError_t launch_unload(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double *x,
                          double *y, double *z, double *ux, double *uy, double *uz, double *w, uint32_t *id,
                          int32_t *alive, cudaStream_t st);
cudaError_t launch_field_to_f64(const Grid &g, const void *src, double *dst, cudaStream_t st);
// Box [lo, hi) of grid positions or cells (output capture).
struct OutBox {
  int lo[3], hi[3];
};
// Copy a box of one field (FP64 if f64, else the grid's precision) into an
// FP64 frame, x fastest.
cudaError_t launch_out_field(const Grid &g, const void *f, bool f64, const OutBox &b, double *out, cudaStream_t st);
// Records (x, y, z, ux, uy, uz, w, id as doubles) of the particles whose cell
// is in the box; *count (zeroed by the caller) receives how many were found,
// at most cap are written.
cudaError_t launch_out_particles(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax,
                                 const OutBox &b, double *out, unsigned long long *count, int64_t cap,
                                 cudaStream_t st);
// Current smoothing of one field in place: `passes` binomial passes along
// every axis, then (compensate) one compensating pass.  f64 selects the
// element type (double, else the grid's precision); tmp holds ncell elements
// of that type.  *nlaunch receives the kernels launched.
cudaError_t launch_smooth(const Grid &g, void *f, bool f64, void *tmp, int passes, int compensate, cudaStream_t st,
                          int *nlaunch);
// n values between an array of the run's real type (prec: PIC_FP32 or
// PIC_FP64) and FP64, on the device.
cudaError_t launch_to_f64(int prec, const void *src, double *dst, int64_t n, cudaStream_t st);
cudaError_t launch_from_f64(int prec, const double *src, void *dst, int64_t n, cudaStream_t st);
cudaError_t launch_field_from_f64(const Grid &g, const double *src, void *dst, cudaStream_t st);
cudaError_t launch_rho(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double q,
                       double *rho, cudaStream_t st);
// Reductions into out[] (double): 0 sum E^2, 1 sum B^2, 2 sum rho, 3 max|divE-rho|,
// 4 max|(rho-rho_prev)/dt + div J| (if rho_prev), 5 nonfinite count (fields)
cudaError_t launch_field_diag(const Grid &g, void *const E[3], void *const B[3], void *const J[3],
                              const double *rho, const double *rho_prev, double *out, cudaStream_t st);
// out[0] += sum E^2, out[1] += sum B^2
cudaError_t launch_field_energy(const Grid &g, void *const E[3], void *const B[3], double *out, cudaStream_t st);
// out[0] += sum w m (gamma-1), out[1] += live count, out[2] += nonfinite count
cudaError_t launch_particle_diag(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, double m,
                                 double *out, cudaStream_t st);

// ---- adjoint (adjoint.cu) ----
// pend (may be null): the Mur transpose's old-time terms, added to lamE at the
// wall nodes in the same pass (the second B half of the reversed step).
cudaError_t launch_adj_yee_b(const Grid &g, void *const lE[3], void *const lB[3], double h, const double *pend,
                             cudaStream_t st);
cudaError_t launch_adj_yee_e(const Grid &g, void *const lE[3], void *const lB[3], void *const lJ[3], double h,
                             cudaStream_t st);
cudaError_t launch_adj_mur(const Grid &g, void *const lE[3], double *pend, const LaserStep &ls_unit, double *da0,
                           cudaStream_t st);
// Work items of a recorded particle buffer (those of the sort in effect when
// it was recorded, see WorkSplit) for the windowed adjoint kernel;
// esc_total counts the particles that had drifted beyond their tile window
// (a running sum).
struct AdjTiles {
  const int32_t *work_tile = nullptr;
  const int64_t *work_pb = nullptr;
  const int64_t *tile_start = nullptr;
  int64_t nwork = 0, chunk = 0;
  unsigned long long *esc_total = nullptr;
};
// Per-particle adjoint of one recorded step (2D3V TSC only): tp/d_count
// is the particle state at the start of the step, E/B the fields gathered.
// With tt (and tiles of at most 16x16 cells) one block per work item stages
// its tile window in shared memory; without, one pass over all slots with
// the nodes in global memory.  *nlaunch receives the kernel launches.
cudaError_t launch_adj_push(const Grid &g, const Particles &tp, const int64_t *d_count, int64_t nmax,
                            void *const E[3], void *const B[3], void *const lJ[3], void *const lE[3],
                            void *const lB[3], void *const lx[3], void *const lu[3], double *lw, int64_t id_cap,
                            unsigned long long *err, double q, double m, const AdjTiles *tt, cudaStream_t st,
                            int *nlaunch);
// Objective sum over particles with x column in [c_lo, c_hi) of
// w dV m (gamma - 1) into *F; seeds lam_u and dF/dw (by id).
// out[b] += sum of w[i] over i < n with bin[i] == b in [0, nbins).
cudaError_t launch_sum_by_bin(const double *w, const int32_t *bin, int64_t n, int nbins, double *out,
                              cudaStream_t st);
cudaError_t launch_adj_seed(const Grid &g, const Particles &p, const int64_t *d_count, int64_t nmax, int c_lo,
                            int c_hi, double dVm, void *const lu[3], double *lw, double *F, int64_t id_cap,
                            unsigned long long *err, cudaStream_t st);

}  // namespace pic
