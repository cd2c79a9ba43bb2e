/*
 * pic.h -- C ABI of the GB300 particle-in-cell library (libpic.so).
 *
 * The library runs the standard relativistic PIC cycle of section 2 of
 * "Optimising PICCANTE -- an Open Source Particle-in-Cell Code for Advanced
 * Simulations on Tier-0 Systems" on one GPU (sm_103a):
 *
 *   field gather   force from the g-weighted average of the Yee fields (§2)
 *   Boris push     dp/dt = q(E + v x B), v = p / sqrt(p^2 + m^2)  (§2 eqs. 1, 3, ref [8])
 *   leap-frog move dr/dt = v                                       (§2 eq. 3)
 *   deposit        J = sum q v g, charge-conserving (Esirkepov)    (§2 eq. 4 and the
 *                  continuity requirement of §2)
 *   Yee FDTD       dE/dt = curl B - J, dB/dt = -curl E             (§2, ref [9])
 *
 * Units are the paper's normalised ones (§2): c = 1, time in 1/omega_r, length
 * in c/omega_r, momentum u = p/(m c) = gamma v, fields in m c omega_r / e,
 * densities in epsilon_0 m omega_r^2 / e^2.  Then div E = rho and an electron
 * has q = -1, m = 1.
 *
 * Conventions shared by every call
 *  - Every call returns an int status: PIC_OK (0) or one of the PIC_E* codes.
 *    pic_last_error() gives a one-line description of the last failure.
 *  - The library owns every simulation buffer (allocated on the device with
 *    cudaMalloc at pic_create / pic_add_species time).  Pointers passed in are
 *    borrowed for the duration of the call only; output buffers belong to the
 *    caller.  mem_kind says whether a pointer is host (PIC_MEM_HOST) or device
 *    (PIC_MEM_DEVICE) memory.
 *  - Work is enqueued on config.stream (a cudaStream_t, NULL = legacy default
 *    stream).  pic_step is asynchronous; pic_fields, pic_particles, pic_diag and
 *    pic_sync synchronise that stream and report errors latched on the device.
 *  - A handle must not be used from two host threads at once.
 *
 * Grid and staggering (Yee lattice): cells i in [0,n[0]), j in [0,n[1]),
 * k in [0,n[2]); a field array is indexed i + n[0]*(j + n[1]*k) (x fastest).
 * Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2)
 * Bz(i+1/2,j+1/2,k); J sits with E; rho at the nodes (i,j,k).  dims = 2 is the
 * 2D3V case: n[2] = 1, three field and momentum components, nothing depends
 * on z.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PIC_OK 0
#define PIC_EINVAL 1    /* bad argument or configuration                       */
#define PIC_ECOURANT 2  /* dt above the Yee stability limit (sum dx^-2)^(-1/2)  */
#define PIC_ENOMEM 3    /* device allocation failed or capacity exceeded         */
#define PIC_ECUDA 4     /* a CUDA runtime call or kernel launch failed           */
#define PIC_EOVERFLOW 5 /* an internal bound was exceeded on the device          */
#define PIC_ETIMEOUT 6  /* a bounded device-side wait gave up (reserved: no
                           kernel of this library waits on another block or
                           on an asynchronous copy)                          */
#define PIC_ENAN 7      /* a non-finite value was found by a diagnostic          */

/* ---- enumerations ---- */
#define PIC_FP32 0 /* FP32 push/gather/deposit on cell-relative offsets */
#define PIC_FP64 1 /* the same cycle in FP64                            */

#define PIC_BC_PERIODIC 0
#define PIC_BC_ABSORBING 1 /* x walls only: first-order Mur fields, particles removed */

#define PIC_MEM_HOST 0
#define PIC_MEM_DEVICE 1

#define PIC_EX 0
#define PIC_EY 1
#define PIC_EZ 2
#define PIC_BX 3
#define PIC_BY 4
#define PIC_BZ 5
#define PIC_JX 6
#define PIC_JY 7
#define PIC_JZ 8
#define PIC_RHO 9 /* charge density of the particles plus the background */

/* Laser entering through the x = 0 wall (laser-plasma runs, §1-§2; the
 * paper gives no source formula -- see the boundary reading in the design
 * notes).  Field amplitude a0 (normalised vector potential), Gaussian
 * transverse profile exp(-r^2/waist^2) about (y_center, z_center), sin^2
 * envelope of total length `duration`, carrier frequency 1 (omega_r = omega
 * of the laser).  polarization 1 = E in the x-y plane (E along y at normal
 * incidence), 2 = E along z.  angle tilts the propagation direction in the
 * x-y plane to (cos angle, sin angle, 0), |angle| < pi/2: the incoming wave
 * is a0 A exp(-r^2/waist^2) T(tau) with r the distance from the beam axis
 * through (0, y_center, z_center), tau = t - x cos(angle) - (y - y0)
 * sin(angle), y0 the wall edge the tilted fronts reach first (0 for
 * angle > 0, the box height for angle < 0), and A = cos(angle) on Ey
 * (polarization 1) or 1 on Ez (polarization 2).  angle = 0 is normal
 * incidence. */
typedef struct {
  int enabled;
  double a0;
  double waist;
  double duration;
  double y_center;
  double z_center;
  int polarization;
  double angle;
} pic_laser;

typedef struct {
  int dims;            /* 2 (2D3V) or 3                                        */
  int n[3];            /* cells per axis; n[2] = 1 when dims = 2               */
  double dx[3];        /* cell sizes                                           */
  double dt;           /* time step; must satisfy dt <= (sum dx^-2)^(-1/2)     */
  int shape_order;     /* 1 = CIC (linear), 2 = TSC (quadratic) shape g (§2)   */
  int precision;       /* PIC_FP32 or PIC_FP64                                 */
  int bc_lo[3];        /* PIC_BC_* per axis; only x may be absorbing           */
  int bc_hi[3];
  int sort_every;      /* steps between particle sorts (0 = 20); a species is also
                          sorted early when its last push sent more than 0.5 %
                          of its particles down the escape path               */
  int tile[3];         /* cell-tile shape of the push kernel (0 = default)     */
  int drift_guard;     /* cells a particle may stray from its tile between sorts
                          and still use the tile's shared-memory window (0 = 1) */
  pic_laser laser;
  void *stream;        /* cudaStream_t                                         */
  /* Current smoothing after the deposit, before the E update (a standard
   * PIC step the paper's §2 does not detail): filter_passes three-point
   * binomial passes J(i) <- J(i)/2 + (J(i-1) + J(i+1))/4 along every axis
   * (periodic), each multiplying a Fourier mode by cos^2(k dx/2); with
   * filter_compensate one more pass with weights alpha = 1 + passes/2 and
   * (1 - alpha)/2 cancels the k^2 term.  0..8 passes; 0 = off.  The FP64
   * diagnostics then test Gauss's law and continuity on the equally smoothed
   * charge (the filter commutes with the Yee differences). */
  int filter_passes;
  int filter_compensate;
  /* Field gather (§2: the g-weighted average of the grid fields):
   * PIC_GATHER_MOMENTUM uses the shape of order shape_order at every Yee
   * location; PIC_GATHER_ENERGY lowers the order by one along each axis on
   * which a component sits at a half-integer position (CIC -> nearest grid
   * point, TSC -> CIC there), the energy-conserving variant. */
  int gather;
} pic_config;

#define PIC_GATHER_MOMENTUM 0
#define PIC_GATHER_ENERGY 1

/* FP64 diagnostics.  Sums across threads accumulate in double; FP32 runs sum
 * each thread's terms with compensated FP32 sums, and rho is deposited in
 * exact fixed point per cell tile (each particle's contributions adding up
 * to its charge exactly) before the FP64 adds. */
typedef struct {
  double energy_field;    /* 1/2 sum (E^2 + B^2) dV at the current integer time  */
  double energy_e;        /* electric part                                        */
  double energy_b;        /* magnetic part                                        */
  double energy_kinetic;  /* sum w dV m (gamma - 1) at the stored momenta         */
  double charge;          /* sum rho dV (particles + background)                  */
  double gauss_max;       /* max |div E - rho|                                    */
  double continuity_max;  /* max |(rho - rho_prev)/dt + div J| when the previous
                             pic_diag call was exactly one step earlier, else -1  */
  int64_t n_alive;        /* live macro-particles, all species                    */
  int64_t n_escaped;      /* particle-steps that left their tile window (slow path)*/
  int64_t n_clamped;      /* FP32 offsets clamped below 1 after a cell carry      */
  int64_t n_absorbed;     /* particles removed at absorbing walls                 */
  int64_t n_sorts_adaptive; /* sorts made ahead of the sort_every cadence because
                             a push sent more than 0.5 % of a species (at least
                             1024 particles) down the escape path              */
  int64_t step;           /* completed time steps                                 */
  int64_t n_push_mid_drain; /* species pushes that took the kernel variant which
                             deposits its deferred shape-changing particles
                             between chunks (chosen when the previous push of
                             the species averaged more than 168 of them per
                             work item, e.g. fast beams)                      */
  int64_t n_adj_escaped;  /* particle adjoints since pic_adjoint_begin computed
                             on the global-memory path: the particle had moved
                             more than 2 cells out of the tile it was sorted
                             into (the rest use the tile's window in shared
                             memory)                                          */
} pic_diag_t;

/* Per-step energy read-back: per-element terms in the storage precision,
 * summed per thread (FP32 runs: compensated FP32 sums, exact to a few FP32
 * ulps of the summed magnitudes) and across threads in FP64. */
typedef struct {
  double energy_e;        /* 1/2 sum E^2 dV                                       */
  double energy_b;        /* 1/2 sum B^2 dV                                       */
  double energy_kinetic;  /* sum w dV m (gamma - 1), all species                  */
  int64_t n_alive;        /* live macro-particles, all species                    */
  int64_t step;           /* completed time steps                                 */
} pic_energy_t;

typedef struct pic_handle pic_handle;

/* Create a simulation.  Validates sizes, shape order, precision, boundary
 * kinds and the Courant condition of the Yee scheme (§2 states dx_i >= c dt;
 * the limit enforced is the sharper (sum dx_i^-2)^(-1/2)).  Allocates and
 * zeroes E, B, J.  Returns PIC_EINVAL / PIC_ECOURANT / PIC_ENOMEM / PIC_ECUDA.
 * On failure *out is NULL.  Checkpoints, tape entries and load staging are
 * stream-ordered allocations from the device's default memory pool; the
 * first pic_create of the process lets that pool keep up to a quarter of
 * the device's memory after frees, for reuse (a process-wide pool
 * attribute), and a particle allocation that finds the device full returns
 * the kept memory first. */
int pic_create(const pic_config *cfg, pic_handle **out);

/* Release every device buffer and the handle (NULL is accepted). */
int pic_destroy(pic_handle *h);

/* Text of the last error on this handle (or of the last failed pic_create
 * when h is NULL).  Owned by the library; valid until the next call. */
const char *pic_last_error(const pic_handle *h);

/* Add a species of charge q and mass m with room for `capacity`
 * macro-particles (§2: each species a has q_a, m_a).  *species receives its
 * index (0, 1, ...).  Up to 8 species. */
int pic_add_species(pic_handle *h, double q, double m, int64_t capacity, int *species);

/* Append n particles to a species.  x, y, z are global positions (physical
 * units; z ignored in 2D), ux, uy, uz the momenta u = p/(m c) at time
 * t - dt/2 (leap-frog), w the weight (density carried, so rho = sum q w g),
 * id an optional tag (NULL = running index) kept through sorts.  Seven values
 * per particle as in §3.3, converted on the device to an integer cell plus an
 * in-cell offset.  Positions outside the box wrap on periodic axes.  A
 * particle outside the absorbing walls' [3, n[0] - 4) cells, or with a
 * non-finite position, momentum or weight, is stored dead and the call
 * returns PIC_EINVAL after loading the others.  Exceeding capacity:
 * PIC_ENOMEM (nothing loaded).  Host arrays are copied in chunks of 4M
 * particles through two device staging buffers (about 0.5 GB, freed before
 * the call returns), copy engine and conversion kernel overlapped; page-locked
 * arrays (cudaHostAlloc, cudaHostRegister) move at the host link's DMA rate.
 * Synchronises. */
int pic_load_particles(pic_handle *h, int species, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy, const double *uz,
                       const double *w, const uint32_t *id, int mem_kind);

/* Immobile neutralising background: rho_bg = -rho of the particles loaded so
 * far (so that E = 0 satisfies Gauss's law).  Used by the diagnostics only:
 * an immobile background carries no current.  Species loaded since their
 * last sort are sorted first, as the next pic_step would do (slot order
 * changes, dead slots are dropped). */
int pic_neutralize(pic_handle *h);

/* Set the immobile background charge density at the nodes (i, j, k):
 * rho_bg holds n[0]*n[1]*n[2] doubles, x fastest (host or device memory per
 * mem_kind, borrowed for the call).  It replaces any earlier background
 * (pic_neutralize included).  Like pic_neutralize it enters rho and the
 * Gauss-law diagnostics only; an immobile background carries no current, so
 * the particle cycle of section 2 is unchanged.  PIC_EINVAL for a NULL
 * pointer or a non-finite value (the background is then left unchanged). */
int pic_set_background(pic_handle *h, const double *rho_bg, int mem_kind);

/* Advance nsteps PIC cycles (enqueued on the stream; asynchronous).
 * Per step: sort (every sort_every steps) -> J = 0 -> per species one fused
 * gather/Boris/move/deposit launch -> Yee B half step -> E step -> B half
 * step (-> wall and laser boundary kernels when enabled). */
int pic_step(pic_handle *h, int nsteps);

/* Copy one field (PIC_EX .. PIC_RHO) as FP64 into out (n[0]*n[1]*n[2]
 * doubles, x fastest).  Synchronises.  J holds the current of the last step.
 * PIC_RHO deposits the particles' charge (plus background) first. */
int pic_fields(pic_handle *h, int which, double *out, int mem_kind);

/* Overwrite one field component (PIC_EX .. PIC_JZ) from FP64 data. */
int pic_set_field(pic_handle *h, int which, const double *in, int mem_kind);

/* Number of particle slots of a species (live particles plus dead ones not
 * yet compacted by a sort). */
int pic_num_particles(pic_handle *h, int species, int64_t *n);

/* Copy a species out in global FP64 coordinates, slot order.  Any pointer
 * may be NULL to skip that array.  alive[i] = 1 for a live slot.
 * Synchronises. */
int pic_particles(pic_handle *h, int species, double *x, double *y, double *z, double *ux,
                  double *uy, double *uz, double *w, uint32_t *id, int32_t *alive, int mem_kind);

/* FP64 diagnostics of the current state.  Synchronises; reports device-side
 * errors (PIC_EOVERFLOW, PIC_ENAN). */
int pic_diag(pic_handle *h, pic_diag_t *out);

/* The field and kinetic energies of the current state without the charge
 * density, Gauss and continuity checks of pic_diag (so it costs one pass
 * over the field arrays and one over the particles).  Synchronises. */
int pic_energy(pic_handle *h, pic_energy_t *out);

/* Wait for all enqueued work and report latched device errors. */
int pic_sync(pic_handle *h);

/* Per-kernel timing with CUDA events on the simulation stream.  enable = 1
 * starts recording (clearing previous records), 0 stops.  pic_timings
 * synchronises and writes, for up to nmax kernel classes, total milliseconds
 * (ms) and launch counts (launches) into caller-owned arrays of nmax
 * entries (either may be NULL); class order: 0 sort, 1 zero J, 2 push,
 * 3 Yee B, 4 Yee E, 5 boundary, 6 current smoothing, 7 adjoint field
 * updates, 8 adjoint particle kernel, 9 checkpoint, restore and tape copies
 * (device-to-device).  The number of classes written goes
 * to *ncls (NULL allowed).  PIC_EINVAL for a NULL handle. */
int pic_profile(pic_handle *h, int enable);
int pic_timings(pic_handle *h, double *ms, int64_t *launches, int nmax, int *ncls);

/* Number of kernels this handle has launched since creation. */
int pic_launch_count(pic_handle *h, int64_t *count);

/* ---- differentiable runs (2D3V, TSC) ----------------------------------
 * Reverse-mode gradients of an objective with respect to the laser
 * amplitude a0 and the particle weights w (hence an initial density
 * profile): hand-written adjoint kernels of the Yee update and its Mur
 * walls with the laser source, of the gather, the Boris push, the move and
 * the Esirkepov deposit (the transposes of the §2 step), FP32 or FP64 like
 * the forward, with the gradients accumulated in FP64.  A reverse sweep
 * needs the forward states of the steps it reverses: take checkpoints during
 * the forward run, and before reversing a segment restore its checkpoint and
 * re-run it with the tape on.  Checkpoints and tapes hold every species
 * added so far; add all species first. */

/* Save (restore) the full state -- fields, particles of every species, step
 * count -- in slot `slot` (0..4096; device memory, owned by the handle,
 * allocated on first use).  pic_restore marks the species for a sort at the
 * next step; it returns PIC_EINVAL for a slot never saved, PIC_ENOMEM when
 * pic_checkpoint cannot allocate the slot. */
int pic_checkpoint(pic_handle *h, int slot);
int pic_restore(pic_handle *h, int slot);

/* Record the state at the start of each of the next nsteps calls to the
 * step loop (after its sort), for pic_adjoint_step.  nsteps = 0 stops.  The
 * handle keeps two tape buffers and alternates between them at each call, so
 * that a segment can be recorded while the previous one is being reversed;
 * the recording waits (on the device) for the last reversal of the buffer it
 * reuses. */
int pic_tape_begin(pic_handle *h, int nsteps);

/* Record the current state as the next tape entry without taking the step
 * (a reverse sweep needs a step's start state, not its result: the last
 * step of a recomputed segment need not run).  The entry holds the state as
 * it is now, before any sort the next step would make; the adjoint kernels
 * index particles by id, so the slot order does not matter.  PIC_EINVAL
 * when no tape entry is left (pic_tape_begin). */
int pic_tape_record(pic_handle *h);

/* Allocate (first call) and zero the adjoint state: field adjoints, and per
 * species particle adjoints indexed by particle id (ids must be below
 * id_capacity), the FP64 weight gradients and dF/da0.  PIC_EINVAL unless
 * dims = 2 and shape_order = 2. */
int pic_adjoint_begin(pic_handle *h, int64_t id_capacity);

/* Objective F = sum over live particles of `species` whose x cell column is
 * in [col_lo, col_hi) of w dV m (gamma - 1) at the current state (FP64),
 * written to *F; seeds the adjoint with dF/du and dF/dw. */
int pic_adjoint_seed_kinetic(pic_handle *h, int species, int col_lo, int col_hi, double *F);

/* Reverse the last nsteps recorded steps (most recent first), accumulating
 * dF/da0 and dF/dw.  PIC_EINVAL if fewer steps are on the tape.  The
 * adjoint kernels run on a stream of the handle's own, after the work
 * enqueued on the simulation stream so far; the call returns once they are
 * enqueued, so the next pic_restore / pic_step calls overlap them.  Every
 * call that reads or writes the adjoint state (pic_adjoint_*, pic_grad,
 * pic_grad_binned, pic_sync, pic_timings) first waits for them. */
int pic_adjoint_step(pic_handle *h, int nsteps);

/* Copy dF/da0 (one double, may be NULL) and dF/dw of `species` indexed by
 * particle id (id_capacity doubles, may be NULL) to host or device memory.
 * Synchronises. */
int pic_grad(pic_handle *h, double *d_a0, int species, double *d_w, int mem_kind);

/* dF/dw of `species` summed over bins of particle ids (row A16: the gradient
 * with respect to an initial density profile, the bins its columns):
 * out[b] = sum of dF/dw over the ids i < n_ids with bin_of_id[i] == b, for
 * b in [0, nbins); ids with a bin outside that range are left out.
 * bin_of_id (n_ids int32) and out (nbins doubles) are both in host or both
 * in device memory per mem_kind (a host map is copied to the device per
 * call).  The sums run on the device in FP64; a warp's ids are summed in
 * lane order, the warps' partial sums by atomics, so the last bits may
 * differ between calls.  Synchronises.  PIC_EINVAL: NULL arguments, no
 * pic_adjoint_begin, bad species or memory kind, n_ids outside
 * [0, id_capacity], nbins < 1; PIC_ENOMEM, PIC_ECUDA. */
int pic_grad_binned(pic_handle *h, int species, const int32_t *bin_of_id, int64_t n_ids, int nbins, double *out,
                    int mem_kind);

/* Adjoint state, for objectives of the caller's own and for checks of the
 * transposes (the adjoint of §2's cycle as above; this access has no
 * counterpart in the paper).  All need pic_adjoint_begin first and
 * synchronise.  The adjoint arrays are of the run's precision; values pass
 * as FP64.  Errors: PIC_EINVAL for NULL arguments, a bad selector, species
 * or memory kind, or no pic_adjoint_begin; PIC_ECUDA.
 *
 * pic_adjoint_field: the adjoint of field component `which` (PIC_EX ..
 *   PIC_BZ: of E, B at the current adjoint time; PIC_JX .. PIC_JZ: of the
 *   current density of the last reversed step) into out (ncell doubles,
 *   index i + n0 (j + n1 k) as in pic_fields), host or device per mem_kind.
 * pic_adjoint_set_field: replace the adjoint of E or B component `which`
 *   (PIC_EX .. PIC_BZ) by in (ncell doubles): dF/dE, dF/dB of an objective
 *   F of the fields at the last recorded step.
 * pic_adjoint_momenta / pic_adjoint_set_momenta: the adjoint of the
 *   momenta u of a species, one array per component of id_capacity doubles
 *   indexed by particle id (a NULL pointer skips that component): dF/du of
 *   an objective of the particles' momenta at the last recorded step. */
int pic_adjoint_field(pic_handle *h, int which, double *out, int mem_kind);
int pic_adjoint_set_field(pic_handle *h, int which, const double *in, int mem_kind);
int pic_adjoint_momenta(pic_handle *h, int species, double *lux, double *luy, double *luz, int mem_kind);
int pic_adjoint_set_momenta(pic_handle *h, int species, const double *lux, const double *luy, const double *luz,
                            int mem_kind);

/* ---- state save / resume ----------------------------------------------
 * A run's complete state as one byte blob: fields E, B, J, the background
 * charge, every species' particle storage (in the library's own cell +
 * offset form, so a resumed run continues exactly where the saved one
 * stopped), the step count and the device counters.  The blob starts with a
 * header recording the configuration; pic_state_load accepts it only into a
 * handle created with the same configuration and the same species (charge,
 * mass, capacity) added in the same order.  Output requests, checkpoints and
 * adjoint state are not part of it. */

/* Bytes of the state blob of this handle (header, fields, every species'
 * storage, counters) into *bytes.  PIC_EINVAL for a NULL argument. */
int pic_state_size(pic_handle *h, int64_t *bytes);

/* Write the state into buf (host or device memory per mem_kind, `bytes` =
 * pic_state_size).  Synchronises.  PIC_EINVAL for a short buffer. */
int pic_state_save(pic_handle *h, void *buf, int64_t bytes, int mem_kind);

/* Replace the state by a saved one.  PIC_EINVAL (state unchanged) when the
 * blob's header does not match this handle, or when a particle slot in use
 * is neither dead nor valid (cell outside the grid, offset outside [0, 1),
 * non-finite momentum or weight, position beyond an absorbing wall): the
 * particle storage is checked on the device before anything is replaced.
 * The species are re-sorted at the next step. */
int pic_state_load(pic_handle *h, const void *buf, int64_t bytes, int mem_kind);

/* ---- output manager (§3.1) --------------------------------------------
 * The paper's output manager writes reduced-dimension outputs (a plane of a
 * 3D run, a line of a multidimensional one) and sub-domain outputs (a small
 * box of a large run), restricted in time to a window and a frequency.  A
 * request here captures frames on the device, inside pic_step, into a
 * device buffer it owns (reserved by pic_output_add); pic_output_read copies
 * one frame out.  Frames are taken after a step completes: after step s
 * (s = completed steps, 1, 2, ...) when first <= s <= last and
 * (s - first) % every == 0 (pic_output_due).
 *
 * PIC_OUT_FIELD: field `which` (PIC_EX .. PIC_RHO) at the grid positions
 *   (i, j, k) with lo <= (i, j, k) < hi (each component at its own Yee
 *   location, index (i, j, k) as in pic_fields), FP64, x fastest;
 *   count = box size.  PIC_RHO deposits the charge first.
 * PIC_OUT_PARTICLES: the live particles of species `which` whose cell
 *   (i, j, k) lies in the box, as records of 8 doubles (x, y, z, ux, uy, uz,
 *   w, id) in the units of pic_load_particles; the record order is not
 *   defined.  count = particles found; when it exceeds max_particles only
 *   max_particles records are kept and pic_output_read returns
 *   PIC_EOVERFLOW (the frame's count still says how many there were).
 * In 2D lo[2] = 0, hi[2] = 1.  Frames past max_frames are dropped and
 * counted (pic_output_count). */
#define PIC_OUT_FIELD 0
#define PIC_OUT_PARTICLES 1

typedef struct {
  int kind;              /* PIC_OUT_FIELD or PIC_OUT_PARTICLES                  */
  int which;             /* field id or species index                           */
  int lo[3], hi[3];      /* box [lo, hi), 0 <= lo < hi <= n per axis            */
  int64_t first, last;   /* window of completed steps, 1 <= first <= last       */
  int64_t every;         /* frame period in steps, >= 1                         */
  int64_t max_frames;    /* frames reserved, >= 1                               */
  int64_t max_particles; /* PIC_OUT_PARTICLES: records per frame, >= 1          */
} pic_output_t;

/* 1 if the request's schedule takes a frame after `step` completed steps,
 * else 0.  Pure host function (no handle, no device). */
int pic_output_due(const pic_output_t *req, int64_t step);

/* Register a request and reserve its device buffer (max_frames frames of
 * box-size doubles, or of 8 * max_particles doubles); *id receives its
 * handle.  PIC_EINVAL for a bad kind, field, species, box or schedule;
 * PIC_ENOMEM when the buffer cannot be reserved. */
int pic_output_add(pic_handle *h, const pic_output_t *req, int *id);

/* Take one frame of request id now, at the current step, outside the
 * schedule (e.g. the initial state). */
int pic_output_capture(pic_handle *h, int id);

/* Frames held (*nframes) and frames dropped for lack of room (*dropped,
 * may be NULL).  Synchronises. */
int pic_output_count(pic_handle *h, int id, int64_t *nframes, int64_t *dropped);

/* Copy frame `frame` (0 = oldest) of request id into out (host or device
 * per mem_kind; room for the box size, or 8 * max_particles doubles);
 * *count receives the values' count (FIELD) or the particles found
 * (PARTICLES), *step (may be NULL) the completed steps at capture.
 * Synchronises.  PIC_EOVERFLOW when a particle frame lost records. */
int pic_output_read(pic_handle *h, int id, int64_t frame, double *out, int64_t *count, int64_t *step,
                    int mem_kind);

/* Release request id and its buffer (its id is not reused). */
int pic_output_remove(pic_handle *h, int id);

/* Measured FMA throughput of the current device, the denominators of the
 * arithmetic rooflines a throughput report gives beside the HBM one (the
 * paper has no counterpart: §4 quotes BlueGene/Q scaling, not per-node
 * rates).  Times, with CUDA events on `stream` (cudaStream_t, NULL = the
 * default stream), a kernel of eight independent FMA chains per thread on
 * every SM in FP32 and in FP64, best of three launches each, and writes the
 * rates in TFLOP/s (an FMA counts 2 flops) to *fp32_tflops, *fp64_tflops
 * (host memory).  Synchronises; takes about 0.1 s; changes no clock or power
 * setting.  PIC_EINVAL for NULL outputs, PIC_ECUDA if a launch failed. */
int pic_alu_peak(double *fp32_tflops, double *fp64_tflops, void *stream);

/* FP64 field energies without any device allocation.  The paper has no
 * counterpart: this is a library service for callers that must not call
 * cudaMalloc/cudaFree (which can synchronise the device), e.g. code embedded
 * in an application whose device memory belongs to its own pool or fixed
 * budget, or code running on a host-callback or latency-critical thread.
 * Computes out[0] = 1/2 sum(Ex^2+Ey^2+Ez^2) dV and out[1] = 1/2 sum(Bx^2+
 * By^2+Bz^2) dV -- pic_diag's energy_e and energy_b -- over ncell cells of the
 * caller's device arrays E[0..2], B[0..2] (float for PIC_FP32, double for
 * PIC_FP64), summed in a fixed order (bitwise reproducible).  out (2 doubles)
 * is host (the call then synchronises the stream) or device memory
 * (asynchronous) per mem_kind.  Scratch lives in a static device array of
 * 32 KB that every GPU loading the library keeps until exit; ncell above
 * 33,554,432 is rejected with PIC_EINVAL.  All calls share that array, so
 * calls that overlap on the GPU race.  The first call on each device looks up
 * the array's device address (it must run with that device current, and
 * before any stream capture).  Errors: PIC_EINVAL, PIC_ECUDA; text via
 * pic_last_error(NULL). */
int pic_field_energy_noalloc(int precision, const void *const E[3], const void *const B[3], int64_t ncell,
                             double cell_volume, double *out, int mem_kind, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
