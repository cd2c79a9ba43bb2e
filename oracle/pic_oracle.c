/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle of the relativistic PIC cycle.
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by tests/, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg; the product
 * library never links, calls or includes it, and it shares no code with the
 * CUDA path.
 *
 * What it computes follows section 2 of "Optimising PICCANTE -- an Open
 * Source Particle-in-Cell Code for Advanced Simulations on Tier-0 Systems":
 *   - normalised units with c = 1, v = p / sqrt(p^2 + m^2)        (§2, eq. 1)
 *   - macro-particles with a compact positive shape g              (§2, eq. 2)
 *   - equations of motion dp/dt = q(E + v x B), dr/dt = v          (§2, eq. 3)
 *   - current density J = sum q v g(r - r_n)                       (§2, eq. 4)
 *   - Maxwell curl equations dE/dt = curl B - J, dB/dt = -curl E   (§2)
 *   - force = g-weighted average of the grid fields                (§2)
 *   - leap-frog + Boris pusher, FDTD on the Yee lattice            (§2, refs [8],[9])
 *   - particle record of seven doubles (x,y,z,px,py,pz,w)          (§3.3)
 * The paper leaves the continuity-preserving deposit, the boundary
 * conditions and the laser source unstated (§2); the readings taken here are:
 *   - Esirkepov's charge-conserving current (Comput. Phys. Commun. 135, 2001)
 *   - periodic boundaries; absorbing x walls with a first-order Mur
 *     condition and an incoming laser wave at x = 0.
 *
 * Data layout (deliberately unlike the GPU path): particles are an array of
 * structs holding global positions in physical units and momenta p = m u;
 * every field component is a full nx*ny*nz array of doubles, index
 * i + nx*(j + ny*k).  Staggering (Yee): Ex(i+1/2,j,k) Ey(i,j+1/2,k)
 * Ez(i,j,k+1/2) Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k); J sits
 * with E; rho at nodes (i,j,k).  In 2D (2D3V) nz = 1 and nothing depends on z.
 * Shape sums run over a generous window of nodes and every weight is taken
 * from the shape function itself, so zero weights simply drop out.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EX 0
#define ORC_EY 1
#define ORC_EZ 2
#define ORC_BX 3
#define ORC_BY 4
#define ORC_BZ 5
#define ORC_JX 6
#define ORC_JY 7
#define ORC_JZ 8
#define ORC_RHO 9
#define ORC_NFIELD 10

typedef struct {
  double x, y, z;    /* global position, physical units            */
  double px, py, pz; /* momentum p = m u (u = gamma v), §2 eq. 1   */
  double w;          /* weight: density carried by the particle    */
  uint32_t id;
  int alive;
} orc_particle;

typedef struct {
  double q, m;
  long n;
  orc_particle *p;
} orc_species;

typedef struct {
  int dims;
  int n[3];
  double d[3];
  double dt;
  int order;
  long ncell;
  double *f[ORC_NFIELD]; /* E, B, J, and a scratch rho */
  double *rho_bg;        /* immobile background charge density (nodes) */
  int nsp;
  orc_species sp[8];
  long step;
  /* x boundaries: 0 periodic, 1 absorbing (first-order Mur) */
  int absorb_x;
  /* laser entering through x = 0 (section on boundary readings) */
  int laser_on;
  double a0, waist, duration, yc, zc;
  int pol; /* 1: E in the x-y plane (Ey at the wall), 2: E along z */
  double angle; /* propagation direction (cos angle, sin angle, 0) */
  double *mur_prev; /* previous boundary samples kept by the Mur condition */
  /* gather variant: 0 = the same shape at every Yee location; 1 = one order
   * lower along each axis on which the component sits at a half-integer
   * position ("energy-conserving" gather) */
  int gather_ec;
  /* current smoothing after the deposit: filter_passes three-point binomial
   * passes per axis, then (filter_comp) one compensating pass */
  int filter_passes, filter_comp;
} orc_sim;

/* ------------------------------------------------------------------ */
/* Boundary readings (the paper names boundary conditions but gives   */
/* none, §2).  With absorbing x walls the field domain is the nodes    */
/* i = 0 .. nx-1; tangential E (Ey, Ez) on the wall nodes i = 0 and    */
/* nx-1 follows the first-order Mur condition applied to the field     */
/* minus the incoming laser wave; By, Bz and Ex at i = nx-1 (a half    */
/* cell beyond the last node) are never updated.  A particle whose new */
/* position leaves [3, nx-4) cells is removed after its move has       */
/* deposited its current, so no stencil reaches past the arrays.       */
/* ------------------------------------------------------------------ */
#define ORC_WALL_LO 3.0
#define ORC_WALL_HI_MARGIN 4.0

void oracle_set_boundary(void *h, int absorb_x) { ((orc_sim *)h)->absorb_x = absorb_x; }

/* Laser through x = 0, travelling along k = (cos a, sin a, 0) (a = angle,
 * 0 for normal incidence): a Gaussian beam of waist `waist` about the axis
 * through (0, yc, zc) along k, times the waveform env(tau) sin(tau),
 * env(tau) = sin^2(pi tau / duration) on [0, duration] (carrier frequency
 * 1: times are in 1/omega_laser).  The phase tau = t - k.(x, y - y0) counts
 * time from the wall edge y0 the tilted fronts reach first (y0 = 0 for
 * a > 0, the box height for a < 0).  The field is the component tangential
 * to the wall: along z (pol 2, amplitude a0) or, for E in the x-y plane
 * (pol 1, E along (-sin a, cos a, 0)), its y component a0 cos a. */
void oracle_set_laser(void *h, int on, double a0, double waist, double duration, double yc, double zc, int pol,
                      double angle) {
  orc_sim *s = (orc_sim *)h;
  s->laser_on = on;
  s->a0 = a0;
  s->waist = waist;
  s->duration = duration;
  s->yc = yc;
  s->zc = zc;
  s->pol = pol;
  s->angle = angle;
}

/* Incoming laser field at (x, y, z, t) for the polarised component. */
double oracle_laser_field(void *h, double x, double y, double z, double t) {
  orc_sim *s = (orc_sim *)h;
  if (!s->laser_on) return 0.0;
  double ca = cos(s->angle), sa = sin(s->angle);
  double y0 = s->angle > 0.0 ? 0.0 : s->n[1] * s->d[1];
  double tau = t - (x * ca + (y - y0) * sa);
  if (tau <= 0.0 || tau >= s->duration) return 0.0;
  double env = sin(M_PI * tau / s->duration);
  /* distance from the beam axis: the part of (x, y - yc, z - zc) across k */
  double across = (y - s->yc) * ca - x * sa;
  double r2 = across * across + (s->dims == 3 ? (z - s->zc) * (z - s->zc) : 0.0);
  double amp = s->pol == 1 ? s->a0 * ca : s->a0;
  return amp * exp(-r2 / (s->waist * s->waist)) * env * env * sin(tau);
}

/* ------------------------------------------------------------------ */
/* Shape functions (§2: g compact and positive).                       */
/* order 1: cloud-in-cell (linear B-spline); order 2: triangular-      */
/* shaped cloud (quadratic B-spline).  xi is measured in cells.        */
/* ------------------------------------------------------------------ */
double oracle_shape(int order, double xi) {
  if (order == 0) return (xi >= -0.5 && xi < 0.5) ? 1.0 : 0.0; /* nearest grid point, half-open cell */
  double a = fabs(xi);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a <= 0.5) return 0.75 - a * a;
  if (a < 1.5) {
    double b = 1.5 - a;
    return 0.5 * b * b;
  }
  return 0.0;
}

static long wrapi(long i, int n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

static long idx(const orc_sim *s, long i, long j, long k) {
  return wrapi(i, s->n[0]) + (long)s->n[0] * (wrapi(j, s->n[1]) + (long)s->n[1] * wrapi(k, s->n[2]));
}

/* ------------------------------------------------------------------ */
/* Creation / teardown                                                 */
/* ------------------------------------------------------------------ */
void *oracle_create(int dims, const int *n, const double *d, double dt, int order) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  s->dims = dims;
  for (int a = 0; a < 3; ++a) {
    s->n[a] = n[a];
    s->d[a] = d[a];
  }
  if (dims == 2) {
    s->n[2] = 1;
    if (s->d[2] <= 0) s->d[2] = 1.0;
  }
  s->dt = dt;
  s->order = order;
  s->ncell = (long)s->n[0] * s->n[1] * s->n[2];
  for (int c = 0; c < ORC_NFIELD; ++c) s->f[c] = (double *)calloc(s->ncell, sizeof(double));
  s->rho_bg = (double *)calloc(s->ncell, sizeof(double));
  s->mur_prev = (double *)calloc(8 * (size_t)s->n[1] * s->n[2], sizeof(double));
  return s;
}

void oracle_destroy(void *h) {
  orc_sim *s = (orc_sim *)h;
  if (!s) return;
  for (int c = 0; c < ORC_NFIELD; ++c) free(s->f[c]);
  free(s->rho_bg);
  free(s->mur_prev);
  for (int i = 0; i < s->nsp; ++i) free(s->sp[i].p);
  free(s);
}

/* Species are given momenta as u = p/m (the generator's convention); the
 * oracle stores p = m u, the paper's variable (§2 eq. 1, §3.3). */
int oracle_add_species(void *h, double q, double m, long n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy, const double *uz,
                       const double *w, const uint32_t *id) {
  orc_sim *s = (orc_sim *)h;
  if (s->nsp >= 8) return -1;
  orc_species *sp = &s->sp[s->nsp];
  sp->q = q;
  sp->m = m;
  sp->n = n;
  sp->p = (orc_particle *)calloc(n > 0 ? n : 1, sizeof(orc_particle));
  for (long i = 0; i < n; ++i) {
    orc_particle *p = &sp->p[i];
    p->x = x[i];
    p->y = y[i];
    p->z = (s->dims == 3) ? z[i] : 0.0;
    p->px = m * ux[i];
    p->py = m * uy[i];
    p->pz = m * uz[i];
    p->w = w[i];
    p->id = id ? id[i] : (uint32_t)i;
    p->alive = 1;
  }
  return s->nsp++;
}

long oracle_num_particles(void *h, int isp) {
  orc_sim *s = (orc_sim *)h;
  long c = 0;
  for (long i = 0; i < s->sp[isp].n; ++i) c += s->sp[isp].p[i].alive;
  return c;
}

/* Output: for each live particle, x y z ux uy uz w (u = p/m). */
long oracle_get_particles(void *h, int isp, double *out7, uint32_t *id) {
  orc_sim *s = (orc_sim *)h;
  orc_species *sp = &s->sp[isp];
  long c = 0;
  for (long i = 0; i < sp->n; ++i) {
    orc_particle *p = &sp->p[i];
    if (!p->alive) continue;
    double *o = out7 + 7 * c;
    o[0] = p->x;
    o[1] = p->y;
    o[2] = p->z;
    o[3] = p->px / sp->m;
    o[4] = p->py / sp->m;
    o[5] = p->pz / sp->m;
    o[6] = p->w;
    id[c] = p->id;
    ++c;
  }
  return c;
}

void oracle_get_field(void *h, int which, double *out) {
  orc_sim *s = (orc_sim *)h;
  memcpy(out, s->f[which], sizeof(double) * s->ncell);
}

void oracle_set_field(void *h, int which, const double *in) {
  orc_sim *s = (orc_sim *)h;
  memcpy(s->f[which], in, sizeof(double) * s->ncell);
}

long oracle_step_count(void *h) { return ((orc_sim *)h)->step; }

/* ------------------------------------------------------------------ */
/* Field gather (§2: "spatial average of the EM fields weighted with   */
/* g").  Each component is sampled with the shape centred on the       */
/* particle, using that component's own Yee location; stag[a] is 0 for */
/* an integer position and 0.5 for a half-integer one along axis a.    */
/* ------------------------------------------------------------------ */
static double gather_component(const orc_sim *s, const double *F, const double X[3], const double stag[3]) {
  /* shape order per axis: one lower at half-integer positions in the
   * energy-conserving variant */
  int ox = s->order - (s->gather_ec && stag[0] != 0.0);
  int oy = s->order - (s->gather_ec && stag[1] != 0.0);
  int oz = s->order - (s->gather_ec && stag[2] != 0.0);
  if (s->dims == 2) {
    double sum = 0.0;
    long i0 = (long)floor(X[0] - stag[0]), j0 = (long)floor(X[1] - stag[1]);
    for (long j = j0 - 2; j <= j0 + 3; ++j) {
      double sy = oracle_shape(oy, X[1] - stag[1] - (double)j);
      if (sy == 0.0) continue;
      for (long i = i0 - 2; i <= i0 + 3; ++i) {
        double sx = oracle_shape(ox, X[0] - stag[0] - (double)i);
        if (sx == 0.0) continue;
        sum += F[idx(s, i, j, 0)] * sx * sy;
      }
    }
    return sum;
  }
  double sum = 0.0;
  long i0 = (long)floor(X[0] - stag[0]), j0 = (long)floor(X[1] - stag[1]), k0 = (long)floor(X[2] - stag[2]);
  for (long k = k0 - 2; k <= k0 + 3; ++k) {
    double sz = oracle_shape(oz, X[2] - stag[2] - (double)k);
    if (sz == 0.0) continue;
    for (long j = j0 - 2; j <= j0 + 3; ++j) {
      double sy = oracle_shape(oy, X[1] - stag[1] - (double)j);
      if (sy == 0.0) continue;
      for (long i = i0 - 2; i <= i0 + 3; ++i) {
        double sx = oracle_shape(ox, X[0] - stag[0] - (double)i);
        if (sx == 0.0) continue;
        sum += F[idx(s, i, j, k)] * sx * sy * sz;
      }
    }
  }
  return sum;
}

/* Yee locations of the six components (in cells). */
static const double STAG_E[3][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
static const double STAG_B[3][3] = {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};

static void gather_at(const orc_sim *s, double x, double y, double z, double E[3], double B[3]) {
  double X[3] = {x / s->d[0], y / s->d[1], s->dims == 3 ? z / s->d[2] : 0.0};
  for (int c = 0; c < 3; ++c) {
    E[c] = gather_component(s, s->f[ORC_EX + c], X, STAG_E[c]);
    B[c] = gather_component(s, s->f[ORC_BX + c], X, STAG_B[c]);
  }
}

void oracle_gather_point(void *h, double x, double y, double z, double *E, double *B) {
  gather_at((orc_sim *)h, x, y, z, E, B);
}

/* ------------------------------------------------------------------ */
/* Boris pusher in the paper's variables (§2 eq. 3, ref [8]):           */
/* half electric kick, magnetic rotation, half electric kick.  Written */
/* for momentum p with gamma m = sqrt(p^2 + m^2).                      */
/* ------------------------------------------------------------------ */
void oracle_boris(double q, double m, double dt, const double *E, const double *B, double *p) {
  double h = 0.5 * q * dt;
  double pm[3] = {p[0] + h * E[0], p[1] + h * E[1], p[2] + h * E[2]};
  double gm = sqrt(pm[0] * pm[0] + pm[1] * pm[1] + pm[2] * pm[2] + m * m); /* gamma * m */
  double t[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double sv[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
  double pp[3] = {pm[0] + (pm[1] * t[2] - pm[2] * t[1]), pm[1] + (pm[2] * t[0] - pm[0] * t[2]),
                  pm[2] + (pm[0] * t[1] - pm[1] * t[0])};
  double pl[3] = {pm[0] + (pp[1] * sv[2] - pp[2] * sv[1]), pm[1] + (pp[2] * sv[0] - pp[0] * sv[2]),
                  pm[2] + (pp[0] * sv[1] - pp[1] * sv[0])};
  p[0] = pl[0] + h * E[0];
  p[1] = pl[1] + h * E[1];
  p[2] = pl[2] + h * E[2];
}

/* ------------------------------------------------------------------ */
/* Esirkepov charge-conserving current for one particle moving from    */
/* X0 to X1 (positions in cells, unwrapped).  With S0, S1 the shapes   */
/* at the two positions and DS = S1 - S0 on a common run of nodes:     */
/*  3D: Wx = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3), cyclic  */
/*      for Wy, Wz; Jx(i+1/2) - Jx(i-1/2) = -q w (dx/dt) Wx(i), the run */
/*      starting from zero below the stencil.                          */
/*  2D: Wx = DSx (S0y + DSy/2), Wy = DSy (S0x + DSx/2) with the same    */
/*      running sums; Jz(i,j) += q w vz (S0x S0y + DSx S0y/2 +          */
/*      S0x DSy/2 + DSx DSy/3).                                         */
/* This makes (rho1 - rho0)/dt + div J = 0 with rho = sum q w S (§2     */
/* eq. 4 and the continuity requirement stated in §2).                 */
/* ------------------------------------------------------------------ */
#define ORC_SW 10
static void esirkepov(orc_sim *s, double *const J3[3], double q, double w, const double X0[3], const double X1[3],
                      double vz) {
  int o = s->order;
  int na = s->dims;
  long lo[3] = {0, 0, 0};
  int wdt[3] = {1, 1, 1};
  double S0[3][ORC_SW], S1[3][ORC_SW], DS[3][ORC_SW];
  for (int a = 0; a < na; ++a) {
    double mn = X0[a] < X1[a] ? X0[a] : X1[a];
    double mx = X0[a] < X1[a] ? X1[a] : X0[a];
    lo[a] = (long)floor(mn) - 2;
    wdt[a] = (int)((long)floor(mx) + 3 - lo[a] + 1);
    if (wdt[a] > ORC_SW) wdt[a] = ORC_SW; /* moves of more than a cell are outside CFL */
    for (int i = 0; i < wdt[a]; ++i) {
      S0[a][i] = oracle_shape(o, (double)(lo[a] + i) - X0[a]);
      S1[a][i] = oracle_shape(o, (double)(lo[a] + i) - X1[a]);
      DS[a][i] = S1[a][i] - S0[a][i];
    }
  }
  double *Jx = J3[0], *Jy = J3[1], *Jz = J3[2];
  double cx = -q * w * s->d[0] / s->dt, cy = -q * w * s->d[1] / s->dt, cz = -q * w * s->d[2] / s->dt;
  if (s->dims == 2) {
    for (int j = 0; j < wdt[1]; ++j) {
      double acc = 0.0;
      for (int i = 0; i < wdt[0]; ++i) {
        acc += DS[0][i] * (S0[1][j] + 0.5 * DS[1][j]);
        Jx[idx(s, lo[0] + i, lo[1] + j, 0)] += cx * acc;
      }
    }
    for (int i = 0; i < wdt[0]; ++i) {
      double acc = 0.0;
      for (int j = 0; j < wdt[1]; ++j) {
        acc += DS[1][j] * (S0[0][i] + 0.5 * DS[0][i]);
        Jy[idx(s, lo[0] + i, lo[1] + j, 0)] += cy * acc;
      }
    }
    for (int j = 0; j < wdt[1]; ++j)
      for (int i = 0; i < wdt[0]; ++i) {
        double sm = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +
                    DS[0][i] * DS[1][j] / 3.0;
        Jz[idx(s, lo[0] + i, lo[1] + j, 0)] += q * w * vz * sm;
      }
    return;
  }
  /* 3D */
  for (int k = 0; k < wdt[2]; ++k)
    for (int j = 0; j < wdt[1]; ++j) {
      double acc = 0.0;
      for (int i = 0; i < wdt[0]; ++i) {
        acc += DS[0][i] * (S0[1][j] * S0[2][k] + 0.5 * DS[1][j] * S0[2][k] + 0.5 * S0[1][j] * DS[2][k] +
                           DS[1][j] * DS[2][k] / 3.0);
        Jx[idx(s, lo[0] + i, lo[1] + j, lo[2] + k)] += cx * acc;
      }
    }
  for (int k = 0; k < wdt[2]; ++k)
    for (int i = 0; i < wdt[0]; ++i) {
      double acc = 0.0;
      for (int j = 0; j < wdt[1]; ++j) {
        acc += DS[1][j] * (S0[2][k] * S0[0][i] + 0.5 * DS[2][k] * S0[0][i] + 0.5 * S0[2][k] * DS[0][i] +
                           DS[2][k] * DS[0][i] / 3.0);
        Jy[idx(s, lo[0] + i, lo[1] + j, lo[2] + k)] += cy * acc;
      }
    }
  for (int j = 0; j < wdt[1]; ++j)
    for (int i = 0; i < wdt[0]; ++i) {
      double acc = 0.0;
      for (int k = 0; k < wdt[2]; ++k) {
        acc += DS[2][k] * (S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +
                           DS[0][i] * DS[1][j] / 3.0);
        Jz[idx(s, lo[0] + i, lo[1] + j, lo[2] + k)] += cz * acc;
      }
    }
}

/* Deposit the current of one move from global positions r0 to r1. */
void oracle_deposit_move(void *h, double q, double w, const double *r0, const double *r1, double vz) {
  orc_sim *s = (orc_sim *)h;
  double X0[3] = {r0[0] / s->d[0], r0[1] / s->d[1], s->dims == 3 ? r0[2] / s->d[2] : 0.0};
  double X1[3] = {r1[0] / s->d[0], r1[1] / s->d[1], s->dims == 3 ? r1[2] / s->d[2] : 0.0};
  esirkepov(s, s->f + ORC_JX, q, w, X0, X1, vz);
}

/* ------------------------------------------------------------------ */
/* Yee FDTD (§2, ref [9]), split so that B is known at integer times:  */
/*   B^{n+1/2} = B^n - dt/2 curl E^n                                   */
/*   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})                 */
/*   B^{n+1}   = B^{n+1/2} - dt/2 curl E^{n+1}                         */
/* Differences wrap periodically; with nz = 1 every z difference is    */
/* zero, which is the 2D case.                                         */
/* ------------------------------------------------------------------ */
static void yee_b(orc_sim *s, double h) {
  double *Ex = s->f[ORC_EX], *Ey = s->f[ORC_EY], *Ez = s->f[ORC_EZ];
  double *Bx = s->f[ORC_BX], *By = s->f[ORC_BY], *Bz = s->f[ORC_BZ];
  double dx = s->d[0], dy = s->d[1], dz = s->d[2];
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long c = idx(s, i, j, k);
        /* curl E at the B locations */
        double cx = (Ez[idx(s, i, j + 1, k)] - Ez[c]) / dy - (Ey[idx(s, i, j, k + 1)] - Ey[c]) / dz;
        double cy = (Ex[idx(s, i, j, k + 1)] - Ex[c]) / dz - (Ez[idx(s, i + 1, j, k)] - Ez[c]) / dx;
        double cz = (Ey[idx(s, i + 1, j, k)] - Ey[c]) / dx - (Ex[idx(s, i, j + 1, k)] - Ex[c]) / dy;
        Bx[c] -= h * cx;
        if (s->absorb_x && i == s->n[0] - 1) continue; /* By, Bz beyond the last node */
        By[c] -= h * cy;
        Bz[c] -= h * cz;
      }
}

static void yee_e(orc_sim *s, double h) {
  double *Ex = s->f[ORC_EX], *Ey = s->f[ORC_EY], *Ez = s->f[ORC_EZ];
  double *Bx = s->f[ORC_BX], *By = s->f[ORC_BY], *Bz = s->f[ORC_BZ];
  double *Jx = s->f[ORC_JX], *Jy = s->f[ORC_JY], *Jz = s->f[ORC_JZ];
  double dx = s->d[0], dy = s->d[1], dz = s->d[2];
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long c = idx(s, i, j, k);
        /* curl B at the E locations */
        double cx = (Bz[c] - Bz[idx(s, i, j - 1, k)]) / dy - (By[c] - By[idx(s, i, j, k - 1)]) / dz;
        double cy = (Bx[c] - Bx[idx(s, i, j, k - 1)]) / dz - (Bz[c] - Bz[idx(s, i - 1, j, k)]) / dx;
        double cz = (By[c] - By[idx(s, i - 1, j, k)]) / dx - (Bx[c] - Bx[idx(s, i, j - 1, k)]) / dy;
        if (s->absorb_x && i == s->n[0] - 1) continue; /* wall node: Mur; Ex beyond the last node */
        Ex[c] += h * (cx - Jx[c]);
        if (s->absorb_x && i == 0) continue; /* wall node: Mur */
        Ey[c] += h * (cy - Jy[c]);
        Ez[c] += h * (cz - Jz[c]);
      }
}

/* First-order Mur condition on the tangential E of both x walls, applied to
 * the scattered field E - E_laser:
 *   E(0)^{n+1} = E(1)^n + k (E(1)^{n+1} - E(0)^n),  k = (dt - dx)/(dt + dx)
 * and the mirror image at the right wall.  `old` holds E^n of the nodes
 * 0, 1, nx-2, nx-1 (components y, z) saved before the E update. */
static double laser_comp(orc_sim *s, int comp, long i, long j, long k, double t) {
  /* Ey at (i, j+1/2, k), Ez at (i, j, k+1/2) */
  if (!s->laser_on) return 0.0;
  if ((comp == 0 && s->pol != 1) || (comp == 1 && s->pol != 2)) return 0.0;
  double x = i * s->d[0];
  double y = (j + (comp == 0 ? 0.5 : 0.0)) * s->d[1];
  double z = (k + (comp == 1 ? 0.5 : 0.0)) * s->d[2];
  return oracle_laser_field(s, x, y, z, t);
}

static void mur_save(orc_sim *s) {
  long nyz = (long)s->n[1] * s->n[2], nx = s->n[0];
  long nodes[4] = {0, 1, nx - 2, nx - 1};
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q < 4; ++q)
      for (long jk = 0; jk < nyz; ++jk) {
        long j = jk % s->n[1], k = jk / s->n[1];
        s->mur_prev[((c * 4 + q) * nyz) + jk] = s->f[ORC_EY + c][idx(s, nodes[q], j, k)];
      }
}

static void mur_apply(orc_sim *s, double t_old, double t_new) {
  long nyz = (long)s->n[1] * s->n[2], nx = s->n[0];
  double kc = (s->dt - s->d[0]) / (s->dt + s->d[0]);
  for (int c = 0; c < 2; ++c)
    for (long jk = 0; jk < nyz; ++jk) {
      long j = jk % s->n[1], k = jk / s->n[1];
      double *E = s->f[ORC_EY + c];
      const double *o = s->mur_prev + (long)c * 4 * nyz;
      /* left wall (node 0, neighbour node 1): scattered field leaves towards -x */
      double s0_old = o[0 * nyz + jk] - laser_comp(s, c, 0, j, k, t_old);
      double s1_old = o[1 * nyz + jk] - laser_comp(s, c, 1, j, k, t_old);
      double s1_new = E[idx(s, 1, j, k)] - laser_comp(s, c, 1, j, k, t_new);
      E[idx(s, 0, j, k)] = laser_comp(s, c, 0, j, k, t_new) + s1_old + kc * (s1_new - s0_old);
      /* right wall (node nx-1, neighbour nx-2): no laser term there */
      double r0_old = o[3 * nyz + jk], r1_old = o[2 * nyz + jk];
      double r1_new = E[idx(s, nx - 2, j, k)];
      E[idx(s, nx - 1, j, k)] = r1_old + kc * (r1_new - r0_old);
    }
}

/* Field-only update, exposed for the Yee dispersion and Courant pins. */
/* ------------------------------------------------------------------ */
/* Current smoothing (a standard PIC addition; the paper's §2 leaves   */
/* such details out).  One pass along axis a replaces every value by   */
/*   alpha f(i) + (1 - alpha)/2 (f(i-1) + f(i+1))   (periodic),        */
/* which multiplies a Fourier mode exp(i k x) by alpha + (1 - alpha)    */
/* cos(k dx).  The binomial pass is alpha = 1/2 (factor cos^2(k dx/2)); */
/* after n of them the compensating pass alpha = 1 + n/2 cancels the    */
/* k^2 term of the product.                                            */
/* ------------------------------------------------------------------ */
static void smooth_axis(orc_sim *s, double *f, int axis, double alpha) {
  double *tmp = (double *)malloc(sizeof(double) * s->ncell);
  memcpy(tmp, f, sizeof(double) * s->ncell);
  double side = 0.5 * (1.0 - alpha);
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long lo = axis == 0 ? idx(s, i - 1, j, k) : axis == 1 ? idx(s, i, j - 1, k) : idx(s, i, j, k - 1);
        long hi = axis == 0 ? idx(s, i + 1, j, k) : axis == 1 ? idx(s, i, j + 1, k) : idx(s, i, j, k + 1);
        f[idx(s, i, j, k)] = alpha * tmp[idx(s, i, j, k)] + side * (tmp[lo] + tmp[hi]);
      }
  free(tmp);
}

static void smooth_field(orc_sim *s, double *f) {
  for (int p = 0; p < s->filter_passes; ++p)
    for (int a = 0; a < s->dims; ++a) smooth_axis(s, f, a, 0.5);
  if (s->filter_comp && s->filter_passes > 0)
    for (int a = 0; a < s->dims; ++a) smooth_axis(s, f, a, 1.0 + 0.5 * s->filter_passes);
}

void oracle_set_filter(void *h, int passes, int compensate) {
  orc_sim *s = (orc_sim *)h;
  s->filter_passes = passes;
  s->filter_comp = compensate;
}

void oracle_set_gather(void *h, int energy_conserving) { ((orc_sim *)h)->gather_ec = energy_conserving; }

/* Apply the configured smoothing to one stored field (test hook). */
void oracle_smooth(void *h, int which) {
  orc_sim *s = (orc_sim *)h;
  smooth_field(s, s->f[which]);
}

static void field_cycle(orc_sim *s) {
  double t_old = s->step * s->dt, t_new = (s->step + 1) * s->dt;
  yee_b(s, 0.5 * s->dt);
  if (s->absorb_x) mur_save(s);
  yee_e(s, s->dt);
  if (s->absorb_x) mur_apply(s, t_old, t_new);
  yee_b(s, 0.5 * s->dt);
}

void oracle_field_step(void *h, int nsteps) {
  orc_sim *s = (orc_sim *)h;
  for (int t = 0; t < nsteps; ++t) {
    field_cycle(s);
    s->step++;
  }
}

/* ------------------------------------------------------------------ */
/* One PIC cycle: gather -> Boris -> move -> deposit, then Yee.        */
/* ------------------------------------------------------------------ */
/* Gather, Boris, move and deposit (into J3) of one live particle. */
static void advance_particle(orc_sim *s, const orc_species *sp, orc_particle *p, const double L[3],
                             double *const J3[3]) {
  double E[3], B[3];
  gather_at(s, p->x, p->y, p->z, E, B);
  double mom[3] = {p->px, p->py, p->pz};
  oracle_boris(sp->q, sp->m, s->dt, E, B, mom);
  p->px = mom[0];
  p->py = mom[1];
  p->pz = mom[2];
  double gm = sqrt(mom[0] * mom[0] + mom[1] * mom[1] + mom[2] * mom[2] + sp->m * sp->m);
  double v[3] = {mom[0] / gm, mom[1] / gm, mom[2] / gm}; /* §2 eq. 1 */
  double r0[3] = {p->x, p->y, p->z};
  double r1[3] = {p->x + s->dt * v[0], p->y + s->dt * v[1], s->dims == 3 ? p->z + s->dt * v[2] : 0.0};
  double X0[3] = {r0[0] / s->d[0], r0[1] / s->d[1], r0[2] / s->d[2]};
  double X1[3] = {r1[0] / s->d[0], r1[1] / s->d[1], r1[2] / s->d[2]};
  esirkepov(s, J3, sp->q, p->w, X0, X1, v[2]);
  if (s->absorb_x && (X1[0] < ORC_WALL_LO || X1[0] >= s->n[0] - ORC_WALL_HI_MARGIN)) {
    p->alive = 0; /* removed at the wall after depositing its last move */
    return;
  }
  /* periodic wrap of the stored position */
  for (int a = 0; a < s->dims; ++a) {
    if (r1[a] >= L[a]) r1[a] -= L[a];
    else if (r1[a] < 0.0) r1[a] += L[a];
  }
  p->x = r1[0];
  p->y = r1[1];
  p->z = r1[2];
}

#ifdef _OPENMP
/* The particle loop of one step on all OpenMP threads (the library built
 * with -fopenmp).  Each thread deposits into J arrays of its own; they are
 * then summed node by node in thread order, so the result depends only on
 * the thread count and differs from the serial loop by the order of the
 * additions alone (round-off). */
static void push_all_parallel(orc_sim *s, const double L[3]) {
  const int nt = omp_get_max_threads();
  const long nc = s->ncell;
  double *buf = (double *)calloc((size_t)nt * 3 * (size_t)nc, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    double *J3[3] = {buf + ((size_t)t * 3 + 0) * nc, buf + ((size_t)t * 3 + 1) * nc, buf + ((size_t)t * 3 + 2) * nc};
    for (int isp = 0; isp < s->nsp; ++isp) {
      orc_species *sp = &s->sp[isp];
#pragma omp for schedule(static)
      for (long ip = 0; ip < sp->n; ++ip)
        if (sp->p[ip].alive) advance_particle(s, sp, &sp->p[ip], L, J3);
    }
#pragma omp for schedule(static)
    for (long c = 0; c < nc; ++c)
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int u = 0; u < nt; ++u) acc += buf[((size_t)u * 3 + a) * nc + c];
        s->f[ORC_JX + a][c] = acc;
      }
  }
  free(buf);
}
#endif

/* Threads the particle loop runs on (1 for the serial build). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_step(void *h, int nsteps) {
  orc_sim *s = (orc_sim *)h;
  double L[3] = {s->n[0] * s->d[0], s->n[1] * s->d[1], s->n[2] * s->d[2]};
  for (int t = 0; t < nsteps; ++t) {
    memset(s->f[ORC_JX], 0, sizeof(double) * s->ncell);
    memset(s->f[ORC_JY], 0, sizeof(double) * s->ncell);
    memset(s->f[ORC_JZ], 0, sizeof(double) * s->ncell);
#ifdef _OPENMP
    push_all_parallel(s, L);
#else
    for (int isp = 0; isp < s->nsp; ++isp) {
      orc_species *sp = &s->sp[isp];
      for (long ip = 0; ip < sp->n; ++ip)
        if (sp->p[ip].alive) advance_particle(s, sp, &sp->p[ip], L, s->f + ORC_JX);
    }
#endif
    if (s->filter_passes > 0)
      for (int c = 0; c < 3; ++c) smooth_field(s, s->f[ORC_JX + c]);
    field_cycle(s);
    s->step++;
  }
}

/* ------------------------------------------------------------------ */
/* Charge density at the nodes: rho = sum q w S (+ background), §2.    */
/* ------------------------------------------------------------------ */
static void deposit_rho(orc_sim *s, double *rho) {
  int o = s->order;
  memcpy(rho, s->rho_bg, sizeof(double) * s->ncell);
  for (int isp = 0; isp < s->nsp; ++isp) {
    orc_species *sp = &s->sp[isp];
    for (long ip = 0; ip < sp->n; ++ip) {
      orc_particle *p = &sp->p[ip];
      if (!p->alive) continue;
      double X[3] = {p->x / s->d[0], p->y / s->d[1], s->dims == 3 ? p->z / s->d[2] : 0.0};
      long i0 = (long)floor(X[0]), j0 = (long)floor(X[1]), k0 = (long)floor(X[2]);
      long kr = s->dims == 3 ? 2 : 0;
      for (long k = k0 - kr; k <= k0 + kr + (s->dims == 3); ++k) {
        double sz = s->dims == 3 ? oracle_shape(o, X[2] - (double)k) : 1.0;
        if (sz == 0.0) continue;
        for (long j = j0 - 2; j <= j0 + 3; ++j) {
          double sy = oracle_shape(o, X[1] - (double)j);
          if (sy == 0.0) continue;
          for (long i = i0 - 2; i <= i0 + 3; ++i) {
            double sx = oracle_shape(o, X[0] - (double)i);
            if (sx == 0.0) continue;
            rho[idx(s, i, j, k)] += sp->q * p->w * sx * sy * sz;
          }
        }
      }
    }
  }
}

/* rho of the particles (+ background) into the scratch rho field. */
void oracle_compute_rho(void *h) {
  orc_sim *s = (orc_sim *)h;
  deposit_rho(s, s->f[ORC_RHO]);
}

/* Immobile background charge density at the nodes, given explicitly. */
void oracle_set_background(void *h, const double *rho) {
  orc_sim *s = (orc_sim *)h;
  memcpy(s->rho_bg, rho, sizeof(double) * s->ncell);
}

/* Immobile neutralising background: rho_bg = -rho of the current particles. */
void oracle_neutralize(void *h) {
  orc_sim *s = (orc_sim *)h;
  memset(s->rho_bg, 0, sizeof(double) * s->ncell);
  double *tmp = (double *)calloc(s->ncell, sizeof(double));
  deposit_rho(s, tmp);
  for (long c = 0; c < s->ncell; ++c) s->rho_bg[c] = -tmp[c];
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* Diagnostics in FP64.  out[0] field energy 1/2 sum(E^2+B^2) dV,       */
/* out[1] kinetic energy sum w dV (sqrt(p^2+m^2) - m) at the stored    */
/* momenta, out[2] total charge sum rho dV (incl. background),         */
/* out[3] max |div E - rho|, out[4] live particle count,               */
/* out[5] electric part, out[6] magnetic part of the field energy.     */
/* ------------------------------------------------------------------ */
void oracle_diag(void *h, double *out) {
  orc_sim *s = (orc_sim *)h;
  double dV = s->d[0] * s->d[1] * (s->dims == 3 ? s->d[2] : 1.0);
  double ue = 0, ub = 0;
  for (long c = 0; c < s->ncell; ++c) {
    for (int a = 0; a < 3; ++a) {
      ue += s->f[ORC_EX + a][c] * s->f[ORC_EX + a][c];
      ub += s->f[ORC_BX + a][c] * s->f[ORC_BX + a][c];
    }
  }
  ue *= 0.5 * dV;
  ub *= 0.5 * dV;
  double uk = 0;
  long nalive = 0;
  for (int isp = 0; isp < s->nsp; ++isp) {
    orc_species *sp = &s->sp[isp];
    for (long ip = 0; ip < sp->n; ++ip) {
      orc_particle *p = &sp->p[ip];
      if (!p->alive) continue;
      double gm = sqrt(p->px * p->px + p->py * p->py + p->pz * p->pz + sp->m * sp->m);
      uk += p->w * dV * (gm - sp->m);
      ++nalive;
    }
  }
  double *rho = s->f[ORC_RHO];
  deposit_rho(s, rho);
  /* with current smoothing, Gauss's law holds for the equally smoothed
   * charge (the filter commutes with the difference operators) */
  if (s->filter_passes > 0) smooth_field(s, rho);
  double q = 0, gmax = 0;
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long c = idx(s, i, j, k);
        q += rho[c] * dV;
        double div = (s->f[ORC_EX][c] - s->f[ORC_EX][idx(s, i - 1, j, k)]) / s->d[0] +
                     (s->f[ORC_EY][c] - s->f[ORC_EY][idx(s, i, j - 1, k)]) / s->d[1] +
                     (s->f[ORC_EZ][c] - s->f[ORC_EZ][idx(s, i, j, k - 1)]) / s->d[2];
        double r = fabs(div - rho[c]);
        if (r > gmax) gmax = r;
      }
  out[0] = ue + ub;
  out[1] = uk;
  out[2] = q;
  out[3] = gmax;
  out[4] = (double)nalive;
  out[5] = ue;
  out[6] = ub;
}
