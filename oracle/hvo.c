/*
 * Hybrid PIC oracle: a plain, slow, FP64 CPU restatement of the per-step ion
 * loop of the kinetic-ion / massless-fluid-electron hybrid PIC method of
 * Hybrid-VPIC (arXiv 2305.05600).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path and must never be used
 * as a fallback for it.
 *
 * Every routine is written as plain loops in the order the paper states the
 * method; there is no blocking, fusion or reordering.  Sections and equations
 * cited below are those of the paper:
 *   Sec. 2.1  hybrid model equations: Ohm's law (Eq. 2), R_ei (Eq. 3),
 *             Ampere (Eq. 4), Faraday (Eq. 5), equation of state (Eq. 6),
 *             density floor n_e = max(n_e, n_f), whistler CFL and subcycling.
 *   Sec. 2.2  PIC implementation: leapfrog / Boris (Eqs. 9-10), linear
 *             extrapolation of J_i (Eq. 11), cell-centred grid and centred
 *             differences (Eq. 12), particle storage as cell index + relative
 *             coordinates in [-1,1]^3, NGP shape (Eq. 13), smoothing.
 *   App. B    QS particle shape: deposit weights (Eq. 17), interpolation
 *             coefficients (Eq. 18) and field at the particle (Eq. 19).
 *   Sec. 2.3  boundaries: fully periodic (the simplest case, named at the
 *             start of the section).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   R1 relative coordinates are taken in [-1,1): a particle exactly on the
 *      upper face belongs to the next cell; x = x_c + d * Delta / 2.
 *   R2 the half-time-step position used for deposit (App. B, after Eq. 17)
 *      is used for every shape and for both n and J.
 *   R3 n is extrapolated like J (Eq. 11 states it for J only).
 *   R4 smoothing is the separable (1/4,1/2,1/4) binomial filter applied to
 *      the deposited moments.
 *   R16 the optional electron energy equation (Sec. 2.1, Eq. dpdt) makes
 *      p_e a field: dp_e/dt = -gamma div(p_e u_e) + (gamma - 1) u_e . grad p_e
 *      + (gamma - 1) div(kappa grad T_e), with u_e = -(J - J_i) / n_f,
 *      T_e = p_e / n_f, a constant kappa, H_ei = 0 (no collisions) and the
 *      centred operators of Eq. 12 (the Laplacian of R6 for the heat flux).
 *      It is advanced with B in each explicit-midpoint subcycle (R7), with
 *      the moments held at their half-step values; Ohm's law takes grad p_e
 *      from the field.  At start-up p_e = Te n_f^gamma of the start-up
 *      moments (Eq. 6).
 *   R17 the optional electrostatic model (Sec. 4, Eq. esohm): Ohm's law
 *      keeps only E = -grad p_e / n_f (R_ei = 0: no collision model here);
 *      B is not advanced and stays at its initial value, which the ions
 *      still feel; with the electron energy equation u_e = J_i / n_f (no
 *      magnetic current).
 *   R18 the optional resistive-background model (App. A, kinetic-electron
 *      beam): E = eta (curl B - J_k), J_k the deposited current of the
 *      kinetic species; B advances with Faraday's law in the same subcycles.
 *   R19 the optional relativistic push (Sec. 2.2, App. A): a particle
 *      carries u = gamma v; Boris with t = (q dt / 2m) B / gamma^-,
 *      gamma^- = sqrt(1 + |u^-|^2 / c^2); positions and currents use
 *      v = u / gamma; the kinetic energy is m w (gamma - 1) c^2, written as
 *      m w |u|^2 / (gamma + 1), and the momentum m w u.
 *   R15 the optional field smoothing (Sec. 2.2: a self-consistent field and
 *      moment smoother) applies the same operator S, field_smooth_passes
 *      times, to copies of E^n and B^n that the ions gather in the push;
 *      the field state is not smoothed.  S is symmetric, so with as many
 *      field passes as moment passes the smoothed gather is the transpose
 *      of the smoothed deposit and an ion exerts no force on itself.
 *   R5 the floor n_f = max(n, n_floor) is applied wherever n enters Ohm's
 *      law (pressure, ion flow and Hall term).
 *   R6 the Laplacian in the hyper-resistive term is the 3-point-per-axis
 *      cell-centred Laplacian.
 *   R7 each field subcycle of length h = dt/nsub is an explicit-midpoint
 *      (RK2) step; the moments are held at their half-step values
 *      n^{n+1/2}, J^{n+1/2} during the subcycle B^n -> B^{n+1}.
 *   R8 start-up: loaded velocities are v^{-1/2}; the previous moments are the
 *      deposit at x^0; E^0 = Ohm(B^0, those moments).
 *   R20 the optional split B = B0 + B1 (Sec. 2.3): B0 is a fixed external
 *      field given on the cells; only B1 is advanced by Faraday's law; the
 *      current in Ohm's law (Hall, resistive and hyper-resistive terms) is
 *      J = curl B1, the cross products with B and the push use the total
 *      B0 + B1; W_B is taken of the total field and max |div B| of B1 (the
 *      advanced part, whose discrete divergence Faraday's law keeps).
 *   R21 open faces (Sec. 2.3): the part of an ion's shape that falls beyond
 *      an open face is deposited in the interior cell next to the face, so
 *      the deposited charge stays the sum of q w over the ions inside.
 *   R22 open faces: one ghost cell beyond each open face; B1, B0 and the
 *      moments there equal those of the interior neighbour; J, lap J,
 *      grad p_e and so E are evaluated in the ghost cell with derivatives
 *      normal to the face set to zero; an ion ending a step beyond an open
 *      face is removed.
 *   R23 open faces are built for the hybrid Ohm's law with the equation of
 *      state and without smoothing.
 *   R24 injection through an open face (Sec. 2.3, after Daughton et al.
 *      2006): a drifting Maxwellian (n, u, T) and a weight w per species
 *      and face; per face cell and step the count is N = Gamma A dt / w
 *      rounded stochastically, each ion's inward speed follows the
 *      flux-weighted distribution, its tangential velocity the Maxwellian,
 *      it enters at a uniform time within the step and is appended after
 *      the push (it deposits from the next step on); random numbers from
 *      Philox4x32-10 keyed by the run's seed.
 *   R9 an axis with one cell (2D runs use ny = 1) is periodic with period one
 *      cell, so shapes fold onto the same cell and centred differences along
 *      it vanish.  Offsets along such an axis are never moved.
 *
 * Units: normalised Alfvenic units, e = m_p = mu_0 = 1, lengths in d_i,
 * time in 1/Omega_ci.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the particle loop and the cell loops (1 by default: the
 * parity reference runs on one thread).  With T > 1 the particles are split
 * into T contiguous ranges, each thread deposits into private grids, and the
 * private grids and energy sums are added in thread order, so results are
 * deterministic for a given T and differ from T = 1 only in FP64 summation
 * order.  Cell loops write one output per cell and are unchanged by T. */
static int g_threads = 1;

void hvo_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int hvo_get_threads(void) { return g_threads; }

/* Threads available to OpenMP (1 when built without it). */
int hvo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

typedef struct {
  int64_t nx, ny, nz;
  double dx, dy, dz, dt;
  int64_t nsub;
  double Te, gamma_e, eta, eta_h, n_floor;
  int64_t shape; /* 0 NGP (Eq. 13), 1 QS (Eq. 17), 2 CIC (tensor-linear) */
  int64_t smooth_passes;
  int64_t field_smooth_passes; /* R15 */
  int64_t pe_eq;                /* R16: 1 = electron energy equation */
  double kappa;                 /* R16: heat conductivity */
  int64_t ohm_model;            /* 0 hybrid (Eq. 2), 1 electrostatic (R17),
                                   2 resistive background (R18) */
  int64_t relativistic;         /* R19: relativistic Boris push */
  double c_light;               /* R19: speed of light */
  int64_t open[3];              /* R22: 1 = the axis has open faces (Sec. 2.3) */
  const double *B0;             /* R20: fixed external field [3][ncell] or NULL */
} hvo_grid;

typedef struct {
  int64_t n;
  double q, m;
  int64_t *cell;
  double *ox, *oy, *oz;
  double *vx, *vy, *vz;
  double *w;
} hvo_species;

typedef struct {
  double W_K;   /* sum 1/2 m w |v^{n+1/2}|^2 */
  double P[3];  /* sum m w v^{n+1/2} */
  double charge;/* sum n^{n+1/2} V_c over cells (deposited, unsmoothed) */
  double W_B;   /* sum 1/2 |B|^2 V_c */
  double max_divB;
} hvo_diag;

static int64_t ncell_of(const hvo_grid *g) { return g->nx * g->ny * g->nz; }

static int64_t wrapi(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

/* linear cell index I <-> (i,j,k), x fastest (Sec. 2.2), periodic wrap */
static int64_t cidx(const hvo_grid *g, int64_t i, int64_t j, int64_t k) {
  return wrapi(i, g->nx) + g->nx * (wrapi(j, g->ny) + g->ny * wrapi(k, g->nz));
}

static void cdecode(const hvo_grid *g, int64_t c, int64_t *i, int64_t *j, int64_t *k) {
  *i = c % g->nx;
  *j = (c / g->nx) % g->ny;
  *k = c / (g->nx * g->ny);
}

/* ------------------------------------------------------------------------ */
/* Particle shapes.  Returns the number of target cells; fills the cell     */
/* shifts (si,sj,sk) relative to the particle's cell and the weights.       */
/* ------------------------------------------------------------------------ */
int hvo_shape(int64_t shape, double dx, double dy, double dz,
              int32_t *si, int32_t *sj, int32_t *sk, double *wt) {
  if (shape == 0) {
    /* NGP (Eq. 13): all weight to the particle's own cell. */
    si[0] = sj[0] = sk[0] = 0;
    wt[0] = 1.0;
    return 1;
  }
  if (shape == 1) {
    /* QS (Eq. 17): own cell and its six face neighbours. */
    int t = 0;
    si[t] = 0;  sj[t] = 0;  sk[t] = 0;  wt[t++] = (3.0 - dx * dx - dy * dy - dz * dz) / 6.0;
    si[t] = 1;  sj[t] = 0;  sk[t] = 0;  wt[t++] = (1.0 + dx) * (1.0 + dx) / 12.0;
    si[t] = 0;  sj[t] = 1;  sk[t] = 0;  wt[t++] = (1.0 + dy) * (1.0 + dy) / 12.0;
    si[t] = 0;  sj[t] = 0;  sk[t] = 1;  wt[t++] = (1.0 + dz) * (1.0 + dz) / 12.0;
    si[t] = -1; sj[t] = 0;  sk[t] = 0;  wt[t++] = (1.0 - dx) * (1.0 - dx) / 12.0;
    si[t] = 0;  sj[t] = -1; sk[t] = 0;  wt[t++] = (1.0 - dy) * (1.0 - dy) / 12.0;
    si[t] = 0;  sj[t] = 0;  sk[t] = -1; wt[t++] = (1.0 - dz) * (1.0 - dz) / 12.0;
    return t;
  }
  /* CIC on cell centres: per axis, weight 1 - |d|/2 to the own cell and
   * |d|/2 to the neighbour on the side of d; tensor product over axes. */
  {
    double d[3] = {dx, dy, dz};
    int side[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      side[a] = d[a] >= 0.0 ? 1 : -1;
      f[a] = fabs(d[a]) / 2.0;
    }
    int t = 0;
    for (int c = 0; c < 8; ++c) {
      int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
      si[t] = ox ? side[0] : 0;
      sj[t] = oy ? side[1] : 0;
      sk[t] = oz ? side[2] : 0;
      wt[t] = (ox ? f[0] : 1.0 - f[0]) * (oy ? f[1] : 1.0 - f[1]) * (oz ? f[2] : 1.0 - f[2]);
      ++t;
    }
    return t;
  }
}

/* Field at a particle: F(x_p) = sum_t S_t F_t, the same weights as the
 * deposit (App. B: Eqs. 17 and 19 together are self-force free).
 * F is component-major [nc][ncell]. */
void hvo_gather(const hvo_grid *g, const double *F, int64_t nc, int64_t cell,
                double dx, double dy, double dz, double *out) {
  int32_t si[8], sj[8], sk[8];
  double wt[8];
  int64_t i, j, k, nce = ncell_of(g);
  cdecode(g, cell, &i, &j, &k);
  int nt = hvo_shape(g->shape, dx, dy, dz, si, sj, sk, wt);
  for (int64_t a = 0; a < nc; ++a) out[a] = 0.0;
  for (int t = 0; t < nt; ++t) {
    int64_t c = cidx(g, i + si[t], j + sj[t], k + sk[t]);
    for (int64_t a = 0; a < nc; ++a) out[a] += wt[t] * F[a * nce + c];
  }
}

/* Non-relativistic Boris push (Sec. 2.2, Eq. 9): half electric kick over
 * dt/2, magnetic rotation over dt, half electric kick over dt/2.
 * qmdt = (q/m) dt.  v enters as v^{n-1/2} and leaves as v^{n+1/2}. */
void hvo_boris(double qmdt, const double *E, const double *B, double *v) {
  double h = 0.5 * qmdt;
  double vm[3], t[3], s[3], vp[3], vq[3];
  for (int a = 0; a < 3; ++a) vm[a] = v[a] + h * E[a];
  for (int a = 0; a < 3; ++a) t[a] = h * B[a];
  double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
  /* v' = v- + v- x t */
  vp[0] = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
  vp[1] = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
  vp[2] = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
  /* v+ = v- + v' x s */
  vq[0] = vm[0] + (vp[1] * s[2] - vp[2] * s[1]);
  vq[1] = vm[1] + (vp[2] * s[0] - vp[0] * s[2]);
  vq[2] = vm[2] + (vp[0] * s[1] - vp[1] * s[0]);
  for (int a = 0; a < 3; ++a) v[a] = vq[a] + h * E[a];
}

/* Relativistic Boris push (reading R19): u = gamma v in place,
 *   u- = u + h E,  gamma- = sqrt(1 + |u-|^2 / c^2),  t = h B / gamma-,
 *   rotation as in hvo_boris,  u <- u+ + h E,  h = q dt / 2m. */
void hvo_boris_rel(double qmdt, double c, const double *E, const double *B, double *u) {
  double h = 0.5 * qmdt;
  double um[3], t[3], s[3], up[3], uq[3];
  for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
  double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) / (c * c));
  for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
  double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
  up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
  uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
  uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
  for (int a = 0; a < 3; ++a) u[a] = uq[a] + h * E[a];
}

/* Lorentz factor of u = gamma v (R19). */
static double lorentz(double c, const double *u) {
  return sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (c * c));
}

/* Move a particle by v * (frac * dt) (Sec. 2.2, Eq. 10) in cell-index +
 * relative-coordinate form (reading R1): d <- d + 2 v frac dt / Delta,
 * shift m = floor((d+1)/2), d <- d - 2m, cell <- cell + m (periodic).
 * Axes with a single cell are not moved (reading R9). */
void hvo_move(const hvo_grid *g, int64_t *cell, double *d, const double *v, double frac) {
  int64_t n[3] = {g->nx, g->ny, g->nz};
  double del[3] = {g->dx, g->dy, g->dz};
  int64_t idx[3];
  cdecode(g, *cell, &idx[0], &idx[1], &idx[2]);
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 1) continue;
    double x = d[a] + 2.0 * v[a] * frac * g->dt / del[a];
    double m = floor((x + 1.0) / 2.0);
    x -= 2.0 * m;
    if (x >= 1.0) { x -= 2.0; m += 1.0; }
    if (x < -1.0) { x += 2.0; m -= 1.0; }
    d[a] = x;
    idx[a] = wrapi(idx[a] + (int64_t)m, n[a]);
  }
  *cell = cidx(g, idx[0], idx[1], idx[2]);
}

/* Add one particle's contribution q w S_t / V_c to n and q w v S_t / V_c to
 * J at position (cell, d) (Eqs. 13 and 17). */
static void deposit_one(const hvo_grid *g, int64_t cell, const double *d, const double *v,
                        double qw, double *n, double *J) {
  int32_t si[8], sj[8], sk[8];
  double wt[8];
  int64_t i, j, k, nce = ncell_of(g);
  double vc = g->dx * g->dy * g->dz;
  cdecode(g, cell, &i, &j, &k);
  int nt = hvo_shape(g->shape, d[0], d[1], d[2], si, sj, sk, wt);
  for (int t = 0; t < nt; ++t) {
    int64_t c = cidx(g, i + si[t], j + sj[t], k + sk[t]);
    double s = qw * wt[t] / vc;
    n[c] += s;
    J[0 * nce + c] += s * v[0];
    J[1 * nce + c] += s * v[1];
    J[2 * nce + c] += s * v[2];
  }
}

/* Deposit every particle at its current position with its current velocity,
 * without pushing (start-up, reading R8).  n, J are accumulated into. */
void hvo_deposit(const hvo_grid *g, const hvo_species *sp, int64_t nsp, double *n, double *J) {
  for (int64_t s = 0; s < nsp; ++s) {
    for (int64_t p = 0; p < sp[s].n; ++p) {
      double d[3] = {sp[s].ox[p], sp[s].oy[p], sp[s].oz[p]};
      double v[3] = {sp[s].vx[p], sp[s].vy[p], sp[s].vz[p]};
      if (g->relativistic) {  /* R19: the stored u = gamma v */
        double gi = 1.0 / lorentz(g->c_light, v);
        for (int a = 0; a < 3; ++a) v[a] *= gi;
      }
      deposit_one(g, sp[s].cell[p], d, v, sp[s].q * sp[s].w[p], n, J);
    }
  }
}

/* One ion of the particle part of a step: gather E^n, B^n at x^n,
 * Boris-push v^{n-1/2} -> v^{n+1/2}, deposit n, J at the half-step position
 * x^{n+1/2} (App. B; reading R2), then move to x^{n+1}.  n_acc, J_acc, kin
 * are accumulated into (kin: sum 1/2 m w |v|^2 and sum m w v). */
static void push_one(const hvo_grid *g, hvo_species *sp, int64_t p, double qmdt,
                     const double *E, const double *B, double *n_acc, double *J_acc,
                     double *kin) {
  int64_t cell = sp->cell[p];
  double d[3] = {sp->ox[p], sp->oy[p], sp->oz[p]};
  double v[3] = {sp->vx[p], sp->vy[p], sp->vz[p]};
  double Ep[3], Bp[3];
  hvo_gather(g, E, 3, cell, d[0], d[1], d[2], Ep);
  hvo_gather(g, B, 3, cell, d[0], d[1], d[2], Bp);
  double u[3] = {v[0], v[1], v[2]}, gam = 1.0;
  if (g->relativistic) {  /* R19 */
    hvo_boris_rel(qmdt, g->c_light, Ep, Bp, u);
    gam = lorentz(g->c_light, u);
    for (int a = 0; a < 3; ++a) v[a] = u[a] / gam;
  } else {
    hvo_boris(qmdt, Ep, Bp, v);
    for (int a = 0; a < 3; ++a) u[a] = v[a];
  }
  /* half-step position for the deposit */
  int64_t ch = cell;
  double dh[3] = {d[0], d[1], d[2]};
  hvo_move(g, &ch, dh, v, 0.5);
  deposit_one(g, ch, dh, v, sp->q * sp->w[p], n_acc, J_acc);
  /* full move */
  hvo_move(g, &cell, d, v, 1.0);
  sp->cell[p] = cell;
  sp->ox[p] = d[0];
  sp->oy[p] = d[1];
  sp->oz[p] = d[2];
  sp->vx[p] = u[0];
  sp->vy[p] = u[1];
  sp->vz[p] = u[2];
  double mw = sp->m * sp->w[p];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  kin[0] += g->relativistic ? mw * uu / (gam + 1.0) : 0.5 * mw * uu;
  kin[1] += mw * u[0];
  kin[2] += mw * u[1];
  kin[3] += mw * u[2];
}

/* The particle part of one step over every ion (push_one); n_acc, J_acc
 * are accumulated into and kin[0..3] receive the energy and momentum sums.
 * With more than one thread each thread takes a contiguous range of ions
 * and its own grids, added in thread order afterwards. */
void hvo_push_deposit(const hvo_grid *g, hvo_species *sp, int64_t nsp,
                      const double *E, const double *B, double *n_acc, double *J_acc,
                      double *kin) {
  int64_t nce = ncell_of(g);
  for (int a = 0; a < 4; ++a) kin[a] = 0.0;
  for (int64_t s = 0; s < nsp; ++s) {
    double qmdt = sp[s].q / sp[s].m * g->dt;
    int nt = g_threads;
    if (nt <= 1 || sp[s].n < 2) {
      for (int64_t p = 0; p < sp[s].n; ++p) push_one(g, &sp[s], p, qmdt, E, B, n_acc, J_acc, kin);
      continue;
    }
    double *priv = (double *)calloc((size_t)nt * (size_t)(4 * nce + 4), sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
      int tid = 0, team = 1;
#ifdef _OPENMP
      tid = omp_get_thread_num();
      team = omp_get_num_threads();
#endif
      /* range t of nt whatever the team size OpenMP grants */
      for (int t = tid; t < nt; t += team) {
        double *pn = priv + (size_t)t * (4 * nce + 4);
        int64_t p0 = sp[s].n * t / nt, p1 = sp[s].n * (t + 1) / nt;
        for (int64_t p = p0; p < p1; ++p)
          push_one(g, &sp[s], p, qmdt, E, B, pn, pn + nce, pn + 4 * nce);
      }
    }
    for (int t = 0; t < nt; ++t) {
      const double *pn = priv + (size_t)t * (4 * nce + 4);
      for (int64_t c = 0; c < nce; ++c) n_acc[c] += pn[c];
      for (int64_t c = 0; c < 3 * nce; ++c) J_acc[c] += pn[nce + c];
      for (int a = 0; a < 4; ++a) kin[a] += pn[4 * nce + a];
    }
    free(priv);
  }
}

/* ------------------------------------------------------------------------ */
/* Grid operators on the cell-centred grid (Sec. 2.2, Eq. 12).              */
/* ------------------------------------------------------------------------ */

/* centred derivative of scalar field f along axis a at cell (i,j,k) */
static double dcen(const hvo_grid *g, const double *f, int a, int64_t i, int64_t j, int64_t k) {
  if (a == 0) return (f[cidx(g, i + 1, j, k)] - f[cidx(g, i - 1, j, k)]) / (2.0 * g->dx);
  if (a == 1) return (f[cidx(g, i, j + 1, k)] - f[cidx(g, i, j - 1, k)]) / (2.0 * g->dy);
  return (f[cidx(g, i, j, k + 1)] - f[cidx(g, i, j, k - 1)]) / (2.0 * g->dz);
}

/* out = curl A (centred), A and out component-major [3][ncell] */
void hvo_curl(const hvo_grid *g, const double *A, double *out) {
  int64_t nce = ncell_of(g);
  const double *Ax = A, *Ay = A + nce, *Az = A + 2 * nce;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (int64_t c = 0; c < nce; ++c) {
    int64_t i, j, k;
    cdecode(g, c, &i, &j, &k);
    out[0 * nce + c] = dcen(g, Az, 1, i, j, k) - dcen(g, Ay, 2, i, j, k);
    out[1 * nce + c] = dcen(g, Ax, 2, i, j, k) - dcen(g, Az, 0, i, j, k);
    out[2 * nce + c] = dcen(g, Ay, 0, i, j, k) - dcen(g, Ax, 1, i, j, k);
  }
}

/* out = grad f (centred) [3][ncell] */
void hvo_grad(const hvo_grid *g, const double *f, double *out) {
  int64_t nce = ncell_of(g);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (int64_t c = 0; c < nce; ++c) {
    int64_t i, j, k;
    cdecode(g, c, &i, &j, &k);
    for (int a = 0; a < 3; ++a) out[a * nce + c] = dcen(g, f, a, i, j, k);
  }
}

/* out = div A (centred) [ncell] */
void hvo_div(const hvo_grid *g, const double *A, double *out) {
  int64_t nce = ncell_of(g);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (int64_t c = 0; c < nce; ++c) {
    int64_t i, j, k;
    cdecode(g, c, &i, &j, &k);
    out[c] = dcen(g, A, 0, i, j, k) + dcen(g, A + nce, 1, i, j, k) + dcen(g, A + 2 * nce, 2, i, j, k);
  }
}

/* out = Laplacian of each of nc components (3 points per axis, reading R6) */
void hvo_lap(const hvo_grid *g, const double *A, int64_t nc, double *out) {
  int64_t nce = ncell_of(g);
  for (int64_t a = 0; a < nc; ++a) {
    const double *f = A + a * nce;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (int64_t c = 0; c < nce; ++c) {
      int64_t i, j, k;
      cdecode(g, c, &i, &j, &k);
      double fc = f[c];
      out[a * nce + c] =
          (f[cidx(g, i + 1, j, k)] - 2.0 * fc + f[cidx(g, i - 1, j, k)]) / (g->dx * g->dx) +
          (f[cidx(g, i, j + 1, k)] - 2.0 * fc + f[cidx(g, i, j - 1, k)]) / (g->dy * g->dy) +
          (f[cidx(g, i, j, k + 1)] - 2.0 * fc + f[cidx(g, i, j, k - 1)]) / (g->dz * g->dz);
    }
  }
}

/* Ohm's law for massless electrons (Eq. 2) with R_ei = eta J - eta_H lap J
 * (Eq. 3), J = curl B (Eq. 4, mu_0 = 1), p_e = Te n^gamma (Eq. 6, p_0 = n_0
 * Te, n_0 = 1) and the density floor n_f = max(n, n_floor) (Sec. 2.1):
 *   E = -grad p_e / n_f - (J_i / n_f) x B + (J x B) / n_f + eta J - eta_H lap J
 * Inputs: B [3][ncell], n [ncell], Ji [3][ncell]; output E [3][ncell].
 * With an external field (R20) B is B1: J = curl B1 and the cross products
 * take B0 + B1. */
static void ohm_with(const hvo_grid *g, const double *B, const double *n, const double *Ji,
                     const double *pe_field, double *E) {
  int64_t nce = ncell_of(g);
  double *J = (double *)malloc(sizeof(double) * 3 * nce);
  double *LJ = (double *)malloc(sizeof(double) * 3 * nce);
  double *nf = (double *)malloc(sizeof(double) * nce);
  double *pe = (double *)malloc(sizeof(double) * nce);
  double *gp = (double *)malloc(sizeof(double) * 3 * nce);
  hvo_curl(g, B, J);
  hvo_lap(g, J, 3, LJ);
  for (int64_t c = 0; c < nce; ++c) {
    nf[c] = n[c] > g->n_floor ? n[c] : g->n_floor;
    pe[c] = pe_field ? pe_field[c] : g->Te * pow(nf[c], g->gamma_e);
  }
  hvo_grad(g, pe, gp);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (int64_t c = 0; c < nce; ++c) {
    if (g->ohm_model == 1) {  /* R17: E = -grad p_e / n_f */
      for (int a = 0; a < 3; ++a) E[a * nce + c] = -gp[a * nce + c] / nf[c];
      continue;
    }
    if (g->ohm_model == 2) {  /* R18: E = eta (curl B - J_k) */
      for (int a = 0; a < 3; ++a) E[a * nce + c] = g->eta * (J[a * nce + c] - Ji[a * nce + c]);
      continue;
    }
    double b[3] = {B[c], B[nce + c], B[2 * nce + c]};
    if (g->B0) /* R20: B holds B1; the cross products take B0 + B1 */
      for (int a = 0; a < 3; ++a) b[a] += g->B0[a * nce + c];
    double jt[3] = {J[c], J[nce + c], J[2 * nce + c]};
    double ui[3] = {Ji[c] / nf[c], Ji[nce + c] / nf[c], Ji[2 * nce + c] / nf[c]};
    double uixb[3] = {ui[1] * b[2] - ui[2] * b[1], ui[2] * b[0] - ui[0] * b[2], ui[0] * b[1] - ui[1] * b[0]};
    double jxb[3] = {jt[1] * b[2] - jt[2] * b[1], jt[2] * b[0] - jt[0] * b[2], jt[0] * b[1] - jt[1] * b[0]};
    for (int a = 0; a < 3; ++a) {
      E[a * nce + c] = -gp[a * nce + c] / nf[c] - uixb[a] + jxb[a] / nf[c] +
                       g->eta * jt[a] - g->eta_h * LJ[a * nce + c];
    }
  }
  free(J);
  free(LJ);
  free(nf);
  free(pe);
  free(gp);
}

void hvo_ohm(const hvo_grid *g, const double *B, const double *n, const double *Ji, double *E) {
  ohm_with(g, B, n, Ji, NULL, E);
}

/* Ohm's law with p_e taken from the field pe [ncell] (R16). */
void hvo_ohm_pe(const hvo_grid *g, const double *B, const double *n, const double *Ji,
                const double *pe, double *E) {
  ohm_with(g, B, n, Ji, pe, E);
}

/* Electron energy equation (Sec. 2.1, Eq. dpdt; reading R16):
 *   out = -gamma div(p_e u_e) + (gamma - 1) u_e . grad p_e
 *         + (gamma - 1) kappa lap(T_e),
 *   u_e = -(curl B - J_i) / n_f,  T_e = p_e / n_f. */
void hvo_dpdt(const hvo_grid *g, const double *B, const double *pe, const double *n,
              const double *Ji, double *out) {
  int64_t nce = ncell_of(g);
  double gam = g->gamma_e;
  double *J = (double *)malloc(sizeof(double) * 3 * nce);
  double *ue = (double *)malloc(sizeof(double) * 3 * nce);
  double *pu = (double *)malloc(sizeof(double) * 3 * nce);
  double *T = (double *)malloc(sizeof(double) * nce);
  double *divpu = (double *)malloc(sizeof(double) * nce);
  double *gp = (double *)malloc(sizeof(double) * 3 * nce);
  double *lT = (double *)malloc(sizeof(double) * nce);
  hvo_curl(g, B, J);
  if (g->ohm_model == 1) memset(J, 0, sizeof(double) * 3 * nce); /* R17: no magnetic current */
  for (int64_t c = 0; c < nce; ++c) {
    double nf = n[c] > g->n_floor ? n[c] : g->n_floor;
    for (int a = 0; a < 3; ++a) {
      ue[a * nce + c] = -(J[a * nce + c] - Ji[a * nce + c]) / nf;
      pu[a * nce + c] = pe[c] * ue[a * nce + c];
    }
    T[c] = pe[c] / nf;
  }
  hvo_div(g, pu, divpu);
  hvo_grad(g, pe, gp);
  hvo_lap(g, T, 1, lT);
  for (int64_t c = 0; c < nce; ++c) {
    double ugp = ue[c] * gp[c] + ue[nce + c] * gp[nce + c] + ue[2 * nce + c] * gp[2 * nce + c];
    out[c] = -gam * divpu[c] + (gam - 1.0) * ugp + (gam - 1.0) * g->kappa * lT[c];
  }
  free(J);
  free(ue);
  free(pu);
  free(T);
  free(divpu);
  free(gp);
  free(lT);
}

/* Faraday's law (Eq. 5) subcycled nsub times per particle step (Sec. 2.1),
 * each subcycle an explicit-midpoint step of h = dt / nsub (reading R7):
 *   B* = B - (h/2) curl E(B),   B <- B - h curl E(B*).
 * n, Ji are held fixed (the half-step moments). */
void hvo_field_advance(const hvo_grid *g, double *B, const double *n, const double *Ji) {
  if (g->ohm_model == 1) return; /* R17: B is not advanced */
  int64_t nce = ncell_of(g);
  double h = g->dt / (double)g->nsub;
  double *E = (double *)malloc(sizeof(double) * 3 * nce);
  double *cE = (double *)malloc(sizeof(double) * 3 * nce);
  double *Bs = (double *)malloc(sizeof(double) * 3 * nce);
  for (int64_t s = 0; s < g->nsub; ++s) {
    hvo_ohm(g, B, n, Ji, E);
    hvo_curl(g, E, cE);
    for (int64_t c = 0; c < 3 * nce; ++c) Bs[c] = B[c] - 0.5 * h * cE[c];
    hvo_ohm(g, Bs, n, Ji, E);
    hvo_curl(g, E, cE);
    for (int64_t c = 0; c < 3 * nce; ++c) B[c] = B[c] - h * cE[c];
  }
  free(E);
  free(cE);
  free(Bs);
}

/* The same subcycles with the electron energy equation (R16): B and p_e
 * advance together,
 *   B* = B - (h/2) curl E(B, p_e),  p_e* = p_e + (h/2) dpdt(B, p_e),
 *   B <- B - h curl E(B*, p_e*),    p_e <- p_e + h dpdt(B*, p_e*). */
void hvo_field_advance_pe(const hvo_grid *g, double *B, double *pe, const double *n,
                          const double *Ji) {
  int64_t nce = ncell_of(g);
  double h = g->dt / (double)g->nsub;
  double *E = (double *)malloc(sizeof(double) * 3 * nce);
  double *cE = (double *)malloc(sizeof(double) * 3 * nce);
  double *Bs = (double *)malloc(sizeof(double) * 3 * nce);
  double *dp = (double *)malloc(sizeof(double) * nce);
  double *ps = (double *)malloc(sizeof(double) * nce);
  for (int64_t s = 0; s < g->nsub; ++s) {
    hvo_ohm_pe(g, B, n, Ji, pe, E);
    hvo_curl(g, E, cE);
    hvo_dpdt(g, B, pe, n, Ji, dp);
    if (g->ohm_model == 1) memset(cE, 0, sizeof(double) * 3 * nce); /* R17: B is not advanced */
    for (int64_t c = 0; c < 3 * nce; ++c) Bs[c] = B[c] - 0.5 * h * cE[c];
    for (int64_t c = 0; c < nce; ++c) ps[c] = pe[c] + 0.5 * h * dp[c];
    hvo_ohm_pe(g, Bs, n, Ji, ps, E);
    hvo_curl(g, E, cE);
    hvo_dpdt(g, Bs, ps, n, Ji, dp);
    if (g->ohm_model == 1) memset(cE, 0, sizeof(double) * 3 * nce);
    for (int64_t c = 0; c < 3 * nce; ++c) B[c] = B[c] - h * cE[c];
    for (int64_t c = 0; c < nce; ++c) pe[c] = pe[c] + h * dp[c];
  }
  free(E);
  free(cE);
  free(Bs);
  free(dp);
  free(ps);
}

/* Separable binomial (1/4, 1/2, 1/4) smoothing, `passes` times, of nc
 * component-major grids (reading R4). */
void hvo_smooth(const hvo_grid *g, double *q, int64_t nc, int64_t passes) {
  int64_t nce = ncell_of(g);
  double *tmp = (double *)malloc(sizeof(double) * nce);
  for (int64_t p = 0; p < passes; ++p) {
    for (int64_t a = 0; a < nc; ++a) {
      double *f = q + a * nce;
      for (int ax = 0; ax < 3; ++ax) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
        for (int64_t c = 0; c < nce; ++c) {
          int64_t i, j, k;
          cdecode(g, c, &i, &j, &k);
          int64_t cm, cp;
          if (ax == 0) { cm = cidx(g, i - 1, j, k); cp = cidx(g, i + 1, j, k); }
          else if (ax == 1) { cm = cidx(g, i, j - 1, k); cp = cidx(g, i, j + 1, k); }
          else { cm = cidx(g, i, j, k - 1); cp = cidx(g, i, j, k + 1); }
          tmp[c] = 0.25 * f[cm] + 0.5 * f[c] + 0.25 * f[cp];
        }
        memcpy(f, tmp, sizeof(double) * nce);
      }
    }
  }
  free(tmp);
}

/* Linear extrapolation (Eq. 11): out = 3/2 half - 1/2 prev. */
void hvo_extrapolate(int64_t len, const double *half, const double *prev, double *out) {
  for (int64_t c = 0; c < len; ++c) out[c] = 1.5 * half[c] - 0.5 * prev[c];
}

/* Grid diagnostics: W_B = sum 1/2 |B|^2 V_c, charge = sum n V_c,
 * max |div B|. */
void hvo_diag_grid(const hvo_grid *g, const double *B, const double *n, double *wb,
                   double *charge, double *maxdiv) {
  int64_t nce = ncell_of(g);
  double vc = g->dx * g->dy * g->dz;
  double *dv = (double *)malloc(sizeof(double) * nce);
  hvo_div(g, B, dv);
  *wb = 0.0;
  *charge = 0.0;
  *maxdiv = 0.0;
  for (int64_t c = 0; c < nce; ++c) {
    *wb += 0.5 * (B[c] * B[c] + B[nce + c] * B[nce + c] + B[2 * nce + c] * B[2 * nce + c]) * vc;
    *charge += n[c] * vc;
    if (fabs(dv[c]) > *maxdiv) *maxdiv = fabs(dv[c]);
  }
  free(dv);
}

/* Start-up (reading R8): n_prev, J_prev := deposit at x^0 with v^{-1/2}
 * (smoothed like every deposit); E = Ohm(B, n_prev, J_prev). */
void hvo_init(const hvo_grid *g, const hvo_species *sp, int64_t nsp, const double *B,
              double *E, double *n_prev, double *J_prev) {
  int64_t nce = ncell_of(g);
  memset(n_prev, 0, sizeof(double) * nce);
  memset(J_prev, 0, sizeof(double) * 3 * nce);
  hvo_deposit(g, sp, nsp, n_prev, J_prev);
  hvo_smooth(g, n_prev, 1, g->smooth_passes);
  hvo_smooth(g, J_prev, 3, g->smooth_passes);
  hvo_ohm(g, B, n_prev, J_prev, E);
}

/* Start-up with the electron energy equation (R16): as hvo_init, and
 * p_e = Te n_f^gamma of the start-up moments (Eq. 6). */
void hvo_init_pe(const hvo_grid *g, const hvo_species *sp, int64_t nsp, const double *B,
                 double *E, double *pe, double *n_prev, double *J_prev) {
  int64_t nce = ncell_of(g);
  hvo_init(g, sp, nsp, B, E, n_prev, J_prev);
  for (int64_t c = 0; c < nce; ++c) {
    double nf = n_prev[c] > g->n_floor ? n_prev[c] : g->n_floor;
    pe[c] = g->Te * pow(nf, g->gamma_e);
  }
  hvo_ohm_pe(g, B, n_prev, J_prev, pe, E);
}

/* One full step n -> n+1 in the paper's order (Sec. 2.2):
 *   [field smoothing of the gathered copies of E, B (R15)],
 *   push + half-step deposit,  smoothing,  extrapolation (Eq. 11),
 *   subcycled field advance B^n -> B^{n+1} with the half-step moments,
 *   E^{n+1} = Ohm(B^{n+1}, n^{n+1}, J^{n+1}),  prev := half-step moments.
 * On return n_prev, J_prev hold n^{n+1/2}, J^{n+1/2}.  n_ext, J_ext (may be
 * NULL) receive the extrapolated n^{n+1}, J^{n+1}. */
static void step_impl(const hvo_grid *g, hvo_species *sp, int64_t nsp, double *B, double *E,
                      double *pe, double *n_prev, double *J_prev, double *n_ext, double *J_ext,
                      hvo_diag *dg) {
  int64_t nce = ncell_of(g);
  double *nh = (double *)calloc((size_t)nce, sizeof(double));
  double *Jh = (double *)calloc((size_t)(3 * nce), sizeof(double));
  double *ne = (double *)malloc(sizeof(double) * nce);
  double *Je = (double *)malloc(sizeof(double) * 3 * nce);
  double kin[4];
  /* the ions feel the total field: B0 + B1 with an external field (R20) */
  double *Bt = NULL;
  const double *Bg = B;
  if (g->B0) {
    Bt = (double *)malloc(sizeof(double) * 3 * nce);
    for (int64_t c = 0; c < 3 * nce; ++c) Bt[c] = B[c] + g->B0[c];
    Bg = Bt;
  }
  if (g->field_smooth_passes > 0) {
    double *Eg = (double *)malloc(sizeof(double) * 3 * nce);
    double *Bs = (double *)malloc(sizeof(double) * 3 * nce);
    memcpy(Eg, E, sizeof(double) * 3 * nce);
    memcpy(Bs, Bg, sizeof(double) * 3 * nce);
    hvo_smooth(g, Eg, 3, g->field_smooth_passes);
    hvo_smooth(g, Bs, 3, g->field_smooth_passes);
    hvo_push_deposit(g, sp, nsp, Eg, Bs, nh, Jh, kin);
    free(Eg);
    free(Bs);
  } else {
    hvo_push_deposit(g, sp, nsp, E, Bg, nh, Jh, kin);
  }
  double charge_raw = 0.0, vc = g->dx * g->dy * g->dz;
  for (int64_t c = 0; c < nce; ++c) charge_raw += nh[c] * vc;
  hvo_smooth(g, nh, 1, g->smooth_passes);
  hvo_smooth(g, Jh, 3, g->smooth_passes);
  hvo_extrapolate(nce, nh, n_prev, ne);
  hvo_extrapolate(3 * nce, Jh, J_prev, Je);
  if (pe) {
    hvo_field_advance_pe(g, B, pe, nh, Jh);
    hvo_ohm_pe(g, B, ne, Je, pe, E);
  } else {
    hvo_field_advance(g, B, nh, Jh);
    hvo_ohm(g, B, ne, Je, E);
  }
  memcpy(n_prev, nh, sizeof(double) * nce);
  memcpy(J_prev, Jh, sizeof(double) * 3 * nce);
  if (n_ext) memcpy(n_ext, ne, sizeof(double) * nce);
  if (J_ext) memcpy(J_ext, Je, sizeof(double) * 3 * nce);
  if (dg) {
    double wb, ch, md;
    hvo_diag_grid(g, B, nh, &wb, &ch, &md);
    if (Bt) { /* R20: W_B of the total field, max |div B| of B1 */
      double md1 = md;
      for (int64_t c = 0; c < 3 * nce; ++c) Bt[c] = B[c] + g->B0[c];
      hvo_diag_grid(g, Bt, nh, &wb, &ch, &md);
      md = md1;
    }
    dg->W_K = kin[0];
    dg->P[0] = kin[1];
    dg->P[1] = kin[2];
    dg->P[2] = kin[3];
    dg->charge = charge_raw;
    dg->W_B = wb;
    dg->max_divB = md;
  }
  free(Bt);
  free(nh);
  free(Jh);
  free(ne);
  free(Je);
}

void hvo_step(const hvo_grid *g, hvo_species *sp, int64_t nsp, double *B, double *E,
              double *n_prev, double *J_prev, double *n_ext, double *J_ext, hvo_diag *dg) {
  step_impl(g, sp, nsp, B, E, NULL, n_prev, J_prev, n_ext, J_ext, dg);
}

/* One step with the electron energy equation (R16): p_e [ncell] is advanced
 * with B and enters Ohm's law. */
void hvo_step_pe(const hvo_grid *g, hvo_species *sp, int64_t nsp, double *B, double *E,
                 double *pe, double *n_prev, double *J_prev, double *n_ext, double *J_ext,
                 hvo_diag *dg) {
  step_impl(g, sp, nsp, B, E, pe, n_prev, J_prev, n_ext, J_ext, dg);
}

/* Stable counting sort of keys in [0, nkeys): counts[k], exclusive offsets
 * offsets[k] (nkeys+1 entries) and perm such that key[perm[0..n)] is
 * non-decreasing with equal keys kept in input order. */
int hvo_sort_stable(const int64_t *key, int64_t n, int64_t nkeys, int64_t *perm,
                    int64_t *counts, int64_t *offsets) {
  for (int64_t k = 0; k < nkeys; ++k) counts[k] = 0;
  for (int64_t p = 0; p < n; ++p) {
    if (key[p] < 0 || key[p] >= nkeys) return -1;
    counts[key[p]] += 1;
  }
  offsets[0] = 0;
  for (int64_t k = 0; k < nkeys; ++k) offsets[k + 1] = offsets[k] + counts[k];
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nkeys > 0 ? nkeys : 1));
  for (int64_t k = 0; k < nkeys; ++k) next[k] = offsets[k];
  for (int64_t p = 0; p < n; ++p) perm[next[key[p]]++] = p;
  free(next);
  return 0;
}

/* ======================================================================== */
/* Open boundaries (Sec. 2.3; readings R21-R23).                            */
/*                                                                          */
/* An axis with open faces carries one ghost cell beyond each face (the     */
/* paper's single ghost layer).  In a ghost cell                            */
/*  - B1, B0 and the moments n, J_i equal those of the interior cell next   */
/*    to it (no normal gradient, Sec. 2.3), and                             */
/*  - the derived quantities of Ohm's law (J = curl B1, lap J, grad p_e and */
/*    so E) are evaluated with every derivative normal to that face set to  */
/*    zero, the tangential ones kept (Sec. 2.3: no normal gradients in the  */
/*    ghost-cell Ohm's law).                                                */
/* Interior cells next to a face take their centred differences across it   */
/* from the ghost values.  Faraday's law advances the interior B1 only.     */
/* The part of a deposit that falls beyond an open face is added to the     */
/* interior cell next to it (R21), and an ion that ends a step beyond an    */
/* open face leaves the simulation (absorbed, Sec. 2.3).  Periodic axes     */
/* wrap as before.  These routines cover the hybrid Ohm's law with the      */
/* equation of state, without smoothing (R23).                              */
/* ======================================================================== */

typedef struct {
  int64_t n[3]; /* interior cells per axis */
  int64_t o[3]; /* ghost cells per side: 1 on an open axis, 0 on a periodic one */
  int64_t N[3]; /* extended extent n + 2 o */
  double d[3];  /* cell sizes */
} xgrid;

static xgrid xgrid_of(const hvo_grid *g) {
  xgrid x;
  int64_t n[3] = {g->nx, g->ny, g->nz};
  double d[3] = {g->dx, g->dy, g->dz};
  for (int a = 0; a < 3; ++a) {
    x.n[a] = n[a];
    x.o[a] = g->open[a] ? 1 : 0;
    x.N[a] = n[a] + 2 * x.o[a];
    x.d[a] = d[a];
  }
  return x;
}

static int64_t xcount(const xgrid *x) { return x->N[0] * x->N[1] * x->N[2]; }

/* coordinate along axis a as an extended-grid position: shifted by the ghost
 * width on an open axis (the caller keeps it within the ghost layer),
 * wrapped on a periodic one */
static int64_t xcoord(const xgrid *x, int a, int64_t c) {
  return x->o[a] ? c + x->o[a] : wrapi(c, x->n[a]);
}

static int64_t xidx(const xgrid *x, int64_t i, int64_t j, int64_t k) {
  return xcoord(x, 0, i) + x->N[0] * (xcoord(x, 1, j) + x->N[1] * xcoord(x, 2, k));
}

/* interior coordinates of extended cell e */
static void xdecode(const xgrid *x, int64_t e, int64_t *c) {
  int64_t r = e;
  for (int a = 0; a < 3; ++a) {
    c[a] = r % x->N[a] - x->o[a];
    r /= x->N[a];
  }
}

/* interior cell nearest to (i, j, k): clamped on open axes, wrapped on
 * periodic ones (the ghost-cell copy rule and the deposit fold, R21) */
static int64_t cidx_near(const hvo_grid *g, const xgrid *x, int64_t i, int64_t j, int64_t k) {
  int64_t c[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (x->o[a]) c[a] = c[a] < 0 ? 0 : (c[a] >= x->n[a] ? x->n[a] - 1 : c[a]);
    else c[a] = wrapi(c[a], x->n[a]);
  }
  return c[0] + g->nx * (c[1] + g->ny * c[2]);
}

static int xghost(const xgrid *x, int a, int64_t c) { return x->o[a] && (c < 0 || c >= x->n[a]); }

/* extended copy of nc interior fields (ghost = nearest interior cell) */
static void xfill(const hvo_grid *g, const xgrid *x, const double *src, int64_t nc, double *dst) {
  int64_t nce = ncell_of(g), ne = xcount(x);
  for (int64_t e = 0; e < ne; ++e) {
    int64_t c[3];
    xdecode(x, e, c);
    int64_t s = cidx_near(g, x, c[0], c[1], c[2]);
    for (int64_t m = 0; m < nc; ++m) dst[m * ne + e] = src[m * nce + s];
  }
}

/* centred derivative along axis a of extended field f at extended cell with
 * interior coordinates c: zero in a cell that is a ghost along a (no normal
 * gradient there), a centred difference otherwise */
static double xd(const xgrid *x, const double *f, int a, const int64_t *c) {
  if (xghost(x, a, c[a])) return 0.0;
  int64_t p[3] = {c[0], c[1], c[2]}, m[3] = {c[0], c[1], c[2]};
  p[a] += 1;
  m[a] -= 1;
  return (f[xidx(x, p[0], p[1], p[2])] - f[xidx(x, m[0], m[1], m[2])]) / (2.0 * x->d[a]);
}

static double xd2(const xgrid *x, const double *f, int a, const int64_t *c) {
  if (xghost(x, a, c[a])) return 0.0;
  int64_t p[3] = {c[0], c[1], c[2]}, m[3] = {c[0], c[1], c[2]};
  p[a] += 1;
  m[a] -= 1;
  return (f[xidx(x, p[0], p[1], p[2])] - 2.0 * f[xidx(x, c[0], c[1], c[2])] +
          f[xidx(x, m[0], m[1], m[2])]) / (x->d[a] * x->d[a]);
}

/* Ohm's law (Eq. 2, as ohm_with) on every extended cell from extended B1,
 * the external field (extended, or NULL), moments and their floor. */
static void xohm(const hvo_grid *g, const xgrid *x, const double *B1, const double *B0,
                 const double *n, const double *Ji, double *E) {
  int64_t ne = xcount(x);
  double *J = (double *)malloc(sizeof(double) * 3 * ne);
  double *pe = (double *)malloc(sizeof(double) * ne);
  for (int64_t e = 0; e < ne; ++e) {
    int64_t c[3];
    xdecode(x, e, c);
    J[e] = xd(x, B1 + 2 * ne, 1, c) - xd(x, B1 + ne, 2, c);
    J[ne + e] = xd(x, B1, 2, c) - xd(x, B1 + 2 * ne, 0, c);
    J[2 * ne + e] = xd(x, B1 + ne, 0, c) - xd(x, B1, 1, c);
    double nf = n[e] > g->n_floor ? n[e] : g->n_floor;
    pe[e] = g->Te * pow(nf, g->gamma_e);
  }
  for (int64_t e = 0; e < ne; ++e) {
    int64_t c[3];
    xdecode(x, e, c);
    double nf = n[e] > g->n_floor ? n[e] : g->n_floor;
    double b[3], jt[3], ui[3], lj[3], gp[3];
    for (int a = 0; a < 3; ++a) {
      b[a] = B1[a * ne + e] + (B0 ? B0[a * ne + e] : 0.0);
      jt[a] = J[a * ne + e];
      ui[a] = Ji[a * ne + e] / nf;
      lj[a] = xd2(x, J + a * ne, 0, c) + xd2(x, J + a * ne, 1, c) + xd2(x, J + a * ne, 2, c);
      gp[a] = xd(x, pe, a, c);
    }
    double uixb[3] = {ui[1] * b[2] - ui[2] * b[1], ui[2] * b[0] - ui[0] * b[2], ui[0] * b[1] - ui[1] * b[0]};
    double jxb[3] = {jt[1] * b[2] - jt[2] * b[1], jt[2] * b[0] - jt[0] * b[2], jt[0] * b[1] - jt[1] * b[0]};
    for (int a = 0; a < 3; ++a)
      E[a * ne + e] = -gp[a] / nf - uixb[a] + jxb[a] / nf + g->eta * jt[a] - g->eta_h * lj[a];
  }
  free(J);
  free(pe);
}

/* E on the extended grid from interior B1 [3][ncell], n, Ji; Eext [3][next] */
void hvo_ohm_open(const hvo_grid *g, const double *B1, const double *n, const double *Ji,
                  double *Eext) {
  xgrid x = xgrid_of(g);
  int64_t ne = xcount(&x);
  double *Bx = (double *)malloc(sizeof(double) * 3 * ne);
  double *B0x = g->B0 ? (double *)malloc(sizeof(double) * 3 * ne) : NULL;
  double *nx = (double *)malloc(sizeof(double) * ne);
  double *Jx = (double *)malloc(sizeof(double) * 3 * ne);
  xfill(g, &x, B1, 3, Bx);
  if (B0x) xfill(g, &x, g->B0, 3, B0x);
  xfill(g, &x, n, 1, nx);
  xfill(g, &x, Ji, 3, Jx);
  xohm(g, &x, Bx, B0x, nx, Jx, Eext);
  free(Bx);
  free(B0x);
  free(nx);
  free(Jx);
}

/* curl of extended E at the interior cells, out [3][ncell] */
static void xcurl_interior(const hvo_grid *g, const xgrid *x, const double *E, double *out) {
  int64_t nce = ncell_of(g), ne = xcount(x);
  for (int64_t q = 0; q < nce; ++q) {
    int64_t c[3];
    cdecode(g, q, &c[0], &c[1], &c[2]);
    out[q] = xd(x, E + 2 * ne, 1, c) - xd(x, E + ne, 2, c);
    out[nce + q] = xd(x, E, 2, c) - xd(x, E + 2 * ne, 0, c);
    out[2 * nce + q] = xd(x, E + ne, 0, c) - xd(x, E, 1, c);
  }
}

/* The subcycled Faraday advance of B1 (as hvo_field_advance, reading R7)
 * with the open-boundary Ohm's law. */
void hvo_field_advance_open(const hvo_grid *g, double *B1, const double *n, const double *Ji) {
  xgrid x = xgrid_of(g);
  int64_t nce = ncell_of(g), ne = xcount(&x);
  double h = g->dt / (double)g->nsub;
  double *E = (double *)malloc(sizeof(double) * 3 * ne);
  double *cE = (double *)malloc(sizeof(double) * 3 * nce);
  double *Bs = (double *)malloc(sizeof(double) * 3 * nce);
  for (int64_t s = 0; s < g->nsub; ++s) {
    hvo_ohm_open(g, B1, n, Ji, E);
    xcurl_interior(g, &x, E, cE);
    for (int64_t c = 0; c < 3 * nce; ++c) Bs[c] = B1[c] - 0.5 * h * cE[c];
    hvo_ohm_open(g, Bs, n, Ji, E);
    xcurl_interior(g, &x, E, cE);
    for (int64_t c = 0; c < 3 * nce; ++c) B1[c] = B1[c] - h * cE[c];
  }
  free(E);
  free(cE);
  free(Bs);
}

/* A move without the wrap on open axes: raw cell coordinates c[3] (which may
 * leave [0, n) on an open axis), offsets d updated; periodic axes wrap. */
static void move_raw(const hvo_grid *g, const xgrid *x, int64_t *c, double *d, const double *v,
                     double frac) {
  for (int a = 0; a < 3; ++a) {
    if (x->n[a] == 1) continue;
    double y = d[a] + 2.0 * v[a] * frac * g->dt / x->d[a];
    double m = floor((y + 1.0) / 2.0);
    y -= 2.0 * m;
    if (y >= 1.0) { y -= 2.0; m += 1.0; }
    if (y < -1.0) { y += 2.0; m -= 1.0; }
    d[a] = y;
    c[a] += (int64_t)m;
    if (!x->o[a]) c[a] = wrapi(c[a], x->n[a]);
  }
}

/* gather of extended fields at a particle in interior cell c with offsets d:
 * shape targets one cell beyond a face read the ghost cell */
static void xgather(const hvo_grid *g, const xgrid *x, const double *F, int64_t nc, const int64_t *c,
                    const double *d, double *out) {
  int32_t si[8], sj[8], sk[8];
  double wt[8];
  int64_t ne = xcount(x);
  int nt = hvo_shape(g->shape, d[0], d[1], d[2], si, sj, sk, wt);
  for (int64_t m = 0; m < nc; ++m) out[m] = 0.0;
  for (int t = 0; t < nt; ++t) {
    int64_t e = xidx(x, c[0] + si[t], c[1] + sj[t], c[2] + sk[t]);
    for (int64_t m = 0; m < nc; ++m) out[m] += wt[t] * F[m * ne + e];
  }
}

/* deposit at raw position (c, d): targets beyond an open face fold onto the
 * interior cell next to it (R21) */
static void deposit_near(const hvo_grid *g, const xgrid *x, const int64_t *c, const double *d,
                         const double *v, double qw, double *n, double *J) {
  int32_t si[8], sj[8], sk[8];
  double wt[8];
  int64_t nce = ncell_of(g);
  double vc = g->dx * g->dy * g->dz;
  int nt = hvo_shape(g->shape, d[0], d[1], d[2], si, sj, sk, wt);
  for (int t = 0; t < nt; ++t) {
    int64_t q = cidx_near(g, x, c[0] + si[t], c[1] + sj[t], c[2] + sk[t]);
    double s = qw * wt[t] / vc;
    n[q] += s;
    J[q] += s * v[0];
    J[nce + q] += s * v[1];
    J[2 * nce + q] += s * v[2];
  }
}

static int outside(const xgrid *x, const int64_t *c) {
  for (int a = 0; a < 3; ++a)
    if (xghost(x, a, c[a])) return 1;
  return 0;
}

/* The particle part of a step with open faces: every ion gathers E and the
 * total B at x^n from the extended fields (Eext, Btx), is pushed (Boris,
 * non-relativistic), deposits at its half-step position (folded, R21) and
 * moves; an ion whose new cell lies beyond an open face is absorbed.  The
 * survivors are compacted in order; sp[s].n is updated.  kin as in
 * hvo_push_deposit (absorbed ions included: they were pushed). */
void hvo_push_deposit_open(const hvo_grid *g, hvo_species *sp, int64_t nsp, const double *Eext,
                           const double *Btx, double *n_acc, double *J_acc, double *kin) {
  xgrid x = xgrid_of(g);
  for (int a = 0; a < 4; ++a) kin[a] = 0.0;
  for (int64_t s = 0; s < nsp; ++s) {
    double qmdt = sp[s].q / sp[s].m * g->dt;
    int64_t kept = 0;
    for (int64_t p = 0; p < sp[s].n; ++p) {
      int64_t c[3];
      cdecode(g, sp[s].cell[p], &c[0], &c[1], &c[2]);
      double d[3] = {sp[s].ox[p], sp[s].oy[p], sp[s].oz[p]};
      double v[3] = {sp[s].vx[p], sp[s].vy[p], sp[s].vz[p]};
      double Ep[3], Bp[3];
      xgather(g, &x, Eext, 3, c, d, Ep);
      xgather(g, &x, Btx, 3, c, d, Bp);
      hvo_boris(qmdt, Ep, Bp, v);
      int64_t ch[3] = {c[0], c[1], c[2]};
      double dh[3] = {d[0], d[1], d[2]};
      move_raw(g, &x, ch, dh, v, 0.5);
      deposit_near(g, &x, ch, dh, v, sp[s].q * sp[s].w[p], n_acc, J_acc);
      move_raw(g, &x, c, d, v, 1.0);
      double mw = sp[s].m * sp[s].w[p];
      kin[0] += 0.5 * mw * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      kin[1] += mw * v[0];
      kin[2] += mw * v[1];
      kin[3] += mw * v[2];
      if (outside(&x, c)) continue; /* absorbed at an open face */
      sp[s].cell[kept] = c[0] + g->nx * (c[1] + g->ny * c[2]);
      sp[s].ox[kept] = d[0];
      sp[s].oy[kept] = d[1];
      sp[s].oz[kept] = d[2];
      sp[s].vx[kept] = v[0];
      sp[s].vy[kept] = v[1];
      sp[s].vz[kept] = v[2];
      sp[s].w[kept] = sp[s].w[p];
      ++kept;
    }
    sp[s].n = kept;
  }
}

/* Start-up with open faces (R8): deposit at x^0 (folded), E^0 on the
 * extended grid. */
void hvo_init_open(const hvo_grid *g, const hvo_species *sp, int64_t nsp, const double *B1,
                   double *Eext, double *n_prev, double *J_prev) {
  xgrid x = xgrid_of(g);
  int64_t nce = ncell_of(g);
  memset(n_prev, 0, sizeof(double) * nce);
  memset(J_prev, 0, sizeof(double) * 3 * nce);
  for (int64_t s = 0; s < nsp; ++s)
    for (int64_t p = 0; p < sp[s].n; ++p) {
      int64_t c[3];
      cdecode(g, sp[s].cell[p], &c[0], &c[1], &c[2]);
      double d[3] = {sp[s].ox[p], sp[s].oy[p], sp[s].oz[p]};
      double v[3] = {sp[s].vx[p], sp[s].vy[p], sp[s].vz[p]};
      deposit_near(g, &x, c, d, v, sp[s].q * sp[s].w[p], n_prev, J_prev);
    }
  hvo_ohm_open(g, B1, n_prev, J_prev, Eext);
}

/* One step with open faces, in the order of step_impl: push + half-step
 * deposit (absorbing), extrapolation (Eq. 11), subcycled advance of B1 with
 * the half-step moments, E^{n+1} on the extended grid from the extrapolated
 * moments.  Diagnostics: W_B of the total interior field, the deposited
 * charge, max |div B1| over interior cells (ghosts by the copy rule). */
void hvo_step_open(const hvo_grid *g, hvo_species *sp, int64_t nsp, double *B1, double *Eext,
                   double *n_prev, double *J_prev, double *n_ext, double *J_ext, hvo_diag *dg) {
  xgrid x = xgrid_of(g);
  int64_t nce = ncell_of(g), ne = xcount(&x);
  double *nh = (double *)calloc((size_t)nce, sizeof(double));
  double *Jh = (double *)calloc((size_t)(3 * nce), sizeof(double));
  double *ne_ = (double *)malloc(sizeof(double) * nce);
  double *Je = (double *)malloc(sizeof(double) * 3 * nce);
  double *Bt = (double *)malloc(sizeof(double) * 3 * nce);
  double *Btx = (double *)malloc(sizeof(double) * 3 * ne);
  double kin[4];
  for (int64_t c = 0; c < 3 * nce; ++c) Bt[c] = B1[c] + (g->B0 ? g->B0[c] : 0.0);
  xfill(g, &x, Bt, 3, Btx);
  hvo_push_deposit_open(g, sp, nsp, Eext, Btx, nh, Jh, kin);
  double charge_raw = 0.0, vc = g->dx * g->dy * g->dz;
  for (int64_t c = 0; c < nce; ++c) charge_raw += nh[c] * vc;
  hvo_extrapolate(nce, nh, n_prev, ne_);
  hvo_extrapolate(3 * nce, Jh, J_prev, Je);
  hvo_field_advance_open(g, B1, nh, Jh);
  hvo_ohm_open(g, B1, ne_, Je, Eext);
  memcpy(n_prev, nh, sizeof(double) * nce);
  memcpy(J_prev, Jh, sizeof(double) * 3 * nce);
  if (n_ext) memcpy(n_ext, ne_, sizeof(double) * nce);
  if (J_ext) memcpy(J_ext, Je, sizeof(double) * 3 * nce);
  if (dg) {
    double wb = 0.0, md = 0.0;
    double *B1x = (double *)malloc(sizeof(double) * 3 * ne);
    xfill(g, &x, B1, 3, B1x);
    for (int64_t q = 0; q < nce; ++q) {
      double bt2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double b = B1[a * nce + q] + (g->B0 ? g->B0[a * nce + q] : 0.0);
        bt2 += b * b;
      }
      wb += 0.5 * bt2 * vc;
      int64_t c[3];
      cdecode(g, q, &c[0], &c[1], &c[2]);
      double dv = xd(&x, B1x, 0, c) + xd(&x, B1x + ne, 1, c) + xd(&x, B1x + 2 * ne, 2, c);
      if (fabs(dv) > md) md = fabs(dv);
    }
    free(B1x);
    dg->W_K = kin[0];
    dg->P[0] = kin[1];
    dg->P[1] = kin[2];
    dg->P[2] = kin[3];
    dg->charge = charge_raw;
    dg->W_B = wb;
    dg->max_divB = md;
  }
  free(nh);
  free(Jh);
  free(ne_);
  free(Je);
  free(Bt);
  free(Btx);
}

/* ------------------------------------------------------------------------ */
/* Injection through open faces (Sec. 2.3: particles re-injected with the   */
/* flux of a drifting Maxwellian; reading R24).                             */
/*                                                                          */
/* Random numbers come from the counter-based generator Philox4x32-10       */
/* (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1,  */
/* 2, 3", SC 2011): 10 rounds of two 32x32 -> 64-bit products of the        */
/* counter words with fixed multipliers, the key added back each round and  */
/* bumped by two Weyl constants between rounds.  The GPU path implements    */
/* the same generator; both draw the same words for the same counter.       */
/* ------------------------------------------------------------------------ */

void hvo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  for (int a = 0; a < 4; ++a) out[a] = c[a];
}

/* a 32-bit word as a uniform in [0, 1) with 24 bits (exact in float) */
#define HVO_PI 3.14159265358979323846

static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

typedef struct {
  int64_t face;     /* 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z (must be an open axis) */
  double n;         /* density of the drifting Maxwellian */
  double u[3];      /* its flow */
  double T;         /* its temperature (thermal speed sqrt(T / m)) */
  double w;         /* weight of every injected ion */
} hvo_inject_face;

/* Expected injected ions per face cell and step, N = Gamma A dt / w, with
 * the one-sided flux Gamma = n [vt/sqrt(2 pi) exp(-U^2/2vt^2) +
 * U/2 (1 + erf(U/(sqrt2 vt)))] of the drifting Maxwellian (U the inward
 * flow), as a 40.24 fixed-point number (the count decision is integer
 * arithmetic on both sides). */
uint64_t hvo_inject_nfix(const hvo_grid *g, double m, const hvo_inject_face *f) {
  int ax = (int)(f->face / 2);
  double sgn = (f->face % 2 == 0) ? 1.0 : -1.0;
  double vt = sqrt(f->T / m), U = sgn * f->u[ax];
  double flux;
  if (vt > 0.0)
    flux = f->n * (vt / sqrt(2.0 * HVO_PI) * exp(-U * U / (2.0 * vt * vt)) +
                   0.5 * U * (1.0 + erf(U / (sqrt(2.0) * vt))));
  else
    flux = f->n * (U > 0.0 ? U : 0.0);
  double d[3] = {g->dx, g->dy, g->dz};
  double area = d[(ax + 1) % 3] * d[(ax + 2) % 3];
  double N = flux * area * g->dt / f->w;
  return (uint64_t)floor(N * 16777216.0 + 0.5);
}

/* Inverse of the flux-weighted CDF of the inward speed, in units of vt:
 * F(t) = g(t) / g(inf), g(t) = exp(-a^2/2) - exp(-(t-a)^2/2)
 *        + a sqrt(pi/2) [erf((t-a)/sqrt2) + erf(a/sqrt2)],  a = U / vt,
 * by 40 bisections of [0, max(a, 0) + 12]. */
static double flux_speed(double a, double u) {
  double ginf = exp(-0.5 * a * a) + a * sqrt(HVO_PI / 2.0) * (1.0 + erf(a / sqrt(2.0)));
  double lo = 0.0, hi = (a > 0.0 ? a : 0.0) + 12.0;
  for (int it = 0; it < 40; ++it) {
    double mid = 0.5 * (lo + hi);
    double gm = exp(-0.5 * a * a) - exp(-0.5 * (mid - a) * (mid - a)) +
                a * sqrt(HVO_PI / 2.0) * (erf((mid - a) / sqrt(2.0)) + erf(a / sqrt(2.0)));
    if (gm < u * ginf) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Ions injected through face f of species s_idx at step `step`: for every
 * face cell c (the tangential cell index, x before y before z), in order,
 * count = (nfix + (r >> 8)) >> 24 with r word 0 of Philox at counter
 * (step, c, 0xffffffff, tag), tag = s_idx << 8 | face << 4; ion k of the
 * cell takes words (u0..u3) at (step, c, k, tag) and (u4..u7) at
 * (step, c, k, tag | 1): inward speed from u0 (flux_speed), tangential
 * velocities by Box-Muller from u1, u2 (first tangential axis cos, second
 * sin), tangential offsets 2 u4 - 1, 2 u5 - 1 (axes with one cell: 0), depth
 * v_n dt u6 from the face (entered at a uniform time in the step).  An ion
 * whose depth reaches beyond the grid is not placed.  Returns the number of
 * ions; fills cell/off/v (cap entries at most) when cell != NULL. */
int64_t hvo_inject(const hvo_grid *g, int64_t s_idx, double m, const hvo_inject_face *f,
                   uint64_t seed, int64_t step, int64_t *cell, double *off, double *v,
                   int64_t cap) {
  int ax = (int)(f->face / 2), low = f->face % 2 == 0;
  int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2; /* tangential axes, ascending */
  int64_t n[3] = {g->nx, g->ny, g->nz};
  double d[3] = {g->dx, g->dy, g->dz};
  double vt = sqrt(f->T / m), sgn = low ? 1.0 : -1.0;
  double a = vt > 0.0 ? sgn * f->u[ax] / vt : 0.0;
  uint64_t nfix = hvo_inject_nfix(g, m, f);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t tag = ((uint32_t)s_idx << 8) | ((uint32_t)f->face << 4);
  int64_t count = 0;
  for (int64_t c = 0; c < n[t1] * n[t2]; ++c) {
    int64_t i1 = c % n[t1], i2 = c / n[t1];
    uint32_t ctr[4] = {(uint32_t)step, (uint32_t)c, 0xffffffffu, tag}, r[4];
    hvo_philox4x32_10(ctr, key, r);
    uint64_t k_n = (nfix + (uint64_t)(r[0] >> 8)) >> 24;
    for (uint64_t k = 0; k < k_n; ++k) {
      uint32_t ca[4] = {(uint32_t)step, (uint32_t)c, (uint32_t)k, tag}, ra[4];
      uint32_t cb[4] = {(uint32_t)step, (uint32_t)c, (uint32_t)k, tag | 1u}, rb[4];
      hvo_philox4x32_10(ca, key, ra);
      hvo_philox4x32_10(cb, key, rb);
      double vn = vt > 0.0 ? vt * flux_speed(a, u24(ra[0])) : sgn * f->u[ax];
      double rr = sqrt(-2.0 * log(1.0 - u24(ra[1]))), th = 2.0 * HVO_PI * u24(ra[2]);
      double depth = vn * g->dt * u24(rb[2]) / d[ax]; /* cells from the face */
      double xr = low ? depth : (double)n[ax] - depth;
      double fl = floor(xr);
      if (fl < 0.0 || fl >= (double)n[ax]) continue;
      if (cell && count < cap) {
        int64_t ci[3];
        double o[3], vv[3];
        ci[ax] = (int64_t)fl;
        o[ax] = 2.0 * (xr - fl) - 1.0;
        vv[ax] = sgn * vn;
        ci[t1] = i1;
        ci[t2] = i2;
        o[t1] = n[t1] > 1 ? 2.0 * u24(rb[0]) - 1.0 : 0.0;
        o[t2] = n[t2] > 1 ? 2.0 * u24(rb[1]) - 1.0 : 0.0;
        vv[t1] = f->u[t1] + vt * rr * cos(th);
        vv[t2] = f->u[t2] + vt * rr * sin(th);
        cell[count] = ci[0] + g->nx * (ci[1] + g->ny * ci[2]);
        for (int q = 0; q < 3; ++q) {
          off[q * cap + count] = o[q];
          v[q * cap + count] = vv[q];
        }
      }
      ++count;
    }
  }
  return count;
}

/* max |div B| over the interior cells, with the ghost copies of open faces
 * (the same rule as the open-face diagnostics) or periodic neighbours. */
double hvo_max_div(const hvo_grid *g, const double *B) {
  xgrid x = xgrid_of(g);
  int64_t nce = ncell_of(g), ne = xcount(&x);
  double *Bx = (double *)malloc(sizeof(double) * 3 * ne);
  xfill(g, &x, B, 3, Bx);
  double md = 0.0;
  for (int64_t q = 0; q < nce; ++q) {
    int64_t c[3];
    cdecode(g, q, &c[0], &c[1], &c[2]);
    double dv = xd(&x, Bx, 0, c) + xd(&x, Bx + ne, 1, c) + xd(&x, Bx + 2 * ne, 2, c);
    if (fabs(dv) > md) md = fabs(dv);
  }
  free(Bx);
  return md;
}

/* Number of cells of the extended grid (for the caller's Eext). */
int64_t hvo_xcount(const hvo_grid *g) {
  xgrid x = xgrid_of(g);
  return xcount(&x);
}

/* ------------------------------------------------------------------------ */
/* Learned moment filter (not in the paper: a residual convolutional filter */
/* of the deposited moments, with the paper's binomial smoothing (Sec. 2.2) */
/* as the fallback).  Written for the x-z layout (ny = 1).                  */
/*   x_c = m_c / s_c  (c = n, Jx, Jy, Jz)                                   */
/*   h1 = bf16(relu(conv3x3(bf16(x); W1, b1)))       4 -> 16 channels      */
/*   h2 = bf16(relu(conv3x3(h1; W2, b2)))            16 -> 16               */
/*   f  = conv3x3(h2; W3, b3)                        16 -> 4                */
/*   y_c = m_c + s_c f_c                                                   */
/* conv3x3 is a periodic cross-correlation: out[o](i,k) = b[o] +            */
/* sum_c sum_{a,b in -1..1} W[o][c][b+1][a+1] in[c](i+a, k+b).              */
/* Gate: a cell keeps the binomial-smoothed moments (one (1/4,1/2,1/4)      */
/* pass per axis of the raw deposit) where n < nmin or |s_n f_n| >          */
/* rmax * max(n, n_floor).  `round` = 0 disables the bf16 rounding (used    */
/* by the finite-difference gradient pins).                                 */
/* Parameter layout (floats): W1[16][4][3][3] b1[16] W2[16][16][3][3]       */
/* b2[16] W3[4][16][3][3] b3[4]  (3492 values).                             */
/* ------------------------------------------------------------------------ */

static double bf16_round(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan */
  uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7fffu + lsb) & 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static void conv3x3(const hvo_grid *g, const double *in, int cin, const double *W,
                    const double *b, int cout, double *out) {
  int64_t nx = g->nx, nz = g->nz, nc = nx * nz;
  for (int o = 0; o < cout; ++o)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i) {
        double s = b[o];
        for (int c = 0; c < cin; ++c)
          for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
              int64_t ii = wrapi(i + da, nx), kk = wrapi(k + db, nz);
              s += W[((o * cin + c) * 3 + (db + 1)) * 3 + (da + 1)] * in[c * nc + kk * nx + ii];
            }
        out[o * nc + k * nx + i] = s;
      }
}

/* Forward pass of the network on x [4][ncell]; writes f [4][ncell] and (if
 * non-NULL) the layer outputs h1, h2 [16][ncell]. */
void hvo_filter_net(const hvo_grid *g, const double *P, const double *x, int round_bf16,
                    double *f, double *h1o, double *h2o) {
  int64_t nc = g->nx * g->nz;
  const double *W1 = P, *b1 = W1 + 16 * 4 * 9, *W2 = b1 + 16, *b2 = W2 + 16 * 16 * 9;
  const double *W3 = b2 + 16, *b3 = W3 + 4 * 16 * 9;
  double *xb = (double *)malloc(sizeof(double) * 4 * nc);
  double *h1 = (double *)malloc(sizeof(double) * 16 * nc);
  double *h2 = (double *)malloc(sizeof(double) * 16 * nc);
  for (int64_t t = 0; t < 4 * nc; ++t) xb[t] = round_bf16 ? bf16_round(x[t]) : x[t];
  conv3x3(g, xb, 4, W1, b1, 16, h1);
  for (int64_t t = 0; t < 16 * nc; ++t) {
    double v = h1[t] > 0.0 ? h1[t] : 0.0;
    h1[t] = round_bf16 ? bf16_round(v) : v;
  }
  conv3x3(g, h1, 16, W2, b2, 16, h2);
  for (int64_t t = 0; t < 16 * nc; ++t) {
    double v = h2[t] > 0.0 ? h2[t] : 0.0;
    h2[t] = round_bf16 ? bf16_round(v) : v;
  }
  conv3x3(g, h2, 16, W3, b3, 4, f);
  if (h1o) memcpy(h1o, h1, sizeof(double) * 16 * nc);
  if (h2o) memcpy(h2o, h2, sizeof(double) * 16 * nc);
  free(xb);
  free(h1);
  free(h2);
}

/* The filter with its gate: m [4][ncell] (n, Jx, Jy, Jz) in, y [4][ncell]
 * out.  Parameters are used as given (the caller passes bf16 values when
 * emulating the device); s[4] are the channel scales. */
void hvo_filter_apply(const hvo_grid *g, const double *P, const double *s, double nmin,
                      double rmax, int round_bf16, const double *m, double *y) {
  int64_t nc = g->nx * g->nz;
  double *x = (double *)malloc(sizeof(double) * 4 * nc);
  double *f = (double *)malloc(sizeof(double) * 4 * nc);
  double *sm = (double *)malloc(sizeof(double) * 4 * nc);
  for (int c = 0; c < 4; ++c)
    for (int64_t t = 0; t < nc; ++t) x[c * nc + t] = m[c * nc + t] / s[c];
  hvo_filter_net(g, P, x, round_bf16, f, NULL, NULL);
  memcpy(sm, m, sizeof(double) * 4 * nc);
  hvo_smooth(g, sm, 4, 1);
  for (int64_t t = 0; t < nc; ++t) {
    double n = m[t];
    double r = fabs(s[0] * f[t]);
    double ref = n > g->n_floor ? n : g->n_floor;
    int fallback = (n < nmin) || (r > rmax * ref);
    for (int c = 0; c < 4; ++c)
      y[c * nc + t] = fallback ? sm[c * nc + t] : m[c * nc + t] + s[c] * f[c * nc + t];
  }
  free(x);
  free(f);
  free(sm);
}

/* Loss and gradient for one training pair (no gate): loss = mean over
 * cells and channels of ((x + f(x)) - t)^2 with x = m / s, t = target / s.
 * grad [3492] receives d loss / d P.  Backward in FP64 through the same
 * rounded activations as the forward (straight-through at the bf16
 * rounding points). */
double hvo_filter_loss_grad(const hvo_grid *g, const double *P, const double *s,
                            int round_bf16, const double *m, const double *target,
                            double *grad) {
  int64_t nx = g->nx, nz = g->nz, nc = nx * nz;
  const double *W2 = P + 16 * 4 * 9 + 16, *W3 = W2 + 16 * 16 * 9 + 16;
  double *x = (double *)malloc(sizeof(double) * 4 * nc);
  double *xb = (double *)malloc(sizeof(double) * 4 * nc);
  double *f = (double *)malloc(sizeof(double) * 4 * nc);
  double *h1 = (double *)malloc(sizeof(double) * 16 * nc);
  double *h2 = (double *)malloc(sizeof(double) * 16 * nc);
  double *df = (double *)malloc(sizeof(double) * 4 * nc);
  double *dh2 = (double *)calloc((size_t)(16 * nc), sizeof(double));
  double *dh1 = (double *)calloc((size_t)(16 * nc), sizeof(double));
  for (int c = 0; c < 4; ++c)
    for (int64_t t = 0; t < nc; ++t) x[c * nc + t] = m[c * nc + t] / s[c];
  for (int64_t t = 0; t < 4 * nc; ++t) xb[t] = round_bf16 ? bf16_round(x[t]) : x[t];
  hvo_filter_net(g, P, x, round_bf16, f, h1, h2);
  double loss = 0.0, norm = 1.0 / (double)(4 * nc);
  for (int c = 0; c < 4; ++c)
    for (int64_t t = 0; t < nc; ++t) {
      double e = x[c * nc + t] + f[c * nc + t] - target[c * nc + t] / s[c];
      loss += e * e * norm;
      df[c * nc + t] = 2.0 * e * norm;
    }
  for (int q = 0; q < 3492; ++q) grad[q] = 0.0;
  double *gW1 = grad, *gb1 = gW1 + 16 * 4 * 9, *gW2 = gb1 + 16, *gb2 = gW2 + 16 * 16 * 9;
  double *gW3 = gb2 + 16, *gb3 = gW3 + 4 * 16 * 9;
  /* layer 3: f = conv(h2; W3) + b3 */
  for (int o = 0; o < 4; ++o)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i) {
        double d = df[o * nc + k * nx + i];
        gb3[o] += d;
        for (int c = 0; c < 16; ++c)
          for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
              int64_t src = c * nc + wrapi(k + db, nz) * nx + wrapi(i + da, nx);
              int w = ((o * 16 + c) * 3 + (db + 1)) * 3 + (da + 1);
              gW3[w] += d * h2[src];
              dh2[src] += d * W3[w];
            }
      }
  for (int64_t t = 0; t < 16 * nc; ++t)
    if (h2[t] <= 0.0) dh2[t] = 0.0; /* relu' (h2 is post-relu) */
  /* layer 2: h2 = relu(conv(h1; W2) + b2) */
  for (int o = 0; o < 16; ++o)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i) {
        double d = dh2[o * nc + k * nx + i];
        gb2[o] += d;
        for (int c = 0; c < 16; ++c)
          for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
              int64_t src = c * nc + wrapi(k + db, nz) * nx + wrapi(i + da, nx);
              int w = ((o * 16 + c) * 3 + (db + 1)) * 3 + (da + 1);
              gW2[w] += d * h1[src];
              dh1[src] += d * W2[w];
            }
      }
  for (int64_t t = 0; t < 16 * nc; ++t)
    if (h1[t] <= 0.0) dh1[t] = 0.0;
  /* layer 1: h1 = relu(conv(xb; W1) + b1) */
  for (int o = 0; o < 16; ++o)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i) {
        double d = dh1[o * nc + k * nx + i];
        gb1[o] += d;
        for (int c = 0; c < 4; ++c)
          for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
              int64_t src = c * nc + wrapi(k + db, nz) * nx + wrapi(i + da, nx);
              gW1[((o * 4 + c) * 3 + (db + 1)) * 3 + (da + 1)] += d * xb[src];
            }
      }
  free(x);
  free(xb);
  free(f);
  free(h1);
  free(h2);
  free(df);
  free(dh2);
  free(dh1);
  return loss;
}
