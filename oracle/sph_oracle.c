/*
 * FP64 CPU oracle of the SPH fluid / rigid-body / heat method of arXiv:2103.07925
 * (Fuchs, Meier, Wall, Cyron).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the
 * smoke check and the timed CPU baseline, never by the product library.
 *
 * Plain double-precision loops, one function per step of the time integrator of
 * Sec. 3.7, compiled with -ffp-contract=off.  Neighbour lists are rebuilt every
 * step (brute force, or a plain bucket list over cells of edge >= r_c, Sec. 3.2)
 * and every list is sorted by particle index, so each sum runs in a fixed order.
 *
 * Readings taken where the paper is silent or ambiguous (each also listed in the
 * design notes of the repository):
 *  R1  kernel: quintic spline of Morris (1997), W = s_d [(3-q)^5 - 6(2-q)^5 + 15(1-q)^5]
 *      (terms dropped when negative), q = r/h, s_2 = 7/(478 pi h^2), s_3 = 1/(120 pi h^3),
 *      support r_c = 3h (Remark on the applied kernel, Sec. 3.1.1).
 *  R2  neighbour set N(a) = { b != a : r_ab^2 < r_c^2 }, r^2 = (dx*dx + dy*dy) + dz*dz,
 *      minimum image on periodic axes.  Cells: n_d = max(1, floor(L_d / (r_c + skin))),
 *      edge L_d / n_d, c_d = clamp(floor((x_d - lo_d) / edge_d), 0, n_d - 1).
 *  R3  density summation (Eq. densum) over fluid targets, self term W(0) included,
 *      neighbours of every kind contribute; rigid and wall particles keep the density
 *      they were given (constant).
 *  R4  boundary extrapolation after Adami et al. 2012 (cited in Sec. 3.3.4, not printed):
 *      p_w = [sum_f p_f W_wf + (g - a_w) . sum_f rho_f r_wf W_wf] / sum_f W_wf,
 *      v_w = 2 u_w - sum_f u_f W_wf / sum_f W_wf; no fluid neighbour: p_w = 0, v_w = u_w.
 *      u_w is the prescribed wall velocity or the rigid particle velocity; a_w = 0 for
 *      walls and a_k + alpha_k x r_rk + w_k x (w_k x r_rk) for rigid particles, with the
 *      body accelerations of the previous evaluation.
 *  R5  momentum (Eq. momentum) fluid-wall and fluid-rigid pairs: p_j = p_w, rho_j from the
 *      inverse equation of state of fluid i, rho_j = rho0_i (p_w / p0_i + 1), V_j = m_j/rho_j
 *      with the particle's own (constant) density, eta_j = eta_i, u_j = v_w.  The rigid
 *      particle receives f_ri = -m_i a_ir (Eq. couplingforce).  No pair term between
 *      particles of the same body; rigid-rigid (other body) and rigid-wall pairs give only
 *      the contact force (Eq. contactforce) with v_rr' = u_r - u_r'.
 *  R6  heat (Eq. heat_equation) for fluid and rigid targets; wall neighbours carry a
 *      prescribed temperature (Dirichlet, kappa_b := kappa_a) or, when it is NaN, do
 *      not take part (adiabatic).  V_b = m_b / rho_b.  T^{n+1} = T^n + dt dT/dt.
 *  R7  rigid-particle inertia I_r = 0.5 m_r r_eff^2 (2D) and 0.4 m_r r_eff^2 (3D): the
 *      remark prints r_eff without the square; only the square reproduces the disk
 *      inertia the paper plots as converging to 3.83495197e-9 (Sec. 4.1).
 *  R8  quaternions scalar-first (w,x,y,z), Hamilton product; the increment of
 *      phi = dt w^{n+1/2} is (cos|phi|/2, sin(|phi|/2) phi/|phi|), identity at phi = 0;
 *      the product is renormalised.  Angular acceleration alpha = I_k^{-1} m_k with the
 *      world inertia I_k = R I_body R^T and no gyroscopic term (Eq. angularmomentum).
 *  R9  initial accelerations come from one full evaluation at t = 0.
 *  R10 phase transitions are evaluated at the end of a step, for all particles at once
 *      against T^{n+1}: a rigid particle above T_t melts, a fluid particle below T_t
 *      solidifies (Sec. 3.6).  A solidifying particle joins the body of its nearest
 *      rigid (non-melting) neighbour (ties: smaller body id, then smaller index);
 *      solidifying particles without one form new bodies, one per connected component
 *      of the neighbour graph among themselves, numbered in order of their smallest
 *      index.  Changed bodies get new m_k, r_k, I_k (Sec. 3.4.2) and
 *      u_k = u'_k + w_k x (r_k - r'_k) (the printed r_rk - r'_rk differs only in sign
 *      convention: r_rk - r'_rk = r'_k - r_k would move the body against the shift of
 *      its centre).  Empty bodies retire.  New bodies: q = 1, u = mass-weighted mean
 *      velocity, w = 0.  A melting particle keeps its velocity and takes the rigid
 *      acceleration of R4 as its a^n.  Particle mass and density (hence volume) do not
 *      change at a transition; a solidified particle keeps its current density.
 *  R11 latent heat (Remark on latent heat; apparent capacity): for materials with L > 0
 *      the state is the specific enthalpy H with dH/dt = c_p dT/dt of Eq. heat_equation,
 *      and T(H) is piecewise linear: solid capacity below T_t - w/2, capacity
 *      c_s + L/w inside the interval of width w, liquid capacity above.  H = 0 at
 *      T_t - w/2.  L = 0 materials use the paper's T update.
 *  R12 optional surface heat source (not in the paper): q = Q0 exp(-2 |x_par - x_s(t)|^2
 *      / r_s^2) for particles with z_top - z < depth, per unit volume, added as q/rho to
 *      dH/dt of particles whose material takes part in a phase transition.
 *  R13 dt (Eq. timestepcond) is fixed when given, otherwise the minimum of the five
 *      conditions with |u|max over fluid particles at the start of the step.
 *  R14 wall particles with a prescribed velocity move with it (the moving boundary
 *      particles of the shear-flow examples, Sec. 4.2): x += dt u_w in the drift.
 *  R15 transport-velocity formulation (Sec. 3.3.2 applies it after Adami, Hu and Adams
 *      2013, without printing it), on when the background pressure p_b > 0: fluid
 *      particles are advected with u~ = u^{n+1/2} + dt/2 a~^n, where
 *      a~_i = -(p_b / m_i) sum_j (V_i^2 + V_j^2) dW/dr e_ij over neighbours of every kind;
 *      the momentum equation gains (1/m_i) sum_j (V_i^2 + V_j^2) 1/2 (A_i + A_j) . e_ij dW/dr
 *      with A = rho u (u~ - u) (an outer product; A = 0 for wall and rigid particles), which
 *      enters the coupling force on rigid particles like every other term of a_ir.
 *      A particle that melts starts with a~ = 0.  p_b = 0 gives the scheme without it.
 *      Pins: a~ = 0 on a regular lattice, exact momentum with the A term (antisymmetry),
 *      regularisation growing with p_b, Couette profile; the overall sign of the A term
 *      follows Adami et al. and is pinned only through these (parity partially unpinned).
 *  R16 concentration (the remark on chemically induced transitions): fluid and rigid
 *      particles carry C with dC_a/dt = (1/rho_a) sum_b V_b 4 D_a D_b / (D_a + D_b)
 *      (C_a - C_b) / r_ab dW/dr, the form of the heat equation of Sec. 3.5 with the
 *      diffusivity in place of kappa and no capacity; wall particles do not take part.  A
 *      phase with a fixed concentration (not NaN) keeps it at all times and acts as a
 *      reservoir.  A phase with transition_by = 1 changes phase when C crosses C_transition
 *      (rigid above, fluid below), evaluated with the temperature rule at the step's end.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static double* dalloc(int64_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static __thread char g_err[512];
static void set_err(const char* m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char* orc_error(void) { return g_err; }

struct orc_scene {
  orc_params P;
  double rc, rc2, dt_ref;
  int64_t n;
  double *x, *u, *a, *rho, *p, *T, *dT, *m, *H, *vext, *f, *rb, *wu, *wT;
  double *ab, *tv; /* R15: background acceleration a~ and u~ - u of the current half step */
  double *C, *dC;  /* R16: concentration and its rate */
  int tvf;
  int32_t *mat, *body;
  /* bodies */
  int32_t K, Kcap;
  double *bm, *br, *bq, *bu, *bw, *ba, *bal, *bf, *bt, *bIb, *bIw;
  int32_t* alive;
  /* neighbours (CSR, sorted) */
  int64_t* nstart;
  int32_t* nlist;
  int64_t ncap;
  int32_t ncell[3];
  double ell[3];
  double time, dt;
  int64_t step;
  double pairs_force;
  int enthalpy;
};

/* ------------------------------------------------------------------ kernel (R1) */

static double sigma_d(int dim, double h) {
  if (dim == 2) return 7.0 / (478.0 * M_PI * h * h);
  return 1.0 / (120.0 * M_PI * h * h * h);
}

double orc_kernel_w(int32_t dim, double r, double h) {
  double q = r / h;
  double w = 0.0;
  if (q < 3.0) w += pow(3.0 - q, 5);
  if (q < 2.0) w -= 6.0 * pow(2.0 - q, 5);
  if (q < 1.0) w += 15.0 * pow(1.0 - q, 5);
  return sigma_d(dim, h) * w;
}

double orc_kernel_dw(int32_t dim, double r, double h) {
  double q = r / h;
  double w = 0.0;
  if (q < 3.0) w -= 5.0 * pow(3.0 - q, 4);
  if (q < 2.0) w += 30.0 * pow(2.0 - q, 4);
  if (q < 1.0) w -= 75.0 * pow(1.0 - q, 4);
  return sigma_d(dim, h) * w / h;
}

/* ------------------------------------------------------------------ small vector helpers */

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_quat_mul(const double* a, const double* b, double* o) {
  /* Hamilton product a o b, scalar first (R8) */
  double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

void orc_quat_rot(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void matvec(const double* M, const double* v, double* o) {
  for (int i = 0; i < 3; i++) o[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
}
static void matTvec(const double* M, const double* v, double* o) {
  for (int i = 0; i < 3; i++) o[i] = M[i] * v[0] + M[3 + i] * v[1] + M[6 + i] * v[2];
}
static void inv3(const double* A, double* B) {
  double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  double id = 1.0 / det;
  B[0] = c00 * id; B[1] = (A[2] * A[7] - A[1] * A[8]) * id; B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  B[3] = c01 * id; B[4] = (A[0] * A[8] - A[2] * A[6]) * id; B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  B[6] = c02 * id; B[7] = (A[1] * A[6] - A[0] * A[7]) * id; B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}
/* world inertia R Ib R^T */
static void rot_inertia(const double* R, const double* Ib, double* Iw) {
  double T[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) T[3 * i + j] = R[3 * i] * Ib[j] + R[3 * i + 1] * Ib[3 + j] + R[3 * i + 2] * Ib[6 + j];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Iw[3 * i + j] = T[3 * i] * R[3 * j] + T[3 * i + 1] * R[3 * j + 1] + T[3 * i + 2] * R[3 * j + 2];
}
/* body inertia R^T Iw R */
static void unrot_inertia(const double* R, const double* Iw, double* Ib) {
  double T[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) T[3 * i + j] = R[i] * Iw[j] + R[3 + i] * Iw[3 + j] + R[6 + i] * Iw[6 + j];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Ib[3 * i + j] = T[3 * i] * R[j] + T[3 * i + 1] * R[3 + j] + T[3 * i + 2] * R[6 + j];
}

/* ------------------------------------------------------------------ geometry (R2) */

static double period(const orc_scene* s, int d) { return s->P.box_max[d] - s->P.box_min[d]; }

static void min_image(const orc_scene* s, const double* xi, const double* xj, double* d) {
  for (int k = 0; k < 3; k++) {
    d[k] = xi[k] - xj[k];
    if (k < s->P.dim && s->P.periodic[k]) {
      double L = period(s, k);
      if (d[k] > 0.5 * L) d[k] -= L;
      else if (d[k] < -0.5 * L) d[k] += L;
    }
  }
}

static double norm2(const orc_scene* s, const double* d) {
  if (s->P.dim == 2) return d[0] * d[0] + d[1] * d[1];
  return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

static void wrap(const orc_scene* s, double* x) {
  for (int k = 0; k < s->P.dim; k++)
    if (s->P.periodic[k]) {
      double L = period(s, k);
      if (x[k] >= s->P.box_max[k]) x[k] -= L;
      else if (x[k] < s->P.box_min[k]) x[k] += L;
    }
}

static void cell_of(const orc_scene* s, const double* x, int32_t* c) {
  for (int k = 0; k < 3; k++) {
    if (k >= s->P.dim) { c[k] = 0; continue; }
    double v = floor((x[k] - s->P.box_min[k]) / s->ell[k]);
    int32_t ci;
    if (v < 0.0) ci = 0;
    else if (v > (double)(s->ncell[k] - 1)) ci = s->ncell[k] - 1;
    else ci = (int32_t)v;
    c[k] = ci;
  }
}

static int is_kind(const orc_scene* s, int64_t i, int kind) { return s->P.materials[s->mat[i]].kind == kind; }
static const orc_material* M(const orc_scene* s, int64_t i) { return &s->P.materials[s->mat[i]]; }

/* ------------------------------------------------------------------ neighbour lists (R2) */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static int is_nb(const orc_scene* s, int64_t i, int64_t j) {
  if (i == j) return 0;
  double d[3];
  min_image(s, &s->x[3 * i], &s->x[3 * j], d);
  return norm2(s, d) < s->rc2;
}

static int build_neighbors(orc_scene* s) {
  int64_t n = s->n;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int brute = s->P.force_brute || n <= 2000;
  for (int k = 0; k < s->P.dim; k++)
    if (s->P.periodic[k] && s->ncell[k] < 3) brute = 1;
  int64_t nc = (int64_t)s->ncell[0] * s->ncell[1] * s->ncell[2];
  int64_t *cstart = NULL, *citems = NULL;
  int32_t* pc = NULL;
  if (!brute) {
    /* bucket list: particles of each cell in increasing index order */
    cstart = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    citems = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    pc = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
      cell_of(s, &s->x[3 * i], &pc[3 * i]);
      int64_t lin = pc[3 * i] + (int64_t)s->ncell[0] * (pc[3 * i + 1] + (int64_t)s->ncell[1] * pc[3 * i + 2]);
      cstart[lin + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) cstart[c + 1] += cstart[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    memcpy(fill, cstart, sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < n; i++) {
      int64_t lin = pc[3 * i] + (int64_t)s->ncell[0] * (pc[3 * i + 1] + (int64_t)s->ncell[1] * pc[3 * i + 2]);
      citems[fill[lin]++] = i;
    }
    free(fill);
  }
  for (int pass = 0; pass < 2; pass++) {
    if (pass == 1) {
      for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
      int64_t tot = cnt[n];
      if (tot > s->ncap) {
        free(s->nlist);
        s->ncap = tot + tot / 8 + 16;
        s->nlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->ncap);
        if (!s->nlist) { set_err("oracle: out of memory (neighbour list)"); return -2; }
      }
      memcpy(s->nstart, cnt, sizeof(int64_t) * ((size_t)n + 1));
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
      int64_t c = 0;
      int64_t out = pass ? s->nstart[i] : 0;
      if (brute) {
        for (int64_t j = 0; j < n; j++)
          if (is_nb(s, i, j)) {
            if (pass) s->nlist[out + c] = (int32_t)j;
            c++;
          }
      } else {
        int32_t ci[3] = {pc[3 * i], pc[3 * i + 1], pc[3 * i + 2]};
        int lo[3], hi[3];
        for (int k = 0; k < 3; k++) {
          lo[k] = (k < s->P.dim) ? -1 : 0;
          hi[k] = (k < s->P.dim) ? 1 : 0;
        }
        for (int oz = lo[2]; oz <= hi[2]; oz++)
          for (int oy = lo[1]; oy <= hi[1]; oy++)
            for (int ox = lo[0]; ox <= hi[0]; ox++) {
              int32_t cc[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz};
              int skip = 0;
              for (int k = 0; k < 3; k++) {
                if (cc[k] < 0 || cc[k] >= s->ncell[k]) {
                  if (k < s->P.dim && s->P.periodic[k]) cc[k] = (cc[k] + s->ncell[k]) % s->ncell[k];
                  else skip = 1;
                }
              }
              if (skip) continue;
              int64_t lin = cc[0] + (int64_t)s->ncell[0] * (cc[1] + (int64_t)s->ncell[1] * cc[2]);
              for (int64_t q = cstart[lin]; q < cstart[lin + 1]; q++) {
                int64_t j = citems[q];
                if (is_nb(s, i, j)) {
                  if (pass) s->nlist[out + c] = (int32_t)j;
                  c++;
                }
              }
            }
      }
      if (!pass) cnt[i + 1] = c;
      else qsort(&s->nlist[out], (size_t)c, sizeof(int32_t), cmp_i32);
    }
  }
  free(cnt);
  free(cstart);
  free(citems);
  free(pc);
  return 0;
}

/* ------------------------------------------------------------------ rigid-body mass quantities (Sec. 3.4.2) */

static double particle_inertia(int dim, double dx, double m) {
  /* R7: rigid particle as a disc / sphere of the lattice volume */
  if (dim == 2) {
    double reff = dx / sqrt(M_PI);
    return 0.5 * m * reff * reff;
  }
  double reff = cbrt(0.75 / M_PI) * dx;
  return 0.4 * m * reff * reff;
}

/* processor-wise mass, centre of mass and inertia of a set of particles (Eqs. procwise_*) */
static void mass_quantities(int dim, double dx, int64_t cnt, const double* pos, const double* mass,
                            double* m_out, double* c_out, double* I_out) {
  double mt = 0.0, c[3] = {0, 0, 0};
  for (int64_t r = 0; r < cnt; r++) {
    mt += mass[r];
    for (int k = 0; k < 3; k++) c[k] += mass[r] * pos[3 * r + k];
  }
  for (int k = 0; k < 3; k++) c[k] /= mt;
  double I[9] = {0};
  for (int64_t r = 0; r < cnt; r++) {
    double d[3] = {c[0] - pos[3 * r], c[1] - pos[3 * r + 1], c[2] - pos[3 * r + 2]};
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double Ir = particle_inertia(dim, dx, mass[r]);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) I[3 * i + j] += Ir * (i == j) + ((i == j) * d2 - d[i] * d[j]) * mass[r];
  }
  *m_out = mt;
  memcpy(c_out, c, sizeof c);
  memcpy(I_out, I, sizeof I);
}

/* two-level evaluation: chunks play the processors of Eqs. procwise_* and global_* */
void orc_body_mass_chunked(int32_t dim, double dx, int64_t n, const double* pos, const double* mass,
                           int64_t chunk, double* m_out, double* com_out, double* inertia_out) {
  int64_t np = (n + chunk - 1) / chunk;
  double* pm = (double*)malloc(sizeof(double) * (size_t)np);
  double* pr = (double*)malloc(sizeof(double) * 3 * (size_t)np);
  double* pI = (double*)malloc(sizeof(double) * 9 * (size_t)np);
  for (int64_t p = 0; p < np; p++) {
    int64_t s0 = p * chunk, cnt = (s0 + chunk <= n) ? chunk : n - s0;
    mass_quantities(dim, dx, cnt, pos + 3 * s0, mass + s0, &pm[p], &pr[3 * p], &pI[9 * p]);
  }
  double mt = 0.0, c[3] = {0, 0, 0};
  for (int64_t p = 0; p < np; p++) {
    mt += pm[p];
    for (int k = 0; k < 3; k++) c[k] += pm[p] * pr[3 * p + k];
  }
  for (int k = 0; k < 3; k++) c[k] /= mt;
  double I[9] = {0};
  for (int64_t p = 0; p < np; p++) {
    double d[3] = {c[0] - pr[3 * p], c[1] - pr[3 * p + 1], c[2] - pr[3 * p + 2]};
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) I[3 * i + j] += pI[9 * p + 3 * i + j] + ((i == j) * d2 - d[i] * d[j]) * pm[p];
  }
  *m_out = mt;
  memcpy(com_out, c, sizeof c);
  memcpy(inertia_out, I, sizeof I);
  free(pm); free(pr); free(pI);
}

/* members of every body: CSR over body ids, particles in increasing index order */
static void body_members(const orc_scene* s, int64_t** start, int64_t** items) {
  int64_t* st = (int64_t*)calloc((size_t)s->Kcap + 1, sizeof(int64_t));
  for (int64_t i = 0; i < s->n; i++)
    if (s->P.materials[s->mat[i]].kind == ORC_RIGID) st[s->body[i] + 1]++;
  for (int32_t k = 0; k < s->Kcap; k++) st[k + 1] += st[k];
  int64_t* it = (int64_t*)malloc(sizeof(int64_t) * (size_t)(st[s->Kcap] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->Kcap + 1));
  memcpy(fill, st, sizeof(int64_t) * (size_t)(s->Kcap + 1));
  for (int64_t i = 0; i < s->n; i++)
    if (s->P.materials[s->mat[i]].kind == ORC_RIGID) it[fill[s->body[i]]++] = i;
  free(fill);
  *start = st;
  *items = it;
}

/* (re)derive m_k, r_k, I_k of body k from its particles (serial case, Remark serial) and
 * the body-frame offsets r_rk of its particles under the current orientation. */
static void body_rebuild(orc_scene* s, int32_t k, const int64_t* idx, int64_t cnt) {
  if (cnt == 0) {
    s->alive[k] = 0;
    return;
  }
  double* pos = (double*)malloc(sizeof(double) * 3 * (size_t)cnt);
  double* mass = (double*)malloc(sizeof(double) * (size_t)cnt);
  int64_t first = idx[0];
  for (int64_t c = 0; c < cnt; c++) {
    int64_t i = idx[c];
    /* unwrap relative to the first particle (minimum image) */
    double d[3];
    min_image(s, &s->x[3 * i], &s->x[3 * first], d);
    for (int q = 0; q < 3; q++) pos[3 * c + q] = s->x[3 * first + q] + d[q];
    mass[c] = s->m[i];
  }
  mass_quantities(s->P.dim, s->P.dx, cnt, pos, mass, &s->bm[k], &s->br[3 * k], &s->bIw[9 * k]);
  double R[9];
  orc_quat_rot(&s->bq[4 * k], R);
  unrot_inertia(R, &s->bIw[9 * k], &s->bIb[9 * k]);
  for (int64_t r = 0; r < cnt; r++) {
    double d[3] = {pos[3 * r] - s->br[3 * k], pos[3 * r + 1] - s->br[3 * k + 1], pos[3 * r + 2] - s->br[3 * k + 2]};
    matTvec(R, d, &s->rb[3 * idx[r]]);
  }
  s->alive[k] = 1;
  free(pos); free(mass);
}

/* ------------------------------------------------------------------ enthalpy (R11) */

static double T_of_H(const orc_scene* s, int32_t mat, double H) {
  const orc_material* A = &s->P.materials[mat];
  const orc_material* S = A;
  const orc_material* Lq = A;
  if (A->transitions_to >= 0) {
    const orc_material* B = &s->P.materials[A->transitions_to];
    if (A->kind == ORC_RIGID) Lq = B; else S = B;
  }
  double w = A->mushy_width, Tlo = A->T_transition - 0.5 * w;
  double cs = S->cp, cl = Lq->cp, L = A->latent_heat;
  double Hhi = (cs + L / w) * w;
  if (H <= 0.0) return Tlo + H / cs;
  if (H <= Hhi) return Tlo + H / (cs + L / w);
  return Tlo + w + (H - Hhi) / cl;
}

static double H_of_T(const orc_scene* s, int32_t mat, double T) {
  const orc_material* A = &s->P.materials[mat];
  const orc_material* S = A;
  const orc_material* Lq = A;
  if (A->transitions_to >= 0) {
    const orc_material* B = &s->P.materials[A->transitions_to];
    if (A->kind == ORC_RIGID) Lq = B; else S = B;
  }
  double w = A->mushy_width, Tlo = A->T_transition - 0.5 * w;
  double cs = S->cp, cl = Lq->cp, L = A->latent_heat;
  double Hhi = (cs + L / w) * w;
  if (T <= Tlo) return cs * (T - Tlo);
  if (T <= Tlo + w) return (cs + L / w) * (T - Tlo);
  return Hhi + cl * (T - Tlo - w);
}

static int uses_enthalpy(const orc_scene* s, int32_t mat) { return s->P.materials[mat].latent_heat > 0.0; }

/* ------------------------------------------------------------------ evaluation of the rates */

static double wij(const orc_scene* s, double r) { return orc_kernel_w(s->P.dim, r, s->P.h); }
static double dwij(const orc_scene* s, double r) { return orc_kernel_dw(s->P.dim, r, s->P.h); }

/* Eq. densum + Eq. eos for every fluid particle (R3) */
static void density_eos(orc_scene* s) {
  double w0 = wij(s, 0.0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < s->n; i++) {
    if (!is_kind(s, i, ORC_FLUID)) continue;
    double sum = w0;
    for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
      int64_t j = s->nlist[q];
      double d[3];
      min_image(s, &s->x[3 * i], &s->x[3 * j], d);
      sum += wij(s, sqrt(norm2(s, d)));
    }
    s->rho[i] = s->m[i] * sum;
    const orc_material* A = M(s, i);
    s->p[i] = A->c * A->c * (s->rho[i] - A->rho0);
  }
}

/* relative position r_rk (world frame) of a rigid particle */
static void rigid_arm(const orc_scene* s, int64_t i, double* rr) {
  double R[9];
  int32_t k = s->body[i];
  orc_quat_rot(&s->bq[4 * k], R);
  matvec(R, &s->rb[3 * i], rr);
}

/* acceleration of the material point of rigid particle i in its body's motion:
 * a_k + alpha_k x r_rk + w_k x (w_k x r_rk), with the body accelerations of the last
 * evaluation (R4, R10) */
static void rigid_point_acc(const orc_scene* s, int64_t i, double* a) {
  int32_t b = s->body[i];
  double rr[3], t1[3], t2[3], t3[3];
  rigid_arm(s, i, rr);
  cross3(&s->bal[3 * b], rr, t1);
  cross3(&s->bw[3 * b], rr, t2);
  cross3(&s->bw[3 * b], t2, t3);
  for (int k = 0; k < 3; k++) a[k] = s->ba[3 * b + k] + t1[k] + t3[k];
}

/* boundary / rigid extrapolation (R4) */
static void extrapolate(orc_scene* s) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t w = 0; w < s->n; w++) {
    int kind = M(s, w)->kind;
    if (kind == ORC_FLUID) continue;
    double uw[3], aw[3] = {0, 0, 0};
    if (kind == ORC_WALL) {
      for (int k = 0; k < 3; k++) uw[k] = s->wu[3 * w + k];
    } else {
      rigid_point_acc(s, w, aw);
      for (int k = 0; k < 3; k++) uw[k] = s->u[3 * w + k];
    }
    double S = 0.0, P = 0.0, Rv[3] = {0, 0, 0}, U[3] = {0, 0, 0};
    for (int64_t q = s->nstart[w]; q < s->nstart[w + 1]; q++) {
      int64_t f = s->nlist[q];
      if (!is_kind(s, f, ORC_FLUID)) continue;
      double d[3];
      min_image(s, &s->x[3 * w], &s->x[3 * f], d); /* r_wf = r_w - r_f */
      double W = wij(s, sqrt(norm2(s, d)));
      S += W;
      P += s->p[f] * W;
      for (int k = 0; k < 3; k++) {
        Rv[k] += s->rho[f] * d[k] * W;
        U[k] += s->u[3 * f + k] * W;
      }
    }
    if (S > 0.0) {
      double ga = 0.0;
      for (int k = 0; k < 3; k++) ga += (s->P.gravity[k] - aw[k]) * Rv[k];
      s->p[w] = (P + ga) / S;
      for (int k = 0; k < 3; k++) s->vext[3 * w + k] = 2.0 * uw[k] - U[k] / S;
    } else {
      s->p[w] = 0.0;
      for (int k = 0; k < 3; k++) s->vext[3 * w + k] = uw[k];
    }
  }
}

/* temperature rate of fluid and rigid particles (Eq. heat_equation, R6, R11, R12) */
static void heat_rates(orc_scene* s, double t) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t a = 0; a < s->n; a++) {
    const orc_material* A = M(s, a);
    if (A->kind == ORC_WALL) { s->dT[a] = 0.0; continue; }
    double Ta = s->T[a], ka = A->kappa;
    double sum = 0.0;
    for (int64_t q = s->nstart[a]; q < s->nstart[a + 1]; q++) {
      int64_t b = s->nlist[q];
      const orc_material* B = M(s, b);
      double Tb, kb;
      if (B->kind == ORC_WALL) {
        if (isnan(s->wT[b])) continue;
        Tb = s->wT[b];
        kb = ka;
      } else {
        Tb = s->T[b];
        kb = B->kappa;
      }
      double kab = (ka + kb > 0.0) ? 4.0 * ka * kb / (ka + kb) : 0.0;
      double d[3];
      min_image(s, &s->x[3 * a], &s->x[3 * b], d);
      double r = sqrt(norm2(s, d));
      double Vb = s->m[b] / s->rho[b];
      sum += Vb * kab * (Ta - Tb) / r * dwij(s, r);
    }
    double rate = sum / s->rho[a]; /* = c_p dT/dt = dH/dt */
    if (s->P.src_power > 0.0 && A->transitions_to >= 0) {
      double xs[3];
      for (int k = 0; k < 3; k++) xs[k] = s->P.src_origin[k] + s->P.src_speed[k] * t;
      int vz = s->P.dim - 1;
      double dd = 0.0;
      for (int k = 0; k < s->P.dim; k++)
        if (k != vz) dd += (s->x[3 * a + k] - xs[k]) * (s->x[3 * a + k] - xs[k]);
      if (s->P.src_ztop - s->x[3 * a + vz] < s->P.src_depth) {
        double qv = s->P.src_power * exp(-2.0 * dd / (s->P.src_radius * s->P.src_radius));
        rate += qv / s->rho[a];
      }
    }
    s->dT[a] = uses_enthalpy(s, s->mat[a]) ? rate : rate / A->cp;
  }
}

/* R16: dC/dt of fluid and rigid particles (walls do not take part) */
static void conc_rates(orc_scene* s) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t a = 0; a < s->n; a++) {
    const orc_material* A = M(s, a);
    if (A->kind == ORC_WALL) { s->dC[a] = 0.0; continue; }
    double Ca = s->C[a], Da = A->diffusivity, sum = 0.0;
    for (int64_t q = s->nstart[a]; q < s->nstart[a + 1]; q++) {
      int64_t b = s->nlist[q];
      const orc_material* B = M(s, b);
      if (B->kind == ORC_WALL) continue;
      double Db = B->diffusivity;
      double Dab = (Da + Db > 0.0) ? 4.0 * Da * Db / (Da + Db) : 0.0;
      double d[3];
      min_image(s, &s->x[3 * a], &s->x[3 * b], d);
      double r = sqrt(norm2(s, d));
      double Vb = s->m[b] / s->rho[b];
      sum += Vb * Dab * (Ca - s->C[b]) / r * dwij(s, r);
    }
    s->dC[a] = sum / s->rho[a];
  }
}

/* one pair term (V_i^2 + V_j^2)[-p~ dW e + eta~ u_ij / r dW] seen from fluid particle i (R5) */
static void pair_term(const orc_scene* s, int64_t i, int64_t j, double* out) {
  const orc_material* A = M(s, i);
  const orc_material* B = M(s, j);
  double d[3];
  min_image(s, &s->x[3 * i], &s->x[3 * j], d);
  double r = sqrt(norm2(s, d));
  double e[3] = {d[0] / r, d[1] / r, d[2] / r};
  double dW = dwij(s, r);
  double rhoi = s->rho[i], pi = s->p[i], Vi = s->m[i] / rhoi, etai = A->eta;
  double rhoj, pj, Vj, etaj, uj[3];
  if (B->kind == ORC_FLUID) {
    rhoj = s->rho[j];
    pj = s->p[j];
    Vj = s->m[j] / rhoj;
    etaj = B->eta;
    for (int k = 0; k < 3; k++) uj[k] = s->u[3 * j + k];
  } else {
    pj = s->p[j];
    double p0i = A->rho0 * A->c * A->c;
    rhoj = A->rho0 * (pj / p0i + 1.0);
    Vj = s->m[j] / s->rho[j];
    etaj = etai;
    for (int k = 0; k < 3; k++) uj[k] = s->vext[3 * j + k];
  }
  double pt = (rhoj * pi + rhoi * pj) / (rhoi + rhoj);
  double et = (etai + etaj > 0.0) ? 2.0 * etai * etaj / (etai + etaj) : 0.0;
  double coef = (Vi * Vi + Vj * Vj) * dW;
  for (int k = 0; k < 3; k++) {
    double uij = s->u[3 * i + k] - uj[k];
    out[k] = coef * (-pt * e[k] + et * uij / r);
  }
  if (s->tvf) { /* R15: 1/2 (A_i + A_j) . e_ij, A = rho u (u~ - u); A_j = 0 for boundaries */
    double si = 0.0, sj = 0.0;
    for (int k = 0; k < 3; k++) si += s->tv[3 * i + k] * e[k];
    if (B->kind == ORC_FLUID)
      for (int k = 0; k < 3; k++) sj += s->tv[3 * j + k] * e[k];
    for (int k = 0; k < 3; k++) {
      double Ae = rhoi * s->u[3 * i + k] * si + (B->kind == ORC_FLUID ? s->rho[j] * s->u[3 * j + k] * sj : 0.0);
      out[k] += coef * 0.5 * Ae;
    }
  }
}

/* R15: -(p_b / m_i) sum_j (V_i^2 + V_j^2) dW/dr e_ij for fluid particle i, all neighbours */
static void background_acc(orc_scene* s, int64_t i, double* out) {
  double sum[3] = {0, 0, 0};
  double Vi = s->m[i] / s->rho[i];
  for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
    int64_t j = s->nlist[q];
    double d[3];
    min_image(s, &s->x[3 * i], &s->x[3 * j], d);
    double r = sqrt(norm2(s, d));
    double Vj = s->m[j] / s->rho[j];
    double c = (Vi * Vi + Vj * Vj) * dwij(s, r) / r;
    for (int k = 0; k < 3; k++) sum[k] += c * d[k];
  }
  for (int k = 0; k < 3; k++) out[k] = -s->P.p_background / s->m[i] * sum[k];
}

/* Eq. contactforce for the rigid particle r against particle j (rigid of another body or wall) */
static void contact_force(const orc_scene* s, int64_t r, int64_t j, double* out) {
  double d[3];
  min_image(s, &s->x[3 * r], &s->x[3 * j], d);
  double dist = sqrt(norm2(s, d));
  out[0] = out[1] = out[2] = 0.0;
  if (!(dist < s->P.dx)) return;
  double e[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  double uj[3];
  for (int k = 0; k < 3; k++) uj[k] = is_kind(s, j, ORC_WALL) ? s->wu[3 * j + k] : s->u[3 * j + k];
  double ev = 0.0;
  for (int k = 0; k < 3; k++) ev += e[k] * (s->u[3 * r + k] - uj[k]);
  double fn = s->P.k_contact * (dist - s->P.dx) + s->P.d_contact * ev;
  double mn = fn < 0.0 ? fn : 0.0;
  for (int k = 0; k < 3; k++) out[k] = -mn * e[k];
}

/* accelerations of fluid particles and forces on rigid particles (Eqs. momentum,
 * couplingforce, rigidparticle_force) */
static void forces(orc_scene* s) {
  double pairs = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : pairs)
  for (int64_t i = 0; i < s->n; i++) {
    const orc_material* A = M(s, i);
    if (A->kind == ORC_WALL) continue;
    pairs += (double)(s->nstart[i + 1] - s->nstart[i]);
    double acc[3] = {0, 0, 0}, t[3];
    if (A->kind == ORC_FLUID) {
      for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
        pair_term(s, i, s->nlist[q], t);
        for (int k = 0; k < 3; k++) acc[k] += t[k];
      }
      for (int k = 0; k < 3; k++) {
        s->a[3 * i + k] = s->P.gravity[k] + acc[k] / s->m[i];
        s->f[3 * i + k] = 0.0;
      }
      if (s->tvf) background_acc(s, i, &s->ab[3 * i]);
    } else {
      for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
        int64_t j = s->nlist[q];
        const orc_material* B = M(s, j);
        if (B->kind == ORC_FLUID) {
          pair_term(s, j, i, t); /* m_j a_ji, seen from the fluid particle */
          for (int k = 0; k < 3; k++) acc[k] -= t[k];
        } else if (B->kind == ORC_WALL || s->body[j] != s->body[i]) {
          contact_force(s, i, j, t);
          for (int k = 0; k < 3; k++) acc[k] += t[k];
        }
      }
      for (int k = 0; k < 3; k++) {
        s->f[3 * i + k] = acc[k];
        s->a[3 * i + k] = 0.0;
      }
    }
  }
  s->pairs_force = pairs;
}

/* resultant force and torque on each body (Eq. procwise_force, serial case) and the body
 * accelerations (Eqs. linearmomentum, angularmomentum).  One pass over the particles in
 * index order accumulates every body. */
static void body_accelerations(orc_scene* s) {
  int32_t K = s->K;
  double* F = dalloc(3 * (int64_t)K);
  double* Tq = dalloc(3 * (int64_t)K);
  double* R = dalloc(9 * (int64_t)K);
  for (int32_t k = 0; k < K; k++) orc_quat_rot(&s->bq[4 * k], &R[9 * k]);
  for (int64_t i = 0; i < s->n; i++) {
    if (!is_kind(s, i, ORC_RIGID)) continue;
    int32_t k = s->body[i];
    double rr[3], c[3];
    matvec(&R[9 * k], &s->rb[3 * i], rr);
    cross3(rr, &s->f[3 * i], c);
    for (int q = 0; q < 3; q++) {
      F[3 * k + q] += s->f[3 * i + q];
      Tq[3 * k + q] += c[q];
    }
  }
  for (int32_t k = 0; k < K; k++) {
    if (!s->alive[k]) continue;
    double Ibinv[9], t1[3], t2[3];
    const double* Rk = &R[9 * k];
    inv3(&s->bIb[9 * k], Ibinv);
    matTvec(Rk, &Tq[3 * k], t1);
    matvec(Ibinv, t1, t2);
    matvec(Rk, t2, &s->bal[3 * k]);
    for (int q = 0; q < 3; q++) {
      s->bf[3 * k + q] = F[3 * k + q] + s->bm[k] * s->P.gravity[q];
      s->bt[3 * k + q] = Tq[3 * k + q];
      s->ba[3 * k + q] = s->bf[3 * k + q] / s->bm[k];
    }
    if (s->P.dim == 2) {
      s->bal[3 * k] = 0.0;
      s->bal[3 * k + 1] = 0.0;
    }
    rot_inertia(Rk, &s->bIb[9 * k], &s->bIw[9 * k]);
  }
  free(F); free(Tq); free(R);
}

static int evaluate(orc_scene* s, double t) {
  int rc = build_neighbors(s);
  if (rc) return rc;
  density_eos(s);
  extrapolate(s);
  heat_rates(s, t);
  conc_rates(s);
  forces(s);
  body_accelerations(s);
  return 0;
}

/* ------------------------------------------------------------------ time step (Sec. 3.7) */

static double time_step(const orc_scene* s) {
  if (s->P.dt_mode == 0) return s->P.dt_fixed;
  double h = s->P.h, umax = 0.0, cmax = 0.0, numax = 0.0, gmag = 0.0, mr = INFINITY, cond = INFINITY;
  for (int64_t i = 0; i < s->n; i++) {
    if (is_kind(s, i, ORC_FLUID)) {
      const double* u = &s->u[3 * i];
      double v = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      if (v > umax) umax = v;
    } else if (is_kind(s, i, ORC_RIGID)) {
      if (s->m[i] < mr) mr = s->m[i];
    }
  }
  for (int q = 0; q < s->P.n_materials; q++) {
    const orc_material* A = &s->P.materials[q];
    if (A->kind == ORC_FLUID) {
      if (A->c > cmax) cmax = A->c;
      if (A->eta / A->rho0 > numax) numax = A->eta / A->rho0;
    }
    if (A->kind != ORC_WALL && A->kappa > 0.0) {
      double c5 = 0.1 * A->rho0 * A->cp * h * h / A->kappa;
      if (c5 < cond) cond = c5;
    }
  }
  for (int k = 0; k < 3; k++) gmag += s->P.gravity[k] * s->P.gravity[k];
  gmag = sqrt(gmag);
  double dt = INFINITY;
  if (cmax + umax > 0.0) dt = fmin(dt, 0.25 * h / (cmax + umax));
  if (numax > 0.0) dt = fmin(dt, 0.125 * h * h / numax);
  if (gmag > 0.0) dt = fmin(dt, 0.25 * sqrt(h / gmag));
  if (mr < INFINITY && s->P.k_contact > 0.0) dt = fmin(dt, 0.22 * sqrt(mr / s->P.k_contact));
  dt = fmin(dt, cond);
  if (!(dt < INFINITY)) dt = s->P.dt_fixed;
  return dt;
}

static void rigid_kinematics(orc_scene* s) {
  for (int64_t i = 0; i < s->n; i++) {
    if (!is_kind(s, i, ORC_RIGID)) continue;
    int32_t k = s->body[i];
    double rr[3], c[3];
    rigid_arm(s, i, rr);
    cross3(&s->bw[3 * k], rr, c);
    for (int q = 0; q < 3; q++) {
      s->x[3 * i + q] = s->br[3 * k + q] + rr[q];
      s->u[3 * i + q] = s->bu[3 * k + q] + c[q];
    }
    wrap(s, &s->x[3 * i]);
  }
}

static void rigid_velocities(orc_scene* s) {
  for (int64_t i = 0; i < s->n; i++) {
    if (!is_kind(s, i, ORC_RIGID)) continue;
    int32_t k = s->body[i];
    double rr[3], c[3];
    rigid_arm(s, i, rr);
    cross3(&s->bw[3 * k], rr, c);
    for (int q = 0; q < 3; q++) s->u[3 * i + q] = s->bu[3 * k + q] + c[q];
  }
}

/* ------------------------------------------------------------------ phase transitions (Sec. 3.6, R10) */

static int64_t uf_find(int64_t* par, int64_t x) {
  while (par[x] != x) x = par[x];
  return x;
}

static int relabel(orc_scene* s) {
  int64_t n = s->n;
  int8_t* flag = (int8_t*)calloc((size_t)n, 1); /* 1 melt, 2 solidify */
  int64_t nflag = 0;
  for (int64_t i = 0; i < n; i++) {
    const orc_material* A = M(s, i);
    if (A->transitions_to < 0) continue;
    double Ti = uses_enthalpy(s, s->mat[i]) ? T_of_H(s, s->mat[i], s->H[i]) : s->T[i];
    double v = A->transition_by == 1 ? s->C[i] : Ti;              /* R16 */
    double vt = A->transition_by == 1 ? A->C_transition : A->T_transition;
    if (A->kind == ORC_RIGID && v > vt) { flag[i] = 1; nflag++; }
    else if (A->kind == ORC_FLUID && v < vt) { flag[i] = 2; nflag++; }
  }
  if (!nflag) { free(flag); return 0; }
  int8_t* changed = (int8_t*)calloc((size_t)s->Kcap, 1);
  double* old_com = (double*)malloc(sizeof(double) * 3 * (size_t)s->Kcap);
  memcpy(old_com, s->br, sizeof(double) * 3 * (size_t)s->K);
  int32_t* join = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  /* solidifying particles pick the nearest rigid neighbour that does not melt */
  for (int64_t i = 0; i < n; i++) {
    join[i] = -1;
    if (flag[i] != 2) continue;
    double best = INFINITY;
    int32_t bk = -1;
    int64_t bj = -1;
    for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
      int64_t j = s->nlist[q];
      if (!is_kind(s, j, ORC_RIGID) || flag[j] == 1) continue;
      double d[3];
      min_image(s, &s->x[3 * i], &s->x[3 * j], d);
      double r2 = norm2(s, d);
      int32_t kj = s->body[j];
      if (r2 < best || (r2 == best && (kj < bk || (kj == bk && j < bj)))) {
        best = r2; bk = kj; bj = j;
      }
    }
    join[i] = bk;
  }
  /* melting particles: rigid -> fluid, keep velocity, take the rigid acceleration */
  for (int64_t i = 0; i < n; i++) {
    if (flag[i] != 1) continue;
    int32_t k = s->body[i];
    rigid_point_acc(s, i, &s->a[3 * i]);
    for (int q = 0; q < 3; q++) {
      s->ab[3 * i + q] = 0.0; /* R15 */
      s->tv[3 * i + q] = 0.0;
    }
    changed[k] = 1;
    s->mat[i] = M(s, i)->transitions_to;
    s->body[i] = -1;
  }
  /* new bodies: connected components of solidifying particles without a rigid neighbour */
  int64_t* par = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) par[i] = i;
  for (int64_t i = 0; i < n; i++) {
    if (flag[i] != 2 || join[i] >= 0) continue;
    for (int64_t q = s->nstart[i]; q < s->nstart[i + 1]; q++) {
      int64_t j = s->nlist[q];
      if (flag[j] != 2 || join[j] >= 0) continue;
      int64_t a = uf_find(par, i), b = uf_find(par, j);
      if (a != b) { if (a < b) par[b] = a; else par[a] = b; }
    }
  }
  int64_t* newid = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) newid[i] = -1;
  int rc = 0;
  for (int64_t i = 0; i < n; i++) {
    if (flag[i] != 2 || join[i] >= 0) continue;
    int64_t root = uf_find(par, i); /* the smallest index of the component */
    if (newid[root] < 0) {
      if (s->K >= s->Kcap) { set_err("oracle: body capacity exceeded"); rc = -6; break; }
      int32_t k = s->K++;
      newid[root] = k;
      s->alive[k] = 1;
      double q0[4] = {1, 0, 0, 0};
      memcpy(&s->bq[4 * k], q0, sizeof q0);
      for (int q = 0; q < 3; q++) {
        s->bu[3 * k + q] = s->bw[3 * k + q] = s->ba[3 * k + q] = s->bal[3 * k + q] = 0.0;
        s->bf[3 * k + q] = s->bt[3 * k + q] = 0.0;
      }
      changed[k] = 2;
    }
    join[i] = (int32_t)newid[root];
  }
  if (rc == 0) {
    /* new bodies start with the mass-weighted mean velocity of their particles */
    double* mom = (double*)calloc(4 * (size_t)s->Kcap, sizeof(double));
    for (int64_t i = 0; i < n; i++) {
      if (flag[i] != 2) continue;
      int32_t k = join[i];
      if (changed[k] == 2) {
        for (int q = 0; q < 3; q++) mom[4 * k + q] += s->m[i] * s->u[3 * i + q];
        mom[4 * k + 3] += s->m[i];
      }
      const orc_material* A = M(s, i);
      int32_t to = A->transitions_to;
      s->mat[i] = to;
      s->body[i] = k;
      for (int q = 0; q < 3; q++) s->a[3 * i + q] = 0.0;
      if (changed[k] == 0) changed[k] = 1;
    }
    for (int32_t k = 0; k < s->K; k++)
      if (changed[k] == 2)
        for (int q = 0; q < 3; q++) s->bu[3 * k + q] = mom[4 * k + q] / mom[4 * k + 3];
    free(mom);
    /* rebuild the mass quantities of changed bodies, then correct their velocity */
    int64_t *bst, *bit;
    body_members(s, &bst, &bit);
    for (int32_t k = 0; k < s->K; k++) {
      if (!changed[k]) continue;
      body_rebuild(s, k, &bit[bst[k]], bst[k + 1] - bst[k]);
      if (!s->alive[k] || changed[k] == 2) continue;
      double dr[3] = {s->br[3 * k] - old_com[3 * k], s->br[3 * k + 1] - old_com[3 * k + 1],
                      s->br[3 * k + 2] - old_com[3 * k + 2]};
      double c[3];
      cross3(&s->bw[3 * k], dr, c);
      for (int q = 0; q < 3; q++) s->bu[3 * k + q] += c[q];
    }
    free(bst);
    free(bit);
    rigid_velocities(s);
  }
  free(flag); free(changed); free(old_com); free(join); free(par); free(newid);
  return rc;
}

/* ------------------------------------------------------------------ public API */

orc_scene* orc_create(const orc_params* P, int64_t n, const double* pos, const double* vel,
                      const double* mass, const double* density, const double* temperature,
                      const int32_t* material, const int32_t* body, const double* wall_velocity,
                      const double* wall_temperature, int32_t k, const double* quat,
                      const double* bvel, const double* bomega, const double* concentration) {
  if (P->dim != 2 && P->dim != 3) { set_err("oracle: dim must be 2 or 3"); return NULL; }
  if (P->n_materials < 1 || P->n_materials > ORC_MAXMAT) { set_err("oracle: bad material count"); return NULL; }
  for (int q = 0; q < P->n_materials; q++) {
    const orc_material* A = &P->materials[q];
    if (A->kind == ORC_FLUID && !(A->c > 0.0 && A->rho0 > 0.0)) { set_err("oracle: fluid needs c > 0, rho0 > 0"); return NULL; }
    if (A->latent_heat > 0.0 && !(A->mushy_width > 0.0)) { set_err("oracle: latent heat needs a mushy width"); return NULL; }
  }
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  s->P = *P;
  s->rc = P->kernel_support * P->h;
  s->rc2 = s->rc * s->rc;
  s->n = n;
  for (int d = 0; d < 3; d++) {
    if (d < P->dim) {
      double L = P->box_max[d] - P->box_min[d];
      int32_t nc = (int32_t)floor(L / (s->rc + (P->skin > 0.0 ? P->skin : 0.0)));
      if (nc < 1) nc = 1;
      s->ncell[d] = nc;
      s->ell[d] = L / nc;
    } else {
      s->ncell[d] = 1;
      s->ell[d] = 1.0;
    }
  }
  s->x = dalloc(3 * n); s->u = dalloc(3 * n); s->a = dalloc(3 * n); s->rho = dalloc(n);
  s->p = dalloc(n); s->T = dalloc(n); s->dT = dalloc(n); s->m = dalloc(n); s->H = dalloc(n);
  s->vext = dalloc(3 * n); s->f = dalloc(3 * n); s->rb = dalloc(3 * n); s->wu = dalloc(3 * n);
  s->wT = dalloc(n);
  s->ab = dalloc(3 * n); s->tv = dalloc(3 * n);
  s->C = dalloc(n); s->dC = dalloc(n);
  if (concentration) memcpy(s->C, concentration, sizeof(double) * (size_t)n);
  s->tvf = P->p_background > 0.0;
  s->mat = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->body = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->nstart = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  memcpy(s->x, pos, sizeof(double) * 3 * (size_t)n);
  memcpy(s->u, vel, sizeof(double) * 3 * (size_t)n);
  memcpy(s->m, mass, sizeof(double) * (size_t)n);
  memcpy(s->rho, density, sizeof(double) * (size_t)n);
  memcpy(s->T, temperature, sizeof(double) * (size_t)n);
  memcpy(s->mat, material, sizeof(int32_t) * (size_t)n);
  memcpy(s->body, body, sizeof(int32_t) * (size_t)n);
  if (wall_velocity) memcpy(s->wu, wall_velocity, sizeof(double) * 3 * (size_t)n);
  if (wall_temperature) memcpy(s->wT, wall_temperature, sizeof(double) * (size_t)n);
  else for (int64_t i = 0; i < n; i++) s->wT[i] = NAN;
  for (int64_t i = 0; i < n; i++) {
    if (material[i] < 0 || material[i] >= P->n_materials) { set_err("oracle: bad material"); orc_destroy(s); return NULL; }
    if (M(s, i)->kind == ORC_RIGID && (body[i] < 0 || body[i] >= k)) { set_err("oracle: bad body id"); orc_destroy(s); return NULL; }
    if (M(s, i)->kind != ORC_RIGID) s->body[i] = -1;
    wrap(s, &s->x[3 * i]);
    if (uses_enthalpy(s, s->mat[i])) s->H[i] = H_of_T(s, s->mat[i], s->T[i]);
    if (M(s, i)->kind == ORC_WALL) s->C[i] = 0.0;
    else if (!isnan(M(s, i)->C_fixed)) s->C[i] = M(s, i)->C_fixed;
  }
  /* bodies */
  s->K = k;
  s->Kcap = P->body_capacity > k ? P->body_capacity : k + 1024;
  int32_t kc = s->Kcap;
  s->bm = dalloc(kc); s->br = dalloc(3 * kc); s->bq = dalloc(4 * kc); s->bu = dalloc(3 * kc);
  s->bw = dalloc(3 * kc); s->ba = dalloc(3 * kc); s->bal = dalloc(3 * kc); s->bf = dalloc(3 * kc);
  s->bt = dalloc(3 * kc); s->bIb = dalloc(9 * kc); s->bIw = dalloc(9 * kc);
  s->alive = (int32_t*)calloc((size_t)kc, sizeof(int32_t));
  int64_t *bst, *bit;
  body_members(s, &bst, &bit);
  for (int32_t b = 0; b < k; b++) {
    double qn = sqrt(quat[4 * b] * quat[4 * b] + quat[4 * b + 1] * quat[4 * b + 1] +
                     quat[4 * b + 2] * quat[4 * b + 2] + quat[4 * b + 3] * quat[4 * b + 3]);
    for (int q = 0; q < 4; q++) s->bq[4 * b + q] = quat[4 * b + q] / qn;
    for (int q = 0; q < 3; q++) {
      s->bu[3 * b + q] = bvel[3 * b + q];
      s->bw[3 * b + q] = bomega[3 * b + q];
    }
    body_rebuild(s, b, &bit[bst[b]], bst[b + 1] - bst[b]);
  }
  free(bst);
  free(bit);
  /* contact constants (defaults when not given): k_c = m_r (0.22 / dt_ref)^2 with
   * dt_ref = 0.25 h / c_max, so that the contact condition of Eq. timestepcond equals the
   * CFL condition; d_c = 0.2 sqrt(k_c m_r / 2) */
  double cmax = 0.0, mr = INFINITY;
  for (int q = 0; q < P->n_materials; q++)
    if (P->materials[q].kind == ORC_FLUID && P->materials[q].c > cmax) cmax = P->materials[q].c;
  for (int64_t i = 0; i < n; i++)
    if (M(s, i)->kind == ORC_RIGID && s->m[i] < mr) mr = s->m[i];
  s->dt_ref = cmax > 0.0 ? 0.25 * P->h / cmax : P->dt_fixed;
  if (!(mr < INFINITY)) mr = 0.0;
  if (s->P.k_contact <= 0.0) s->P.k_contact = mr * (0.22 / s->dt_ref) * (0.22 / s->dt_ref);
  if (s->P.d_contact < 0.0) s->P.d_contact = 0.2 * sqrt(s->P.k_contact * mr * 0.5);
  /* rigid particle positions and velocities follow their bodies */
  rigid_velocities(s);
  /* R9: accelerations at t = 0 */
  int rc = evaluate(s, 0.0);
  if (rc) { orc_destroy(s); return NULL; }
  return s;
}

static int step_once(orc_scene* s) {
  int64_t n = s->n;
  double dt = time_step(s);
  double half = 0.5 * dt;
  s->dt = dt;
  /* kick and drift of fluid particles; wall particles move with their prescribed
   * velocity (R14) */
  for (int64_t i = 0; i < n; i++) {
    if (is_kind(s, i, ORC_WALL)) {
      const double* w = &s->wu[3 * i];
      if (w[0] == 0.0 && w[1] == 0.0 && w[2] == 0.0) continue;
      for (int q = 0; q < 3; q++) s->x[3 * i + q] = s->x[3 * i + q] + dt * w[q];
      wrap(s, &s->x[3 * i]);
      continue;
    }
    if (!is_kind(s, i, ORC_FLUID)) continue;
    for (int q = 0; q < 3; q++) {
      s->u[3 * i + q] = s->u[3 * i + q] + half * s->a[3 * i + q];
      if (s->tvf) { /* R15: advection with u~ = u^{n+1/2} + dt/2 a~^n */
        s->tv[3 * i + q] = half * s->ab[3 * i + q];
        s->x[3 * i + q] = s->x[3 * i + q] + dt * (s->u[3 * i + q] + s->tv[3 * i + q]);
      } else {
        s->x[3 * i + q] = s->x[3 * i + q] + dt * s->u[3 * i + q];
      }
    }
    wrap(s, &s->x[3 * i]);
  }
  /* kick and drift of rigid bodies, orientation update by the transition quaternion */
  for (int32_t k = 0; k < s->K; k++) {
    if (!s->alive[k]) continue;
    double phi[3];
    for (int q = 0; q < 3; q++) {
      s->bu[3 * k + q] = s->bu[3 * k + q] + half * s->ba[3 * k + q];
      s->bw[3 * k + q] = s->bw[3 * k + q] + half * s->bal[3 * k + q];
      s->br[3 * k + q] = s->br[3 * k + q] + dt * s->bu[3 * k + q];
      phi[q] = dt * s->bw[3 * k + q];
    }
    double ang = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double qi[4] = {1, 0, 0, 0}, qn[4];
    if (ang > 0.0) {
      double sh = sin(0.5 * ang) / ang;
      qi[0] = cos(0.5 * ang); qi[1] = sh * phi[0]; qi[2] = sh * phi[1]; qi[3] = sh * phi[2];
    }
    orc_quat_mul(qi, &s->bq[4 * k], qn);
    double nq = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int q = 0; q < 4; q++) s->bq[4 * k + q] = qn[q] / nq;
  }
  rigid_kinematics(s);
  int rc = evaluate(s, s->time + dt);
  if (rc) return rc;
  /* temperature (or enthalpy) update */
  for (int64_t i = 0; i < n; i++) {
    if (is_kind(s, i, ORC_WALL)) continue;
    if (uses_enthalpy(s, s->mat[i])) {
      s->H[i] = s->H[i] + dt * s->dT[i];
      s->T[i] = T_of_H(s, s->mat[i], s->H[i]);
    } else {
      s->T[i] = s->T[i] + dt * s->dT[i];
    }
  }
  /* concentration update (R16): reservoirs keep their value */
  for (int64_t i = 0; i < n; i++) {
    if (is_kind(s, i, ORC_WALL)) continue;
    s->C[i] = isnan(M(s, i)->C_fixed) ? s->C[i] + dt * s->dC[i] : M(s, i)->C_fixed;
  }
  /* final kick */
  for (int64_t i = 0; i < n; i++) {
    if (!is_kind(s, i, ORC_FLUID)) continue;
    for (int q = 0; q < 3; q++) s->u[3 * i + q] = s->u[3 * i + q] + half * s->a[3 * i + q];
  }
  for (int32_t k = 0; k < s->K; k++) {
    if (!s->alive[k]) continue;
    for (int q = 0; q < 3; q++) {
      s->bu[3 * k + q] = s->bu[3 * k + q] + half * s->ba[3 * k + q];
      s->bw[3 * k + q] = s->bw[3 * k + q] + half * s->bal[3 * k + q];
    }
  }
  rigid_velocities(s);
  rc = relabel(s);
  s->time += dt;
  s->step++;
  return rc;
}

int orc_step(orc_scene* s, int32_t nsteps) {
  for (int32_t i = 0; i < nsteps; i++) {
    int rc = step_once(s);
    if (rc) return rc;
  }
  return 0;
}

int64_t orc_n(orc_scene* s) { return s->n; }
int32_t orc_nbodies(orc_scene* s) { return s->K; }

void orc_get(orc_scene* s, int32_t field, void* out) {
  int64_t n = s->n;
  double* d = (double*)out;
  int32_t* o = (int32_t*)out;
  switch (field) {
    case ORC_F_POS: memcpy(d, s->x, sizeof(double) * 3 * (size_t)n); break;
    case ORC_F_VEL: /* walls report their prescribed velocity */
      for (int64_t i = 0; i < n; i++)
        for (int q = 0; q < 3; q++) d[3 * i + q] = is_kind(s, i, ORC_WALL) ? s->wu[3 * i + q] : s->u[3 * i + q];
      break;
    case ORC_F_ACC: memcpy(d, s->a, sizeof(double) * 3 * (size_t)n); break;
    case ORC_F_RHO: memcpy(d, s->rho, sizeof(double) * (size_t)n); break;
    case ORC_F_PRES: memcpy(d, s->p, sizeof(double) * (size_t)n); break;
    case ORC_F_TEMP: /* walls report their prescribed temperature (NaN: adiabatic) */
      for (int64_t i = 0; i < n; i++) d[i] = is_kind(s, i, ORC_WALL) ? s->wT[i] : s->T[i];
      break;
    case ORC_F_DTEMP: memcpy(d, s->dT, sizeof(double) * (size_t)n); break;
    case ORC_F_MAT: memcpy(o, s->mat, sizeof(int32_t) * (size_t)n); break;
    case ORC_F_BODY: memcpy(o, s->body, sizeof(int32_t) * (size_t)n); break;
    case ORC_F_FORCE: /* f_r of particles that are rigid now */
      for (int64_t i = 0; i < n; i++)
        for (int q = 0; q < 3; q++) d[3 * i + q] = is_kind(s, i, ORC_RIGID) ? s->f[3 * i + q] : 0.0;
      break;
    case ORC_F_VEXT: /* extrapolated velocity of particles that are wall or rigid now */
      for (int64_t i = 0; i < n; i++)
        for (int q = 0; q < 3; q++) d[3 * i + q] = is_kind(s, i, ORC_FLUID) ? 0.0 : s->vext[3 * i + q];
      break;
    case ORC_F_ENTH: memcpy(d, s->H, sizeof(double) * (size_t)n); break;
    case ORC_F_CONC: memcpy(d, s->C, sizeof(double) * (size_t)n); break;
    case ORC_F_DCONC: memcpy(d, s->dC, sizeof(double) * (size_t)n); break;
    case ORC_F_BACC: /* R15: background acceleration a~ of fluid particles */
      for (int64_t i = 0; i < n; i++)
        for (int q = 0; q < 3; q++) d[3 * i + q] = is_kind(s, i, ORC_FLUID) ? s->ab[3 * i + q] : 0.0;
      break;
    case ORC_F_CELL:
      for (int64_t i = 0; i < n; i++) {
        int32_t c[3];
        cell_of(s, &s->x[3 * i], c);
        o[i] = c[0] + s->ncell[0] * (c[1] + s->ncell[1] * c[2]);
      }
      break;
    default: break;
  }
}

void orc_get_bodies(orc_scene* s, double* com, double* quat, double* vel, double* omega,
                    double* mass, double* inertia, double* force, double* torque, int32_t* alive) {
  for (int32_t k = 0; k < s->K; k++) {
    for (int q = 0; q < 3; q++) {
      if (com) com[3 * k + q] = s->br[3 * k + q];
      if (vel) vel[3 * k + q] = s->bu[3 * k + q];
      if (omega) omega[3 * k + q] = s->bw[3 * k + q];
      if (force) force[3 * k + q] = s->bf[3 * k + q];
      if (torque) torque[3 * k + q] = s->bt[3 * k + q];
    }
    for (int q = 0; q < 4; q++)
      if (quat) quat[4 * k + q] = s->bq[4 * k + q];
    for (int q = 0; q < 9; q++)
      if (inertia) inertia[9 * k + q] = s->bIw[9 * k + q];
    if (mass) mass[k] = s->bm[k];
    if (alive) alive[k] = s->alive[k];
  }
}

int64_t orc_neighbors(orc_scene* s, int64_t* counts, int32_t* list, int64_t cap) {
  if (build_neighbors(s)) return -1;
  int64_t tot = s->nstart[s->n];
  for (int64_t i = 0; i < s->n; i++) counts[i] = s->nstart[i + 1] - s->nstart[i];
  if (list && cap >= tot) memcpy(list, s->nlist, sizeof(int32_t) * (size_t)tot);
  return tot;
}

void orc_diagnostics(orc_scene* s, double out[16]) {
  memset(out, 0, sizeof(double) * 16);
  double nf = 0, nr = 0, nb = 0;
  for (int64_t i = 0; i < s->n; i++) {
    const orc_material* A = M(s, i);
    if (A->kind == ORC_WALL) continue;
    double mi = s->m[i];
    if (A->kind == ORC_FLUID) {
      const double* u = &s->u[3 * i];
      const double* x = &s->x[3 * i];
      double c[3], mu[3] = {mi * u[0], mi * u[1], mi * u[2]};
      cross3(x, mu, c);
      for (int q = 0; q < 3; q++) { out[q] += mu[q]; out[3 + q] += c[q]; }
      out[6] += 0.5 * mi * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      nf++;
    } else {
      nr++;
    }
    out[7] += uses_enthalpy(s, s->mat[i]) ? mi * s->H[i] : mi * A->cp * s->T[i];
    out[8] += mi;
  }
  for (int32_t k = 0; k < s->K; k++) {
    if (!s->alive[k]) continue;
    nb++;
    double mk = s->bm[k];
    const double* u = &s->bu[3 * k];
    const double* w = &s->bw[3 * k];
    double mu[3] = {mk * u[0], mk * u[1], mk * u[2]}, c[3], Iw[3];
    cross3(&s->br[3 * k], mu, c);
    matvec(&s->bIw[9 * k], w, Iw);
    for (int q = 0; q < 3; q++) { out[q] += mu[q]; out[3 + q] += c[q] + Iw[q]; }
    out[6] += 0.5 * mk * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + 0.5 * (w[0] * Iw[0] + w[1] * Iw[1] + w[2] * Iw[2]);
  }
  out[9] = s->time;
  out[10] = (double)s->step;
  out[11] = s->dt;
  out[12] = nf;
  out[13] = nr;
  out[14] = nb;
  out[15] = s->pairs_force;
}

/* ------------------------------------------------------------------ post-processing (Eq. postprocessing) */

int orc_interpolate(orc_scene* s, int64_t nq, const double* query, int32_t field, uint32_t material_mask,
                    double* out) {
  int comps = field == ORC_F_VEL ? 3 : 1;
  if (field != ORC_F_VEL && field != ORC_F_RHO && field != ORC_F_PRES && field != ORC_F_TEMP &&
      field != ORC_F_CONC)
    return -1;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < nq; q++) {
    double xq[3] = {query[3 * q], query[3 * q + 1], s->P.dim == 3 ? query[3 * q + 2] : 0.0};
    wrap(s, xq);
    double num[3] = {0, 0, 0}, den = 0.0;
    for (int64_t j = 0; j < s->n; j++) {
      if (!((material_mask >> s->mat[j]) & 1u)) continue;
      double d[3];
      min_image(s, xq, &s->x[3 * j], d);
      double r2 = norm2(s, d);
      if (!(r2 < s->rc2)) continue;
      double w = wij(s, sqrt(r2)) * s->m[j] / s->rho[j];
      den += w;
      double f[3] = {0, 0, 0};
      switch (field) {
        case ORC_F_VEL:
          for (int k = 0; k < 3; k++) f[k] = is_kind(s, j, ORC_WALL) ? s->wu[3 * j + k] : s->u[3 * j + k];
          break;
        case ORC_F_RHO: f[0] = s->rho[j]; break;
        case ORC_F_PRES: f[0] = s->p[j]; break;
        case ORC_F_TEMP: f[0] = is_kind(s, j, ORC_WALL) ? s->wT[j] : s->T[j]; break;
        default: f[0] = s->C[j]; break;
      }
      for (int k = 0; k < comps; k++) num[k] += w * f[k];
    }
    for (int k = 0; k < comps; k++) out[comps * q + k] = den > 0.0 ? num[k] / den : NAN;
  }
  return 0;
}

void orc_destroy(orc_scene* s) {
  if (!s) return;
  double* arrs[] = {s->x, s->u, s->a, s->rho, s->p, s->T, s->dT, s->m, s->H, s->vext, s->f, s->rb,
                    s->wu, s->wT, s->bm, s->br, s->bq, s->bu, s->bw, s->ba, s->bal, s->bf, s->bt,
                    s->bIb, s->bIw, s->ab, s->tv, s->C, s->dC};
  for (size_t q = 0; q < sizeof arrs / sizeof arrs[0]; q++) free(arrs[q]);
  free(s->mat); free(s->body); free(s->alive); free(s->nstart); free(s->nlist);
  free(s);
}
