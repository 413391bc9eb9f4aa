// Import / export, diagnostics and the neighbour-set export of libsph.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_kernels.cuh"

namespace sph {

struct ImportArgs {
  const double *pos, *vel, *mass, *dens, *temp, *wvel, *wtemp;
  const int *mat, *body, *slot;
  const double* conc;  // nullable: zero
};

// specific enthalpy of the apparent-capacity extension (H = 0 at T_t - w/2)
__device__ __forceinline__ double enthalpy_of(const MatD* mats, int mt, double T) {
  const MatD& M = mats[mt];
  int so = mt, li = mt;
  if (M.to >= 0) {
    so = M.kind == KRIGID ? mt : M.to;
    li = M.kind == KRIGID ? M.to : mt;
  }
  double cs = mats[so].cp, cl = mats[li].cp, w = M.w, Tlo = M.Tt - 0.5 * w;
  double Hh = (cs + M.L / w) * w;
  if (T <= Tlo) return cs * (T - Tlo);
  if (T <= Tlo + w) return (cs + M.L / w) * (T - Tlo);
  return Hh + cl * (T - Tlo - w);
}

// input (original order, FP64) -> bank P of the scene, unsorted; the forced rebin that
// follows orders the particles by cell
template <class R>
__global__ void k_import(Scene<R>* const* sc, ImportArgs a) {
  const Scene<R>& S = **sc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
    int mt = a.mat[i];
    int kind = S.mat[mt].kind;
    double x[3] = {a.pos[3 * i], a.pos[3 * i + 1], S.dim == 3 ? a.pos[3 * i + 2] : 0.0};
    for (int k = 0; k < S.dim; k++)
      if (S.per[k]) {
        if (x[k] >= S.hi[k]) x[k] -= S.L[k];
        else if (x[k] < S.lo[k]) x[k] += S.L[k];
      }
    int c[3] = {0, 0, 0};
    for (int k = 0; k < S.dim; k++) {
      double v = floor(__ddiv_rn(__dsub_rn(x[k], S.lo[k]), S.ell[k]));
      c[k] = clamp_cell(v, S.ncell[k]);
    }
    int lin = c[0] + S.ncell[0] * (c[1] + S.ncell[1] * c[2]);
    S.key[i] = part_key(S, kind, lin);
    if (sizeof(R) == 8) {
      S.P.px[i] = (R)x[0]; S.P.py[i] = (R)x[1]; S.P.pz[i] = (R)x[2];
    } else {
      S.P.px[i] = (R)(x[0] - (S.lo[0] + c[0] * S.ell[0]));
      S.P.py[i] = (R)(x[1] - (S.lo[1] + c[1] * S.ell[1]));
      S.P.pz[i] = S.dim == 3 ? (R)(x[2] - (S.lo[2] + c[2] * S.ell[2])) : R(0);
    }
    double v[3] = {0, 0, 0};
    if (kind == KFLUID) { v[0] = a.vel[3 * i]; v[1] = a.vel[3 * i + 1]; v[2] = a.vel[3 * i + 2]; }
    else if (kind == KWALL && a.wvel) { v[0] = a.wvel[3 * i]; v[1] = a.wvel[3 * i + 1]; v[2] = a.wvel[3 * i + 2]; }
    S.P.vx[i] = (R)v[0]; S.P.vy[i] = (R)v[1]; S.P.vz[i] = (R)v[2];
    S.P.ax[i] = R(0); S.P.ay[i] = R(0); S.P.az[i] = R(0);
    double T = kind == KWALL ? (a.wtemp ? a.wtemp[i] : (double)NAN) : a.temp[i];
    S.P.T[i] = (R)T;
    S.P.H[i] = (kind != KWALL && S.mat[mt].enth) ? (R)enthalpy_of(S.mat, mt, T) : R(0);
    S.P.m[i] = (R)a.mass[i];
    S.P.rho[i] = (R)a.dens[i];
    S.P.mt[i] = mt;
    if (S.any_conc) {  // walls carry none; reservoir phases start at their fixed value
      double c = a.conc ? a.conc[i] : 0.0;
      if (kind == KWALL) c = 0.0;
      else if (!isnan(S.mat[mt].Cfix)) c = S.mat[mt].Cfix;
      S.P.C[i] = (R)c;
    }
    S.P.body[i] = kind == KRIGID ? a.body[i] : -1;
    S.P.slot[i] = a.slot[i];
    S.P.orig[i] = i;
    S.where[i] = i;
    S.prs[i] = R(0);
    S.dT[i] = R(0);
    S.vex[i] = R(0); S.vey[i] = R(0); S.vez[i] = R(0);
    if (a.slot[i] >= 0) S.slot_part[a.slot[i]] = i;
  }
}

// overwrite position / velocity / temperature of fluid particles (input order)
template <class R>
__global__ void k_import_fluid(Scene<R>* const* sc, const double* pos, const double* vel, const double* temp) {
  const Scene<R>& S = **sc;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < S.n; o += gridDim.x * blockDim.x) {
    int i = S.where[o];
    int mt = S.P.mt[i];
    if (S.mat[mt].kind != KFLUID) continue;
    if (pos) {
      double x[3] = {pos[3 * o], pos[3 * o + 1], S.dim == 3 ? pos[3 * o + 2] : 0.0};
      for (int k = 0; k < S.dim; k++)
        if (S.per[k]) {
          if (x[k] >= S.hi[k]) x[k] -= S.L[k];
          else if (x[k] < S.lo[k]) x[k] += S.L[k];
        }
      if (sizeof(R) == 8) {
        S.P.px[i] = (R)x[0]; S.P.py[i] = (R)x[1]; S.P.pz[i] = (R)x[2];
      } else {
        // offset from the origin of the particle's current cell (minimum image), as the
        // drift leaves it: the lists and the displacement since their build stay in one
        // frame, and the next rebin moves the particle to its new cell
        int c[3] = {0, 0, 0};
        lin_xyz(S, key_lin(S, S.key[i]), c[0], c[1], c[2]);
        double o[3] = {0.0, 0.0, 0.0};
        bool far = false;
        for (int k = 0; k < S.dim; k++) {
          o[k] = x[k] - (S.lo[k] + c[k] * S.ell[k]);
          if (S.per[k]) {
            if (o[k] > 0.5 * S.L[k]) o[k] -= S.L[k];
            else if (o[k] < -0.5 * S.L[k]) o[k] += S.L[k];
          }
          far |= fabs(o[k]) > 64.0 * S.ell[k];
        }
        if (far) {  // a jump across the box: new cell, and the lists are rebuilt next step
          for (int k = 0; k < S.dim; k++) {
            double v = floor((x[k] - S.lo[k]) / S.ell[k]);
            c[k] = clamp_cell(v, S.ncell[k]);
            o[k] = x[k] - (S.lo[k] + c[k] * S.ell[k]);
          }
          S.key[i] = part_key(S, S.matR[S.P.mt[i]].kind, c[0] + S.ncell[0] * (c[1] + S.ncell[1] * c[2]));
          S.status[10] = 1;
        }
        S.P.px[i] = (R)o[0];
        S.P.py[i] = (R)o[1];
        S.P.pz[i] = (R)o[2];
      }
    }
    if (vel) { S.P.vx[i] = (R)vel[3 * o]; S.P.vy[i] = (R)vel[3 * o + 1]; S.P.vz[i] = (R)vel[3 * o + 2]; }
    if (temp) {
      S.P.T[i] = (R)temp[o];
      if (S.mat[mt].enth) S.P.H[i] = (R)enthalpy_of(S.mat, mt, temp[o]);
    }
  }
}

struct ExportArgs {
  double* f[SPH_F_COUNT];  // double fields (null: not requested)
  int* fi[SPH_F_COUNT];    // int fields
  int original;
};

template <class R>
__global__ void k_export(Scene<R>* const* sc, ExportArgs a) {
  const Scene<R>& S = **sc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
    int o = a.original ? S.P.orig[i] : i;
    int mt = S.P.mt[i];
    int kind = S.mat[mt].kind;
    if (a.f[SPH_F_POS]) {
      double x[3];
      abs_pos<R>(S, i, x);
      for (int q = 0; q < 3; q++) a.f[SPH_F_POS][3 * o + q] = x[q];
    }
    if (a.f[SPH_F_VEL]) {
      a.f[SPH_F_VEL][3 * o] = S.P.vx[i]; a.f[SPH_F_VEL][3 * o + 1] = S.P.vy[i]; a.f[SPH_F_VEL][3 * o + 2] = S.P.vz[i];
    }
    if (a.f[SPH_F_ACC]) {
      bool fl = kind == KFLUID;
      a.f[SPH_F_ACC][3 * o] = fl ? (double)S.P.ax[i] : 0.0;
      a.f[SPH_F_ACC][3 * o + 1] = fl ? (double)S.P.ay[i] : 0.0;
      a.f[SPH_F_ACC][3 * o + 2] = fl ? (double)S.P.az[i] : 0.0;
    }
    if (a.f[SPH_F_RHO]) a.f[SPH_F_RHO][o] = S.P.rho[i];
    if (a.f[SPH_F_PRES]) a.f[SPH_F_PRES][o] = S.prs[i];
    if (a.f[SPH_F_TEMP]) a.f[SPH_F_TEMP][o] = S.P.T[i];
    if (a.f[SPH_F_DTEMP]) a.f[SPH_F_DTEMP][o] = kind == KWALL ? 0.0 : (double)S.dT[i];
    if (a.fi[SPH_F_MAT]) a.fi[SPH_F_MAT][o] = mt;
    if (a.fi[SPH_F_BODY]) a.fi[SPH_F_BODY][o] = S.P.body[i];
    if (a.f[SPH_F_FORCE]) {
      int sl = S.P.slot[i];
      bool rg = kind == KRIGID && sl >= 0;
      for (int q = 0; q < 3; q++) a.f[SPH_F_FORCE][3 * o + q] = rg ? (double)S.fr[3 * sl + q] : 0.0;
    }
    if (a.f[SPH_F_VEXT]) {
      bool b = kind != KFLUID;
      a.f[SPH_F_VEXT][3 * o] = b ? (double)S.vex[i] : 0.0;
      a.f[SPH_F_VEXT][3 * o + 1] = b ? (double)S.vey[i] : 0.0;
      a.f[SPH_F_VEXT][3 * o + 2] = b ? (double)S.vez[i] : 0.0;
    }
    if (a.fi[SPH_F_CELL]) a.fi[SPH_F_CELL][o] = key_lin(S, S.key[i]);
    if (a.f[SPH_F_ENTH]) a.f[SPH_F_ENTH][o] = S.P.H[i];
    if (a.f[SPH_F_CONC]) a.f[SPH_F_CONC][o] = S.any_conc ? (double)S.P.C[i] : 0.0;
    if (a.f[SPH_F_DCONC]) a.f[SPH_F_DCONC][o] = (S.any_conc && kind != KWALL) ? (double)S.dC[i] : 0.0;
    if (a.f[SPH_F_BACC]) {
      bool b = S.tvf && kind == KFLUID;
      a.f[SPH_F_BACC][3 * o] = b ? (double)S.P.bx[i] : 0.0;
      a.f[SPH_F_BACC][3 * o + 1] = b ? (double)S.P.by[i] : 0.0;
      a.f[SPH_F_BACC][3 * o + 2] = b ? (double)S.P.bz[i] : 0.0;
    }
  }
}

// ------------------------------------------------------------------ FP64 diagnostics
// deterministic two-pass reduction: block partials in a fixed order, then one block
constexpr int NDIAG = 11;
template <class R>
__global__ void __launch_bounds__(256) k_diag_part(Scene<R>* const* sc, double* part) {
  const Scene<R>& S = **sc;
  __shared__ double red[NDIAG][256];
  double v[NDIAG];
  for (int q = 0; q < NDIAG; q++) v[q] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
    int mt = S.P.mt[i];
    const MatD& A = S.mat[mt];
    if (A.kind == KWALL) continue;
    double m = (double)S.P.m[i];
    if (A.kind == KFLUID) {
      double u[3] = {(double)S.P.vx[i], (double)S.P.vy[i], (double)S.P.vz[i]};
      double x[3], mu[3] = {m * u[0], m * u[1], m * u[2]}, c[3];
      abs_pos<R>(S, i, x);
      cross(x, mu, c);
      for (int q = 0; q < 3; q++) { v[q] += mu[q]; v[3 + q] += c[q]; }
      v[6] += 0.5 * m * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      v[9] += 1.0;
    } else {
      v[10] += 1.0;
    }
    v[7] += A.enth ? m * (double)S.P.H[i] : m * A.cp * (double)S.P.T[i];
    v[8] += m;
  }
  for (int q = 0; q < NDIAG; q++) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < NDIAG; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < NDIAG; q++) part[NDIAG * blockIdx.x + q] = red[q][0];
}

template <class R>
__global__ void k_diag_fin(Scene<R>* const* sc, const double* part, int nblk, double* out) {
  const Scene<R>& S = **sc;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double v[NDIAG];
  for (int q = 0; q < NDIAG; q++) v[q] = 0.0;
  for (int b = 0; b < nblk; b++)
    for (int q = 0; q < NDIAG; q++) v[q] += part[NDIAG * b + q];
  double nb = 0;
  for (int k = 0; k < *S.K; k++) {
    if (!S.balive[k]) continue;
    nb += 1.0;
    double mk = S.bm[k];
    const double* u = &S.bu[3 * k];
    const double* w = &S.bw[3 * k];
    double mu[3] = {mk * u[0], mk * u[1], mk * u[2]}, c[3], Iw[3];
    cross(&S.br[3 * k], mu, c);
    mv(&S.bIw[9 * k], w, Iw);
    for (int q = 0; q < 3; q++) { v[q] += mu[q]; v[3 + q] += c[q] + Iw[q]; }
    v[6] += 0.5 * mk * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + 0.5 * (w[0] * Iw[0] + w[1] * Iw[1] + w[2] * Iw[2]);
  }
  for (int q = 0; q < 9; q++) out[q] = v[q];
  out[9] = S.st[1];
  out[10] = S.st[2];
  out[11] = S.st[3];
  out[12] = v[9];
  out[13] = v[10];
  out[14] = nb;
  out[15] = (double)S.pairs[0];
}

// ------------------------------------------------------------------ neighbour-set export
template <class R, int DIM>
struct NbPol {
  R *sx, *sy, *sz;
  float4* s4;
  int* sox;
  float *fx, *fy, *fz;
  float tf[3];
  int* so;
  unsigned cmask;
  int cox, cdy, cdz;
  bool active;
  int idx;
  R tp[3];
  int64_t cnt, off;
  int32_t* list;
  static constexpr bool kExact = true;
  static constexpr bool kEntry = false;
  __device__ void stage(const Scene<R>& S, int j, int lane) {
    sx[lane] = S.P.px[j]; sy[lane] = S.P.py[j]; sz[lane] = S.P.pz[j];
    if (sizeof(R) == 8) { fx[lane] = (float)sx[lane]; fy[lane] = (float)sy[lane]; fz[lane] = (float)sz[lane]; }
    so[lane] = S.P.orig[j];
  }
  __device__ void pair(const Scene<R>&, int k, int, R, R, R, R) {
    if (list) list[off + cnt] = so[k];
    cnt++;
  }
};

template <class R, int DIM>
__global__ void __launch_bounds__(128) k_neighbors(Scene<R>* const* sc, int ngroups, int64_t* counts,
                                                   const int64_t* offs, int32_t* list) {
  __shared__ R sm[4][3][32];
  __shared__ float smf[4][3][32];
  __shared__ float4 sm4[sizeof(R) == 4 ? 4 : 1][32];
  __shared__ int smo[4][32], smx[4][32];
  const Scene<R>& S = **sc;
  int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  NbPol<R, DIM> pol;
  pol.sx = sm[wib][0]; pol.sy = sm[wib][1]; pol.sz = sm[wib][2]; pol.so = smo[wib];
  pol.s4 = sm4[sizeof(R) == 4 ? wib : 0]; pol.sox = smx[wib];
  pol.fx = smf[wib][0]; pol.fy = smf[wib][1]; pol.fz = smf[wib][2];
  pol.list = list;
  pol.cmask = (1u << NCLS) - 1u;  // every neighbour, whatever its kind
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < ngroups; g += nw) {
    GroupIter<R, DIM> it(S, g);
    Group<R, DIM> G;
    while (it.next(S, g, lane, G))
    for (int tb = G.ts; tb < G.te; tb += 32) {
      int i = tb + lane;
      bool valid = i < G.te;
      pol.active = valid;
      if (!__any_sync(FULL, pol.active)) continue;
      pol.idx = valid ? i : -1;
      if (valid) target_pos(S, i, G.cx0, pol.tp);
      pol.tf[0] = (float)pol.tp[0]; pol.tf[1] = (float)pol.tp[1]; pol.tf[2] = (float)pol.tp[2];
      pol.cnt = 0;
      pol.off = (valid && offs) ? offs[S.P.orig[i]] : 0;
      traverse<R, DIM>(S, G, pol, lane, S.rc2R, S.rc2f);
      if (valid && !offs) counts[S.P.orig[i]] = pol.cnt;
    }
  }
}

static __global__ void k_sort_segments(const int64_t* offs, int n, int32_t* list) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    int64_t a = offs[o], e = offs[o + 1];
    for (int64_t p = a + 1; p < e; p++) {
      int32_t v = list[p];
      int64_t q = p - 1;
      while (q >= a && list[q] > v) { list[q + 1] = list[q]; q--; }
      list[q + 1] = v;
    }
  }
}

}  // namespace sph

namespace sph {

// ------------------------------------------------------------------ post-processing
// Shepard-filtered field at query points (Eq. postprocessing): sum_j V_j f_j W / sum_j V_j W
// over particles of the selected materials closer than r_c, one thread per query, FP64
// accumulation on both paths.  The 3^d cells around the query's cell hold every such
// particle: cells have edge >= r_c + skin and no particle has moved more than skin / 2
// since it was binned.
template <class R, int DIM>
__global__ void k_interpolate(Scene<R>* const* sc, int nq, const double* q, int field, unsigned mask,
                              double* out) {
  const Scene<R>& S = **sc;
  const double sig = DIM == 2 ? 7.0 / (478.0 * M_PI * S.h * S.h) : 1.0 / (120.0 * M_PI * S.h * S.h * S.h);
  const int comps = field == SPH_F_VEL ? 3 : 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
    double xq[3] = {q[3 * t], q[3 * t + 1], DIM == 3 ? q[3 * t + 2] : 0.0};
    int c[3] = {0, 0, 0};
    for (int k = 0; k < DIM; k++) {
      if (S.per[k]) {
        if (xq[k] >= S.hi[k]) xq[k] -= S.L[k];
        else if (xq[k] < S.lo[k]) xq[k] += S.L[k];
      }
      double v = floor((xq[k] - S.lo[k]) / S.ell[k]);
      c[k] = clamp_cell(v, S.ncell[k]);
    }
    double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
    const int zl = DIM == 3 ? -1 : 0, zh = DIM == 3 ? 1 : 0;
    for (int dz = zl; dz <= zh; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          int cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
          bool skip = false;
          for (int k = 0; k < DIM; k++)
            if (cc[k] < 0 || cc[k] >= S.ncell[k]) {
              if (!S.per[k] || S.ncell[k] < 3) { skip = true; break; }
              cc[k] = (cc[k] + S.ncell[k]) % S.ncell[k];
            }
          if (skip) continue;
          int key = cell_key(S, cc[0] + S.ncell[0] * (cc[1] + S.ncell[1] * cc[2]));
          for (int kc = 0; kc < NCLS; kc++) {
            int a = max(S.cstart[kc * S.ncells + key], 0), e = min(S.cstart[kc * S.ncells + key + 1], S.n);
            for (int j = a; j < e; j++) {
              int mt = S.P.mt[j];
              if (!((mask >> mt) & 1u)) continue;
              double xj[3];
              abs_pos<R>(S, j, xj);
              double r2 = 0.0;
              for (int k = 0; k < DIM; k++) {
                double d = xq[k] - xj[k];
                if (S.per[k]) {
                  if (d > 0.5 * S.L[k]) d -= S.L[k];
                  else if (d < -0.5 * S.L[k]) d += S.L[k];
                }
                r2 += d * d;
              }
              if (!(r2 < S.rc2)) continue;
              double w = sig * quintic_w<double>(sqrt(r2) / S.h) * (double)S.P.m[j] / (double)S.P.rho[j];
              den += w;
              if (field == SPH_F_VEL) {
                num[0] += w * (double)S.P.vx[j];
                num[1] += w * (double)S.P.vy[j];
                num[2] += w * (double)S.P.vz[j];
              } else {
                double f = field == SPH_F_RHO ? (double)S.P.rho[j]
                         : field == SPH_F_PRES ? (double)S.prs[j]
                         : field == SPH_F_TEMP ? (double)S.P.T[j]
                         : (S.any_conc ? (double)S.P.C[j] : 0.0);
                num[0] += w * f;
              }
            }
          }
        }
    for (int k = 0; k < comps; k++) out[comps * t + k] = den > 0.0 ? num[k] / den : (double)NAN;
  }
}

}  // namespace sph
