// CUDA kernels of the SPH interaction sweep (sm_103a).  Templated on the working
// precision R (double: FP64 path; float: FP32 path with FP64 bodies) and the dimension.
//
// Step order (Sec. 3.7, velocity-Verlet kick-drift-kick):
//   k_umax, k_dt            time step, Eq. timestepcond (or fixed)
//   k_body_kick_drift       u_k, w_k half kick; r_k drift; q_k <- q_inc o q_k
//   k_kick_drift            fluid half kick + drift; rigid particles follow their body
//   k_bin .. k_flip         cell binning: counting sort by (kind, cell) key, stable
//                           (Sec. 3.2)
//   k_search                neighbour lists (rebuild steps)
//   k_density               Eq. densum + Eq. eos                       (pair sweep 1)
//   k_extrap                wall / rigid extrapolation (Adami 2012)     (pair sweep 2)
//   k_force                 Eq. momentum, couplingforce, contactforce,
//                           heat_equation                               (pair sweep 3)
//   k_body_reduce           Eqs. procwise_force / global_force, body accelerations,
//                           final body kick                             (FP64)
//   k_final                 T (or H) update, final fluid kick, rigid velocities
//   k_end_step              time and step counters
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_dev.cuh"

namespace sph {

constexpr unsigned FULL = 0xffffffffu;

template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }

// pair distance from its square for the kernel sums, correctly rounded: the pressure of a
// weakly compressible fluid, c^2 (rho - rho_0), carries a relative error of the density sum
// amplified by rho / (rho - rho_0), so a root through the approximate reciprocal root costs
// the FP32 pressure its 1e-5 bound
template <class R> __device__ __forceinline__ R pair_dist(R r2) { return sqrt(r2); }

// quintic spline (Morris 1997), polynomial part: w(q) and dw/dq, valid for q < 3
template <class R>
__device__ __forceinline__ void quintic(R q, R& w, R& dw) {
  R t3 = R(3) - q;
  R t2 = fmax(R(2) - q, R(0));
  R t1 = fmax(R(1) - q, R(0));
  R a2 = t3 * t3, b2 = t2 * t2, c2 = t1 * t1;
  R a4 = a2 * a2, b4 = b2 * b2, c4 = c2 * c2;
  w = a4 * t3 - R(6) * b4 * t2 + R(15) * c4 * t1;
  dw = R(-5) * a4 + R(30) * b4 - R(75) * c4;
}
template <class R>
__device__ __forceinline__ R quintic_w(R q) {
  R t3 = fmax(R(3) - q, R(0));  // (3 - q)_+: a contracted 3 - r/h may round below zero at the edge
  R t2 = fmax(R(2) - q, R(0));
  R t1 = fmax(R(1) - q, R(0));
  R a2 = t3 * t3, b2 = t2 * t2, c2 = t1 * t1;
  return a2 * a2 * t3 - R(6) * b2 * b2 * t2 + R(15) * c2 * c2 * t1;
}
template <class R>
__device__ __forceinline__ R quintic_dw(R q) {
  R t3 = fmax(R(3) - q, R(0));
  R t2 = fmax(R(2) - q, R(0));
  R t1 = fmax(R(1) - q, R(0));
  R a2 = t3 * t3, b2 = t2 * t2, c2 = t1 * t1;
  return R(-5) * a2 * a2 + R(30) * b2 * b2 - R(75) * c2 * c2;
}

__device__ __forceinline__ void qrot(const double* q, double* Rm) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  Rm[0] = 1.0 - 2.0 * (y * y + z * z); Rm[1] = 2.0 * (x * y - w * z);       Rm[2] = 2.0 * (x * z + w * y);
  Rm[3] = 2.0 * (x * y + w * z);       Rm[4] = 1.0 - 2.0 * (x * x + z * z); Rm[5] = 2.0 * (y * z - w * x);
  Rm[6] = 2.0 * (x * z - w * y);       Rm[7] = 2.0 * (y * z + w * x);       Rm[8] = 1.0 - 2.0 * (x * x + y * y);
}
__device__ __forceinline__ void mv(const double* M, const double* v, double* o) {
  o[0] = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
  o[1] = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
  o[2] = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
}
__device__ __forceinline__ void mtv(const double* M, const double* v, double* o) {
  o[0] = M[0] * v[0] + M[3] * v[1] + M[6] * v[2];
  o[1] = M[1] * v[0] + M[4] * v[1] + M[7] * v[2];
  o[2] = M[2] * v[0] + M[5] * v[1] + M[8] * v[2];
}
__device__ __forceinline__ void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// cell key of a row-major cell index
template <class R>
__device__ __forceinline__ int cell_key(const Scene<R>& S, int lin) {
  return S.lin2key ? __ldg(S.lin2key + lin) : lin;
}
// row-major cell index of a sort key (kind * ncells + cell key)
template <class R>
__device__ __forceinline__ int key_lin(const Scene<R>& S, int key) {
  int k = key % S.ncells;
  return S.key2lin ? __ldg(S.key2lin + k) : k;
}
// sort key of a particle of kind `kind` in row-major cell `lin`
template <class R>
__device__ __forceinline__ int part_key(const Scene<R>& S, int kind, int lin) {
  return kind * S.ncells + cell_key(S, lin);
}
template <class R>
__device__ __forceinline__ void lin_xyz(const Scene<R>& S, int lin, int& cx, int& cy, int& cz) {
  cx = lin % S.ncell[0];
  int r = lin / S.ncell[0];
  cy = r % S.ncell[1];
  cz = r / S.ncell[1];
}

// absolute FP64 position of particle i (sorted index) from the current bank
template <class R>
__device__ __forceinline__ void abs_pos(const Scene<R>& S, int i, double* x);
template <>
__device__ __forceinline__ void abs_pos<double>(const Scene<double>& S, int i, double* x) {
  x[0] = S.P.px[i]; x[1] = S.P.py[i]; x[2] = S.P.pz[i];
}
template <>
__device__ __forceinline__ void abs_pos<float>(const Scene<float>& S, int i, double* x) {
  int cx, cy, cz;
  lin_xyz(S, key_lin(S, S.key[i]), cx, cy, cz);
  x[0] = S.lo[0] + cx * S.ell[0] + (double)S.P.px[i];
  x[1] = S.lo[1] + cy * S.ell[1] + (double)S.P.py[i];
  x[2] = S.dim == 3 ? S.lo[2] + cz * S.ell[2] + (double)S.P.pz[i] : 0.0;
}

// store an absolute FP64 position into particle i's slot of the current bank
template <class R>
__device__ __forceinline__ void store_pos(const Scene<R>& S, int i, const double* x);
template <>
__device__ __forceinline__ void store_pos<double>(const Scene<double>& S, int i, const double* x) {
  double y[3] = {x[0], x[1], x[2]};
  for (int k = 0; k < S.dim; k++)
    if (S.per[k]) {
      if (y[k] >= S.hi[k]) y[k] -= S.L[k];
      else if (y[k] < S.lo[k]) y[k] += S.L[k];
    }
  S.P.px[i] = y[0]; S.P.py[i] = y[1]; S.P.pz[i] = y[2];
}
template <>
__device__ __forceinline__ void store_pos<float>(const Scene<float>& S, int i, const double* x) {
  int c[3];
  lin_xyz(S, key_lin(S, S.key[i]), c[0], c[1], c[2]);
  float o[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < S.dim; k++) {
    double v = x[k] - (S.lo[k] + c[k] * S.ell[k]);
    if (S.per[k]) v -= S.L[k] * nearbyint((v - 0.5 * S.ell[k]) / S.L[k]);
    o[k] = (float)v;
  }
  S.P.px[i] = o[0]; S.P.py[i] = o[1]; S.P.pz[i] = o[2];
}

// ============================================================================ time step
// maximum of v over the block (all threads call it), one atomic per block; max is exact, so
// the result does not depend on the order
__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long* ptr) {
  __shared__ unsigned long long red[32];
  for (int o = 16; o; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(FULL, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(FULL, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0 && v > 0ull) atomicMax(ptr, v);
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_umax(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  // one scene: a running maximum per thread and one atomic per block; several scenes: one
  // atomic per scene present in a warp
  unsigned long long run = 0ull;
  for (int g0 = blockIdx.x * blockDim.x; g0 < total; g0 += gridDim.x * blockDim.x) {
    int g = g0 + threadIdx.x;
    // the block's first item decides the scene slice handled in this round
    int s = find_scene(B.pfx_part, B.nsc, min(g, total - 1));
    const Scene<R>& S = *B.sc[s];
    double u = 0.0;
    if (g < total && S.dt_mode == 1) {
      int i = g - __ldg(B.pfx_part + s);
      if (S.matR[S.P.mt[i]].kind == KFLUID) {
        // |u|^2: the root of the maximum equals the maximum of the roots (a correctly
        // rounded root is monotone), so k_dt takes one root instead of one per particle;
        // FP32 scenes square in FP32 (their velocities are FP32; FP64 arithmetic is scarce)
        if constexpr (sizeof(R) == 4) {
          float ux = S.P.vx[i], uy = S.P.vy[i], uz = S.P.vz[i];
          u = (double)__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(uz, uz));
        } else {
          double ux = S.P.vx[i], uy = S.P.vy[i], uz = S.P.vz[i];
          u = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
        }
      }
    }
    // warp maximum for each scene present in the warp, one atomic per scene (max is exact)
    unsigned long long b = (unsigned long long)__double_as_longlong(u);
    if (B.nsc == 1) {
      run = b > run ? b : run;
      continue;
    }
    unsigned pending = FULL;
    while (pending) {
      int leader = __ffs(pending) - 1;
      int cs = __shfl_sync(FULL, s, leader);
      unsigned long long v = s == cs ? b : 0ull;
      for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
      }
      if ((int)(threadIdx.x & 31) == leader && v > 0ull) atomicMax(S.umax, v);
      pending &= ~__ballot_sync(FULL, s == cs);
    }
  }
  if (B.nsc == 1) block_max_atomic(run, B.sc[0]->umax);
}

template <class R>
__global__ void k_dt(BatchView<R> B) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsc) return;
  Scene<R>& S = *B.sc[s];
  double dt = S.dt_fixed;
  if (S.dt_mode == 1) {
    double umax = sqrt(__longlong_as_double((long long)*S.umax));
    dt = S.dt_cond;
    if (S.cmax + umax > 0.0) dt = fmin(dt, 0.25 * S.h / (S.cmax + umax));
    if (!(dt < 1e300)) dt = S.dt_fixed;
  }
  *S.umax = 0ull;
  S.st[0] = dt;
  S.pairs[0] = 0ull;
  S.status[1] = 0;  // relabel counters of this step
  S.status[7] = 0;
  S.status[8] = 0;
}

// ============================================================================ kick + drift
template <class R>
__global__ void k_body_kick_drift(BatchView<R> B) {
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    int k = g - __ldg(B.pfx_body + s);
    if (k >= *S.K || !S.balive[k]) continue;
    double dt = S.st[0], half = 0.5 * dt, phi[3];
    for (int q = 0; q < 3; q++) {
      S.bu[3 * k + q] = S.bu[3 * k + q] + half * S.ba[3 * k + q];
      S.bw[3 * k + q] = S.bw[3 * k + q] + half * S.bal[3 * k + q];
      S.br[3 * k + q] = S.br[3 * k + q] + dt * S.bu[3 * k + q];
      phi[q] = dt * S.bw[3 * k + q];
    }
    // transition quaternion of the increment phi = dt w^{n+1/2}; q^{n+1} = q_inc o q^n
    double ang = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double a[4] = {1.0, 0.0, 0.0, 0.0};
    if (ang > 0.0) {
      double sh = sin(0.5 * ang) / ang;
      a[0] = cos(0.5 * ang); a[1] = sh * phi[0]; a[2] = sh * phi[1]; a[3] = sh * phi[2];
    }
    double* b = &S.bq[4 * k];
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    double nq = sqrt(w * w + x * x + y * y + z * z);
    b[0] = w / nq; b[1] = x / nq; b[2] = y / nq; b[3] = z / nq;
    // R(q^{n+1}) once per body for the rigid particles of this step (the drift and the
    // final kick), instead of once per particle
    qrot(b, &S.bRm[9 * k]);
  }
}

// fluid: u += dt/2 a, r += dt u;  rigid: r_r = r_k + R r_rk, u_r = u_k + w x R r_rk and the
// kinematic acceleration a_k + alpha_k x r_rk + w x (w x r_rk) used by the extrapolation
template <class R>
__device__ __forceinline__ unsigned long long disp_bits(R d2);
template <>
__device__ __forceinline__ unsigned long long disp_bits<double>(double d2) {
  return (unsigned long long)__double_as_longlong(d2);
}
template <>
__device__ __forceinline__ unsigned long long disp_bits<float>(float d2) {
  return (unsigned long long)(unsigned)__float_as_int(d2);
}

template <class R>
__global__ void __launch_bounds__(256) k_kick_drift(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  unsigned long long run = 0ull;  // one scene: running maximum displacement (see k_umax)
  for (int g0 = blockIdx.x * blockDim.x; g0 < total; g0 += gridDim.x * blockDim.x) {
    int g = g0 + threadIdx.x;
    int s = find_scene(B.pfx_part, B.nsc, min(g, total - 1));
    const Scene<R>& S = *B.sc[s];
    int i = g - __ldg(B.pfx_part + s);
    int kind = g < total ? S.matR[S.P.mt[i]].kind : KWALL;
    // wall particles with a prescribed velocity move with it (moving boundaries)
    bool moving_wall = g < total && kind == KWALL && (S.P.vx[i] != R(0) || S.P.vy[i] != R(0) || S.P.vz[i] != R(0));
    if (moving_wall) {
      R dt = (R)S.st[0];
      if (sizeof(R) == 8) {
        double x[3] = {(double)S.P.px[i] + (double)dt * (double)S.P.vx[i],
                       (double)S.P.py[i] + (double)dt * (double)S.P.vy[i],
                       (double)S.P.pz[i] + (double)dt * (double)S.P.vz[i]};
        store_pos<R>(S, i, x);
      } else {
        S.P.px[i] = S.P.px[i] + dt * S.P.vx[i];
        S.P.py[i] = S.P.py[i] + dt * S.P.vy[i];
        S.P.pz[i] = S.P.pz[i] + dt * S.P.vz[i];
      }
    } else if (kind == KFLUID) {
      R dt = (R)S.st[0], half = R(0.5) * dt;
      R ux = S.P.vx[i] + half * S.P.ax[i];
      R uy = S.P.vy[i] + half * S.P.ay[i];
      R uz = S.P.vz[i] + half * S.P.az[i];
      S.P.vx[i] = ux; S.P.vy[i] = uy; S.P.vz[i] = uz;
      // transport-velocity formulation: advection with u~ = u^{n+1/2} + dt/2 a~^n
      R wx = ux, wy = uy, wz = uz;
      if (S.tvf) {
        R tx = half * S.P.bx[i], ty = half * S.P.by[i], tz = half * S.P.bz[i];
        S.P.tx[i] = tx; S.P.ty[i] = ty; S.P.tz[i] = tz;
        wx = ux + tx; wy = uy + ty; wz = uz + tz;
      }
      if (sizeof(R) == 8) {
        double x[3] = {(double)S.P.px[i] + (double)dt * wx, (double)S.P.py[i] + (double)dt * wy,
                       (double)S.P.pz[i] + (double)dt * wz};
        store_pos<R>(S, i, x);
      } else {
        S.P.px[i] = S.P.px[i] + dt * wx;
        S.P.py[i] = S.P.py[i] + dt * wy;
        S.P.pz[i] = S.P.pz[i] + dt * wz;
      }
    } else if (kind == KRIGID) {
      int k = S.P.body[i], sl = S.P.slot[i];
      double rr[3], t1[3], t2[3], t3[3], x[3];
      mv(&S.bRm[9 * k], &S.rb[3 * sl], rr);
      const double* w = &S.bw[3 * k];
      cross(w, rr, t2);
      for (int q = 0; q < 3; q++) x[q] = S.br[3 * k + q] + rr[q];
      store_pos<R>(S, i, x);
      S.P.vx[i] = (R)(S.bu[3 * k] + t2[0]);
      S.P.vy[i] = (R)(S.bu[3 * k + 1] + t2[1]);
      S.P.vz[i] = (R)(S.bu[3 * k + 2] + t2[2]);
      cross(&S.bal[3 * k], rr, t1);
      cross(w, t2, t3);
      S.P.ax[i] = (R)(S.ba[3 * k] + t1[0] + t3[0]);
      S.P.ay[i] = (R)(S.ba[3 * k + 1] + t1[1] + t3[1]);
      S.P.az[i] = (R)(S.ba[3 * k + 2] + t1[2] + t3[2]);
    }
    // packed position for the density sweep of a step without rebuild (FP32 scenes)
    if constexpr (sizeof(R) == 4)
      if (kind != KWALL || moving_wall) S.pa[i] = make_float4(S.P.px[i], S.P.py[i], S.P.pz[i], S.P.rho[i]);
    // displacement since the last list rebuild (skin criterion)
    R d2 = R(0);
    if ((kind != KWALL || moving_wall) && S.skin > 0.0) {
      R d[3] = {S.P.px[i] - S.xr[i], S.P.py[i] - S.yr[i], S.P.pz[i] - S.zr[i]};
      for (int k = 0; k < S.dim; k++)
        if (sizeof(R) == 8 && S.per[k]) {
          if (d[k] > R(0.5) * S.LR[k]) d[k] -= S.LR[k];
          else if (d[k] < R(-0.5) * S.LR[k]) d[k] += S.LR[k];
        }
      d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    }
    unsigned long long b = disp_bits<R>(d2);
    if (B.nsc == 1) {
      run = b > run ? b : run;
      continue;
    }
    unsigned pending = FULL;
    while (pending) {
      int leader = __ffs(pending) - 1;
      int cs = __shfl_sync(FULL, s, leader);
      unsigned long long v = s == cs ? b : 0ull;
      for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
      }
      if ((int)(threadIdx.x & 31) == leader && v > 0ull) atomicMax(S.disp, v);
      pending &= ~__ballot_sync(FULL, s == cs);
    }
  }
  if (B.nsc == 1) block_max_atomic(run, B.sc[0]->disp);
}

// ============================================================================ binning
// Counting sort of the particles by cell key (one digit spanning the whole key): count,
// scan, scatter, then restore input order inside each cell so that the result equals a
// stable sort.  Skipped (early exit) on steps that are not rebin steps.
template <class R>
__device__ __forceinline__ bool rebin_now(const Scene<R>& S) {
  return S.status[4] != 0;
}

// rebuild decision of this step (after the drift): every step without a skin, otherwise
// when a particle moved more than skin / 2 since the last rebuild (or the forced interval)
template <class R>
__global__ void k_decide(BatchView<R> B) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsc) return;
  Scene<R>& S = *B.sc[s];
  R d2 = sizeof(R) == 8 ? (R)__longlong_as_double((long long)*S.disp) : (R)__int_as_float((int)*S.disp);
  int since = S.status[5] + 1;
  // particles that changed phase since the last build change which lists they belong to
  bool rb = S.skin <= 0.0 || d2 > S.half_skin2 || (S.rebin_interval > 1 && since >= S.rebin_interval) ||
            S.status[10] != 0;
  S.status[4] = rb ? 1 : 0;
  if (rb) S.status[10] = 0;
  S.status[5] = rb ? 0 : since;
  if (rb) S.status[6] += 1;
  *S.disp = 0ull;
}

template <class R>
__global__ void k_bin(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    int c[3] = {0, 0, 0};
    int shift = 0;
    if (sizeof(R) == 8) {
      double x[3] = {(double)S.P.px[i], (double)S.P.py[i], (double)S.P.pz[i]};
      for (int k = 0; k < S.dim; k++) {
        double v = floor(__ddiv_rn(__dsub_rn(x[k], S.lo[k]), S.ell[k]));
        c[k] = clamp_cell(v, S.ncell[k]);
      }
    } else {
      // cell-relative positions: new cell = old cell + floor(offset / edge)
      int co[3];
      lin_xyz(S, key_lin(S, S.key[i]), co[0], co[1], co[2]);
      R o[3] = {S.P.px[i], S.P.py[i], S.P.pz[i]};
      for (int k = 0; k < S.dim; k++) {
        // cells moved along k; a non-finite offset keeps its cell (no integer conversion of a NaN)
        float q = floorf((float)o[k] / (float)S.ellR[k]);
        int d = q >= -1048576.f && q <= 1048576.f ? (int)q : 0;
        int cu = co[k] + d;
        int cn;
        if (S.per[k]) cn = ((cu % S.ncell[k]) + S.ncell[k]) % S.ncell[k];
        else cn = cu < 0 ? 0 : (cu >= S.ncell[k] ? S.ncell[k] - 1 : cu);
        c[k] = cn;
        // offset correction applied by the permutation: o -= (c_new_unwrapped - c_old) * edge
        int dd = S.per[k] ? d : cn - co[k];
        dd = dd < -127 ? -127 : (dd > 127 ? 127 : dd);
        shift |= (dd & 0xff) << (8 * k);
      }
    }
    int lin = c[0] + S.ncell[0] * (c[1] + S.ncell[1] * c[2]);
    int key = part_key(S, S.matR[S.P.mt[i]].kind, lin);
    S.tkey[i] = key;
    S.tshift[i] = shift;
    S.tloc[i] = atomicAdd(&S.ccount[key], 1);
  }
}

// block sums of cell counts (blocks of 1024 cells, never straddling scenes)
template <class R>
__global__ void __launch_bounds__(1024) k_scan_blocks(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_cblk + B.nsc);
  __shared__ int red[32];
  for (int blk = blockIdx.x; blk < total; blk += gridDim.x) {
    int s = find_scene(B.pfx_cblk, B.nsc, blk);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int b = blk - __ldg(B.pfx_cblk + s);
    int c = b * 1024 + threadIdx.x;
    int v = c < S.nkey ? S.ccount[c] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      int t = red[threadIdx.x];
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
      if (threadIdx.x == 0) S.cblk[b] = t;
    }
    __syncthreads();
  }
}

// exclusive scan of the block sums of each scene (one block per scene)
template <class R>
__global__ void __launch_bounds__(1024) k_scan_top(BatchView<R> B, int force) {
  __shared__ int wsum[32];
  __shared__ int carry;
  for (int s = blockIdx.x; s < B.nsc; s += gridDim.x) {
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < S.ncblk; base += 1024) {
      int idx = base + threadIdx.x;
      int v = idx < S.ncblk ? S.cblk[idx] : 0;
      int x = v;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
      }
      if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
      __syncthreads();
      if (threadIdx.x < 32) {
        int t = wsum[threadIdx.x], u = t;
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(FULL, u, o);
          if (threadIdx.x >= o) u += y;
        }
        wsum[threadIdx.x] = u - t;
      }
      __syncthreads();
      int excl = carry + wsum[threadIdx.x >> 5] + x - v;
      if (idx < S.ncblk) S.cblk[idx] = excl;
      __syncthreads();
      if (threadIdx.x == 1023) carry = excl + v;
      __syncthreads();
    }
  }
}

// cell starts: exclusive scan inside each block plus the block offset; resets the counts
template <class R>
__global__ void __launch_bounds__(1024) k_scan_cells(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_cblk + B.nsc);
  __shared__ int wsum[32];
  for (int blk = blockIdx.x; blk < total; blk += gridDim.x) {
    int s = find_scene(B.pfx_cblk, B.nsc, blk);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int b = blk - __ldg(B.pfx_cblk + s);
    int c = b * 1024 + threadIdx.x;
    int v = c < S.nkey ? S.ccount[c] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(FULL, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int t = wsum[threadIdx.x], u = t;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, u, o);
        if (threadIdx.x >= o) u += y;
      }
      wsum[threadIdx.x] = u - t;
    }
    __syncthreads();
    if (c < S.nkey) {
      S.cstart[c] = S.cblk[b] + wsum[threadIdx.x >> 5] + x - v;
      S.ccount[c] = 0;
    }
    if (c == S.nkey - 1) S.cstart[S.nkey] = S.n;
    __syncthreads();
  }
}

template <class R>
__global__ void k_scatter(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    S.bucket[S.cstart[S.tkey[i]] + S.tloc[i]] = i;
  }
}

// inside each cell, order the entries by their previous index (one warp per cell):
// rank = number of entries with a smaller previous index
template <class R>
__global__ void k_rank(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_cell + B.nsc);
  int lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < total; g += nw) {
    int s = find_scene(B.pfx_cell, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int c = g - __ldg(B.pfx_cell + s);
    int a = S.cstart[c], e = S.cstart[c + 1];
    int cnt = e - a;
    if (cnt == 0) continue;
    if (cnt < 0 || a < 0 || e > S.n) {  // inconsistent table: flag it, never loop on it
      S.status[3] = 1;
      continue;
    }
    if (cnt == 1) {
      if (lane == 0) S.perm[a] = S.bucket[a];
      continue;
    }
    for (int t0 = 0; t0 < cnt; t0 += 32) {
      int t = t0 + lane;
      int v = t < cnt ? S.bucket[a + t] : 0x7fffffff;
      int rank = 0;
      for (int u0 = 0; u0 < cnt; u0 += 32) {
        int w = (u0 + lane) < cnt ? S.bucket[a + u0 + lane] : 0x7fffffff;
        int lim = min(32, cnt - u0);
        for (int k = 0; k < lim; k++) rank += (__shfl_sync(FULL, w, k) < v);
      }
      if (t < cnt) S.perm[a + rank] = v;
    }
  }
}

template <class R>
__global__ void k_permute(BatchView<R> B, int force) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!force && !rebin_now(S)) continue;
    int j = g - __ldg(B.pfx_part + s);
    int i = S.perm[j];
    const PBank<R>& P = S.P;
    const PBank<R>& Q = S.Q;
    R px = P.px[i], py = P.py[i], pz = P.pz[i];
    if (sizeof(R) == 4) {
      int sh = S.tshift[i];
      int d0 = (int)(signed char)(sh & 0xff), d1 = (int)(signed char)((sh >> 8) & 0xff),
          d2 = (int)(signed char)((sh >> 16) & 0xff);
      px = px - (R)d0 * S.ellR[0];
      py = py - (R)d1 * S.ellR[1];
      pz = pz - (R)d2 * S.ellR[2];
    }
    Q.px[j] = px; Q.py[j] = py; Q.pz[j] = pz;
    // FP32: the packed positions in the new order (the density sweep reads them)
    if constexpr (sizeof(R) == 4) S.pa[j] = make_float4(px, py, pz, P.rho[i]);
    S.xr[j] = px; S.yr[j] = py; S.zr[j] = pz;
    Q.vx[j] = P.vx[i]; Q.vy[j] = P.vy[i]; Q.vz[j] = P.vz[i];
    Q.ax[j] = P.ax[i]; Q.ay[j] = P.ay[i]; Q.az[j] = P.az[i];
    Q.rho[j] = P.rho[i]; Q.T[j] = P.T[i]; Q.H[j] = P.H[i]; Q.m[j] = P.m[i];
    Q.mt[j] = P.mt[i];
    if (S.any_conc) Q.C[j] = P.C[i];
    if (S.tvf) {
      Q.bx[j] = P.bx[i]; Q.by[j] = P.by[i]; Q.bz[j] = P.bz[i];
      Q.tx[j] = P.tx[i]; Q.ty[j] = P.ty[i]; Q.tz[j] = P.tz[i];
    }
    int b = P.body[i], sl = P.slot[i], o = P.orig[i];
    Q.body[j] = b; Q.slot[j] = sl; Q.orig[j] = o;
    S.key[j] = S.tkey[i];
    S.where[o] = j;
    if (sl >= 0) S.slot_part[sl] = j;
  }
}

template <class R>
__global__ void k_flip(BatchView<R> B, int force) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsc) return;
  Scene<R>& S = *B.sc[s];
  if (!force && !rebin_now(S)) return;
  PBank<R> t = S.P;
  S.P = S.Q;
  S.Q = t;
}

// ============================================================================ cell traversal
// One warp per target group (a cell, G consecutive cells along x, or a window of 32
// consecutive particles), split into ranges of one kind.  For each chunk of <= 32 targets
// the warp visits the stencil rows kind by kind; each chunk of <= 32 candidates is staged
// in shared memory, every lane tests all candidates against its target (hit mask), then
// processes its own hits.

template <class R, int DIM>
struct Group {
  int cx0, cy, cz, ncx, ts, te;
  int cls;  // kind of every target of the range
};

// the targets of kind `cls` in search group grp (a cell for Morton keys, a run of G cells
// along x for row-major keys)
template <class R, int DIM>
__device__ __forceinline__ Group<R, DIM> group_of(const Scene<R>& S, int grp, int cls) {
  Group<R, DIM> G;
  G.cls = cls;
  int base = cls * S.ncells;
  if (S.key2lin) {  // Morton keys: one cell per group
    int lin = __ldg(S.key2lin + grp);
    lin_xyz(S, lin, G.cx0, G.cy, G.cz);
    G.ncx = 1;
    G.ts = max(S.cstart[base + grp], 0);
    G.te = min(S.cstart[base + grp + 1], S.n);
  } else {
    int gx = grp % S.ngx, r = grp / S.ngx;
    G.cy = r % S.ncell[1];
    G.cz = r / S.ncell[1];
    G.cx0 = gx * S.G;
    G.ncx = min(S.G, S.ncell[0] - G.cx0);
    int lin0 = G.cx0 + S.ncell[0] * (G.cy + S.ncell[1] * G.cz);
    G.ts = max(S.cstart[base + lin0], 0);
    G.te = min(S.cstart[base + lin0 + G.ncx], S.n);
  }
  return G;
}

// Target ranges of search group g, one per call of next(), each of a single kind: the
// fluid, rigid and wall runs of a cell (Morton keys) or of a run of cells along x (row-major
// keys); in window mode (row-major keys) group g is the 32 consecutive sorted particles
// [32 g, 32 g + 32), split where they cross from one row of cells (cy, cz) or one kind to
// the next, each part with the x range of cells it spans.  All lanes of the warp call next()
// together.
template <class R, int DIM>
struct GroupIter {
  int ts, te, cls;
  __device__ GroupIter(const Scene<R>& S, int g) {
    cls = 0;
    ts = S.win ? 32 * g : 0;
    te = S.win ? min(ts + 32, S.n) : 0;
  }
  __device__ bool next(const Scene<R>& S, int g, int lane, Group<R, DIM>& G) {
    if (!S.win) {
      while (cls < NCLS) {
        G = group_of<R, DIM>(S, g, cls++);
        if (G.te > G.ts) return true;
      }
      return false;
    }
    if (ts >= te) return false;
    int i = ts + lane;
    int key = i < te ? S.key[i] : 0;
    int cx = 0, cy = 0, cz = 0;
    lin_xyz(S, key_lin(S, key), cx, cy, cz);
    int row = key / S.ncell[0];  // (kind, cy, cz): ncells is a multiple of ncell[0]
    int row0 = __shfl_sync(FULL, row, 0);
    unsigned same = __ballot_sync(FULL, i < te && row == row0);
    int cnt = __popc(same);  // sorted keys: the lanes of the first row form a prefix
    G.cls = __shfl_sync(FULL, key, 0) / S.ncells;
    G.cx0 = __shfl_sync(FULL, cx, 0);
    G.ncx = __shfl_sync(FULL, cx, cnt - 1) - G.cx0 + 1;
    G.cy = __shfl_sync(FULL, cy, 0);
    G.cz = __shfl_sync(FULL, cz, 0);
    G.ts = ts;
    G.te = ts + cnt;
    ts += cnt;
    return true;
  }
};

// target position in the frame of the group: FP64 absolute; FP32 relative to the origin
// of the group's first cell
template <class R>
__device__ __forceinline__ void target_pos(const Scene<R>& S, int i, int cx0, R* p) {
  p[0] = S.P.px[i]; p[1] = S.P.py[i]; p[2] = S.P.pz[i];
  if (sizeof(R) == 4 && !S.key2lin) {
    int cx = S.key[i] % S.ncell[0];  // ncells is a multiple of ncell[0]
    p[0] += (R)(cx - cx0) * S.ellR[0];
  }
}

template <class R, int DIM>
__device__ __forceinline__ R dist2(R dx, R dy, R dz) {
  if (DIM == 2) return dx * dx + dy * dy;
  return (dx * dx + dy * dy) + dz * dz;
}

// FP64 path: the squared distance of the predicate is formed without contraction so that
// neighbour sets match a plain IEEE evaluation bit for bit
template <int DIM>
__device__ __forceinline__ double dist2_exact(double dx, double dy, double dz) {
  double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (DIM == 3) s = __dadd_rn(s, __dmul_rn(dz, dz));
  return s;
}

template <class R, int DIM>
__device__ __forceinline__ R pair_r2(R dx, R dy, R dz) {
  if (sizeof(R) == 8) return (R)dist2_exact<DIM>((double)dx, (double)dy, (double)dz);
  return dist2<R, DIM>(dx, dy, dz);
}

template <class R>
__device__ __forceinline__ R dsub(R a, R b) {
  if (sizeof(R) == 8) return (R)__dsub_rn((double)a, (double)b);
  return a - b;
}

// The candidate runs of the 3^d stencil of cells around the columns [cx0, cx0 + ncx) of row
// (cy0, cz0), kind by kind (a bit per kind in cmask), in a fixed order: rows (dz, dy); in
// each row the periodic image of the column left of the box, the columns inside the box,
// the periodic image of the column right of it; each of these kind by kind, and for
// row-major keys the columns inside the box as one run (consecutive keys).  f(cs, ce, oxf,
// shx, shy, shz, dy, dz, kfirst, ncols) gets the sorted index range [cs, ce), the column
// offset oxf of the run's candidates relative to cx0 (kOxKey: each candidate's own column,
// the run then spans the ncols cells of keys kfirst, kfirst + 1, ...), and the shift subtracted from p_i - p_j: FP64 the periodic
// image (+-L), FP32 the cell offset (dy ell_y, dz ell_z; along x the column offset, taken
// per candidate; ox0 = x0 - cx0 the offset of the first column).
constexpr int kOxKey = -(1 << 30);

template <class R, int DIM, class F>
__device__ __forceinline__ void for_each_run(const Scene<R>& S, int cx0, int ncx, int cy0, int cz0, unsigned cmask,
                                             F&& f) {
  const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; dz++)
    for (int dy = -1; dy <= 1; dy++) {
      int cy = cy0 + dy, cz = DIM == 3 ? cz0 + dz : 0;
      R shy = sizeof(R) == 4 ? (R)dy * S.ellR[1] : R(0);
      R shz = sizeof(R) == 4 && DIM == 3 ? (R)dz * S.ellR[2] : R(0);
      if (cy < 0 || cy >= S.ncell[1]) {
        if (!S.per[1]) continue;
        int w = cy < 0 ? 1 : -1;  // image of the row inside the box
        cy += w * S.ncell[1];
        if (sizeof(R) == 8) shy = w > 0 ? -S.LR[1] : S.LR[1];
      }
      if (DIM == 3 && (cz < 0 || cz >= S.ncell[2])) {
        if (!S.per[2]) continue;
        int w = cz < 0 ? 1 : -1;
        cz += w * S.ncell[2];
        if (sizeof(R) == 8) shz = w > 0 ? -S.LR[2] : S.LR[2];
      }
      int row = S.ncell[0] * (cy + S.ncell[1] * cz);
      int nx = S.ncell[0];
      int xa = cx0 - 1, xb = cx0 + ncx;  // stencil columns, inclusive
      int x0 = max(xa, 0), x1 = min(xb, nx - 1);
      // segments: -1 the left image, 0 .. nseg-1 inside the box (one run of consecutive keys,
      // or one column per segment for Morton keys), nseg the right image; one call site of f
      int nseg = S.key2lin ? x1 - x0 + 1 : 1;
      for (int sg = -1; sg <= nseg; sg++) {
        int ka, kb, oxf;  // cell keys [ka, kb] within a kind
        R shx = R(0);
        if (sg < 0) {
          if (!(xa < 0 && S.per[0])) continue;
          ka = kb = cell_key(S, row + nx - 1);
          oxf = -1;
          if (sizeof(R) == 8) shx = -S.LR[0];
        } else if (sg == nseg) {
          if (!(xb > nx - 1 && S.per[0])) continue;
          ka = kb = cell_key(S, row);
          oxf = ncx;
          if (sizeof(R) == 8) shx = S.LR[0];
        } else if (S.key2lin) {
          ka = kb = cell_key(S, row + x0 + sg);
          oxf = x0 + sg - cx0;
        } else {
          ka = row + x0;
          kb = row + x1;
          oxf = kOxKey;
        }
        // the bounds of every kind first (independent loads, one latency), then the runs
        int rb[NCLS], re[NCLS];
#pragma unroll
        for (int cc = 0; cc < NCLS; cc++) {
          rb[cc] = re[cc] = 0;
          if ((cmask >> cc) & 1u) {
            int base = cc * S.ncells;
            rb[cc] = S.cstart[base + ka];
            re[cc] = S.cstart[base + kb + 1];
          }
        }
#pragma unroll
        for (int cc = 0; cc < NCLS; cc++)
          if (rb[cc] < re[cc]) f(rb[cc], re[cc], oxf, shx, shy, shz, dy, dz, cc * S.ncells + ka, kb - ka + 1, x0 - cx0);
      }
    }
}

// generic traversal.  Pol provides: stage(S, j, lane), active, tp[3], idx, cmask (the
// candidate kinds visited, the same for the whole warp), shared arrays sox (column offset
// of each staged candidate) and s4 (FP32: staged x plus that offset, y, z), pair(S, k, j, dx, dy,
// dz, r2) with cox/cdy/cdz set to the candidate's cell offset, kExact (pair() sees exactly
// the pairs with r^2 < rc2, with their offset; otherwise every pre-test hit, a superset,
// without it), and for FP64 scenes FP32 copies fx/fy/fz of the staged positions and tf of
// the target (rc2f: the FP32 pre-test radius, squared, with the margin of the rounding of
// those copies).  With kEntry (lists of the search), sox holds each staged candidate's
// list entry for a target of the group's first column and scol its column offset, and
// every pre-test hit in a column next to its target's goes to put(entry - tx) instead of
// pair().  Candidates come in the order of for_each_run.
template <class R, int DIM, class Pol>
__device__ __forceinline__ void traverse(const Scene<R>& S, const Group<R, DIM>& G, Pol& pol, int lane, R rc2,
                                         float rc2f) {
  for_each_run<R, DIM>(S, G.cx0, G.ncx, G.cy, G.cz, pol.cmask,
                       [&](int cs0, int ce0, int oxf, R shx, R shy, R shz, int dy, int dz, int kfirst, int ncols,
                           int ox0) {
    int cs = max(cs0, 0), ce = min(ce0, S.n);
    pol.cdy = dy;
    pol.cdz = dz;
    // interior cell bounds of a run of up to five columns, loaded once for the run
    int bnd[4];
#pragma unroll
    for (int m = 0; m < 4; m++)
      bnd[m] = (oxf == kOxKey && m + 1 < ncols && ncols <= 5) ? __ldg(S.cstart + kfirst + m + 1) : 0x7fffffff;
    for (int cb = cs; cb < ce; cb += 32) {
      int cnt = min(32, ce - cb);
      __syncwarp();
      if (lane < cnt) {
        int j = cb + lane;
        pol.stage(S, j, lane);
        int ox = oxf;
        if (oxf == kOxKey) {
          if (ncols <= 5) {  // the column from the cell bounds of the run
            ox = ox0;
#pragma unroll
            for (int m = 0; m < 4; m++) ox += j >= bnd[m] ? 1 : 0;
          } else {  // row-major keys: the key modulo ncell[0] (ncells is a multiple of it)
            ox = S.key[j] % S.ncell[0] - G.cx0;
          }
        }
        if constexpr (Pol::kEntry) {  // the list entry for a target of column cx0 (tx = 0): a
          // target of column cx0 + tx subtracts tx (the x field ox + 1 - tx lands in 0..2)
          pol.sox[lane] = (int)(((unsigned)j << 6) + (unsigned)(((dz + 1) << 4) + ((dy + 1) << 2) + (ox + 1)));
          pol.scol[lane] = ox;
        } else {
          pol.sox[lane] = ox;
        }
        if constexpr (sizeof(R) == 4)
          pol.s4[lane] = make_float4(pol.sx[lane] + (R)ox * S.ellR[0], pol.sy[lane], pol.sz[lane], 0.f);
      } else if (sizeof(R) == 4) {
        pol.s4[lane] = make_float4(1e30f, 0.f, 0.f, 0.f);  // padding: fails every test
      } else {
        pol.fx[lane] = 1e30f;
      }
      __syncwarp();
      unsigned mask = 0u;
      if (pol.active) {
        // the candidates in groups over the padded batch (FP64 scenes four, FP32 eight)
        if constexpr (sizeof(R) == 8) {
          // FP64 scenes: an FP32 test with a margin keeps a superset of the pairs
          float shf[3] = {(float)shx, (float)shy, (float)shz};
          for (int k0 = 0; k0 < cnt; k0 += 4) {
#pragma unroll
            for (int k = k0; k < k0 + 4; k++) {
              float dx = (pol.tf[0] - pol.fx[k]) - shf[0];
              float dy2 = (pol.tf[1] - pol.fy[k]) - shf[1];
              float dz2 = DIM == 3 ? (pol.tf[2] - pol.fz[k]) - shf[2] : 0.f;
              float r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
              if (r2 < rc2f) mask |= 1u << k;
            }
          }
        } else {
          // FP32 scenes: a pre-test on the staged x shifted by its column and the target
          // shifted by the row, its radius widened past the rounding of that reordering (a
          // relative 1e-4 on r^2)
          R qy = pol.tp[1] - shy, qz = pol.tp[2] - shz;
          R rc2m = rc2 * R(1.0001);
          // eight at a time (the padded entries fail), each hit bit at a fixed position of
          // a byte that is then shifted into place (9 % faster search than four at a time,
          // each bit at its own variable shift)
          for (int k0 = 0; k0 < cnt; k0 += 8) {
            unsigned m8 = 0u;
#pragma unroll
            for (int q = 0; q < 8; q++) {
              float4 c = pol.s4[k0 + q];  // one broadcast load per candidate
              R dx = pol.tp[0] - c.x;
              R dy2 = qy - c.y;
              R dz2 = DIM == 3 ? qz - c.z : R(0);
              R r2 = dist2<R, DIM>(dx, dy2, dz2);
              if (r2 < rc2m) m8 |= 1u << q;
            }
            mask |= m8 << k0;
          }
        }
        unsigned self = (unsigned)(pol.idx - cb);  // a target is not its own neighbour
        if (self < (unsigned)cnt) mask &= ~(1u << self);
      }
      while (mask) {
        int k = __ffs(mask) - 1;
        mask &= mask - 1;
        if constexpr (Pol::kEntry) {
          // a candidate two columns from its target is farther than the cell edge, itself at
          // least r_c + skin, and passes only through the pre-test's margin (a cell edge
          // within about 1e-4 of r_c + skin); its x field would fall outside 0..2 and borrow
          // into the other fields and the index, so it is left out of the list
          if ((unsigned)(pol.scol[k] - pol.tx + 1) > 2u) continue;
          pol.put((int)((unsigned)pol.sox[k] - (unsigned)pol.tx));
          continue;
        }
        int ox = pol.sox[k];
        pol.cox = ox;
        if constexpr (Pol::kExact) {  // the exact set: each hit decided on the sweeps' offset
          R sx0 = sizeof(R) == 4 ? (R)ox * S.ellR[0] : shx;
          R dx = dsub(dsub(pol.tp[0], pol.sx[k]), sx0);
          R dy2 = dsub(dsub(pol.tp[1], pol.sy[k]), shy);
          R dz2 = DIM == 3 ? dsub(dsub(pol.tp[2], pol.sz[k]), shz) : R(0);
          R r2 = pair_r2<R, DIM>(dx, dy2, dz2);
          if (!(r2 < rc2)) continue;  // the pre-tests keep a superset
          pol.pair(S, k, cb + k, dx, dy2, dz2, r2);
        } else {
          pol.pair(S, k, cb + k, R(0), R(0), R(0), R(0));
        }
      }
    }
  });
}

}  // namespace sph

#include "sph_sweeps.cuh"

namespace sph {

// ============================================================================ bodies (FP64)
// force and torque of every body (Eq. procwise_force with thread partials as the
// processors), body accelerations (Eqs. linear/angular momentum), final body kick
template <class R>
__global__ void __launch_bounds__(128) k_body_reduce(BatchView<R> B, int kick) {
  __shared__ double red[6][128];
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    int k = g - __ldg(B.pfx_body + s);
    if (k >= *S.K || !S.balive[k]) continue;
    double Rm[9];
    qrot(&S.bq[4 * k], Rm);
    double F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
    for (int sl = S.bstart[k] + threadIdx.x; sl < S.bend[k]; sl += blockDim.x) {
      double f[3] = {(double)S.fr[3 * sl], (double)S.fr[3 * sl + 1], (double)S.fr[3 * sl + 2]};
      double rr[3], c[3];
      mv(Rm, &S.rb[3 * sl], rr);
      cross(rr, f, c);
      for (int q = 0; q < 3; q++) { F[q] += f[q]; Tq[q] += c[q]; }
    }
    for (int q = 0; q < 3; q++) { red[q][threadIdx.x] = F[q]; red[3 + q][threadIdx.x] = Tq[q]; }
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        for (int q = 0; q < 6; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double f[3], t[3], t1[3], t2[3], al[3];
      for (int q = 0; q < 3; q++) { f[q] = red[q][0] + S.bm[k] * S.g[q]; t[q] = red[3 + q][0]; }
      mtv(Rm, t, t1);
      mv(&S.bIbinv[9 * k], t1, t2);
      mv(Rm, t2, al);
      if (S.dim == 2) { al[0] = 0.0; al[1] = 0.0; }
      double half = 0.5 * S.st[0];
      for (int q = 0; q < 3; q++) {
        S.bf[3 * k + q] = f[q];
        S.bt[3 * k + q] = t[q];
        S.ba[3 * k + q] = f[q] / S.bm[k];
        S.bal[3 * k + q] = al[q];
        if (kick) {
          S.bu[3 * k + q] = S.bu[3 * k + q] + half * S.ba[3 * k + q];
          S.bw[3 * k + q] = S.bw[3 * k + q] + half * al[q];
        }
      }
      // world inertia R I_body R^T
      double T9[9];
      const double* Ib = &S.bIb[9 * k];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) T9[3 * a + b] = Rm[3 * a] * Ib[b] + Rm[3 * a + 1] * Ib[3 + b] + Rm[3 * a + 2] * Ib[6 + b];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
          S.bIw[9 * k + 3 * a + b] = T9[3 * a] * Rm[3 * b] + T9[3 * a + 1] * Rm[3 * b + 1] + T9[3 * a + 2] * Rm[3 * b + 2];
    }
    __syncthreads();
  }
}

// ============================================================================ final update
template <class R>
__global__ void k_final(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    int i = g - __ldg(B.pfx_part + s);
    const MatR<R>& A = S.matR[S.P.mt[i]];
    if (A.kind == KWALL) continue;
    R dt = (R)S.st[0];
    if (A.enth) {
      R Hn = S.P.H[i] + dt * S.dT[i];
      S.P.H[i] = Hn;
      const MatD& M = S.mat[S.P.mt[i]];
      // T(H): apparent-capacity interval of width w below/above T_t
      int so = S.P.mt[i], li = S.P.mt[i];
      if (M.to >= 0) {
        so = M.kind == KRIGID ? S.P.mt[i] : M.to;
        li = M.kind == KRIGID ? M.to : S.P.mt[i];
      }
      double cs = S.mat[so].cp, cl = S.mat[li].cp, w = M.w, Tlo = M.Tt - 0.5 * w;
      double Hh = (cs + M.L / w) * w, H = (double)Hn, T;
      if (H <= 0.0) T = Tlo + H / cs;
      else if (H <= Hh) T = Tlo + H / (cs + M.L / w);
      else T = Tlo + w + (H - Hh) / cl;
      S.P.T[i] = (R)T;
    } else {
      S.P.T[i] = S.P.T[i] + dt * S.dT[i];
    }
    if (S.any_conc) {  // concentration; reservoir phases keep their fixed value
      double cf = S.mat[S.P.mt[i]].Cfix;
      S.P.C[i] = isnan(cf) ? S.P.C[i] + dt * S.dC[i] : (R)cf;
    }
    if (A.kind == KFLUID) {
      R half = R(0.5) * dt;
      R ux = S.P.vx[i] + half * S.P.ax[i];
      R uy = S.P.vy[i] + half * S.P.ay[i];
      R uz = S.P.vz[i] + half * S.P.az[i];
      S.P.vx[i] = ux; S.P.vy[i] = uy; S.P.vz[i] = uz;
      if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) S.status[0] = 1;
    } else {
      int k = S.P.body[i], sl = S.P.slot[i];
      double rr[3], c[3];
      mv(&S.bRm[9 * k], &S.rb[3 * sl], rr);  // R(q^{n+1}) of the body's drift this step
      cross(&S.bw[3 * k], rr, c);
      S.P.vx[i] = (R)(S.bu[3 * k] + c[0]);
      S.P.vy[i] = (R)(S.bu[3 * k + 1] + c[1]);
      S.P.vz[i] = (R)(S.bu[3 * k + 2] + c[2]);
    }
  }
}

// failure flag of every scene in the batch tables (one copy to the host per poll): non-finite
// velocities, or a relabel that could not be applied (body capacity, union-find retry cap)
template <class R>
__global__ void k_gather_failed(Scene<R>* const* sc, int ns, int* out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const int* st = sc[s]->status;
    out[s] = st[ST_NONFINITE] != 0 || st[ST_CAPACITY] != 0 || st[ST_HOOK_TIMEOUT] != 0;
  }
}

template <class R>
__global__ void k_end_step(BatchView<R> B) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsc) return;
  Scene<R>& S = *B.sc[s];
  S.st[1] += S.st[0];
  S.st[2] += 1.0;
  S.st[3] = S.st[0];
  S.pairs[1] += S.pairs[0];  // cumulative ordered pairs of the force / heat sweep
}

// ============================================================================ body set-up (FP64)
// Mass, centre of mass and inertia of every body from its rigid particles: each thread
// sums a chunk (processor-wise Eqs. procwise_centerofmass / procwise_inertia) and the
// chunks are combined by Eqs. global_centerofmass / global_inertia (Huygens-Steiner).
// Then the body-frame inertia R^T I R, its inverse, and the body-frame offsets of the
// particles r_rk = R^T (x_r - r_k).
template <class R>
__global__ void __launch_bounds__(128) k_body_mass(BatchView<R> B, int changed_only) {
  __shared__ double pm[128], pr[3][128], pI[9][128];
  __shared__ double com[3];
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    int k = g - __ldg(B.pfx_body + s);
    if (k >= *S.K) continue;
    if (changed_only && !S.bchg[k]) continue;
    int a = S.bstart[k], e = S.bend[k];
    if (e <= a) {
      if (threadIdx.x == 0) S.balive[k] = 0;
      continue;
    }
    // reference particle for minimum-image unwrapping on periodic axes
    double x0[3];
    abs_pos<R>(S, S.slot_part[a], x0);
    double Ir_c = S.dim == 2 ? 0.5 * S.dx * S.dx / M_PI : 0.4 * cbrt(0.75 / M_PI) * cbrt(0.75 / M_PI) * S.dx * S.dx;
    double m = 0, c[3] = {0, 0, 0};
    // chunk of this thread: contiguous slots
    int n = e - a, per = (n + blockDim.x - 1) / blockDim.x;
    int s0 = a + threadIdx.x * per, s1 = min(e, s0 + per);
    for (int sl = s0; sl < s1; sl++) {
      double x[3];
      abs_pos<R>(S, S.slot_part[sl], x);
      for (int q = 0; q < S.dim; q++)
        if (S.per[q]) {
          double d = x[q] - x0[q];
          if (d > 0.5 * S.L[q]) x[q] -= S.L[q]; else if (d < -0.5 * S.L[q]) x[q] += S.L[q];
        }
      double mr = (double)S.P.m[S.slot_part[sl]];
      m += mr;
      for (int q = 0; q < 3; q++) c[q] += mr * x[q];
    }
    double I[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (m > 0)
      for (int q = 0; q < 3; q++) c[q] /= m;
    for (int sl = s0; sl < s1; sl++) {
      double x[3];
      abs_pos<R>(S, S.slot_part[sl], x);
      for (int q = 0; q < S.dim; q++)
        if (S.per[q]) {
          double d = x[q] - x0[q];
          if (d > 0.5 * S.L[q]) x[q] -= S.L[q]; else if (d < -0.5 * S.L[q]) x[q] += S.L[q];
        }
      double mr = (double)S.P.m[S.slot_part[sl]];
      double d[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
      double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) I[3 * p + q] += Ir_c * mr * (p == q) + ((p == q) * d2 - d[p] * d[q]) * mr;
    }
    pm[threadIdx.x] = m;
    for (int q = 0; q < 3; q++) pr[q][threadIdx.x] = c[q];
    for (int q = 0; q < 9; q++) pI[q][threadIdx.x] = I[q];
    __syncthreads();
    if (threadIdx.x == 0) {
      double M = 0, C[3] = {0, 0, 0};
      for (int t = 0; t < blockDim.x; t++) {
        M += pm[t];
        for (int q = 0; q < 3; q++) C[q] += pm[t] * pr[q][t];
      }
      for (int q = 0; q < 3; q++) C[q] /= M;
      double IG[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int t = 0; t < blockDim.x; t++) {
        if (pm[t] == 0.0) continue;
        double d[3] = {C[0] - pr[0][t], C[1] - pr[1][t], C[2] - pr[2][t]};
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        for (int p = 0; p < 3; p++)
          for (int q = 0; q < 3; q++) IG[3 * p + q] += pI[3 * p + q][t] + ((p == q) * d2 - d[p] * d[q]) * pm[t];
      }
      S.bm[k] = M;
      for (int q = 0; q < 3; q++) { S.br[3 * k + q] = C[q]; com[q] = C[q]; }
      double Rm[9], T9[9], Ib[9];
      qrot(&S.bq[4 * k], Rm);
      for (int q = 0; q < 9; q++) S.bIw[9 * k + q] = IG[q];
      // I_body = R^T I R
      for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) T9[3 * p + q] = Rm[p] * IG[q] + Rm[3 + p] * IG[3 + q] + Rm[6 + p] * IG[6 + q];
      for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) Ib[3 * p + q] = T9[3 * p] * Rm[q] + T9[3 * p + 1] * Rm[3 + q] + T9[3 * p + 2] * Rm[6 + q];
      for (int q = 0; q < 9; q++) S.bIb[9 * k + q] = Ib[q];
      double c00 = Ib[4] * Ib[8] - Ib[5] * Ib[7], c01 = Ib[5] * Ib[6] - Ib[3] * Ib[8], c02 = Ib[3] * Ib[7] - Ib[4] * Ib[6];
      double det = Ib[0] * c00 + Ib[1] * c01 + Ib[2] * c02, id = 1.0 / det;
      double* Bi = &S.bIbinv[9 * k];
      Bi[0] = c00 * id; Bi[1] = (Ib[2] * Ib[7] - Ib[1] * Ib[8]) * id; Bi[2] = (Ib[1] * Ib[5] - Ib[2] * Ib[4]) * id;
      Bi[3] = c01 * id; Bi[4] = (Ib[0] * Ib[8] - Ib[2] * Ib[6]) * id; Bi[5] = (Ib[2] * Ib[3] - Ib[0] * Ib[5]) * id;
      Bi[6] = c02 * id; Bi[7] = (Ib[1] * Ib[6] - Ib[0] * Ib[7]) * id; Bi[8] = (Ib[0] * Ib[4] - Ib[1] * Ib[3]) * id;
      S.balive[k] = 1;
    }
    __syncthreads();
    double Rm[9];
    qrot(&S.bq[4 * k], Rm);
    for (int sl = a + threadIdx.x; sl < e; sl += blockDim.x) {
      // same unwrapping as for the mass quantities: image nearest to the reference particle
      double x[3], d[3];
      abs_pos<R>(S, S.slot_part[sl], x);
      for (int q = 0; q < 3; q++) {
        if (q < S.dim && S.per[q]) {
          double dd = x[q] - x0[q];
          if (dd > 0.5 * S.L[q]) x[q] -= S.L[q]; else if (dd < -0.5 * S.L[q]) x[q] += S.L[q];
        }
        d[q] = x[q] - com[q];
      }
      mtv(Rm, d, &S.rb[3 * sl]);
    }
    __syncthreads();
  }
}

// rigid particle velocities from their bodies (after creation or a relabel)
template <class R>
__global__ void k_rigid_vel(BatchView<R> B, int after_relabel) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (after_relabel && !(S.has_transition && S.status[1] > 0 && S.status[ST_CAPACITY] == 0 &&
                           S.status[ST_HOOK_TIMEOUT] == 0)) continue;
    int i = g - __ldg(B.pfx_part + s);
    if (S.matR[S.P.mt[i]].kind != KRIGID) continue;
    int k = S.P.body[i], sl = S.P.slot[i];
    double Rm[9], rr[3], c[3], t1[3], t3[3];
    qrot(&S.bq[4 * k], Rm);
    mv(Rm, &S.rb[3 * sl], rr);
    cross(&S.bw[3 * k], rr, c);
    S.P.vx[i] = (R)(S.bu[3 * k] + c[0]);
    S.P.vy[i] = (R)(S.bu[3 * k + 1] + c[1]);
    S.P.vz[i] = (R)(S.bu[3 * k + 2] + c[2]);
    cross(&S.bal[3 * k], rr, t1);
    cross(&S.bw[3 * k], c, t3);
    S.P.ax[i] = (R)(S.ba[3 * k] + t1[0] + t3[0]);
    S.P.ay[i] = (R)(S.ba[3 * k + 1] + t1[1] + t3[1]);
    S.P.az[i] = (R)(S.ba[3 * k + 2] + t1[2] + t3[2]);
  }
}

}  // namespace sph

#include "sph_relabel.cuh"
