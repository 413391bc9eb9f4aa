// The pair sweeps of a step (warp per target group, candidates staged in shared memory).
//
// The candidates of a target group are the particles of its stencil cells (3^d cells around
// it, Sec. 3.2) taken as one stream: cells in traversal order, particles in index order.
// The stream is cut into chunks of 32 candidates.
//
//  k_search   on list-rebuild steps: for every target and chunk, the 32-bit mask of the
//             candidates closer than r_c + skin (stored at nbm[c * n + i]), and the density
//             summation + EOS of fluid targets (Eq. densum, Eq. eos).
//  k_density  on the other steps: Eq. densum + Eq. eos from the stored masks.
//  k_extrap   wall / rigid targets: extrapolation of pressure and velocity from the fluid
//             (Adami et al. 2012, cited in Sec. 3.3.4).
//  k_force    fluid / rigid targets: Eq. momentum, Eq. couplingforce, Eq. contactforce,
//             Eq. heat_equation.
// The sweeps stage batches of chunks (coalesced loads of packed records), and every lane
// walks the set bits of its own masks, so lanes stay busy however the hits are spread.
// Streams longer than the stored chunks (very dense groups) recompute the masks on the fly.
#pragma once
#include "sph_kernels.cuh"

namespace sph {

template <class R> __device__ __forceinline__ R qdiv(R a, R b);
template <> __device__ __forceinline__ double qdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// density, pressure and the packed records of a fluid particle (Eq. densum, Eq. eos)
template <class R>
__device__ __forceinline__ void fluid_density_out(const Scene<R>& S, int i, R wsum) {
  const MatR<R>& A = S.matR[S.P.mt[i]];
  R rho = S.P.m[i] * (S.w0 + S.sig_w * wsum);
  R p = A.c2 * (rho - A.rho0);
  S.P.rho[i] = rho;
  S.prs[i] = p;
  V4<R> r1, r2;
  r1.x = qdiv<R>(S.P.m[i], rho); r1.y = p; r1.z = rho; r1.w = S.P.T[i];
  r2.x = S.P.vx[i]; r2.y = S.P.vy[i]; r2.z = S.P.vz[i]; r2.w = R(-1);
  S.rec1[i] = r1;
  S.rec2[i] = r2;
}

// d = r_i - r_j.  FP64: absolute positions with the minimum image on periodic axes (the
// arithmetic of the oracle).  FP32: both positions are relative to the origin of the
// group's first cell (staged candidates are shifted into that frame when staged).
template <class R, int DIM>
__device__ __forceinline__ void pair_delta(const Scene<R>& S, const R* ti, const V4<R>& pj, R* d) {
  if (sizeof(R) == 8) {
    d[0] = dsub(ti[0], pj.x);
    d[1] = dsub(ti[1], pj.y);
    d[2] = DIM == 3 ? dsub(ti[2], pj.z) : R(0);
    for (int k = 0; k < DIM; k++)
      if (S.per[k]) {
        R h = R(0.5) * S.LR[k];
        if (d[k] > h) d[k] = dsub(d[k], S.LR[k]);
        else if (d[k] < -h) d[k] = dsub(d[k], -S.LR[k]);
      }
  } else {
    d[0] = ti[0] - pj.x;
    d[1] = ti[1] - pj.y;
    d[2] = DIM == 3 ? ti[2] - pj.z : R(0);
  }
}

// ---------------------------------------------------------------- candidate streams
template <class R> struct TileCap { static constexpr int v = sizeof(R) == 4 ? 192 : 96; };

template <class R>
struct TileSmem {
  V4<R> p[TileCap<R>::v], a[TileCap<R>::v], b[TileCap<R>::v];
  int sj[TileCap<R>::v];
  int cs[32], base[33];
};

template <class R, int DIM>
__device__ __forceinline__ int stencil_cells(const Group<R, DIM>& G) { return (G.ncx + 2) * 3 * (DIM == 3 ? 3 : 1); }

// stencil table of a group: first particle and stream offset of every stencil cell;
// returns the stream length
template <class R, int DIM>
__device__ __forceinline__ int build_stream(const Scene<R>& S, const Group<R, DIM>& G, TileSmem<R>& T, int lane) {
  int ncs = stencil_cells<R, DIM>(G);
  int cnt = 0, start = 0;
  if (lane < ncs) {
    int w = G.ncx + 2;
    int ox = lane % w - 1, dy = (lane / w) % 3 - 1, dz = DIM == 3 ? lane / (3 * w) - 1 : 0;
    int key;
    R sh[3];
    if (stencil_cell<R, DIM>(S, G, ox, dy, dz, key, sh)) {
      start = max(S.cstart[key], 0);
      cnt = max(min(S.cstart[key + 1], S.n) - start, 0);
    }
  }
  int x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  __syncwarp();
  if (lane < ncs) { T.cs[lane] = start; T.base[lane + 1] = x; }
  if (lane == 0) T.base[0] = 0;
  __syncwarp();
  return __shfl_sync(FULL, x, ncs - 1);
}

// stage stream positions [b0, b1) into slots 0..: records selected by WHAT (1 pos4, 2 rec1,
// 4 rec2).  FP32 positions are moved into the frame of the group's first cell.
template <class R, int DIM, int WHAT>
__device__ __forceinline__ void stage_batch(const Scene<R>& S, TileSmem<R>& T, int ncs, int w, int b0, int b1,
                                            int lane) {
  __syncwarp();
  for (int t = b0 + lane; t < b1; t += 32) {
    // stencil cell of stream position t (binary search over the cell offsets)
    int lo = 0, hi = ncs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (T.base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int j = T.cs[lo] + (t - T.base[lo]);
    int q = t - b0;
    T.sj[q] = j;
    if (WHAT & 1) {
      V4<R> pj = S.pos4[j];
      if (sizeof(R) == 4) {
        int ox = lo % w - 1, dy = (lo / w) % 3 - 1, dz = DIM == 3 ? lo / (3 * w) - 1 : 0;
        pj.x += (R)ox * S.ellR[0];
        pj.y += (R)dy * S.ellR[1];
        if (DIM == 3) pj.z += (R)dz * S.ellR[2];
      }
      T.p[q] = pj;
    }
    if (WHAT & 2) T.a[q] = S.rec1[j];
    if (WHAT & 4) T.b[q] = S.rec2[j];
  }
  __syncwarp();
}

// mask of the staged candidates q0..q0+nq-1 closer than sqrt(rad2) to the target, without
// the target itself (stream position tself)
template <class R, int DIM>
__device__ __forceinline__ unsigned test_chunk(const Scene<R>& S, const TileSmem<R>& T, int q0, int nq, int qself,
                                               const R* ti, R rad2) {
  unsigned m = 0u;
  for (int k = 0; k < nq; k++) {
    R d[3];
    pair_delta<R, DIM>(S, ti, T.p[q0 + k], d);
    R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
    if (r2 < rad2) m |= 1u << k;
  }
  int ks = qself - q0;
  if (ks >= 0 && ks < 32) m &= ~(1u << ks);
  return m;
}

template <class R, int DIM>
__device__ __forceinline__ int target_tx(const Scene<R>& S, const Group<R, DIM>& G, int i) {
  return G.ncx > 1 ? key_lin(S, S.key[i]) % S.ncell[0] - G.cx0 : 0;
}

// position of target i in the pair frame, and its own position in the candidate stream
template <class R, int DIM>
__device__ __forceinline__ int target_frame(const Scene<R>& S, const Group<R, DIM>& G, const TileSmem<R>& T, int i,
                                            R* ti) {
  int tx = target_tx(S, G, i);
  ti[0] = S.P.px[i]; ti[1] = S.P.py[i]; ti[2] = S.P.pz[i];
  if (sizeof(R) == 4) ti[0] += (R)tx * S.ellR[0];
  int w = G.ncx + 2;
  int own = (tx + 1) + w * (1 + (DIM == 3 ? 3 : 0));  // stencil cell (tx, 0, 0)
  return T.base[own] + (i - T.cs[own]);
}

// ---------------------------------------------------------------- search + density
template <class R, int DIM>
__global__ void __launch_bounds__(128) k_search(BatchView<R> B) {
  __shared__ TileSmem<R> T4[4];
  TileSmem<R>& T = T4[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  int total = __ldg(B.pfx_grp + B.nsc);
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < total; g += nw) {
    int s = find_scene(B.pfx_grp, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!rebin_now(S)) continue;  // masks of the last rebuild still hold (skin)
    Group<R, DIM> G = group_of<R, DIM>(S, g - __ldg(B.pfx_grp + s));
    int M = build_stream<R, DIM>(S, G, T, lane);
    int ncs = stencil_cells<R, DIM>(G);
    int w = G.ncx + 2;
    int nch = (M + 31) >> 5;
    for (int tb = G.ts; tb < G.te; tb += 32) {
      int i = tb + lane;
      bool valid = i < G.te;
      if (!__any_sync(FULL, valid)) continue;
      bool fluid = valid && S.matR[S.P.mt[i]].kind == KFLUID;
      R ti[3] = {R(0), R(0), R(0)};
      int qself = valid ? target_frame(S, G, T, i, ti) : -1;
      R acc = R(0);
      for (int c = 0; c < nch; c++) {
        int b0 = c * 32, b1 = min(M, b0 + 32);
        stage_batch<R, DIM, 1>(S, T, ncs, w, b0, b1, lane);
        unsigned m = valid ? test_chunk<R, DIM>(S, T, 0, b1 - b0, qself - b0, ti, S.rl2R) : 0u;
        if (valid && c < S.maxch) S.nbm[(size_t)c * S.n + i] = m;
        if (fluid) {
          while (m) {
            int k = __ffs(m) - 1;
            m &= m - 1;
            R d[3];
            pair_delta<R, DIM>(S, ti, T.p[k], d);
            R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
            if (r2 < S.rc2R) acc += quintic_w<R>(sqrt(r2) * S.inv_h);
          }
        }
      }
      if (fluid) fluid_density_out(S, i, acc);
    }
  }
}

// ---------------------------------------------------------------- generic tiled sweep
// Pol provides WHAT (records to stage), want(S, i), begin(S, i), pair(S, T, q, j, d, r2),
// end(S, i), flush(lane).
template <class R, int DIM, class Pol>
__device__ __forceinline__ void tiled_sweep(const Scene<R>& S, const Group<R, DIM>& G, TileSmem<R>& T, Pol& pol,
                                            int lane) {
  constexpr int CAP = TileCap<R>::v;
  constexpr int CPB = CAP / 32;  // chunks per batch
  int M = build_stream<R, DIM>(S, G, T, lane);
  int ncs = stencil_cells<R, DIM>(G);
  int w = G.ncx + 2;
  int nch = (M + 31) >> 5;
  for (int tb = G.ts; tb < G.te; tb += 32) {
    int i = tb + lane;
    bool valid = i < G.te;
    bool active = valid && pol.want(S, i);
    if (!__any_sync(FULL, active)) continue;
    R ti[3] = {R(0), R(0), R(0)};
    int qself = -1;
    if (active) {
      qself = target_frame(S, G, T, i, ti);
      pol.begin(S, i);
    }
    for (int c0 = 0; c0 < nch; c0 += CPB) {
      int nb = min(CPB, nch - c0);
      // stored masks of this batch (coalesced across the lanes)
      unsigned mk[CPB];
      unsigned any = 0u;
#pragma unroll
      for (int k = 0; k < CPB; k++) {
        mk[k] = 0u;
        int c = c0 + k;
        if (k < nb && active && c < S.maxch) mk[k] = __ldg(S.nbm + (size_t)c * S.n + i);
        any |= mk[k];
      }
      bool recompute = c0 + nb > S.maxch;  // chunks beyond the stored masks
      if (!__any_sync(FULL, any != 0u || (recompute && active))) continue;
      int b0 = c0 * 32, b1 = min(M, (c0 + nb) * 32);
      stage_batch<R, DIM, Pol::WHAT>(S, T, ncs, w, b0, b1, lane);
      if (recompute && active) {
#pragma unroll
        for (int k = 0; k < CPB; k++) {
          int c = c0 + k;
          if (k < nb && c >= S.maxch) {
            int q0 = k * 32;
            mk[k] = test_chunk<R, DIM>(S, T, q0, min(32, b1 - b0 - q0), qself - b0, ti, S.rl2R);
          }
        }
      }
      if (active) {
        // the batch's masks as 64-bit words (static indices only, so they stay in registers)
        constexpr int NW = (CPB + 1) / 2;
        unsigned long long mw[NW];
#pragma unroll
        for (int v = 0; v < NW; v++) {
          unsigned lo = mk[2 * v], hi = (2 * v + 1 < CPB) ? mk[2 * v + 1] : 0u;
          mw[v] = (unsigned long long)lo | ((unsigned long long)hi << 32);
        }
        while (true) {
          int q = -1;
#pragma unroll
          for (int v = 0; v < NW; v++)
            if (q < 0 && mw[v]) {
              q = v * 64 + __ffsll((long long)mw[v]) - 1;
              mw[v] &= mw[v] - 1;
            }
          if (q < 0) break;
          R d[3];
          pair_delta<R, DIM>(S, ti, T.p[q], d);
          R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
          if (r2 < S.rc2R) pol.pair(S, T, q, T.sj[q], d, r2);
        }
      }
    }
    if (active) pol.end(S, i);
  }
}

template <class R, int DIM, class Pol>
__device__ __forceinline__ void tiled_kernel_body(BatchView<R> B, Pol& pol, TileSmem<R>& T, bool on_rebuild,
                                                  bool off_rebuild) {
  int lane = threadIdx.x & 31;
  int total = __ldg(B.pfx_grp + B.nsc);
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < total; g += nw) {
    int s = find_scene(B.pfx_grp, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    bool rb = rebin_now(S);
    if ((rb && !on_rebuild) || (!rb && !off_rebuild)) continue;
    Group<R, DIM> G = group_of<R, DIM>(S, g - __ldg(B.pfx_grp + s));
    pol.pairs_scene = S.pairs;
    tiled_sweep<R, DIM>(S, G, T, pol, lane);
    pol.flush(lane);
  }
}

// ---------------------------------------------------------------- density on steps without rebuild
template <class R, int DIM>
struct DensityTile {
  static constexpr int WHAT = 1;
  unsigned long long* pairs_scene;
  R acc;
  __device__ bool want(const Scene<R>& S, int i) const { return S.matR[S.P.mt[i]].kind == KFLUID; }
  __device__ void begin(const Scene<R>&, int) { acc = R(0); }
  __device__ void pair(const Scene<R>& S, const TileSmem<R>&, int, int, const R*, R r2) {
    acc += quintic_w<R>(sqrt(r2) * S.inv_h);
  }
  __device__ void end(const Scene<R>& S, int i) { fluid_density_out(S, i, acc); }
  __device__ void flush(int) {}
};

template <class R, int DIM>
__global__ void __launch_bounds__(128) k_density(BatchView<R> B) {
  __shared__ TileSmem<R> T[4];
  DensityTile<R, DIM> pol;
  tiled_kernel_body<R, DIM>(B, pol, T[threadIdx.x >> 5], false, true);
}

// ---------------------------------------------------------------- extrapolation (walls, rigid)
template <class R, int DIM>
struct ExtrapTile {
  static constexpr int WHAT = 7;
  unsigned long long* pairs_scene;
  R S0, P0, Rv[3], U[3];
  __device__ bool want(const Scene<R>& S, int i) const { return S.matR[S.P.mt[i]].kind != KFLUID; }
  __device__ void begin(const Scene<R>&, int) {
    S0 = P0 = R(0);
    for (int q = 0; q < 3; q++) Rv[q] = U[q] = R(0);
  }
  __device__ void pair(const Scene<R>& S, const TileSmem<R>& T, int q, int, const R* d, R r2) {
    if (S.matR[(int)T.p[q].w].kind != KFLUID) return;
    R W = quintic_w<R>(sqrt(r2) * S.inv_h);
    V4<R> a = T.a[q], b = T.b[q];
    S0 += W;
    P0 += a.y * W;
    R rw = a.z * W;
    Rv[0] += rw * d[0]; Rv[1] += rw * d[1]; Rv[2] += rw * d[2];
    U[0] += b.x * W; U[1] += b.y * W; U[2] += b.z * W;
  }
  __device__ void end(const Scene<R>& S, int i) {
    int kind = S.matR[S.P.mt[i]].kind;
    R uw[3] = {S.P.vx[i], S.P.vy[i], S.P.vz[i]};  // prescribed wall / rigid velocity
    R pw, vw[3];
    if (S0 > R(0)) {
      R aw[3] = {R(0), R(0), R(0)};
      if (kind == KRIGID) { aw[0] = S.P.ax[i]; aw[1] = S.P.ay[i]; aw[2] = S.P.az[i]; }
      R ga = (S.gR[0] - aw[0]) * Rv[0] + (S.gR[1] - aw[1]) * Rv[1] + (S.gR[2] - aw[2]) * Rv[2];
      R inv = R(1) / S0;
      pw = (P0 + ga) * inv;
      for (int q = 0; q < 3; q++) vw[q] = R(2) * uw[q] - U[q] * inv;
    } else {
      pw = R(0);
      for (int q = 0; q < 3; q++) vw[q] = uw[q];
    }
    S.prs[i] = pw;
    S.vex[i] = vw[0]; S.vey[i] = vw[1]; S.vez[i] = vw[2];
    R rho = S.P.rho[i];
    V4<R> r1, r2;
    r1.x = qdiv<R>(S.P.m[i], rho); r1.y = pw; r1.z = rho; r1.w = S.P.T[i];
    r2.x = vw[0]; r2.y = vw[1]; r2.z = vw[2]; r2.w = (R)S.P.body[i];
    S.rec1[i] = r1;
    S.rec2[i] = r2;
  }
  __device__ void flush(int) {}
};

template <class R, int DIM>
__global__ void __launch_bounds__(128) k_extrap(BatchView<R> B) {
  __shared__ TileSmem<R> T[4];
  ExtrapTile<R, DIM> pol;
  tiled_kernel_body<R, DIM>(B, pol, T[threadIdx.x >> 5], true, true);
}

// ---------------------------------------------------------------- forces and heat
template <class R>
struct Target {
  int kind, body;
  const MatR<R>* M;
  R rho, p, V2, eta, kap, T;
  R u[3], ve[3];
};

template <class R, int DIM>
__device__ __forceinline__ void force_pair(const Scene<R>& S, const Target<R>& t, int j, int mj, const V4<R>& a,
                                           const V4<R>& b, const R* d, R r2, R* acc, R& heat) {
  // a = (V_j, p_j, rho_j, T_j), b = (velocity seen by fluid, body_j)
  const MatR<R>& Bm = S.matR[mj];
  int bk = Bm.kind;
  R inv_r = rsqrt_<R>(r2);
  R r = r2 * inv_r;
  R dW = S.sig_dw * quintic_dw<R>(r * S.inv_h);
  R ex = d[0] * inv_r, ey = d[1] * inv_r, ez = d[2] * inv_r;
  R Vj = a.x;
  // heat conduction (Cleary & Monaghan), walls Dirichlet (kappa_b = kappa_a) or adiabatic
  if (S.any_heat) {
    R Tb = a.w;
    if (!(bk == KWALL && isnan(Tb))) {
      R kb = bk == KWALL ? t.kap : Bm.kappa;
      R ks = t.kap + kb;
      R kab = ks > R(0) ? qdiv<R>(R(4) * t.kap * kb, ks) : R(0);
      heat += Vj * kab * (t.T - Tb) * inv_r * dW;
    }
  }
  R pj = a.y;
  if (t.kind == KFLUID) {
    R rhoj, etaj;
    if (bk == KFLUID) {
      rhoj = a.z;
      etaj = Bm.eta;
    } else {  // wall / rigid: inverse EOS of fluid i for the extrapolated pressure
      rhoj = t.M->rho0 * (pj * t.M->inv_p0 + R(1));
      etaj = t.eta;
    }
    R pt = qdiv<R>(rhoj * t.p + t.rho * pj, t.rho + rhoj);
    R es = t.eta + etaj;
    R et = es > R(0) ? qdiv<R>(R(2) * t.eta * etaj, es) : R(0);
    R coef = (t.V2 + Vj * Vj) * dW;
    R vis = et * inv_r;
    acc[0] += coef * (-pt * ex + vis * (t.u[0] - b.x));
    acc[1] += coef * (-pt * ey + vis * (t.u[1] - b.y));
    acc[2] += coef * (-pt * ez + vis * (t.u[2] - b.z));
  } else if (bk == KFLUID) {  // rigid target: -m_j a_jr seen from fluid particle j
    R rhoj = a.z;
    R rs = Bm.rho0 * (t.p * Bm.inv_p0 + R(1));
    R pt = qdiv<R>(rs * pj + rhoj * t.p, rhoj + rs);
    R coef = (Vj * Vj + t.V2) * dW;
    R vis = Bm.eta * inv_r;
    acc[0] -= coef * (pt * ex + vis * (b.x - t.ve[0]));
    acc[1] -= coef * (pt * ey + vis * (b.y - t.ve[1]));
    acc[2] -= coef * (pt * ez + vis * (b.z - t.ve[2]));
  } else if (bk == KWALL || (int)b.w != t.body) {
    if (r < S.dxR) {  // Eq. contactforce with tension cut-off, u_j the particle's own velocity
      R ev = ex * (t.u[0] - S.P.vx[j]) + ey * (t.u[1] - S.P.vy[j]) + ez * (t.u[2] - S.P.vz[j]);
      R fn = S.kcR * (r - S.dxR) + S.dcR * ev;
      R mn = fn < R(0) ? fn : R(0);
      acc[0] -= mn * ex; acc[1] -= mn * ey; acc[2] -= mn * ez;
    }
  }
}

template <class R, int DIM>
struct ForceTile {
  static constexpr int WHAT = 7;
  unsigned long long* pairs_scene;
  Target<R> t;
  R acc[3], heat;
  unsigned long long npairs;
  __device__ bool want(const Scene<R>& S, int i) const { return S.matR[S.P.mt[i]].kind != KWALL; }
  __device__ void begin(const Scene<R>& S, int i) {
    int tm = S.P.mt[i];
    t.kind = S.matR[tm].kind;
    t.body = S.P.body[i];
    t.M = &S.matR[tm];
    V4<R> own = S.rec1[i];
    t.rho = own.z;
    t.p = own.y;
    t.V2 = own.x * own.x;
    t.eta = t.M->eta;
    t.kap = t.M->kappa;
    t.T = S.P.T[i];
    t.u[0] = S.P.vx[i]; t.u[1] = S.P.vy[i]; t.u[2] = S.P.vz[i];
    t.ve[0] = S.vex[i]; t.ve[1] = S.vey[i]; t.ve[2] = S.vez[i];
    acc[0] = acc[1] = acc[2] = R(0);
    heat = R(0);
  }
  __device__ void pair(const Scene<R>& S, const TileSmem<R>& T, int q, int j, const R* d, R r2) {
    force_pair<R, DIM>(S, t, j, (int)T.p[q].w, T.a[q], T.b[q], d, r2, acc, heat);
    npairs++;
  }
  __device__ void end(const Scene<R>& S, int i) {
    int tm = S.P.mt[i];
    if (t.kind == KFLUID) {
      R im = R(1) / S.P.m[i];
      S.P.ax[i] = S.gR[0] + acc[0] * im;
      S.P.ay[i] = S.gR[1] + acc[1] * im;
      S.P.az[i] = S.gR[2] + acc[2] * im;
    } else {
      int sl = S.P.slot[i];
      S.fr[3 * sl] = acc[0];
      S.fr[3 * sl + 1] = acc[1];
      S.fr[3 * sl + 2] = acc[2];
    }
    R rate = heat / t.rho;  // c_p dT/dt = dH/dt
    if (S.has_source && S.mat[tm].src) {
      double x[3];
      abs_pos<R>(S, i, x);
      double tt = S.st[1] + S.st[0];
      int vz = S.dim - 1;
      double dd = 0.0;
      for (int q = 0; q < S.dim; q++)
        if (q != vz) {
          double c = x[q] - (S.src_x0[q] + S.src_v[q] * tt);
          dd += c * c;
        }
      if (S.src_ztop - x[vz] < S.src_depth)
        rate += (R)(S.src_Q * exp(-2.0 * dd / (S.src_r * S.src_r))) / t.rho;
    }
    S.dT[i] = t.M->enth ? rate : rate / t.M->cp;
  }
  __device__ void flush(int lane) {
    unsigned long long x = npairs;
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if (lane == 0 && x) atomicAdd(pairs_scene, x);
    npairs = 0;
  }
};

template <class R, int DIM>
__global__ void __launch_bounds__(128) k_force(BatchView<R> B) {
  __shared__ TileSmem<R> T[4];
  ForceTile<R, DIM> pol;
  pol.npairs = 0;
  tiled_kernel_body<R, DIM>(B, pol, T[threadIdx.x >> 5], true, true);
}

}  // namespace sph
