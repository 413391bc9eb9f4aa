// The neighbour search and the three pair sweeps of a step.
//
//  k_search   on rebuild steps, one warp per target group: cell-list candidate tests
//             (staged in shared memory) and the neighbour list of every particle (index
//             and cell-offset code per entry, layout list[k * n + i] so that a warp of
//             consecutive targets reads one line per k; a wall particle lists its fluid
//             neighbours only, the only ones it reads).  A list holds every pair within
//             its radius r_c + skin and possibly a few just beyond it.
//  k_density  one thread per particle over its list: density summation + EOS of fluid
//             targets (Eq. densum, Eq. eos), and the packed records of every particle.
//  k_extrap   one thread per wall / rigid target over its list: extrapolation of pressure
//             and velocity from the fluid (Adami et al. 2012, cited in Sec. 3.3.4).
//  k_force    one thread per fluid / rigid target over its list: Eq. momentum,
//             Eq. couplingforce, Eq. contactforce, Eq. heat_equation.
// A target whose neighbour count exceeds the list capacity scans its 3^d cells directly
// (same predicate and order, so the result does not depend on the path taken).
#pragma once
#include <type_traits>
#include "sph_kernels.cuh"

namespace sph {

template <class R> __device__ __forceinline__ R qdiv(R a, R b);
template <> __device__ __forceinline__ double qdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// warp-aggregated add to a per-scene counter (one atomic per scene present in the warp)
__device__ __forceinline__ void warp_add(int s, unsigned long long v, unsigned long long* ptr) {
  unsigned pending = FULL;
  while (pending) {
    int leader = __ffs(pending) - 1;
    int cs = __shfl_sync(FULL, s, leader);
    unsigned long long x = s == cs ? v : 0ull;
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if ((int)(threadIdx.x & 31) == leader && x) atomicAdd(ptr, x);
    pending &= ~__ballot_sync(FULL, s == cs);
  }
}

// packed neighbour state of particle i (FP32 scenes), written where its density is final
template <class R>
__device__ __forceinline__ void write_pack(const Scene<R>& S, int i, R rho, R p, R vol, bool with_pos = true) {
  if constexpr (sizeof(R) == 4) {
    int mt = S.P.mt[i];
    if (with_pos)
      S.pa[i] = make_float4(S.P.px[i], S.P.py[i], S.P.pz[i], rho);
    else
      S.pa[i].w = rho;
    S.pb[i] = make_float4(S.P.vx[i], S.P.vy[i], S.P.vz[i], p);
    S.pv[i] = make_float2(vol, __int_as_float(mt | (S.matR[mt].kind << 16)));
    if (S.tvf || S.any_conc)
      S.pd[i] = make_float4(S.tvf ? S.P.tx[i] : 0.f, S.tvf ? S.P.ty[i] : 0.f, S.tvf ? S.P.tz[i] : 0.f,
                            S.any_conc ? S.P.C[i] : 0.f);
  }
}

// ---------------------------------------------------------------- neighbour search
// a list chunk filled as a shift register: the new entry enters at w
__device__ __forceinline__ void chunk_push(int4& b, int e) {
  b.x = b.y;
  b.y = b.z;
  b.z = b.w;
  b.w = e;
}
// a partly filled chunk (its last r entries at the end) moved to the front before it is stored
__device__ __forceinline__ void chunk_align(int4& b, int r) {
  if (r == 1) {
    b.x = b.w;
  } else if (r == 2) {
    b.x = b.z;
    b.y = b.w;
  } else if (r == 3) {
    b.x = b.y;
    b.y = b.z;
    b.z = b.w;
  }
}

template <class R, int DIM>
struct SearchPol {
  R *sx, *sy, *sz;     // staged candidates (see traverse)
  float4* s4;
  int* sox;
  int* scol;           // column offset of each staged candidate (see traverse)
  float *fx, *fy, *fz;    // FP32 copies of the staged positions (FP64 scenes)
  float tf[3];
  unsigned cmask;      // candidate kinds: a wall particle only ever reads its fluid neighbours
                       // (extrapolation of Sec. 3.3.4), the others read all
  bool active;
  int idx, tx, n, maxnb, cnt;
  int cox, cdy, cdz;
  int4* list;          // the target's list chunks (chunk q at list[q * n])
  int4 buf;            // the chunk being filled (entries cnt & ~3 .. cnt - 1)
  R tp[3];
  // a list may hold a few pairs just beyond its radius (the pre-test's margin): every sweep
  // decides r < r_c itself, so the exact per-pair test is skipped here
  static constexpr bool kExact = false;
  // the traversal stages each candidate's list entry relative to the group's first column
  // (see traverse) and hands a hit's entry to put()
  static constexpr bool kEntry = true;
  __device__ void stage(const Scene<R>& S, int j, int lane) {
    if constexpr (sizeof(R) == 4) {  // the packed position record: one 16-byte load
      float4 a = S.pa[j];
      sx[lane] = a.x; sy[lane] = a.y; sz[lane] = a.z;
    } else {
      sx[lane] = S.P.px[j]; sy[lane] = S.P.py[j]; sz[lane] = S.P.pz[j];
      fx[lane] = (float)sx[lane]; fy[lane] = (float)sy[lane]; fz[lane] = (float)sz[lane];
    }
  }
  // entries collect in a register chunk that is stored whole (16 bytes); entries past the
  // capacity are counted, not stored (the sweeps then scan the cells of that target)
  // the chunk is a shift register: each entry enters at w and moves the others down, so a
  // full chunk holds its four entries in order (measured 24 % faster search than writing
  // entry cnt & 3 in place, whose four-way select every hit paid)
  __device__ void put(int e) {
    chunk_push(buf, e);
    cnt++;
    if ((cnt & 3) == 0 && cnt <= maxnb) list[(size_t)((cnt >> 2) - 1) * n] = buf;
  }
  __device__ void pair(const Scene<R>&, int, int j, R, R, R, R) { put(nb_entry(j, nb_code(cox - tx, cdy, cdz))); }
  __device__ void flush() {
    chunk_align(buf, cnt & 3);
    if ((cnt & 3) != 0 && cnt <= maxnb) list[(size_t)(cnt >> 2) * n] = buf;
  }
};

// resident blocks of 128 threads per SM the search is compiled for (register budget; FP32:
// five, with four and six within 1 %, eight and ten slower)
#ifndef SPH_SEARCH_MIN_BLOCKS
#define SPH_SEARCH_MIN_BLOCKS 5
#endif
#ifndef SPH_SEARCH_MIN_BLOCKS_64
#define SPH_SEARCH_MIN_BLOCKS_64 6
#endif

template <class R, int DIM>
__global__ void __launch_bounds__(128, sizeof(R) == 8 ? SPH_SEARCH_MIN_BLOCKS_64 : SPH_SEARCH_MIN_BLOCKS)
    k_search(BatchView<R> B) {
  __shared__ R sm[4][3][32];
  __shared__ float smf[sizeof(R) == 8 ? 4 : 1][3][32];
  __shared__ float4 sm4[sizeof(R) == 4 ? 4 : 1][32];
  __shared__ int smo[4][32];
  __shared__ int smc[4][32];
  int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  SearchPol<R, DIM> pol;
  pol.sx = sm[wib][0]; pol.sy = sm[wib][1]; pol.sz = sm[wib][2];
  pol.s4 = sm4[sizeof(R) == 4 ? wib : 0];
  pol.sox = smo[wib];
  pol.scol = smc[wib];
  int wf = sizeof(R) == 8 ? wib : 0;
  pol.fx = smf[wf][0]; pol.fy = smf[wf][1]; pol.fz = smf[wf][2];
  int total = __ldg(B.pfx_grp + B.nsc);
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < total; g += nw) {
    int s = find_scene(B.pfx_grp, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!rebin_now(S)) continue;  // lists of the last rebuild still hold (skin)
    int gl = g - __ldg(B.pfx_grp + s);
    GroupIter<R, DIM> it(S, gl);
    Group<R, DIM> G;
    pol.n = S.n;
    pol.maxnb = S.maxnb;
    while (it.next(S, gl, lane, G))
    for (int tb = G.ts; tb < G.te; tb += 32) {
      int i = tb + lane;
      bool valid = i < G.te;
      pol.active = valid;
      if (!__any_sync(FULL, valid)) continue;
      pol.idx = valid ? i : -1;
      int tkind = valid ? S.matR[S.P.mt[i]].kind : G.cls;
      if (tkind != G.cls) S.status[3] = 1;  // a kind changed without a rebuild (never expected)
      pol.cmask = G.cls == KWALL ? 1u << KFLUID : (1u << NCLS) - 1u;
      pol.tx = 0;
      if (valid) {
        target_pos(S, i, G.cx0, pol.tp);
        if (G.ncx > 1) pol.tx = key_lin(S, S.key[i]) % S.ncell[0] - G.cx0;
      }
      pol.tf[0] = (float)pol.tp[0]; pol.tf[1] = (float)pol.tp[1]; pol.tf[2] = (float)pol.tp[2];
      pol.cnt = 0;
      pol.list = (int4*)S.nbl + (valid ? i : 0);
      traverse<R, DIM>(S, G, pol, lane, S.rl2R, S.rl2f);
      if (valid) {
        pol.flush();
        S.nbc[i] = pol.cnt;
      }
    }
  }
}

// ---------------------------------------------------------------- pair geometry from a list entry
// d = r_i - r_j: FP64 absolute positions with the minimum image on periodic axes (the same
// arithmetic as the cell traversal); FP32 cell-relative offsets minus the cell offset
template <class R, int DIM>
__device__ __forceinline__ void list_delta(const Scene<R>& S, const R* ti, int j, int code, R* d) {
  if (sizeof(R) == 8) {
    d[0] = dsub(ti[0], S.P.px[j]);
    d[1] = dsub(ti[1], S.P.py[j]);
    d[2] = DIM == 3 ? dsub(ti[2], S.P.pz[j]) : R(0);
    for (int k = 0; k < DIM; k++)
      if (S.per[k]) {
        R h = R(0.5) * S.LR[k];
        if (d[k] > h) d[k] = dsub(d[k], S.LR[k]);
        else if (d[k] < -h) d[k] = dsub(d[k], -S.LR[k]);
      }
  } else {
    d[0] = (ti[0] - S.P.px[j]) - (R)nb_o(code, 0) * S.ellR[0];
    d[1] = (ti[1] - S.P.py[j]) - (R)nb_o(code, 1) * S.ellR[1];
    d[2] = DIM == 3 ? (ti[2] - S.P.pz[j]) - (R)nb_o(code, 2) * S.ellR[2] : R(0);
  }
}

// the same offset from a packed FP32 neighbour record: the cell offset o ell of the entry's
// code is formed exactly (o in {-1, 0, 1} from its two bits, the product one of 0, +-ell),
// so the sum is rounded once, as above.  Decoded in registers: the sweeps are bound by
// their gathers through the L1 data pipe, which a table of the offsets loaded once per
// entry had loaded further (measured 2-4 % slower in each sweep)
template <int DIM>
__device__ __forceinline__ void pack_delta(const SweepK& K, const float* ti, float4 a, int code, float* d) {
  d[0] = (ti[0] - a.x) + nb_of(code, 0) * K.nell[0];
  d[1] = (ti[1] - a.y) + nb_of(code, 1) * K.nell[1];
  d[2] = DIM == 3 ? (ti[2] - a.z) + nb_of(code, 2) * K.nell[2] : 0.f;
}

// compensated FP32 sum (Kahan): the rounding error of each addition is carried into the
// next, so the sum of the positive kernel terms keeps about twice the working precision;
// sum() is the compensated value in FP64
struct KSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double sum() const { return (double)s - (double)c; }
};

// writer of particle i's in-range list (int4 chunks, see SweepK): entries collect in a
// register chunk (a shift register, as in the search) that is stored whole; more than cq
// entries (the capacity) mark the list as not kept (-1), and the force sweep then walks the
// full list itself
struct InRange {
  int4 buf;
  int m = 0;
  __device__ __forceinline__ void put(int4* nbq, size_t n, int i, int cq, int e) {
    chunk_push(buf, e);
    m++;
    if ((m & 3) == 0 && m <= cq) nbq[(size_t)((m >> 2) - 1) * n + i] = buf;
  }
  __device__ __forceinline__ int finish(int4* nbq, size_t n, int i, int cq) {
    chunk_align(buf, m & 3);
    if ((m & 3) != 0 && m <= cq) nbq[(size_t)(m >> 2) * n + i] = buf;
    return m <= cq ? m : -1;
  }
};
template <int DIM>
__device__ __forceinline__ void pack_delta(const Scene<float>& S, const float* ti, float4 a, int code, float* d) {
  pack_delta<DIM>(S.k, ti, a, code, d);
}

// the sweep constants of a launch: the kernel parameter (launches over one scene) or the
// scene descriptor's copy
template <bool ONE>
__device__ __forceinline__ const SweepK& sweep_k(const SweepK& kp, const SweepK& ks) {
  if constexpr (ONE) return kp;
  else return ks;
}

// scan of the 3^d cells around target i (targets whose list overflowed); calls
// f(j, code) for every candidate j != i of the kinds its list holds, in the order of the
// search's traversal (for_each_run)
template <class R, int DIM, class F>
__device__ __forceinline__ void scan_cells(const Scene<R>& S, int i, F&& f) {
  int cx, cy, cz;
  lin_xyz(S, key_lin(S, S.key[i]), cx, cy, cz);
  unsigned cm = S.key[i] / S.ncells == KWALL ? 1u << KFLUID : (1u << NCLS) - 1u;
  for_each_run<R, DIM>(S, cx, 1, cy, cz, cm, [&](int cs, int ce, int oxf, R, R, R, int dy, int dz, int, int, int) {
    int a = max(cs, 0), e = min(ce, S.n);
    for (int j = a; j < e; j++) {
      if (j == i) continue;
      int ox = oxf != kOxKey ? oxf : S.key[j] % S.ncell[0] - cx;
      f(j, nb_code(ox, dy, dz));
    }
  });
}

// ---------------------------------------------------------------- density on steps without rebuild
// Eq. densum + Eq. eos over the list, every step
// ONE: a launch over one scene, its sweep constants by value (kp)
template <class R, int DIM, bool ONE>
__global__ void __launch_bounds__(256, 4) k_density(BatchView<R> B, SweepK kp) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    int i = g - __ldg(B.pfx_part + s);
    const MatR<R>& A = S.matR[S.P.mt[i]];
    R rho = S.P.rho[i];
    if (A.kind == KFLUID) {
      R ti[3] = {S.P.px[i], S.P.py[i], S.P.pz[i]};
      R acc = R(0);
      KSum ks;  // FP32 scenes: the sum, compensated
      auto visit = [&](int j, int code) {
        R d[3];
        if constexpr (sizeof(R) == 4)
          pack_delta<DIM>(S, ti, S.pa[j], code, d);  // positions packed by the drift
        else
          list_delta<R, DIM>(S, ti, j, code, d);
        R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
        if (r2 < S.rc2R) {
          if constexpr (sizeof(R) == 4) ks.add(quintic_w<R>(pair_dist<R>(r2) * S.inv_h));
          else acc += quintic_w<R>(pair_dist<R>(r2) * S.inv_h);
        }
      };
      int cnt = S.nbc[i];
      if (cnt <= S.maxnb) {
        int k = 0;
        if constexpr (sizeof(R) == 4) {
          // one list chunk (four entries) at a time: the four position gathers are in flight
          // together (a latency-bound walk), the next chunk while they are summed; the sum
          // keeps the list order.  The entries inside the support are copied, in list order,
          // into the in-range list the force sweep of this evaluation walks.
          const SweepK& K = sweep_k<ONE>(kp, S.k);
          size_t n = K.n;
          const float4* pa = K.pa;
          const int4* L4 = (const int4*)K.nbl + i;
          InRange ir;
          const int cq = K.cq;
          int4 c = cnt > 0 ? __ldg(L4) : make_int4(0, 0, 0, 0);
          // the full chunks without a bound check per entry, then the partial last one (the
          // unchecked gathers schedule freely: 15 % faster sweep than a check on every entry)
          auto chunk = [&](int4 cc, int kk, auto tail) {
            constexpr bool kTail = decltype(tail)::value;
            int e[4] = {cc.x, cc.y, cc.z, cc.w};
            bool ok[4];
            float4 a[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
              ok[q] = !kTail || kk + q < cnt;
              a[q] = pa[ok[q] ? nb_j(e[q]) : i];
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
              if (!ok[q]) continue;
              R d[3];
              pack_delta<DIM>(K, ti, a[q], nb_cd(e[q]), d);
              R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
              if (r2 < S.rc2R) {
                ks.add(quintic_w<R>(pair_dist<R>(r2) * S.inv_h));
                ir.put((int4*)K.nbq, n, i, cq, e[q]);
              }
            }
          };
          const int full = cnt & ~3;
          for (; k < full; k += 4) {
            int4 cn = k + 4 < cnt ? __ldg(L4 + (size_t)((k >> 2) + 1) * n) : make_int4(0, 0, 0, 0);
            chunk(c, k, std::false_type{});
            c = cn;
          }
          if (k < cnt) {
            chunk(c, k, std::true_type{});
            k = cnt;
          }
          S.nbqc[i] = ir.finish((int4*)K.nbq, n, i, cq);
        }
        for (; k < cnt; k++) {
          int e = __ldg(S.nbl + nb_at(S.n, i, k));
          visit(nb_j(e), nb_cd(e));
        }
      } else {
        scan_cells<R, DIM>(S, i, visit);
        if constexpr (sizeof(R) == 4) S.nbqc[i] = -1;
      }
      if constexpr (sizeof(R) == 4) {
        // FP32 scenes: rho = m (W(0) + sum W) and p = c^2 (rho - rho0) in FP64 from the
        // compensated sum, so that the pressure, a small difference of large numbers, does
        // not carry the rounding of the stored density (Eq. eos)
        double rd = (double)S.P.m[i] * (S.w0d + S.sig_wd * ks.sum());
        const MatD& Ad = S.mat[S.P.mt[i]];
        rho = (R)rd;
        S.P.rho[i] = rho;
        S.prs[i] = (R)(Ad.c * Ad.c * (rd - Ad.rho0));
      } else {
        rho = S.P.m[i] * (S.w0 + S.sig_w * acc);
        S.P.rho[i] = rho;
        S.prs[i] = A.c2 * (rho - A.rho0);
      }
    }
    R vol = qdiv<R>(S.P.m[i], rho);
    S.vol[i] = vol;
    // the positions of the packed records (written by the drift, or by the permutation on
    // rebuild steps) are read by this sweep: write only the density
    write_pack<R>(S, i, rho, A.kind == KFLUID ? S.prs[i] : R(0), vol, false);
  }
}

// ---------------------------------------------------------------- extrapolation (walls, rigid)
// ONE: a launch over one scene, its sweep constants by value (kp).  A minimum of one block
// per SM leaves ptxas the registers it asks for (78-80 FP32, 90 FP64, no spills): 11 %
// faster than the 64 it chose without one, which spilled
template <class R, int DIM, bool ONE>
__global__ void __launch_bounds__(256, 1) k_extrap(BatchView<R> B, SweepK kp) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    // kind-major keys: the wall and rigid particles follow the fluid ones, from the start of
    // the rigid key range on
    int nf = S.cstart[S.ncells];  // fluid particles: sorted indices [0, nf)
    int i = nf + (g - __ldg(B.pfx_part + s));
    if (i >= S.n) continue;
    int kind = S.matR[S.P.mt[i]].kind;
    if (kind == KFLUID) continue;
    // a wall particle's list (and its cell scan) holds fluid neighbours only; a rigid
    // particle's holds all kinds and reads the fluid ones, told apart by their index
    bool wall = kind == KWALL;
    R ti[3] = {S.P.px[i], S.P.py[i], S.P.pz[i]};
    R S0 = R(0), P0 = R(0), Rv[3] = {R(0), R(0), R(0)}, U[3] = {R(0), R(0), R(0)};
    auto visit = [&](int j, int code) {
      if constexpr (sizeof(R) == 4) {
        if (!wall && j >= nf) return;
        float4 a = S.pa[j];
        R d[3];
        pack_delta<DIM>(S, ti, a, code, d);
        R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
        if (!(r2 < S.rc2R)) return;
        float4 b = S.pb[j];
        R W = quintic_w<R>(pair_dist<R>(r2) * S.inv_h);
        S0 += W;
        P0 += b.w * W;
        R rw = a.w * W;
        Rv[0] += rw * d[0]; Rv[1] += rw * d[1]; Rv[2] += rw * d[2];
        U[0] += b.x * W; U[1] += b.y * W; U[2] += b.z * W;
      } else {
        if (!wall && j >= nf) return;
        R d[3];
        list_delta<R, DIM>(S, ti, j, code, d);
        R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
        if (!(r2 < S.rc2R)) return;
        R W = quintic_w<R>(pair_dist<R>(r2) * S.inv_h);
        S0 += W;
        P0 += S.prs[j] * W;
        R rw = S.P.rho[j] * W;
        Rv[0] += rw * d[0]; Rv[1] += rw * d[1]; Rv[2] += rw * d[2];
        U[0] += S.P.vx[j] * W; U[1] += S.P.vy[j] * W; U[2] += S.P.vz[j] * W;
      }
    };
    int cnt = S.nbc[i];
    if (cnt <= S.maxnb) {
      int k = 0;
      if constexpr (sizeof(R) == 4) {
        // one list chunk (four entries) at a time, two entries with both their records in
        // flight together (a latency-bound walk); the sums keep the list order.  A rigid
        // target also copies every entry inside the support (all kinds), in list order, into
        // the in-range list of the force sweep.
        const SweepK& K = sweep_k<ONE>(kp, S.k);
        size_t n = K.n;
        const int4* L4 = (const int4*)K.nbl + i;
        InRange ir;
        const int cq = K.cq;
        int4 c = cnt > 0 ? __ldg(L4) : make_int4(0, 0, 0, 0);
        // full chunks without a bound check per entry, then the partial last one
        auto chunk = [&](int4 cc, int kk, auto tail) {
          constexpr bool kTail = decltype(tail)::value;
          int ec[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
          for (int h = 0; h < 4; h += 2) {
            int e[2] = {ec[h], ec[h + 1]};
            float4 a[2], b[2];
            bool fl[2], ok[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
              ok[q] = !kTail || kk + h + q < cnt;
              int j = ok[q] ? nb_j(e[q]) : i;
              a[q] = K.pa[j];
              b[q] = K.pb[j];
              fl[q] = wall || j < nf;
            }
#pragma unroll
            for (int q = 0; q < 2; q++) {
              if (!ok[q]) continue;
              R d[3];
              pack_delta<DIM>(K, ti, a[q], nb_cd(e[q]), d);
              R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
              if (r2 < S.rc2R) {
                if (!wall) ir.put((int4*)K.nbq, n, i, cq, e[q]);
                if (fl[q]) {
                  R W = quintic_w<R>(pair_dist<R>(r2) * S.inv_h);
                  S0 += W;
                  P0 += b[q].w * W;
                  R rw = a[q].w * W;
                  Rv[0] += rw * d[0]; Rv[1] += rw * d[1]; Rv[2] += rw * d[2];
                  U[0] += b[q].x * W; U[1] += b[q].y * W; U[2] += b[q].z * W;
                }
              }
            }
          }
        };
        const int full = cnt & ~3;
        for (; k < full; k += 4) {
          int4 cn = k + 4 < cnt ? __ldg(L4 + (size_t)((k >> 2) + 1) * n) : make_int4(0, 0, 0, 0);
          chunk(c, k, std::false_type{});
          c = cn;
        }
        if (k < cnt) {
          chunk(c, k, std::true_type{});
          k = cnt;
        }
        if (!wall) S.nbqc[i] = ir.finish((int4*)K.nbq, n, i, cq);
      }
      for (; k < cnt; k++) {
        int e = __ldg(S.nbl + nb_at(S.n, i, k));
        visit(nb_j(e), nb_cd(e));
      }
    } else {
      scan_cells<R, DIM>(S, i, visit);
      if constexpr (sizeof(R) == 4) S.nbqc[i] = -1;
    }
    R uw[3] = {S.P.vx[i], S.P.vy[i], S.P.vz[i]};  // prescribed wall / rigid velocity
    if (S0 > R(0)) {
      R aw[3] = {R(0), R(0), R(0)};
      if (kind == KRIGID) { aw[0] = S.P.ax[i]; aw[1] = S.P.ay[i]; aw[2] = S.P.az[i]; }
      R ga = (S.gR[0] - aw[0]) * Rv[0] + (S.gR[1] - aw[1]) * Rv[1] + (S.gR[2] - aw[2]) * Rv[2];
      // divide by the weight sum rather than multiply by its reciprocal: with only edge
      // neighbours the sum can be subnormal in FP32 and its reciprocal overflow, while each
      // quotient is a weighted mean bounded by the neighbours' values
      S.prs[i] = (P0 + ga) / S0;
      S.vex[i] = R(2) * uw[0] - U[0] / S0;
      S.vey[i] = R(2) * uw[1] - U[1] / S0;
      S.vez[i] = R(2) * uw[2] - U[2] / S0;
    } else {
      S.prs[i] = R(0);
      S.vex[i] = uw[0]; S.vey[i] = uw[1]; S.vez[i] = uw[2];
    }
    if constexpr (sizeof(R) == 4) S.pb[i] = make_float4(S.vex[i], S.vey[i], S.vez[i], S.prs[i]);
  }
}

// ---------------------------------------------------------------- forces and heat
template <class R>
struct Target {
  int i, kind, body, mi;  // index, kind, body id, material index
  const MatR<R>* M;
  R rho, p, V2, eta, kap, T;
  R u[3], ve[3];
  R tv[3];   // u~ - u (transport-velocity formulation)
  R bs[3];   // sum_j (V_i^2 + V_j^2) dW/dr e_ij of the background acceleration
  R C, D;    // concentration and diffusivity
  R cs;      // sum_j V_j D_ij (C_i - C_j) / r dW/dr
};

template <class R, int DIM, bool TVF>
__device__ __forceinline__ void force_pair(const Scene<R>& S, Target<R>& t, int j, const R* d, R r2,
                                           R* acc, R& heat) {
  int mj = S.P.mt[j];
  const MatR<R>& Bm = S.matR[mj];
  int bk = Bm.kind;
  R inv_r = rsqrt_<R>(r2);
  R r = r2 * inv_r;
  R dW = S.sig_dw * quintic_dw<R>(r * S.inv_h);
  R ex = d[0] * inv_r, ey = d[1] * inv_r, ez = d[2] * inv_r;
  R Vj = S.vol[j];
  // heat conduction (Cleary & Monaghan), walls Dirichlet (kappa_b = kappa_a) or adiabatic;
  // the pair mean 4 kappa_a kappa_b / (kappa_a + kappa_b) from the material-pair table
  if (S.any_heat) {
    R Tb = S.P.T[j];
    if (!(bk == KWALL && isnan(Tb))) {
      R kab = (R)S.kap_ab[t.mi][bk == KWALL ? t.mi : mj];
      heat += Vj * kab * (t.T - Tb) * inv_r * dW;
    }
  }
  if (TVF && S.any_conc && bk != KWALL) {  // concentration: the heat form with the diffusivity
    R Db = Bm.D, Ds = t.D + Db;
    R Dab = Ds > R(0) ? qdiv<R>(R(4) * t.D * Db, Ds) : R(0);
    t.cs += Vj * Dab * (t.C - S.P.C[j]) * inv_r * dW;
  }
  if (t.kind == KFLUID) {
    R rhoj, pj, etaj, uj[3];
    pj = S.prs[j];
    if (bk == KFLUID) {
      rhoj = S.P.rho[j];
      etaj = Bm.eta;
      uj[0] = S.P.vx[j]; uj[1] = S.P.vy[j]; uj[2] = S.P.vz[j];
    } else {  // wall / rigid: inverse EOS of fluid i for the extrapolated pressure
      rhoj = t.M->rho0 * (pj * t.M->inv_p0 + R(1));
      etaj = t.eta;
      uj[0] = S.vex[j]; uj[1] = S.vey[j]; uj[2] = S.vez[j];
    }
    R pt = qdiv<R>(rhoj * t.p + t.rho * pj, t.rho + rhoj);
    (void)etaj;  // eta_j = eta_i for boundaries: the table's diagonal
    R et = (R)S.eta_ab[t.mi][bk == KFLUID ? mj : t.mi];
    R coef = (t.V2 + Vj * Vj) * dW;
    R vis = et * inv_r;
    acc[0] += coef * (-pt * ex + vis * (t.u[0] - uj[0]));
    acc[1] += coef * (-pt * ey + vis * (t.u[1] - uj[1]));
    acc[2] += coef * (-pt * ez + vis * (t.u[2] - uj[2]));
    if (TVF && S.tvf) {  // 1/2 (A_i + A_j) . e_ij with A = rho u (u~ - u), zero for boundaries
      R si = t.tv[0] * ex + t.tv[1] * ey + t.tv[2] * ez;
      R sj = bk == KFLUID ? S.P.tx[j] * ex + S.P.ty[j] * ey + S.P.tz[j] * ez : R(0);
      R rj = bk == KFLUID ? rhoj : R(0);
      acc[0] += coef * R(0.5) * (t.rho * t.u[0] * si + rj * uj[0] * sj);
      acc[1] += coef * R(0.5) * (t.rho * t.u[1] * si + rj * uj[1] * sj);
      acc[2] += coef * R(0.5) * (t.rho * t.u[2] * si + rj * uj[2] * sj);
      t.bs[0] += coef * ex; t.bs[1] += coef * ey; t.bs[2] += coef * ez;
    }
  } else if (bk == KFLUID) {  // rigid target: -m_j a_jr seen from fluid particle j
    R rhoj = S.P.rho[j], pj = S.prs[j];
    R rs = Bm.rho0 * (t.p * Bm.inv_p0 + R(1));
    R pt = qdiv<R>(rs * pj + rhoj * t.p, rhoj + rs);
    R coef = (Vj * Vj + t.V2) * dW;
    R vis = Bm.eta * inv_r;
    acc[0] -= coef * (pt * ex + vis * (S.P.vx[j] - t.ve[0]));
    acc[1] -= coef * (pt * ey + vis * (S.P.vy[j] - t.ve[1]));
    acc[2] -= coef * (pt * ez + vis * (S.P.vz[j] - t.ve[2]));
    if (TVF && S.tvf) {  // the A_j term of a_jr (A = 0 for the rigid particle)
      R sj = S.P.tx[j] * ex + S.P.ty[j] * ey + S.P.tz[j] * ez;
      acc[0] += coef * R(0.5) * rhoj * S.P.vx[j] * sj;
      acc[1] += coef * R(0.5) * rhoj * S.P.vy[j] * sj;
      acc[2] += coef * R(0.5) * rhoj * S.P.vz[j] * sj;
    }
  } else if (bk == KWALL || S.P.body[j] != t.body) {
    if (r < S.dxR) {  // Eq. contactforce with tension cut-off
      R ev = ex * (t.u[0] - S.P.vx[j]) + ey * (t.u[1] - S.P.vy[j]) + ez * (t.u[2] - S.P.vz[j]);
      R fn = S.kcR * (r - S.dxR) + S.dcR * ev;
      R mn = fn < R(0) ? fn : R(0);
      acc[0] -= mn * ex; acc[1] -= mn * ey; acc[2] -= mn * ez;
    }
  }
}

// force_pair on packed FP32 neighbour records (same arithmetic in the same order)
template <int DIM, bool TVF>
__device__ __forceinline__ void force_pair_packed(const Scene<float>& S, const SweepK& K, Target<float>& t, int j,
                                                  const float* d, float r2, float4 a, float4 b, float2 c, float* acc,
                                                  float& heat) {
  int mk = __float_as_int(c.y);
  int bk = mk >> 16;
  int mj = mk & 0xffff;
  bool same = mj == t.mi;  // the material constants of a pair of one material are the target's
  float inv_r = rsqrt_<float>(r2);
  float r = r2 * inv_r;
  float dW = K.sig_dw * quintic_dw<float>(r * K.inv_h);
  float ex = d[0] * inv_r, ey = d[1] * inv_r, ez = d[2] * inv_r;
  float Vj = c.x;
  if (K.any_heat) {
    float Tb = S.P.T[j];
    if (!(bk == KWALL && isnan(Tb))) {
      float kb = bk == KWALL || same ? t.kap : S.matR[mj].kappa;
      float ks = t.kap + kb;
      float kab = ks > 0.f ? qdiv<float>(4.f * t.kap * kb, ks) : 0.f;
      heat += Vj * kab * (t.T - Tb) * inv_r * dW;
    }
  }
  if (TVF && K.any_conc && bk != KWALL) {  // concentration: the heat form with the diffusivity
    float Db = same ? t.D : S.matR[mj].D, Ds = t.D + Db;
    float Dab = Ds > 0.f ? qdiv<float>(4.f * t.D * Db, Ds) : 0.f;
    t.cs += Vj * Dab * (t.C - K.pd[j].w) * inv_r * dW;
  }
  if (t.kind == KFLUID) {
    float rhoj, pj = b.w, etaj;
    if (bk == KFLUID) {
      rhoj = a.w;
      etaj = same ? t.eta : S.matR[mj].eta;
    } else {  // wall / rigid: inverse EOS of fluid i for the extrapolated pressure
      rhoj = t.M->rho0 * (pj * t.M->inv_p0 + 1.f);
      etaj = t.eta;
    }
    float pt = qdiv<float>(rhoj * t.p + t.rho * pj, t.rho + rhoj);
    float et;  // 2 eta_i eta_j / (eta_i + eta_j): eta itself for a pair of one material
    if (same || bk != KFLUID) {
      et = t.eta;
    } else {
      float es = t.eta + etaj;
      et = es > 0.f ? qdiv<float>(2.f * t.eta * etaj, es) : 0.f;
    }
    float coef = (t.V2 + Vj * Vj) * dW;
    float vis = et * inv_r;
    acc[0] += coef * (-pt * ex + vis * (t.u[0] - b.x));
    acc[1] += coef * (-pt * ey + vis * (t.u[1] - b.y));
    acc[2] += coef * (-pt * ez + vis * (t.u[2] - b.z));
    if (TVF && K.tvf) {  // 1/2 (A_i + A_j) . e_ij with A = rho u (u~ - u), zero for boundaries
      float si = t.tv[0] * ex + t.tv[1] * ey + t.tv[2] * ez, sj = 0.f, rj = 0.f;
      if (bk == KFLUID) {
        float4 w = K.pd[j];
        sj = w.x * ex + w.y * ey + w.z * ez;
        rj = rhoj;
      }
      acc[0] += coef * 0.5f * (t.rho * t.u[0] * si + rj * b.x * sj);
      acc[1] += coef * 0.5f * (t.rho * t.u[1] * si + rj * b.y * sj);
      acc[2] += coef * 0.5f * (t.rho * t.u[2] * si + rj * b.z * sj);
      t.bs[0] += coef * ex; t.bs[1] += coef * ey; t.bs[2] += coef * ez;
    }
  } else if (bk == KFLUID) {  // rigid target: -m_j a_jr seen from fluid particle j
    const MatR<float>& Bm = S.matR[mj];
    float rhoj = a.w, pj = b.w;
    float rs = Bm.rho0 * (t.p * Bm.inv_p0 + 1.f);
    float pt = qdiv<float>(rs * pj + rhoj * t.p, rhoj + rs);
    float coef = (Vj * Vj + t.V2) * dW;
    float vis = Bm.eta * inv_r;
    float ve[3] = {S.vex[t.i], S.vey[t.i], S.vez[t.i]};
    acc[0] -= coef * (pt * ex + vis * (b.x - ve[0]));
    acc[1] -= coef * (pt * ey + vis * (b.y - ve[1]));
    acc[2] -= coef * (pt * ez + vis * (b.z - ve[2]));
    if (TVF && K.tvf) {  // the A_j term of a_jr (A = 0 for the rigid particle)
      float4 w = K.pd[j];
      float sj = w.x * ex + w.y * ey + w.z * ez;
      acc[0] += coef * 0.5f * rhoj * b.x * sj;
      acc[1] += coef * 0.5f * rhoj * b.y * sj;
      acc[2] += coef * 0.5f * rhoj * b.z * sj;
    }
  } else if (bk == KWALL || S.P.body[j] != t.body) {
    if (r < K.dx) {  // Eq. contactforce with tension cut-off (particle velocities, not v_w)
      float ev = ex * (t.u[0] - S.P.vx[j]) + ey * (t.u[1] - S.P.vy[j]) + ez * (t.u[2] - S.P.vz[j]);
      float fn = K.kc * (r - K.dx) + K.dc * ev;
      float mn = fn < 0.f ? fn : 0.f;
      acc[0] -= mn * ex; acc[1] -= mn * ey; acc[2] -= mn * ez;
    }
  }
}

// resident blocks per SM the force sweep is compiled for (register budget)
#ifndef SPH_FORCE_MIN_BLOCKS
#define SPH_FORCE_MIN_BLOCKS 4
#endif

// TVF: instantiation with the transport-velocity and concentration terms (launched when
// a resident scene uses either; the plain instantiation keeps its register budget).
// ONE: a launch over a single scene, whose sweep constants kp come as a kernel parameter.
template <class R, int DIM, bool TVF, bool ONE>
__global__ void __launch_bounds__(256, TVF ? 3 : SPH_FORCE_MIN_BLOCKS) k_force(BatchView<R> B, SweepK kp) {
  int total = __ldg(B.pfx_part + B.nsc);
  int nthr = gridDim.x * blockDim.x;
  // uniform trip count so that the warp-wide pair counter sees every lane
  for (int g0 = blockIdx.x * blockDim.x; g0 < total; g0 += nthr) {
    int g = g0 + threadIdx.x;
    int s = find_scene(B.pfx_part, B.nsc, min(g, total - 1));
    const Scene<R>& S = *B.sc[s];
    unsigned long long npairs = 0;
    int i = g - __ldg(B.pfx_part + s);
    int tm = g < total ? S.P.mt[i] : 0;
    int kind = S.matR[tm].kind;
    // each instantiation takes the scenes of its own kind, so a scene's arithmetic does not
    // depend on the other scenes of a batch
    bool mine = TVF == (S.tvf != 0 || S.any_conc != 0);
    if (g < total && kind != KWALL && mine) {
      Target<R> t;
      t.i = i;
      t.kind = kind;
      t.mi = tm;
      t.body = S.P.body[i];
      t.M = &S.matR[tm];
      t.rho = S.P.rho[i];
      t.p = S.prs[i];
      R V = S.vol[i];
      t.V2 = V * V;
      t.eta = t.M->eta;
      t.kap = t.M->kappa;
      t.T = S.P.T[i];
      t.u[0] = S.P.vx[i]; t.u[1] = S.P.vy[i]; t.u[2] = S.P.vz[i];
      if constexpr (sizeof(R) == 8) { t.ve[0] = S.vex[i]; t.ve[1] = S.vey[i]; t.ve[2] = S.vez[i]; }
      t.tv[0] = t.tv[1] = t.tv[2] = R(0);
      t.bs[0] = t.bs[1] = t.bs[2] = R(0);
      if (TVF && S.tvf && kind == KFLUID) { t.tv[0] = S.P.tx[i]; t.tv[1] = S.P.ty[i]; t.tv[2] = S.P.tz[i]; }
      t.C = t.D = t.cs = R(0);
      if (TVF && S.any_conc) { t.C = S.P.C[i]; t.D = t.M->D; }
      R ti[3] = {S.P.px[i], S.P.py[i], S.P.pz[i]};
      R acc[3] = {R(0), R(0), R(0)}, heat = R(0);
      const SweepK& K = sweep_k<ONE>(kp, S.k);
      auto visit = [&](int j, int code) {
        if constexpr (sizeof(R) == 4) {
          float4 a = K.pa[j];
          R d[3];
          pack_delta<DIM>(K, ti, a, code, d);
          R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
          if (r2 < K.rc2) {
            float4 b = K.pb[j];
            float2 c = K.pv[j];
            force_pair_packed<DIM, TVF>(S, K, t, j, d, r2, a, b, c, acc, heat);
            npairs++;
          }
        } else {
          R d[3];
          list_delta<R, DIM>(S, ti, j, code, d);
          R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
          if (r2 < S.rc2R) {
            force_pair<R, DIM, TVF>(S, t, j, d, r2, acc, heat);
            npairs++;
          }
        }
      };
      int cnt = S.nbc[i];
      int cin = -1;
      if constexpr (sizeof(R) == 4) cin = __ldg(K.nbqc + i);
      if (cin >= 0) {
        if constexpr (sizeof(R) == 4) {
          // the in-range list of this evaluation (every entry inside the support, in list
          // order): no distance test, every lane has a pair at every entry but the last few;
          // four entries per load, the next four loaded while these are evaluated
          const int4* Q = K.nbq + i;
          int4 cur = cin > 0 ? __ldg(Q) : make_int4(0, 0, 0, 0);
          // full chunks without a bound check per entry, then the partial last one
          auto chunk = [&](int4 cc, int mm, auto tail) {
            constexpr bool kTail = decltype(tail)::value;
            int ee[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int u = 0; u < 4; u++) {
              if (!kTail || mm + u < cin) {
                int e = ee[u], j = nb_j(e);
                float4 a = K.pa[j], b = K.pb[j];
                float2 c = K.pv[j];
                float d[3];
                pack_delta<DIM>(K, ti, a, nb_cd(e), d);
                float r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
                force_pair_packed<DIM, TVF>(S, K, t, j, d, r2, a, b, c, acc, heat);
              }
            }
          };
          const int full = cin & ~3;
          int m = 0;
          for (; m < full; m += 4) {
            int4 nxt = m + 4 < cin ? __ldg(Q + (size_t)((m >> 2) + 1) * K.n) : make_int4(0, 0, 0, 0);
            chunk(cur, m, std::false_type{});
            cur = nxt;
          }
          if (m < cin) chunk(cur, m, std::true_type{});
          npairs += (unsigned long long)cin;
        }
      } else if (cnt <= S.maxnb) {
        int k = 0;
        if constexpr (sizeof(R) == 4) {
          // software pipeline: the next list entry is loaded while this pair is evaluated; the
          // velocity and material records only for pairs inside the support (measured faster
          // than loading them with the position, before the distance test)
          int e = k < cnt ? __ldg(K.nbl + nb_at(K.n, i, k)) : 0;
          for (; k < cnt; k++) {
            int en = k + 1 < cnt ? __ldg(K.nbl + nb_at(K.n, i, k + 1)) : 0;
            int j = nb_j(e);
            float4 a = K.pa[j];
            float d[3];
            pack_delta<DIM>(K, ti, a, nb_cd(e), d);
            float r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
            if (r2 < K.rc2) {
              float4 b = K.pb[j];
              float2 c = K.pv[j];
              force_pair_packed<DIM, TVF>(S, K, t, j, d, r2, a, b, c, acc, heat);
              npairs++;
            }
            e = en;
          }
        }
        for (; k < cnt; k++) {
          int e = __ldg(S.nbl + nb_at(S.n, i, k));
          visit(nb_j(e), nb_cd(e));
        }
      } else {
        scan_cells<R, DIM>(S, i, visit);
      }
      if (kind == KFLUID) {
        R im = R(1) / S.P.m[i];
        S.P.ax[i] = S.gR[0] + acc[0] * im;
        S.P.ay[i] = S.gR[1] + acc[1] * im;
        S.P.az[i] = S.gR[2] + acc[2] * im;
        if (TVF && S.tvf) {  // a~_i = -(p_b / m_i) sum_j (V_i^2 + V_j^2) dW/dr e_ij
          R c = -S.pbgR * im;
          S.P.bx[i] = c * t.bs[0]; S.P.by[i] = c * t.bs[1]; S.P.bz[i] = c * t.bs[2];
        }
      } else {
        int sl = S.P.slot[i];
        S.fr[3 * sl] = acc[0];
        S.fr[3 * sl + 1] = acc[1];
        S.fr[3 * sl + 2] = acc[2];
      }
      if (TVF && S.any_conc) S.dC[i] = t.cs / t.rho;
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
    warp_add(s, npairs, S.pairs);
  }
}

}  // namespace sph
