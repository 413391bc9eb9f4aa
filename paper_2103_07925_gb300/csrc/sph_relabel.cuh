// Reversible phase transitions (Sec. 3.6) at the end of a step, for all particles at once
// against T^{n+1}:
//   k_rl_flag      rigid above T_t melts (1), fluid below T_t solidifies (2)
//   k_rl_join      a solidifying particle joins the body of its nearest rigid, non-melting
//                  neighbour (ties: smaller body id, then smaller input index)
//   k_rl_hook/root the others form new bodies, one per connected component of the
//                  neighbour graph among themselves (union-find; the root of a component is
//                  its smallest sorted index, and the component is numbered by its smallest
//                  input index)
//   k_rl_number    new body ids K + rank in that order
//   k_rl_apply     relabel: materials, body ids, accelerations of melting particles
//   k_rl_slots*    regroup the rigid slots by body: unchanged bodies keep their order, changed
//                  bodies are sorted by input index
//   k_rl_bodies    mass quantities of changed bodies (k_body_mass), velocity correction
//                  u_k = u'_k + w_k x (r_k - r'_k), start state of new bodies
// Every kernel returns at once when no particle changed phase in this step.
#pragma once

namespace sph {

template <class R>
__device__ __forceinline__ bool relabel_now(const Scene<R>& S) {
  return S.has_transition && S.status[1] > 0 && S.status[ST_CAPACITY] == 0 && S.status[ST_HOOK_TIMEOUT] == 0;
}

// neighbours j (r < r_c) of particle i, from its list or a scan of its cells
template <class R, int DIM, class F>
__device__ __forceinline__ void for_each_neighbor(const Scene<R>& S, int i, F&& f) {
  R ti[3] = {S.P.px[i], S.P.py[i], S.P.pz[i]};
  auto visit = [&](int j, int code) {
    R d[3];
    list_delta<R, DIM>(S, ti, j, code, d);
    R r2 = pair_r2<R, DIM>(d[0], d[1], d[2]);
    if (r2 < S.rc2R) f(j, r2);
  };
  int cnt = S.nbc[i];
  if (cnt <= S.maxnb) {
    for (int k = 0; k < cnt; k++) {
      int e = S.nbl[nb_at(S.n, i, k)];
      visit(nb_j(e), nb_cd(e));
    }
  } else {
    scan_cells<R, DIM>(S, i, visit);
  }
}

template <class R>
__global__ void k_rl_flag(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!S.has_transition) continue;
    int i = g - __ldg(B.pfx_part + s);
    const MatD& M = S.mat[S.P.mt[i]];
    int f = 0;
    if (M.to >= 0) {  // temperature, or the concentration for phases that transition on it
      double v = M.tby == 1 ? (double)S.P.C[i] : (double)S.P.T[i];
      double vt = M.tby == 1 ? M.Ct : M.Tt;
      if (M.kind == KRIGID && v > vt) f = 1;
      else if (M.kind == KFLUID && v < vt) f = 2;
    }
    S.tloc[i] = f;
    if (f) atomicAdd(&S.status[1], 1);
  }
}

// squared distance of a join candidate, decided in FP64 on both paths (the FP64 path
// reuses its bit-exact pair distance; the FP32 path rebuilds absolute positions)
template <class R>
__device__ __forceinline__ double join_r2(const Scene<R>& S, int i, int j, R r2) {
  if constexpr (sizeof(R) == 8) {
    return (double)r2;
  } else {
    double xi[3], xj[3];
    abs_pos<R>(S, i, xi);
    abs_pos<R>(S, j, xj);
    double d[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < S.dim; q++) {
      d[q] = xi[q] - xj[q];
      if (S.per[q]) {
        if (d[q] > 0.5 * S.L[q]) d[q] -= S.L[q]; else if (d[q] < -0.5 * S.L[q]) d[q] += S.L[q];
      }
    }
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  }
}

template <class R, int DIM>
__global__ void k_rl_join(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    S.tkey[i] = -1;
    S.bucket[i] = -1;
    if (S.tloc[i] != 2) continue;
    double best = 0.0;
    int bk = -1, bo = 0x7fffffff;
    for_each_neighbor<R, DIM>(S, i, [&](int j, R r2R) {
      if (S.matR[S.P.mt[j]].kind != KRIGID || S.tloc[j] == 1) return;
      int kj = S.P.body[j], oj = S.P.orig[j];
      double r2 = join_r2<R>(S, i, j, r2R);
      if (bk < 0 || r2 < best || (r2 == best && (kj < bk || (kj == bk && oj < bo)))) {
        best = r2; bk = kj; bo = oj;
      }
    });
    S.tkey[i] = bk;
    if (bk < 0) {
      S.bucket[i] = i;  // union-find parent of a solidifying particle without a rigid neighbour
      S.aux[i] = 0x7fffffff;
      atomicAdd(&S.status[7], 1);
    }
  }
}

// retry cap of one union-find hook (CAS contention on a root); compile-time so that a test
// build can lower it and reach the timeout path without any fault
#ifndef SPH_RL_HOOK_TRIES
#define SPH_RL_HOOK_TRIES 1000000
#endif

__device__ __forceinline__ int uf_find(int* par, int x) {
  int p = ((volatile int*)par)[x];
  while (p != x) {
    int gp = ((volatile int*)par)[p];
    if (gp != p) ((volatile int*)par)[x] = gp;  // path halving (benign race)
    x = p;
    p = ((volatile int*)par)[x];
  }
  return x;
}

template <class R, int DIM>
__global__ void k_rl_hook(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S) || S.status[7] == 0) continue;
    int i = g - __ldg(B.pfx_part + s);
    if (S.bucket[i] < 0) continue;
    for_each_neighbor<R, DIM>(S, i, [&](int j, R) {
      if (j < i || S.bucket[j] < 0) return;
      // hook the larger root under the smaller one; only roots are rewritten.  Bounded
      // retries: a hook that still fails after SPH_RL_HOOK_TRIES attempts sets the scene's
      // timeout word, and the relabel of this step is not applied (SPH_ERR_TIMEOUT)
      bool done = false;
      for (int it = 0; it < SPH_RL_HOOK_TRIES && !done; it++) {
        int a = uf_find(S.bucket, i), b = uf_find(S.bucket, j);
        if (a == b) { done = true; break; }
        int hi = a > b ? a : b, lo = a > b ? b : a;
        done = atomicCAS(&S.bucket[hi], hi, lo) == hi;
      }
      if (!done) S.status[ST_HOOK_TIMEOUT] = 1;
    });
  }
}

template <class R>
__global__ void k_rl_root(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S) || S.status[7] == 0) continue;
    int i = g - __ldg(B.pfx_part + s);
    if (S.bucket[i] < 0) continue;
    int r = uf_find(S.bucket, i);
    atomicMin(&S.aux[r], S.P.orig[i]);
    if (r == i) {
      int c = atomicAdd(&S.status[8], 1);
      S.perm[c] = i;  // list of component roots (any order)
    }
  }
}

// new body ids: K + rank of the component's smallest input index (one block per scene)
template <class R>
__global__ void k_rl_number(BatchView<R> B) {
  for (int s = blockIdx.x; s < B.nsc; s += gridDim.x) {
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int C = S.status[8];
    int K = *S.K;
    if (K + C > S.Kcap) {
      if (threadIdx.x == 0) S.status[ST_CAPACITY] = 1;  // body capacity exceeded: no relabel this step
      continue;
    }
    for (int a = threadIdx.x; a < C; a += blockDim.x) {
      int ra = S.perm[a];
      int ka = S.aux[ra], rank = 0;
      for (int b = 0; b < C; b++) rank += S.aux[S.perm[b]] < ka;
      S.tkey[ra] = K + rank;  // the root carries the new body id
      S.bchg[K + rank] = 2;
    }
  }
}

template <class R>
__global__ void k_rl_apply(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    int f = S.tloc[i];
    if (f == 1) {  // melting: keeps its velocity, takes the rigid acceleration as a^n
      int k = S.P.body[i], sl = S.P.slot[i];
      double Rm[9], rr[3], t1[3], t2[3], t3[3];
      qrot(&S.bq[4 * k], Rm);
      mv(Rm, &S.rb[3 * sl], rr);
      cross(&S.bal[3 * k], rr, t1);
      cross(&S.bw[3 * k], rr, t2);
      cross(&S.bw[3 * k], t2, t3);
      S.P.ax[i] = (R)(S.ba[3 * k] + t1[0] + t3[0]);
      S.P.ay[i] = (R)(S.ba[3 * k + 1] + t1[1] + t3[1]);
      S.P.az[i] = (R)(S.ba[3 * k + 2] + t1[2] + t3[2]);
      S.bchg[k] = 1;
      S.P.mt[i] = S.mat[S.P.mt[i]].to;
      S.P.body[i] = -1;
      S.P.slot[i] = -1;
      if (S.tvf) {  // a new fluid particle starts with a~ = 0
        S.P.bx[i] = R(0); S.P.by[i] = R(0); S.P.bz[i] = R(0);
        S.P.tx[i] = R(0); S.P.ty[i] = R(0); S.P.tz[i] = R(0);
      }
      atomicAdd(&S.status[9], 1);
      S.status[10] = 1;
    } else if (f == 2) {
      int k = S.tkey[i];
      if (k < 0) k = S.tkey[uf_find(S.bucket, i)];
      else if (S.bchg[k] == 0) S.bchg[k] = 1;
      S.P.mt[i] = S.mat[S.P.mt[i]].to;
      S.P.body[i] = k;
      S.P.ax[i] = R(0); S.P.ay[i] = R(0); S.P.az[i] = R(0);
      atomicAdd(&S.status[9], 1);
      S.status[10] = 1;
    }
  }
}

// slot regrouping, 1: counts per body (one block per scene clears, then particles count)
template <class R>
__global__ void k_rl_slots_clear(BatchView<R> B) {
  for (int s = blockIdx.x; s < B.nsc; s += gridDim.x) {
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    for (int k = threadIdx.x; k < S.Kcap; k += blockDim.x) S.bcur[k] = 0;
  }
}

template <class R>
__global__ void k_rl_slots_count(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    if (S.matR[S.P.mt[i]].kind == KRIGID) atomicAdd(&S.bcur[S.P.body[i]], 1);
  }
}

// 2: new slot ranges (exclusive scan over bodies, one block per scene) into bst2 (start) and
// bst2 + Kcap (end); bcur becomes the fill cursor; K grows by the new bodies
template <class R>
__global__ void __launch_bounds__(1024) k_rl_slots_scan(BatchView<R> B) {
  __shared__ int wsum[32];
  __shared__ int carry;
  for (int s = blockIdx.x; s < B.nsc; s += gridDim.x) {
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int Knew = *S.K + S.status[8];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < Knew; base += 1024) {
      int k = base + threadIdx.x;
      int v = k < Knew ? S.bcur[k] : 0;
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
      if (k < Knew) {
        S.bst2[k] = excl;
        S.bst2[S.Kcap + k] = excl + v;
        S.bcur[k] = excl;
      }
      __syncthreads();
      if (threadIdx.x == 1023) carry = excl + v;
      __syncthreads();
    }
    if (threadIdx.x == 0) *S.K = Knew;
    __syncthreads();
  }
}

// 3: fill.  A body whose membership did not change keeps its slot order, shifted to its new
// range (offsets and slot forces move along); a changed or new body is filled unordered and
// sorted in step 4.
template <class R>
__global__ void k_rl_slots_fill(BatchView<R> B) {
  int total = __ldg(B.pfx_part + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_part, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int i = g - __ldg(B.pfx_part + s);
    if (S.matR[S.P.mt[i]].kind != KRIGID) continue;
    int k = S.P.body[i];
    if (S.bchg[k] == 0) {
      int old = S.P.slot[i];
      int sl = S.bst2[k] + (old - S.bstart[k]);
      S.slot_part[sl] = i;
      for (int q = 0; q < 3; q++) {
        S.rb2[3 * sl + q] = S.rb[3 * old + q];
        S.fr2[3 * sl + q] = S.fr[3 * old + q];
      }
    } else {
      S.perm[atomicAdd(&S.bcur[k], 1)] = i;
    }
  }
}

// 4: every changed body's slots in input-index order (the order the slots were first built
// in; the first slot is the unwrapping reference): one block per body, bitonic sort of
// (input index, particle) in shared memory up to kSortCap slots, a block-wide rank count
// above that
constexpr int kSortCap = 8192;

template <class R>
__device__ __forceinline__ void rl_place(const Scene<R>& S, int sl, int v) {
  int old = S.P.slot[v];
  S.slot_part[sl] = v;
  for (int q = 0; q < 3; q++) {
    // offsets of particles that were rigid before; a particle that was fluid in this
    // step carries no rigid force (its offset comes from the new mass quantities)
    S.rb2[3 * sl + q] = old >= 0 ? S.rb[3 * old + q] : 0.0;
    S.fr2[3 * sl + q] = old >= 0 ? S.fr[3 * old + q] : R(0);
  }
}

template <class R>
__global__ void __launch_bounds__(512) k_rl_slots_order(BatchView<R> B) {
  extern __shared__ int sm_sort[];
  int* key = sm_sort;
  int* val = sm_sort + kSortCap;
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int k = g - __ldg(B.pfx_body + s);
    if (k >= *S.K || S.bchg[k] == 0) continue;
    int a = S.bst2[k], cnt = S.bst2[S.Kcap + k] - a;
    if (cnt <= 0) continue;
    if (cnt <= kSortCap) {
      int p2 = 1;
      while (p2 < cnt) p2 <<= 1;
      for (int t = threadIdx.x; t < p2; t += blockDim.x) {
        int v = t < cnt ? S.perm[a + t] : -1;
        key[t] = t < cnt ? S.P.orig[v] : 0x7fffffff;
        val[t] = v;
      }
      __syncthreads();
      for (int w = 2; w <= p2; w <<= 1)
        for (int j = w >> 1; j > 0; j >>= 1) {
          for (int t = threadIdx.x; t < p2; t += blockDim.x) {
            int u = t ^ j;
            if (u > t) {
              bool up = (t & w) == 0;
              if ((key[t] > key[u]) == up) {
                int tk = key[t]; key[t] = key[u]; key[u] = tk;
                int tv = val[t]; val[t] = val[u]; val[u] = tv;
              }
            }
          }
          __syncthreads();
        }
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) rl_place(S, a + t, val[t]);
      __syncthreads();
    } else {
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int v = S.perm[a + t], ov = S.P.orig[v], rank = 0;
        for (int u = 0; u < cnt; u++) rank += S.P.orig[S.perm[a + u]] < ov;
        rl_place(S, a + rank, v);
      }
      __syncthreads();
    }
  }
}

// 5: adopt the new slots, offsets, slot forces and slot ranges
template <class R>
__global__ void k_rl_slots_adopt(BatchView<R> B) {
  int total = __ldg(B.pfx_slot + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_slot, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int sl = g - __ldg(B.pfx_slot + s);
    int K = *S.K;
    if (sl < K) {
      S.bstart[sl] = S.bst2[sl];
      S.bend[sl] = S.bst2[S.Kcap + sl];
    }
    if (K == 0 || sl >= S.bst2[S.Kcap + K - 1]) continue;
    int i = S.slot_part[sl];
    S.P.slot[i] = sl;
    for (int q = 0; q < 3; q++) {
      S.rb[3 * sl + q] = S.rb2[3 * sl + q];
      S.fr[3 * sl + q] = S.fr2[3 * sl + q];
    }
  }
}

// bodies before the mass quantities are rebuilt: remember the centre of changed bodies,
// start state of new bodies
template <class R>
__global__ void k_rl_bodies_pre(BatchView<R> B) {
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int k = g - __ldg(B.pfx_body + s);
    int c = S.bchg[k];
    if (c == 1) {
      for (int q = 0; q < 3; q++) S.bold[3 * k + q] = S.br[3 * k + q];
    } else if (c == 2) {
      S.bq[4 * k] = 1.0; S.bq[4 * k + 1] = 0.0; S.bq[4 * k + 2] = 0.0; S.bq[4 * k + 3] = 0.0;
      for (int q = 0; q < 3; q++) {
        S.bu[3 * k + q] = S.bw[3 * k + q] = S.ba[3 * k + q] = S.bal[3 * k + q] = 0.0;
        S.bf[3 * k + q] = S.bt[3 * k + q] = 0.0;
      }
    }
  }
}

// after k_body_mass: u_k = u'_k + w x (r_k - r'_k) for changed bodies, mass-weighted mean
// velocity for new ones (one block per body, slot order); clears the change marks
template <class R>
__global__ void __launch_bounds__(128) k_rl_bodies_post(BatchView<R> B) {
  __shared__ double red[4][128];
  int total = __ldg(B.pfx_body + B.nsc);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int s = find_scene(B.pfx_body, B.nsc, g);
    const Scene<R>& S = *B.sc[s];
    if (!relabel_now(S)) continue;
    int k = g - __ldg(B.pfx_body + s);
    int c = S.bchg[k];
    if (c == 2 && S.balive[k]) {
      double m = 0, mu[3] = {0, 0, 0};
      for (int sl = S.bstart[k] + threadIdx.x; sl < S.bend[k]; sl += blockDim.x) {
        int i = S.slot_part[sl];
        double mi = (double)S.P.m[i];
        m += mi;
        mu[0] += mi * (double)S.P.vx[i];
        mu[1] += mi * (double)S.P.vy[i];
        mu[2] += mi * (double)S.P.vz[i];
      }
      red[0][threadIdx.x] = m;
      for (int q = 0; q < 3; q++) red[1 + q][threadIdx.x] = mu[q];
      __syncthreads();
      for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
          for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) S.bu[3 * k + q] = red[1 + q][0] / red[0][0];
      __syncthreads();
    } else if (c == 1 && S.balive[k] && threadIdx.x == 0) {
      double dr[3] = {S.br[3 * k] - S.bold[3 * k], S.br[3 * k + 1] - S.bold[3 * k + 1],
                      S.br[3 * k + 2] - S.bold[3 * k + 2]};
      double cw[3];
      cross(&S.bw[3 * k], dr, cw);
      for (int q = 0; q < 3; q++) S.bu[3 * k + q] += cw[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) S.bchg[k] = 0;
    __syncthreads();
  }
}

}  // namespace sph
