// Device-side data layout of libsph.
//
// A scene lives in device memory as a Scene<R> descriptor (R = double for the FP64 path,
// float for the FP32 path) that holds constants and pointers to structure-of-arrays
// particle fields.  Particle arrays are kept sorted by cell key (Sec. 3.2: cells of edge
// >= r_c); each rebin permutes them into the second bank and a one-thread kernel swaps
// the banks, so a captured CUDA graph can replay every step with fixed arguments.
//
// FP64 scenes store absolute positions.  FP32 scenes store positions relative to the
// origin of the particle's current cell, so that a pair distance is formed from small
// numbers: d = (o_i - o_j) - (c_j - c_i) * edge.
//
// Kernels address many scenes at once (batches): every launch walks a global item space
// (particles, cells, bodies, warp groups) and finds the scene of an item by binary search
// in a prefix table.  A single scene is a batch of one.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

constexpr int MAXMAT = 16;
enum { KFLUID = 0, KRIGID = 1, KWALL = 2 };
constexpr int NCLS = 3;  // key classes: the particle kinds, in this order

struct MatD {  // material constants, FP64
  int kind, to, enth, src;
  double rho0, c, eta, cp, kappa, Tt, L, w, p0;
  int tby;              // transition driven by 0 temperature, 1 concentration
  double D, Ct, Cfix;   // diffusivity, transition concentration, fixed concentration (NaN: free)
};

template <class R>
struct MatR {  // material constants in the working precision (pair sums)
  int kind, enth;
  R rho0, c2, eta, cp, kappa, inv_p0;
  R D;                  // diffusivity of the concentration
};

template <class R>
struct PBank {  // particle fields (one bank)
  R *px, *py, *pz;     // position (FP64: absolute; FP32: relative to the cell origin)
  R *vx, *vy, *vz;     // velocity (fluid u, rigid u_r, wall prescribed velocity)
  R *ax, *ay, *az;     // fluid acceleration; rigid: kinematic acceleration used by Eq. R4
  R *rho, *T, *H, *m;  // density, temperature (walls: prescribed or NaN), enthalpy, mass
  int *mt, *body, *slot, *orig;  // material, body id, rigid slot, input index
  // transport-velocity formulation (null when off): background acceleration a~ of the
  // last evaluation and u~ - u of the current half step
  R *bx, *by, *bz, *tx, *ty, *tz;
  R* C;                 // concentration (null when no phase carries one)
};

// What the FP32 pair sweeps read for every list entry, besides the neighbour records: a
// copy lives in the scene descriptor, and launches over a single scene also take it by value
// (kernel parameters are read from the constant bank: no cache traffic and no registers to
// hold them across the list walk).  Nothing in it changes after the scene is created.
struct SweepK {
  const float4 *pa, *pb, *pd;       // packed neighbour records (pd: TVF / concentration)
  const float2* pv;                 // (V, material | kind << 16) of every particle
  const int* nbl;                   // neighbour lists, entry k of particle i at nbl[nb_at(n, i, k)]
  // the in-range part of each fluid or rigid particle's list (r < r_c at this evaluation, in
  // list order), written by the density / extrapolation sweep: entries 4q .. 4q + 3 of
  // particle i in nbq[q * n + i]; nbqc[i] entries, or -1 when they did not fit (cq)
  const int4* nbq;
  const int* nbqc;
  int cq;
  int n;
  float ell[3];                     // cell edges (positions are relative to the cell origin)
  float nell[3];                    // -ell: the cell offset of an entry is nb_of(code) nell
  float rc2, sig_dw, inv_h;         // r_c^2, dW/dr = sig_dw w'(r / h)
  float dx, kc, dc;                 // contact: cut-off distance, spring and damper
  int any_heat, any_conc, tvf;
};

template <class R>
struct Scene {
  // ---------------------------------------------------------------- constants
  int dim, n, nmat, key_order, G;
  int win;             // row-major keys searched in windows of 32 consecutive particles
  int ncell[3], ncells, ngroups, ngx, ncblk;
  int nkey;             // key space: NCLS classes (particle kinds) x ncells cells
  int per[3];
  double lo[3], hi[3], L[3], ell[3];
  R ellR[3], LR[3];
  double g[3];
  R gR[3];
  double h, rc, rc2, dx, skin;
  R rc2R, rl2R, inv_h, sig_w, sig_dw, w0;  // W = sig_w w(q), dW/dr = sig_dw w'(q); rl: list radius
  double sig_wd, w0d;  // the same factors in FP64 (the FP32 density is formed in FP64 from its sum)
  R half_skin2;
  float rc2f, rl2f;    // FP64 scenes: FP32 pre-test radii (squared) with the rounding margin
  double kc, dc;
  R kcR, dcR, dxR;
  double src_Q, src_r, src_v[3], src_x0[3], src_depth, src_ztop;
  int dt_mode, rebin_interval, has_transition, has_enthalpy, has_source, any_heat;
  int tvf;             // transport-velocity formulation on (p_background > 0)
  int any_conc;        // some phase diffuses, holds or transitions on a concentration
  double pbg;          // background pressure p_b
  R pbgR;
  double dt_fixed, dt_cond;  // dt_cond: min of the velocity-independent conditions
  double cmax;
  MatD mat[MAXMAT];
  MatR<R> matR[MAXMAT];
  // FP64 scenes: pair means of the material constants, from the per-pair formulas
  // 2 eta_a eta_b / (eta_a + eta_b) and 4 kappa_a kappa_b / (kappa_a + kappa_b) (0 when the
  // denominator is 0), evaluated once on the host
  double eta_ab[MAXMAT][MAXMAT], kap_ab[MAXMAT][MAXMAT];
  // ---------------------------------------------------------------- particles
  PBank<R> P, Q;       // current and alternate bank
  R *prs, *dT;         // pressure, rate (not permuted: recomputed every evaluation)
  R* dC;               // dC/dt of the last evaluation (when any_conc)
  R *vex, *vey, *vez;  // extrapolated velocity of wall and rigid particles
  R* vol;              // particle volume m / rho of the current evaluation
  // FP32 scenes: what a pair sweep gathers from a neighbour, packed per particle after the
  // density summation (two 16-byte and one 8-byte load per neighbour instead of eleven
  // scalar ones): pa = (x, y, z, rho), pb = (u or extrapolated v_w, p or p_w),
  // pv = (V, material | kind << 16); the force sweep reads T (heat) and the body id (rigid
  // targets) from the particle arrays where it needs them
  float4 *pa, *pb;
  float2* pv;
  SweepK k;            // FP32 scenes: the per-entry constants of the pair sweeps
  float4* pd;          // (u~ - u, C): transport-velocity formulation and concentration
  int* nbl;            // neighbour lists: entry k of particle i at nbl[nb_at(n, i, k)] = nb_entry(j, code)
  int* nbc;            // neighbour count of each particle (may exceed maxnb: then cells are scanned)
  int4* nbq;           // FP32 scenes: in-range entries of this evaluation (see SweepK)
  int* nbqc;
  int cq;              // capacity of the in-range lists (entries, a multiple of 4)
  R *xr, *yr, *zr;     // positions at the last list rebuild (same frame as the bank)
  unsigned long long* disp;  // bits of the largest squared displacement since the rebuild
  int maxnb;           // list capacity per particle
  int* key;            // sort key of each (sorted) particle: kind * ncells + cell key, so the
                       // fluid, rigid and wall particles form three runs in cell order (a
                       // particle changes kind only in the relabelling, which forces a
                       // rebuild before the next pair sweep: key class == kind in every sweep)
  int* where;          // input index -> current sorted index
  // rebin scratch
  int *tkey, *tloc, *bucket, *perm, *tshift;
  // ---------------------------------------------------------------- cells
  int *cstart;         // nkey + 1 entries, by key
  int *ccount;         // nkey, kept at zero between rebins
  int *cblk;           // block sums of the counting scan
  const int *lin2key;  // Morton rank of a row-major cell (null for row-major keys)
  const int *key2lin;
  // ---------------------------------------------------------------- bodies (FP64)
  int Kcap, nslot;
  int* K;              // device: bodies in use (ids 0..K-1)
  double *bm, *br, *bq, *bu, *bw, *ba, *bal, *bf, *bt, *bIb, *bIbinv, *bIw;
  double* bRm;         // rotation matrix R(q) of each body after the drift of the step
  int *balive, *bstart, *bend;  // slot ranges of each body
  int *bchg, *bcur;    // relabel: 1 changed body, 2 new body; slot cursor
  double* bold;        // relabel: centre of mass before the change (3 per body)
  double* rb2;         // relabel: body-frame offsets in the new slot order
  R* fr2;              // relabel: slot forces in the new slot order
  int* aux;            // relabel: smallest input index of each new-body component (per root)
  int* bst2;           // relabel: new slot range of every body (start, then end at + Kcap)
  double* rb;          // body-frame offset of every slot (3 per slot)
  int* slot_part;      // slot -> current sorted particle index
  R* fr;               // force on every slot (3 per slot)
  // ---------------------------------------------------------------- per-step state
  double* st;          // [0] dt [1] time [2] step [3] dt of last step
  unsigned long long* umax;  // bits of max |u|^2 over fluid particles (FP64, non-negative)
  int* status;         // [0] non-finite flag [1] relabel count [2] capacity error [3] table error
                       // [4] rebuild in this step [5] steps since rebuild [6] rebuild count
                       // [7] solidifiers without a rigid neighbour [8] new bodies this step
                       // [9] relabelled particles so far [10] lists stale (kinds changed, or a particle was moved
                       // to another cell by a write) since they were built [11] the union-find hooking of
                       // new bodies gave up (retry cap): that step's relabel is not applied
  int* pfx1;           // prefix tables of this scene alone (6 x 2 ints)
  Scene<R>** self;     // device array holding the address of this descriptor
  unsigned long long* pairs;  // [0] force-sweep pairs of the last evaluation
  double* red;         // scratch for deterministic FP64 reductions
};

// batch view handed to every kernel
template <class R>
struct BatchView {
  Scene<R>* const* sc;  // device array of pointers to the scene descriptors
  int nsc;
  const int* pfx_part;   // nsc+1 prefix of particle counts
  const int* pfx_cell;   // cells
  const int* pfx_grp;    // warp groups of the sweeps
  const int* pfx_body;   // body capacities
  const int* pfx_cblk;   // scan blocks of 1024 cells
  const int* pfx_slot;   // rigid slots
};

// cell index along one axis from v = floor((x - lo) / edge), clamped to [0, n - 1]; a NaN
// (a non-finite position) maps to cell 0 explicitly, so no index depends on how a NaN
// converts to an integer
__device__ __forceinline__ int clamp_cell(double v, int n) {
  return v >= 0.0 ? (v < (double)(n - 1) ? (int)v : n - 1) : 0;
}

// status words of a scene that stop its phase relabelling (checked by the host after a step)
enum { ST_NONFINITE = 0, ST_CAPACITY = 2, ST_HOOK_TIMEOUT = 11 };

// neighbour lists in chunks of four entries: entries 4q .. 4q + 3 of particle i form the
// int4 at index q n + i (one 16-byte store by the search, one 16-byte load by a sweep);
// the int offset of entry k of particle i
__device__ __forceinline__ size_t nb_at(size_t n, int i, int k) {
  return 4 * ((size_t)(k >> 2) * n + (size_t)i) + (size_t)(k & 3);
}

// a list entry: the neighbour's sorted index j (26 bits) and the offset o = c_j - c_i of its
// cell from the target's, o + 1 in two bits per axis: e = j << 6 | code (read unsigned)
constexpr int kMaxListIndex = 1 << 26;
__device__ __forceinline__ int nb_code(int ox, int oy, int oz) {
  return (ox + 1) | ((oy + 1) << 2) | ((oz + 1) << 4);
}
__device__ __forceinline__ int nb_entry(int j, int code) { return (int)(((unsigned)j << 6) | (unsigned)code); }
__device__ __forceinline__ int nb_j(int e) { return (int)((unsigned)e >> 6); }
__device__ __forceinline__ int nb_cd(int e) { return e & 63; }
__device__ __forceinline__ int nb_o(int code, int a) { return ((code >> (2 * a)) & 3) - 1; }
// the same offset as an exact float: the two bits b end the mantissa of 1.5 2^23 + b (unit
// in the last place 1), so subtracting 1.5 2^23 + 1 leaves b - 1 exactly
__device__ __forceinline__ float nb_of(int code, int a) {
  return __int_as_float(0x4B400000 | ((code >> (2 * a)) & 3)) - 12582913.0f;
}

__device__ __forceinline__ int find_scene(const int* __restrict__ pfx, int nsc, int g) {
  int lo = 0, hi = nsc - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(pfx + mid) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------- Morton
__host__ __device__ inline uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}
__host__ __device__ inline uint64_t spread2(uint64_t v) {  // 32 bits -> every second bit
  v &= 0xffffffffULL;
  v = (v | v << 16) & 0x0000ffff0000ffffULL;
  v = (v | v << 8) & 0x00ff00ff00ff00ffULL;
  v = (v | v << 4) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v | v << 2) & 0x3333333333333333ULL;
  v = (v | v << 1) & 0x5555555555555555ULL;
  return v;
}

}  // namespace sph
