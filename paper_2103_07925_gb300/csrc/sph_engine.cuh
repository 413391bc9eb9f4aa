// Host runtime of libsph: owns the device memory of every scene, the batch tables that
// the kernels walk, and the captured CUDA graph of one time step.
//
// Engine<R, DIM> holds any number of scenes of one precision and dimension.  A plain
// scene (sph_create_scene) is an engine with one scene; a batch holds one engine per
// dimension.  Every kernel of a step is one launch over all resident scenes; the launch
// sequence is captured once into a CUDA graph and replayed each step.  Adding or
// removing a scene rebuilds the prefix tables and re-captures the graph.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_aux.cuh"
#include "sph_kernels.cuh"

namespace sph {

void set_error(const char* fmt, ...);

#define SPH_CU(call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      set_error("CUDA error %s at %s:%d: %s", cudaGetErrorName(e_), __FILE__, __LINE__,     \
                cudaGetErrorString(e_));                                                    \
      return e_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA;                  \
    }                                                                                       \
  } while (0)

#define SPH_TRY(call)                     \
  do {                                    \
    sph_status s_ = (call);               \
    if (s_ != SPH_OK) return s_;          \
  } while (0)

struct HostScene {
  size_t bytes = 0;
  std::vector<void*> allocs;
  int64_t job_id = -1;
  int32_t nsteps_total = 0, steps_done = 0;
  bool done = false, reported = false, failed = false;
  int n = 0, nfluid = 0, nrigid = 0, nwall = 0, K0 = 0;
};

// geometry and constants derived from the parameters exactly as the checker does
// (cell count floor(L / r_c), edge L / count)
// ------------------------------------------------------------------------------ helpers
// list capacity: 1.3 x the lattice sites inside the list radius, rounded up to 32
inline int list_capacity(int dim, double radius_in_dx) {
  double ball = dim == 3 ? 4.0 / 3.0 * M_PI * radius_in_dx * radius_in_dx * radius_in_dx
                         : M_PI * radius_in_dx * radius_in_dx;
  int c = (int)std::ceil(1.3 * ball / 32.0) * 32;
  return c < 32 ? 32 : c;
}

template <class R>
inline sph_status fill_constants(const sph_params* p, Scene<R>& S) {
  if (p->dim != 2 && p->dim != 3) { set_error("dim must be 2 or 3"); return SPH_ERR_INVALID; }
  if (!(p->h > 0) || !(p->dx > 0) || !(p->kernel_support > 0)) { set_error("h, dx and kernel_support must be > 0"); return SPH_ERR_INVALID; }
  if (p->n_materials < 1 || p->n_materials > MAXMAT || !p->materials) { set_error("1..16 materials required"); return SPH_ERR_INVALID; }
  S.dim = p->dim;
  S.h = p->h;
  S.rc = p->kernel_support * p->h;
  S.rc2 = S.rc * S.rc;
  S.dx = p->dx;
  S.ncells = 1;
  for (int d = 0; d < 3; d++) {
    S.lo[d] = p->box_min[d];
    S.hi[d] = p->box_max[d];
    S.per[d] = d < p->dim ? (p->periodic[d] != 0) : 0;
    S.g[d] = p->gravity[d];
    S.gR[d] = (R)p->gravity[d];
    if (d < p->dim) {
      double L = p->box_max[d] - p->box_min[d];
      if (!(L > 0)) { set_error("box_max must exceed box_min"); return SPH_ERR_INVALID; }
      // the cell count stays a double until it is known to fit (no overflowing conversion)
      double ncd = std::floor(L / (S.rc + (p->skin > 0.0 ? p->skin : 0.0)));
      if (!(ncd <= (double)(1 << 20))) { set_error("too many cells on axis %d", d); return SPH_ERR_INVALID; }
      int nc = ncd < 1.0 ? 1 : (int)ncd;
      if (S.per[d] && nc < 3) { set_error("periodic axis %d needs at least 3 cells of edge >= r_c + skin", d); return SPH_ERR_INVALID; }
      S.ncell[d] = nc;
      S.L[d] = L;
      S.ell[d] = L / nc;
    } else {
      S.ncell[d] = 1;
      S.L[d] = 1.0;
      S.ell[d] = 1.0;
    }
    S.ellR[d] = (R)S.ell[d];
    S.LR[d] = (R)S.L[d];
    if ((double)S.ncells * S.ncell[d] * NCLS > 2.0e9) { set_error("cell lattice too large"); return SPH_ERR_INVALID; }
    S.ncells *= S.ncell[d];
  }
  S.skin = p->skin > 0.0 ? p->skin : 0.0;
  S.rc2R = (R)S.rc2;
  S.rl2R = (R)((S.rc + S.skin) * (S.rc + S.skin));
  {  // FP32 copies of coordinates up to X in magnitude are off by 2^-24 X each; the pre-test
     // distance (two subtractions and a shift) by at most about 1.5e-6 X
    double X = 0.0;
    for (int d = 0; d < 3; d++) X = std::fmax(X, std::fmax(std::fabs(p->box_min[d]), std::fabs(p->box_max[d])));
    X += std::fmax(std::fmax(S.L[0], S.L[1]), S.L[2]);
    double m = 2e-6 * X + 1e-30;
    S.rc2f = (float)((S.rc + m) * (S.rc + m) * (1.0 + 1e-5));
    S.rl2f = (float)((S.rc + S.skin + m) * (S.rc + S.skin + m) * (1.0 + 1e-5));
  }
  S.half_skin2 = (R)(0.25 * S.skin * S.skin);
  S.inv_h = (R)(1.0 / S.h);
  double sig = p->dim == 2 ? 7.0 / (478.0 * M_PI * S.h * S.h) : 1.0 / (120.0 * M_PI * S.h * S.h * S.h);
  S.sig_w = (R)sig;
  S.sig_dw = (R)(sig / S.h);
  S.w0 = (R)(sig * 66.0);  // w(0) = 3^5 - 6 * 2^5 + 15
  S.sig_wd = sig;
  S.w0d = sig * 66.0;
  S.nmat = p->n_materials;
  S.has_transition = S.has_enthalpy = 0;
  S.any_heat = 0;
  S.any_conc = 0;
  S.cmax = 0.0;
  double numax = 0.0, cond = INFINITY;
  for (int q = 0; q < p->n_materials; q++) {
    const sph_material& m = p->materials[q];
    if (m.kind < 0 || m.kind > 2) { set_error("material %d: bad kind", q); return SPH_ERR_INVALID; }
    if (m.kind == SPH_FLUID && !(m.c > 0 && m.rho0 > 0)) { set_error("fluid material %d needs c > 0 and rho0 > 0", q); return SPH_ERR_INVALID; }
    if (m.latent_heat > 0 && !(m.mushy_width > 0)) { set_error("material %d: latent heat needs a mushy width", q); return SPH_ERR_INVALID; }
    if (m.transitions_to >= p->n_materials) { set_error("material %d: bad transitions_to", q); return SPH_ERR_INVALID; }
    if (m.transitions_to >= 0) {
      int k2 = p->materials[m.transitions_to].kind;
      bool ok = (m.kind == SPH_RIGID && k2 == SPH_FLUID) || (m.kind == SPH_FLUID && k2 == SPH_RIGID);
      if (!ok) { set_error("material %d: transitions must pair a fluid and a rigid phase", q); return SPH_ERR_INVALID; }
      S.has_transition = 1;
    }
    MatD& D = S.mat[q];
    D.kind = m.kind; D.to = m.transitions_to; D.enth = m.latent_heat > 0; D.src = m.transitions_to >= 0;
    D.rho0 = m.rho0; D.c = m.c; D.eta = m.eta; D.cp = m.cp; D.kappa = m.kappa; D.Tt = m.T_transition;
    D.L = m.latent_heat; D.w = m.mushy_width; D.p0 = m.rho0 * m.c * m.c;
    D.tby = m.transition_by; D.D = m.diffusivity; D.Ct = m.C_transition; D.Cfix = m.C_fixed;
    if (m.diffusivity > 0.0 || m.transition_by == 1 || !std::isnan(m.C_fixed)) S.any_conc = 1;
    MatR<R>& A = S.matR[q];
    A.kind = m.kind; A.enth = D.enth;
    A.D = (R)m.diffusivity;
    A.rho0 = (R)m.rho0; A.c2 = (R)(m.c * m.c); A.eta = (R)m.eta; A.cp = (R)m.cp; A.kappa = (R)m.kappa;
    A.inv_p0 = D.p0 > 0 ? (R)(1.0 / D.p0) : R(0);
    if (D.enth) S.has_enthalpy = 1;
    if (m.kappa > 0 && m.kind != SPH_WALL) S.any_heat = 1;
    if (m.kind == SPH_FLUID) {
      if (m.c > S.cmax) S.cmax = m.c;
      if (m.eta / m.rho0 > numax) numax = m.eta / m.rho0;
    }
    if (m.kind != SPH_WALL && m.kappa > 0.0) {
      double c5 = 0.1 * m.rho0 * m.cp * S.h * S.h / m.kappa;
      if (c5 < cond) cond = c5;
    }
  }
  for (int a = 0; a < p->n_materials; a++)
    for (int b = 0; b < p->n_materials; b++) {
      double ea = p->materials[a].eta, eb = p->materials[b].eta;
      double ka = p->materials[a].kappa, kb = p->materials[b].kappa;
      S.eta_ab[a][b] = (ea + eb > 0.0) ? 2.0 * ea * eb / (ea + eb) : 0.0;
      S.kap_ab[a][b] = (ka + kb > 0.0) ? 4.0 * ka * kb / (ka + kb) : 0.0;
    }
  S.has_source = p->src_power > 0 ? 1 : 0;
  S.pbg = p->p_background > 0.0 ? p->p_background : 0.0;
  S.pbgR = (R)S.pbg;
  S.tvf = S.pbg > 0.0 ? 1 : 0;
  if (S.has_source) S.any_heat = 1;
  S.src_Q = p->src_power; S.src_r = p->src_radius; S.src_depth = p->src_depth; S.src_ztop = p->src_ztop;
  for (int d = 0; d < 3; d++) { S.src_v[d] = p->src_speed[d]; S.src_x0[d] = p->src_origin[d]; }
  S.dt_mode = p->dt_mode;
  S.dt_fixed = p->dt_fixed;
  if (p->dt_mode != 0 && p->dt_mode != 1) { set_error("dt_mode must be 0 or 1"); return SPH_ERR_INVALID; }
  if (p->dt_mode == 0 && !(p->dt_fixed > 0)) { set_error("dt_fixed must be > 0"); return SPH_ERR_INVALID; }
  double gmag = std::sqrt(p->gravity[0] * p->gravity[0] + p->gravity[1] * p->gravity[1] + p->gravity[2] * p->gravity[2]);
  double dtc = INFINITY;
  if (numax > 0.0) dtc = std::fmin(dtc, 0.125 * S.h * S.h / numax);
  if (gmag > 0.0) dtc = std::fmin(dtc, 0.25 * std::sqrt(S.h / gmag));
  dtc = std::fmin(dtc, cond);
  S.dt_cond = dtc;  // the contact condition is added once k_c and m_r are known
  S.rebin_interval = p->rebin_interval < 1 ? 1 : p->rebin_interval;
  S.key_order = p->key_order;
  return SPH_OK;
}

template <class R, int DIM>
class Engine {
 public:
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int cap = 0;  // scene slots
  std::vector<Scene<R>> hs;       // host copies of the device descriptors
  std::vector<HostScene> meta;
  Scene<R>** d_sc = nullptr;      // device table of descriptor addresses (cap)
  int* d_pfx = nullptr;           // 7 prefix tables of cap+1
  std::vector<int> h_pfx;
  cudaGraphExec_t graph = nullptr;
  bool graph_dirty = true;
  int grid_part = 0, grid_warp = 0, grid_blk = 0;
  // launch shape of the pair sweeps (density, extrapolation, force) and of the search:
  // threads per block of the sweeps, and resident waves of blocks per SM for both
  int sweep_block = 256, sweep_waves = 0, search_waves = 0;
  int grid_sweep = 0;                    // force sweep (plain instantiation)
  int grid_tvf = 0, grid_dens = 0, grid_extrap = 0;  // the other sweeps, each by its own occupancy
  int grid_sweep1 = 0, grid_tvf1 = 0;   // force sweeps of launches over a single scene
  int kernels_per_step = 0;
  int sms = 0;
  int64_t steps_taken = 0;
  int* d_flags = nullptr;          // non-finite flags gathered from the scenes (cap)
  std::vector<int> h_flags;
  // staging for reads
  void* d_stage = nullptr;
  size_t stage_bytes = 0;

  ~Engine() { release_all(); }

  sph_status init(int capacity, cudaStream_t s) {
    cap = capacity;
    if (s) stream = s;
    else {
      SPH_CU(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    int dev;
    SPH_CU(cudaGetDevice(&dev));
    SPH_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SPH_CU(cudaMalloc(&d_sc, sizeof(Scene<R>*) * cap));
    SPH_CU(cudaMalloc(&d_pfx, sizeof(int) * 7 * (cap + 1)));
    SPH_CU(cudaMalloc(&d_flags, sizeof(int) * cap));
    h_flags.assign(cap, 0);
    h_pfx.assign(7 * (cap + 1), 0);
    SPH_CU(cudaMemsetAsync(d_pfx, 0, sizeof(int) * 7 * (cap + 1), stream));
    int b1 = 0, b2 = 0;
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_kick_drift<R>, 256, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_search<R, DIM>, 128, 0));
    grid_part = sms * std::max(1, b1);
    grid_warp = sms * std::max(1, b2);
    grid_blk = sms * 8;
    SPH_CU(cudaFuncSetAttribute(k_rl_slots_order<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * kSortCap * (int)sizeof(int)));
    return apply_launch();
  }

  // grids of the sweeps and the search from the launch shape (0 waves: the occupancy limit)
  sph_status apply_launch() {
    int bs = 0, bw = 0, bt = 0, bd = 0, be = 0, bs1 = 0, bt1 = 0;
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_force<R, DIM, false, false>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bt, k_force<R, DIM, true, false>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs1, k_force<R, DIM, false, true>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bt1, k_force<R, DIM, true, true>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_density<R, DIM, true>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&be, k_extrap<R, DIM, true>, sweep_block, 0));
    SPH_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, k_search<R, DIM>, 128, 0));
    // resident blocks per SM: the kernel's occupancy, capped by the requested waves
    auto waves = [&](int occ, int req) { occ = std::max(1, occ); return sms * (req > 0 ? std::min(req, occ) : occ); };
    grid_sweep = waves(bs, sweep_waves);
    grid_tvf = waves(bt, sweep_waves);
    grid_sweep1 = waves(bs1, sweep_waves);
    grid_tvf1 = waves(bt1, sweep_waves);
    grid_dens = waves(bd, sweep_waves);
    grid_extrap = waves(be, sweep_waves);
    grid_warp = waves(bw, search_waves);
    graph_dirty = true;
    return SPH_OK;
  }

  sph_status set_launch(const int32_t* cfg, int32_t n) {
    int b = n > 0 ? cfg[0] : 256, w = n > 1 ? cfg[1] : 0, v = n > 2 ? cfg[2] : 0;
    if (b < 32 || b > 256 || b % 32 || w < 0 || v < 0) {
      set_error("launch shape: block must be a multiple of 32 in [32, 256], waves >= 0");
      return SPH_ERR_INVALID;
    }
    sweep_block = b;
    sweep_waves = w;
    search_waves = v;
    return apply_launch();
  }

  void get_launch(int32_t* cfg) {
    cfg[0] = sweep_block;
    cfg[1] = grid_sweep / std::max(1, sms);
    cfg[2] = grid_warp / std::max(1, sms);
  }

  // device time of n steps (graph replays) between two events on the engine's stream
  sph_status time_steps(int32_t n, double* ms) {
    if (n < 1 || !ms) { set_error("time_steps needs n >= 1 and an output"); return SPH_ERR_INVALID; }
    cudaEvent_t a, b;
    SPH_CU(cudaEventCreate(&a));
    SPH_CU(cudaEventCreate(&b));
    sph_status st = SPH_OK;
    if (cudaEventRecord(a, stream) != cudaSuccess) st = SPH_ERR_CUDA;
    if (st == SPH_OK) st = step(n, false);
    if (st == SPH_OK && cudaEventRecord(b, stream) != cudaSuccess) st = SPH_ERR_CUDA;
    if (st == SPH_OK && cudaEventSynchronize(b) != cudaSuccess) st = SPH_ERR_CUDA;
    float t = 0.f;
    if (st == SPH_OK && cudaEventElapsedTime(&t, a, b) != cudaSuccess) st = SPH_ERR_CUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st == SPH_ERR_CUDA) set_error("event timing failed");
    *ms = t;
    return st;
  }

  void release_scene(size_t idx) {
    for (void* p : meta[idx].allocs) cudaFree(p);
    meta[idx].allocs.clear();
  }

  void release_all() {
    if (stream) cudaStreamSynchronize(stream);
    for (size_t i = 0; i < meta.size(); i++) release_scene(i);
    hs.clear();
    meta.clear();
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    if (d_sc) cudaFree(d_sc);
    if (d_pfx) cudaFree(d_pfx);
    if (d_flags) cudaFree(d_flags);
    d_flags = nullptr;
    if (d_stage) cudaFree(d_stage);
    d_sc = nullptr; d_pfx = nullptr; d_stage = nullptr;
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }

  BatchView<R> view() const {
    BatchView<R> B;
    B.sc = d_sc;
    B.nsc = (int)act.size();
    int c1 = cap + 1;
    B.pfx_part = d_pfx;
    B.pfx_cell = d_pfx + c1;
    B.pfx_grp = d_pfx + 2 * c1;
    B.pfx_body = d_pfx + 3 * c1;
    B.pfx_cblk = d_pfx + 4 * c1;
    B.pfx_slot = d_pfx + 5 * c1;
    return B;
  }

  // one-scene view (set-up and read-out kernels of a single scene)
  static BatchView<R> view_one(const Scene<R>& S) {
    BatchView<R> B;
    B.sc = S.self;
    B.nsc = 1;
    B.pfx_part = S.pfx1;
    B.pfx_cell = S.pfx1 + 2;
    B.pfx_grp = S.pfx1 + 4;
    B.pfx_body = S.pfx1 + 6;
    B.pfx_cblk = S.pfx1 + 8;
    B.pfx_slot = S.pfx1 + 10;
    return B;
  }

  std::vector<Scene<R>*> h_ptrs;
  std::vector<Scene<R>*> d_self;  // device address of each scene's descriptor
  std::vector<int> act;           // scenes in the batch tables (not finished)

  sph_status upload_tables() {
    act.clear();
    for (int s = 0; s < (int)hs.size(); s++)
      if (!meta[s].done) act.push_back(s);
    int ns = (int)act.size();
    int c1 = cap + 1;
    std::fill(h_pfx.begin(), h_pfx.end(), 0);
    h_ptrs.clear();
    for (int s = 0; s < ns; s++) {
      const Scene<R>& S = hs[act[s]];
      h_ptrs.push_back(d_self[act[s]]);
      h_pfx[0 * c1 + s + 1] = h_pfx[0 * c1 + s] + S.n;
      h_pfx[1 * c1 + s + 1] = h_pfx[1 * c1 + s] + S.nkey;
      h_pfx[2 * c1 + s + 1] = h_pfx[2 * c1 + s] + S.ngroups;
      h_pfx[3 * c1 + s + 1] = h_pfx[3 * c1 + s] + S.Kcap;
      h_pfx[4 * c1 + s + 1] = h_pfx[4 * c1 + s] + S.ncblk;
      h_pfx[5 * c1 + s + 1] = h_pfx[5 * c1 + s] + S.nslot;
    }
    SPH_CU(cudaMemcpyAsync(d_pfx, h_pfx.data(), sizeof(int) * 7 * c1, cudaMemcpyHostToDevice, stream));
    if (ns) SPH_CU(cudaMemcpyAsync(d_sc, h_ptrs.data(), sizeof(Scene<R>*) * ns, cudaMemcpyHostToDevice, stream));
    SPH_CU(cudaStreamSynchronize(stream));
    graph_dirty = true;
    return SPH_OK;
  }

  template <class T>
  sph_status dalloc(HostScene& M, T** p, size_t count) {
    size_t b = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMallocAsync((void**)p, b, stream);
    if (e != cudaSuccess) {
      set_error("device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
      return SPH_ERR_OOM;
    }
    M.allocs.push_back(*p);
    M.bytes += b;
    return SPH_OK;
  }

  // rc_dx, rl_dx: r_c and r_c + skin in units of dx (the capacities of the in-range and the
  // neighbour lists, as add_scene allocates them)
  static size_t footprint(int64_t n, int64_t ncells, int64_t kcap, int64_t nrigid, bool trans, bool tvf,
                          double rc_dx, double rl_dx) {
    // the neighbour list and its count; FP32: the packed records and the in-range lists of
    // each evaluation (capacity at r_c)
    size_t per = 2 * (13 * sizeof(R) + 4 * sizeof(int)) + 9 * sizeof(R) + 8 * sizeof(int) + 8 * sizeof(double) +
                 (size_t)(list_capacity(DIM, rl_dx) + 1) * sizeof(int) +
                 (sizeof(R) == 4 ? 2 * sizeof(float4) + sizeof(float2) + (size_t)(list_capacity(DIM, rc_dx) + 1) * sizeof(int) : 0);
    size_t cells = (size_t)(NCLS * ncells + 1) * 2 * sizeof(int) + (size_t)ncells * 2 * sizeof(int) +
                   (size_t)(NCLS * ncells / 1024 + 2) * sizeof(int);
    size_t bodies = (size_t)kcap * (69 * sizeof(double) + 3 * sizeof(int));
    size_t slots = (size_t)nrigid * (3 * sizeof(double) + 3 * sizeof(R) + sizeof(int));
    // relabel scratch: offsets and forces in the new slot order, one root mark per particle
    size_t relabel = trans ? (size_t)nrigid * (3 * sizeof(double) + 3 * sizeof(R)) + (size_t)n * sizeof(int) +
                                 (size_t)kcap * 2 * sizeof(int) : 0;
    // transport-velocity state: a~ and u~ - u in both banks, and the packed u~ - u (FP32)
    size_t tv = tvf ? (size_t)n * (12 * sizeof(R) + (sizeof(R) == 4 ? sizeof(float4) : 0)) : 0;
    return per * (size_t)n + cells + bodies + slots + relabel + tv + 4096;
  }

  // ---------------------------------------------------------------------------- create
  sph_status add_scene(const sph_params* p, const sph_particles_in* in, const sph_bodies_in* bi,
                       int64_t job_id, int32_t nsteps_total, int* out_idx);
  sph_status remove_scene(int idx);
  sph_status capture();
  sph_status launch_step(cudaEvent_t* ev = nullptr);
  sph_status profile(int32_t reps, double* ms);
  sph_status step(int32_t nsteps, bool sync);
  sph_status advance_jobs(int32_t nsteps);
  int find_job(int64_t id) const {
    for (int i = 0; i < (int)meta.size(); i++)
      if (meta[i].job_id == id) return i;
    return -1;
  }
  size_t bytes_in_use() const {
    size_t b = 0;
    for (auto& M : meta) b += M.bytes;
    return b;
  }
  sph_status evaluate_initial(int idx);
  sph_status read_fields(int idx, uint32_t mask, void* const* dst, int original_order);
  sph_status write_fields(int idx, uint32_t mask, const void* const* src);
  sph_status interpolate(int idx, int64_t nq, const double* query, int32_t field, uint32_t mask, double* out);
  sph_status read_bodies(int idx, const sph_bodies_out* out, int32_t* kout);
  sph_status diagnostics(int idx, double out[16]);
  sph_status neighbors(int idx, int64_t* counts, int32_t* list, int64_t cap_list, int64_t* total);
  sph_status check_status(int idx, bool* nonfinite);
  // jobs whose velocities became non-finite leave the batch tables as failed
  sph_status check_failed() {
    int ns = (int)act.size();
    if (!ns) return SPH_OK;
    k_gather_failed<R><<<(ns + 127) / 128, 128, 0, stream>>>(d_sc, ns, d_flags);
    SPH_CU(cudaGetLastError());
    SPH_CU(cudaMemcpyAsync(h_flags.data(), d_flags, sizeof(int) * ns, cudaMemcpyDeviceToHost, stream));
    SPH_CU(cudaStreamSynchronize(stream));
    bool changed = false;
    for (int s = 0; s < ns; s++)
      if (h_flags[s]) {
        meta[act[s]].done = meta[act[s]].failed = true;
        changed = true;
      }
    return changed ? upload_tables() : SPH_OK;
  }
  sph_status ensure_stage(size_t bytes) {
    if (bytes <= stage_bytes) return SPH_OK;
    if (d_stage) cudaFreeAsync(d_stage, stream);
    d_stage = nullptr;
    cudaError_t e = cudaMallocAsync(&d_stage, bytes, stream);
    if (e != cudaSuccess) { set_error("staging allocation failed"); stage_bytes = 0; return SPH_ERR_OOM; }
    stage_bytes = bytes;
    return SPH_OK;
  }
};

}  // namespace sph

namespace sph {


inline int grid_for(int64_t items, int per_block, int max_grid) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (int)std::min<int64_t>(b, max_grid);
}

// Morton ranks of the cells of an nx x ny x nz lattice: key2lin lists the row-major index
// of the cells in increasing Morton code, lin2key is its inverse
inline void morton_tables(int dim, const int* nc, std::vector<int>& lin2key, std::vector<int>& key2lin) {
  int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
  std::vector<std::pair<uint64_t, int>> codes((size_t)ncells);
  for (int z = 0; z < nc[2]; z++)
    for (int y = 0; y < nc[1]; y++)
      for (int x = 0; x < nc[0]; x++) {
        int lin = x + nc[0] * (y + nc[1] * z);
        uint64_t c = dim == 3 ? (spread3(x) | (spread3(y) << 1) | (spread3(z) << 2)) : (spread2(x) | (spread2(y) << 1));
        codes[(size_t)lin] = {c, lin};
      }
  std::sort(codes.begin(), codes.end());
  lin2key.assign((size_t)ncells, 0);
  key2lin.assign((size_t)ncells, 0);
  for (int64_t k = 0; k < ncells; k++) {
    key2lin[(size_t)k] = codes[(size_t)k].second;
    lin2key[(size_t)codes[(size_t)k].second] = (int)k;
  }
}

template <class R, int DIM>
sph_status Engine<R, DIM>::add_scene(const sph_params* p, const sph_particles_in* in, const sph_bodies_in* bi,
                                     int64_t job_id, int32_t nsteps_total, int* out_idx) {
  if (!p || !in) { set_error("params and particles are required"); return SPH_ERR_INVALID; }
  if ((int)hs.size() >= cap) { set_error("no free scene slot"); return SPH_ERR_CAPACITY; }
  if (p->dim != DIM) { set_error("scene dimension does not match this engine"); return SPH_ERR_INVALID; }
  Scene<R> S;
  memset(&S, 0, sizeof(S));
  SPH_TRY(fill_constants(p, S));
  int64_t n64 = in->n;
  // a list entry holds a sorted index in 26 bits
  if (n64 < 1 || n64 > kMaxListIndex) { set_error("particle count must be in [1, 2^26]"); return SPH_ERR_INVALID; }
  if (!in->pos || !in->vel || !in->mass || !in->density || !in->temperature || !in->material || !in->body) {
    set_error("pos, vel, mass, density, temperature, material and body are required");
    return SPH_ERR_INVALID;
  }
  int n = (int)n64;
  int K = bi ? bi->k : 0;
  if (K < 0 || (K > 0 && (!bi->quat || !bi->vel || !bi->omega))) { set_error("bad body input"); return SPH_ERR_INVALID; }
  // host-side validation and rigid slot order (rigid particles grouped by body)
  HostScene M;
  M.n = n;
  M.job_id = job_id;
  M.nsteps_total = nsteps_total;
  std::vector<int> bodycount((size_t)K + 1, 0);
  double mr = INFINITY;
  for (int i = 0; i < n; i++) {
    int mt = in->material[i];
    if (mt < 0 || mt >= p->n_materials) { set_error("particle %d: material out of range", i); return SPH_ERR_INVALID; }
    int kind = p->materials[mt].kind;
    for (int d = 0; d < 3; d++) {
      double x = in->pos[3 * i + d];
      if (!std::isfinite(x)) { set_error("particle %d: non-finite position", i); return SPH_ERR_INVALID; }
      if (d < p->dim && !S.per[d] && (x < S.lo[d] || x > S.hi[d])) {
        set_error("particle %d lies outside the box on axis %d", i, d);
        return SPH_ERR_INVALID;
      }
    }
    if (!(in->mass[i] > 0) || !(in->density[i] > 0)) { set_error("particle %d: mass and density must be > 0", i); return SPH_ERR_INVALID; }
    if (kind == SPH_FLUID) M.nfluid++;
    else if (kind == SPH_WALL) M.nwall++;
    else {
      M.nrigid++;
      int b = in->body[i];
      if (b < 0 || b >= K) { set_error("rigid particle %d: body id out of range", i); return SPH_ERR_INVALID; }
      bodycount[(size_t)b]++;
      if (in->mass[i] < mr) mr = in->mass[i];
    }
  }
  for (int b = 0; b < K; b++)
    if (bodycount[(size_t)b] == 0) { set_error("body %d has no rigid particle", b); return SPH_ERR_INVALID; }
  std::vector<int> bstart((size_t)std::max(K, 1), 0), bend((size_t)std::max(K, 1), 0), slot((size_t)n, -1);
  {
    int acc = 0;
    for (int b = 0; b < K; b++) { bstart[(size_t)b] = acc; acc += bodycount[(size_t)b]; bend[(size_t)b] = bstart[(size_t)b]; }
    for (int i = 0; i < n; i++)
      if (p->materials[in->material[i]].kind == SPH_RIGID) slot[(size_t)i] = bend[(size_t)in->body[i]]++;
  }
  M.K0 = K;
  S.n = n;
  S.Kcap = std::max(1, p->body_capacity > K ? p->body_capacity : K + (S.has_transition ? 1024 : 0));
  S.nslot = std::max(1, S.has_transition ? n : M.nrigid);
  // contact constants (defaults scale with the CFL step, Eq. timestepcond)
  if (!(mr < INFINITY)) mr = 0.0;
  double dt_ref = S.cmax > 0.0 ? 0.25 * p->h / S.cmax : p->dt_fixed;
  S.kc = p->k_contact > 0.0 ? p->k_contact : mr * (0.22 / dt_ref) * (0.22 / dt_ref);
  S.dc = p->d_contact >= 0.0 ? p->d_contact : 0.2 * std::sqrt(S.kc * mr * 0.5);
  if (M.nrigid > 0 && S.kc > 0.0) S.dt_cond = std::fmin(S.dt_cond, 0.22 * std::sqrt(mr / S.kc));
  S.kcR = (R)S.kc; S.dcR = (R)S.dc; S.dxR = (R)S.dx;
  // cell keys and warp groups
  bool morton = p->key_order == 0;
  S.key_order = morton ? 0 : 1;
  S.G = 1;
  S.win = !morton && p->cells_per_group < 0;
  if (!morton && !S.win) S.G = p->cells_per_group > 0 ? p->cells_per_group : (DIM == 2 ? 3 : 1);
  S.ngx = (S.ncell[0] + S.G - 1) / S.G;
  S.ngroups = morton ? S.ncells : (S.win ? (n + 31) / 32 : S.ngx * S.ncell[1] * S.ncell[2]);
  S.nkey = NCLS * S.ncells;
  S.ncblk = (S.nkey + 1023) / 1024;
  // ------------------------------------------------------------------ allocations
  auto A = [&](auto** ptr, size_t cnt) { return dalloc(M, ptr, cnt); };
  for (PBank<R>* B : {&S.P, &S.Q}) {
    R** rf[] = {&B->px, &B->py, &B->pz, &B->vx, &B->vy, &B->vz, &B->ax, &B->ay, &B->az, &B->rho, &B->T, &B->H, &B->m};
    for (R** f : rf) SPH_TRY(A(f, (size_t)n));
    int** ifs[] = {&B->mt, &B->body, &B->slot, &B->orig};
    for (int** f : ifs) SPH_TRY(A(f, (size_t)n));
    if (S.any_conc) SPH_TRY(A(&B->C, (size_t)n));
    if (S.tvf) {
      R** tf[] = {&B->bx, &B->by, &B->bz, &B->tx, &B->ty, &B->tz};
      for (R** f : tf) {
        SPH_TRY(A(f, (size_t)n));
        SPH_CU(cudaMemsetAsync(*f, 0, sizeof(R) * n, stream));
      }
    }
  }
  R** rx[] = {&S.prs, &S.dT, &S.vex, &S.vey, &S.vez, &S.vol};
  for (R** f : rx) SPH_TRY(A(f, (size_t)n));
  if (sizeof(R) == 4)
  {
    for (float4** f : {&S.pa, &S.pb}) SPH_TRY(A(f, (size_t)n));
    SPH_TRY(A(&S.pv, (size_t)n));
  }
  if (sizeof(R) == 4 && (S.tvf || S.any_conc)) SPH_TRY(A(&S.pd, (size_t)n));
  if (S.any_conc) {
    SPH_TRY(A(&S.dC, (size_t)n));
    SPH_CU(cudaMemsetAsync(S.dC, 0, sizeof(R) * n, stream));
  }
  S.maxnb = list_capacity(DIM, (S.rc + S.skin) / S.dx);
  SPH_TRY(A(&S.nbl, (size_t)S.maxnb * n));
  SPH_TRY(A(&S.nbc, (size_t)n));
  if (sizeof(R) == 4) {  // in-range lists of each evaluation
    S.cq = list_capacity(DIM, S.rc / S.dx);
    SPH_TRY(A(&S.nbq, (size_t)(S.cq / 4) * n));
    SPH_TRY(A(&S.nbqc, (size_t)n));
  }
  SPH_TRY(A(&S.xr, (size_t)n));
  SPH_TRY(A(&S.yr, (size_t)n));
  SPH_TRY(A(&S.zr, (size_t)n));
  SPH_TRY(A(&S.disp, 1));
  SPH_CU(cudaMemsetAsync(S.disp, 0, sizeof(unsigned long long), stream));
  int** ix[] = {&S.key, &S.where, &S.tkey, &S.tloc, &S.bucket, &S.perm, &S.tshift};
  for (int** f : ix) SPH_TRY(A(f, (size_t)n));
  SPH_TRY(A(&S.cstart, (size_t)S.nkey + 1));
  SPH_TRY(A(&S.ccount, (size_t)S.nkey));
  SPH_TRY(A(&S.cblk, (size_t)S.ncblk + 1));
  std::vector<int> l2k, k2l;
  if (morton) {
    morton_tables(DIM, S.ncell, l2k, k2l);
    int *a1, *a2;
    SPH_TRY(A(&a1, (size_t)S.ncells));
    SPH_TRY(A(&a2, (size_t)S.ncells));
    SPH_CU(cudaMemcpyAsync(a1, l2k.data(), sizeof(int) * S.ncells, cudaMemcpyHostToDevice, stream));
    SPH_CU(cudaMemcpyAsync(a2, k2l.data(), sizeof(int) * S.ncells, cudaMemcpyHostToDevice, stream));
    S.lin2key = a1;
    S.key2lin = a2;
  }
  int kc = S.Kcap;
  double** bd[] = {&S.bm, &S.br, &S.bq, &S.bu, &S.bw, &S.ba, &S.bal, &S.bf, &S.bt, &S.bIb, &S.bIbinv, &S.bIw, &S.bRm};
  size_t bdn[] = {1, 3, 4, 3, 3, 3, 3, 3, 3, 9, 9, 9, 9};
  for (int q = 0; q < 13; q++) SPH_TRY(A(bd[q], bdn[q] * (size_t)kc));
  SPH_TRY(A(&S.balive, (size_t)kc));
  SPH_TRY(A(&S.bchg, (size_t)kc));
  SPH_TRY(A(&S.bcur, (size_t)kc));
  SPH_TRY(A(&S.bold, 3 * (size_t)kc));
  SPH_CU(cudaMemsetAsync(S.bchg, 0, sizeof(int) * kc, stream));
  if (S.has_transition) {
    SPH_TRY(A(&S.rb2, 3 * (size_t)S.nslot));
    SPH_TRY(A(&S.fr2, 3 * (size_t)S.nslot));
    SPH_TRY(A(&S.aux, (size_t)n));
    SPH_TRY(A(&S.bst2, 2 * (size_t)S.Kcap));
  }
  SPH_TRY(A(&S.bstart, (size_t)kc));
  SPH_TRY(A(&S.bend, (size_t)kc));
  SPH_TRY(A(&S.K, 1));
  SPH_TRY(A(&S.rb, 3 * (size_t)S.nslot));
  SPH_TRY(A(&S.slot_part, (size_t)S.nslot));
  SPH_TRY(A(&S.fr, 3 * (size_t)S.nslot));
  SPH_TRY(A(&S.st, 8));
  SPH_TRY(A(&S.umax, 1));
  SPH_TRY(A(&S.status, 16));
  SPH_TRY(A(&S.pfx1, 12));
  SPH_TRY(A(&S.self, 1));
  SPH_TRY(A(&S.pairs, 2));
  SPH_TRY(A(&S.red, 64));
  Scene<R>* dself;
  SPH_TRY(A(&dself, 1));
  // ------------------------------------------------------------------ uploads
  SPH_CU(cudaMemsetAsync(S.ccount, 0, sizeof(int) * S.nkey, stream));
  SPH_CU(cudaMemsetAsync(S.st, 0, sizeof(double) * 8, stream));
  SPH_CU(cudaMemsetAsync(S.umax, 0, sizeof(unsigned long long), stream));
  {
    int st0[16] = {0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // [4]: the creation step builds the lists
    SPH_CU(cudaMemcpyAsync(S.status, st0, sizeof(st0), cudaMemcpyHostToDevice, stream));
  }
  SPH_CU(cudaMemsetAsync(S.pairs, 0, sizeof(unsigned long long) * 2, stream));
  for (int q = 0; q < 13; q++) SPH_CU(cudaMemsetAsync(*bd[q], 0, sizeof(double) * bdn[q] * kc, stream));
  SPH_CU(cudaMemsetAsync(S.balive, 0, sizeof(int) * kc, stream));
  SPH_CU(cudaMemsetAsync(S.bstart, 0, sizeof(int) * kc, stream));
  SPH_CU(cudaMemsetAsync(S.bend, 0, sizeof(int) * kc, stream));
  SPH_CU(cudaMemsetAsync(S.fr, 0, sizeof(R) * 3 * S.nslot, stream));
  SPH_CU(cudaMemsetAsync(S.rb, 0, sizeof(double) * 3 * S.nslot, stream));
  SPH_CU(cudaMemsetAsync(S.slot_part, 0xff, sizeof(int) * S.nslot, stream));
  {
    std::vector<double> st(8, 0.0);
    st[0] = p->dt_mode == 0 ? p->dt_fixed : 0.0;
    SPH_CU(cudaMemcpyAsync(S.st, st.data(), sizeof(double) * 8, cudaMemcpyHostToDevice, stream));
    int pf[12] = {0, n, 0, S.nkey, 0, S.ngroups, 0, S.Kcap, 0, S.ncblk, 0, S.nslot};
    SPH_CU(cudaMemcpyAsync(S.pfx1, pf, sizeof(pf), cudaMemcpyHostToDevice, stream));
    SPH_CU(cudaMemcpyAsync(S.self, &dself, sizeof(dself), cudaMemcpyHostToDevice, stream));
    SPH_CU(cudaMemcpyAsync(S.K, &K, sizeof(int), cudaMemcpyHostToDevice, stream));
    if (K > 0) {
      std::vector<double> q((size_t)4 * K);
      for (int b = 0; b < K; b++) {
        double qn = std::sqrt(bi->quat[4 * b] * bi->quat[4 * b] + bi->quat[4 * b + 1] * bi->quat[4 * b + 1] +
                              bi->quat[4 * b + 2] * bi->quat[4 * b + 2] + bi->quat[4 * b + 3] * bi->quat[4 * b + 3]);
        if (!(qn > 0)) { set_error("body %d: zero quaternion", b); return SPH_ERR_INVALID; }
        for (int c = 0; c < 4; c++) q[(size_t)4 * b + c] = bi->quat[4 * b + c] / qn;
      }
      SPH_CU(cudaMemcpyAsync(S.bq, q.data(), sizeof(double) * 4 * K, cudaMemcpyHostToDevice, stream));
      SPH_CU(cudaMemcpyAsync(S.bu, bi->vel, sizeof(double) * 3 * K, cudaMemcpyHostToDevice, stream));
      SPH_CU(cudaMemcpyAsync(S.bw, bi->omega, sizeof(double) * 3 * K, cudaMemcpyHostToDevice, stream));
      SPH_CU(cudaMemcpyAsync(S.bstart, bstart.data(), sizeof(int) * K, cudaMemcpyHostToDevice, stream));
      SPH_CU(cudaMemcpyAsync(S.bend, bend.data(), sizeof(int) * K, cudaMemcpyHostToDevice, stream));
    }
  }
  // raw inputs -> staging -> k_import
  {
    size_t nd = (size_t)n;
    size_t doubles = nd * (3 + 3 + 1 + 1 + 1 + 3 + 1 + 1);
    size_t ints = nd * 3;
    char* stg = nullptr;
    SPH_CU(cudaMallocAsync((void**)&stg, doubles * 8 + ints * 4 + 64, stream));
    double* dpos = (double*)stg;
    double* dvel = dpos + 3 * nd;
    double* dmass = dvel + 3 * nd;
    double* ddens = dmass + nd;
    double* dtemp = ddens + nd;
    double* dwv = dtemp + nd;
    double* dwt = dwv + 3 * nd;
    double* dconc = dwt + nd;
    int* dmat = (int*)(dconc + nd);
    int* dbody = dmat + nd;
    int* dslot = dbody + nd;
    cudaMemcpyAsync(dpos, in->pos, 24 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dvel, in->vel, 24 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dmass, in->mass, 8 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(ddens, in->density, 8 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dtemp, in->temperature, 8 * nd, cudaMemcpyHostToDevice, stream);
    if (in->wall_velocity) cudaMemcpyAsync(dwv, in->wall_velocity, 24 * nd, cudaMemcpyHostToDevice, stream);
    if (in->wall_temperature) cudaMemcpyAsync(dwt, in->wall_temperature, 8 * nd, cudaMemcpyHostToDevice, stream);
    if (in->concentration) cudaMemcpyAsync(dconc, in->concentration, 8 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dmat, in->material, 4 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dbody, in->body, 4 * nd, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dslot, slot.data(), 4 * nd, cudaMemcpyHostToDevice, stream);
    S.k = SweepK{};
    if (sizeof(R) == 4) {
      S.k.pa = S.pa; S.k.pb = S.pb; S.k.pv = S.pv; S.k.pd = S.pd;
      S.k.nbl = S.nbl;
      S.k.nbq = S.nbq;
      S.k.nbqc = S.nbqc;
      S.k.cq = S.cq;
      S.k.n = n;
      for (int d = 0; d < 3; d++) {
        S.k.ell[d] = (float)S.ellR[d];
        S.k.nell[d] = -(float)S.ellR[d];
      }
      S.k.rc2 = (float)S.rc2R; S.k.sig_dw = (float)S.sig_dw; S.k.inv_h = (float)S.inv_h;
      S.k.dx = (float)S.dxR; S.k.kc = (float)S.kcR; S.k.dc = (float)S.dcR;
      S.k.any_heat = S.any_heat; S.k.any_conc = S.any_conc; S.k.tvf = S.tvf;
    }
    SPH_CU(cudaMemcpyAsync(dself, &S, sizeof(S), cudaMemcpyHostToDevice, stream));
    ImportArgs ia{dpos, dvel, dmass, ddens, dtemp, in->wall_velocity ? dwv : nullptr,
                  in->wall_temperature ? dwt : nullptr, dmat, dbody, dslot, in->concentration ? dconc : nullptr};
    k_import<R><<<grid_for(n, 256, sms * 8), 256, 0, stream>>>(S.self, ia);
    SPH_CU(cudaGetLastError());
    SPH_CU(cudaFreeAsync(stg, stream));
  }
  hs.push_back(S);
  meta.push_back(M);
  d_self.push_back(dself);
  int idx = (int)hs.size() - 1;
  SPH_TRY(upload_tables());
  sph_status st = evaluate_initial(idx);
  if (st != SPH_OK) {
    remove_scene(idx);
    return st;
  }
  if (out_idx) *out_idx = idx;
  return SPH_OK;
}

// forced binning, body mass quantities and one full evaluation at t = 0
// the device address of a host buffer the device can address directly (page-locked
// memory): the import kernel then reads it over the host link, with no staging copy; null
// for any other pointer (those go through a staging buffer)
inline void* device_view(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::evaluate_initial(int idx) {
  const Scene<R>& S = hs[idx];
  BatchView<R> B = view_one(S);
  int n = S.n;
  int gp = grid_for(n, 256, grid_part);
  k_bin<R><<<gp, 256, 0, stream>>>(B, 1);
  k_scan_blocks<R><<<grid_for(S.ncblk, 1, grid_blk), 1024, 0, stream>>>(B, 1);
  k_scan_top<R><<<1, 1024, 0, stream>>>(B, 1);
  k_scan_cells<R><<<grid_for(S.ncblk, 1, grid_blk), 1024, 0, stream>>>(B, 1);
  k_scatter<R><<<gp, 256, 0, stream>>>(B, 1);
  k_rank<R><<<grid_for((int64_t)S.nkey * 32, 256, grid_part), 256, 0, stream>>>(B, 1);
  k_permute<R><<<gp, 256, 0, stream>>>(B, 1);
  k_flip<R><<<1, 32, 0, stream>>>(B, 1);
  if (meta[idx].K0 > 0) k_body_mass<R><<<grid_for(S.Kcap, 1, grid_blk), 128, 0, stream>>>(B, 0);
  k_rigid_vel<R><<<gp, 256, 0, stream>>>(B, 0);
  int gw = grid_for((int64_t)S.ngroups * 32, 128, grid_warp);
  k_search<R, DIM><<<gw, 128, 0, stream>>>(B);
  k_density<R, DIM, true><<<grid_for(n, sweep_block, grid_dens), sweep_block, 0, stream>>>(B, S.k);
  k_extrap<R, DIM, true><<<grid_for(n, sweep_block, grid_extrap), sweep_block, 0, stream>>>(B, S.k);
  if (S.tvf || S.any_conc)
    k_force<R, DIM, true, true><<<grid_for(n, sweep_block, grid_tvf1), sweep_block, 0, stream>>>(B, S.k);
  else
    k_force<R, DIM, false, true><<<grid_for(n, sweep_block, grid_sweep1), sweep_block, 0, stream>>>(B, S.k);
  if (meta[idx].K0 > 0) k_body_reduce<R><<<grid_for(S.Kcap, 1, grid_blk), 128, 0, stream>>>(B, 0);
  k_rigid_vel<R><<<gp, 256, 0, stream>>>(B, 0);
  SPH_CU(cudaGetLastError());
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::remove_scene(int idx) {
  SPH_CU(cudaStreamSynchronize(stream));
  release_scene((size_t)idx);
  hs.erase(hs.begin() + idx);
  meta.erase(meta.begin() + idx);
  d_self.erase(d_self.begin() + idx);
  return upload_tables();
}

// stages of a step, in launch order (sph_profile reports one time per stage; the names are
// those of sph_profile_stage_name)
constexpr int kStages = 21;
static_assert(kStages == SPH_PROFILE_STAGES, "profiled stages");

// Launch one step.  With ev != nullptr an event is recorded before the first stage and
// after every stage (stages that do not apply record an empty interval).
template <class R, int DIM>
sph_status Engine<R, DIM>::launch_step(cudaEvent_t* ev) {
  BatchView<R> B = view();
  int ns = (int)act.size();
  if (!ns) return SPH_OK;
  int64_t np = h_pfx[ns], nc = h_pfx[(cap + 1) + ns], ng = h_pfx[2 * (cap + 1) + ns];
  int64_t nb = h_pfx[3 * (cap + 1) + ns], ncb = h_pfx[4 * (cap + 1) + ns];
  bool any_dt = false, any_body = false;
  bool any_transition = false, any_tvf = false, any_plain = false;
  for (int a : act) {
    any_tvf |= hs[a].tvf != 0 || hs[a].any_conc != 0;
    any_plain |= hs[a].tvf == 0 && hs[a].any_conc == 0;
    any_dt |= hs[a].dt_mode == 1;
    any_body |= meta[a].K0 > 0 || hs[a].has_transition != 0;
    any_transition |= hs[a].has_transition != 0;
  }
  int gp = grid_for(np, 256, grid_part);
  int gs = grid_for(ns, 128, 1 << 20);
  int gw = grid_for(ng * 32, 128, grid_warp);
  int gsw = grid_for(np, sweep_block, grid_sweep);
  int gst = grid_for(np, sweep_block, grid_tvf);
  int gsd = grid_for(np, sweep_block, grid_dens);
  int gse = grid_for(np, sweep_block, grid_extrap);
  int gb = grid_for(nb, 1, grid_blk);
  int gcb = grid_for(ncb, 1, grid_blk);
  int kcount = 0, stage = 0;
  auto rec = [&]() {
    if (ev) cudaEventRecord(ev[++stage], stream);
  };
  if (ev) cudaEventRecord(ev[0], stream);
  if (any_dt) { k_umax<R><<<gp, 256, 0, stream>>>(B); kcount++; }
  rec();
  k_dt<R><<<gs, 128, 0, stream>>>(B);
  rec();
  if (any_body) { k_body_kick_drift<R><<<grid_for(nb, 128, grid_part), 128, 0, stream>>>(B); kcount++; }
  rec();
  k_kick_drift<R><<<gp, 256, 0, stream>>>(B);
  rec();
  k_decide<R><<<gs, 128, 0, stream>>>(B);
  rec();
  k_bin<R><<<gp, 256, 0, stream>>>(B, 0);
  rec();
  k_scan_blocks<R><<<gcb, 1024, 0, stream>>>(B, 0);
  rec();
  k_scan_top<R><<<std::min(ns, grid_blk), 1024, 0, stream>>>(B, 0);
  rec();
  k_scan_cells<R><<<gcb, 1024, 0, stream>>>(B, 0);
  rec();
  k_scatter<R><<<gp, 256, 0, stream>>>(B, 0);
  rec();
  k_rank<R><<<grid_for(nc * 32, 256, grid_part), 256, 0, stream>>>(B, 0);
  rec();
  k_permute<R><<<gp, 256, 0, stream>>>(B, 0);
  rec();
  k_flip<R><<<gs, 128, 0, stream>>>(B, 0);
  rec();
  k_search<R, DIM><<<gw, 128, 0, stream>>>(B);
  rec();
  if (ns == 1) k_density<R, DIM, true><<<gsd, sweep_block, 0, stream>>>(B, hs[act[0]].k);
  else k_density<R, DIM, false><<<gsd, sweep_block, 0, stream>>>(B, SweepK{});
  rec();
  if (ns == 1) k_extrap<R, DIM, true><<<gse, sweep_block, 0, stream>>>(B, hs[act[0]].k);
  else k_extrap<R, DIM, false><<<gse, sweep_block, 0, stream>>>(B, SweepK{});
  rec();
  if (ns == 1) {  // one scene: its sweep constants by value
    const SweepK& k1 = hs[act[0]].k;
    if (any_tvf) k_force<R, DIM, true, true><<<grid_for(np, sweep_block, grid_tvf1), sweep_block, 0, stream>>>(B, k1);
    else k_force<R, DIM, false, true><<<grid_for(np, sweep_block, grid_sweep1), sweep_block, 0, stream>>>(B, k1);
    kcount++;
  } else {
    SweepK k0{};
    if (any_tvf) { k_force<R, DIM, true, false><<<gst, sweep_block, 0, stream>>>(B, k0); kcount++; }
    if (any_plain) { k_force<R, DIM, false, false><<<gsw, sweep_block, 0, stream>>>(B, k0); kcount++; }
  }
  kcount--;  // one force launch is counted with the fixed stages
  rec();
  if (any_body) { k_body_reduce<R><<<gb, 128, 0, stream>>>(B, 1); kcount++; }
  rec();
  k_final<R><<<gp, 256, 0, stream>>>(B);
  rec();
  if (any_transition) {
    // phase transitions at the end of the step (Sec. 3.6); every kernel exits at once
    // when no particle of its scene changed phase
    int gsb = std::min(ns, grid_blk);
    int gsl = grid_for(h_pfx[5 * (cap + 1) + ns], 256, grid_part);
    k_rl_flag<R><<<gp, 256, 0, stream>>>(B);
    k_rl_join<R, DIM><<<gp, 256, 0, stream>>>(B);
    k_rl_hook<R, DIM><<<gp, 256, 0, stream>>>(B);
    k_rl_root<R><<<gp, 256, 0, stream>>>(B);
    k_rl_number<R><<<gsb, 256, 0, stream>>>(B);
    k_rl_apply<R><<<gp, 256, 0, stream>>>(B);
    k_rl_slots_clear<R><<<gsb, 256, 0, stream>>>(B);
    k_rl_slots_count<R><<<gp, 256, 0, stream>>>(B);
    k_rl_slots_scan<R><<<gsb, 1024, 0, stream>>>(B);
    k_rl_slots_fill<R><<<gp, 256, 0, stream>>>(B);
    k_rl_slots_order<R><<<gb, 512, 2 * kSortCap * sizeof(int), stream>>>(B);
    k_rl_slots_adopt<R><<<gsl, 256, 0, stream>>>(B);
    k_rl_bodies_pre<R><<<grid_for(nb, 128, grid_part), 128, 0, stream>>>(B);
    k_body_mass<R><<<gb, 128, 0, stream>>>(B, 1);
    k_rl_bodies_post<R><<<gb, 128, 0, stream>>>(B);
    k_rigid_vel<R><<<gp, 256, 0, stream>>>(B, 1);
    kcount += 16;
  }
  rec();
  k_end_step<R><<<gs, 128, 0, stream>>>(B);
  rec();
  kcount += 17;
  kernels_per_step = kcount;
  SPH_CU(cudaGetLastError());
  return SPH_OK;
}

// per-stage device time (ms, averaged over reps steps launched without the graph)
template <class R, int DIM>
sph_status Engine<R, DIM>::profile(int32_t reps, double* ms) {
  cudaEvent_t ev[kStages + 1];
  for (int q = 0; q <= kStages; q++) SPH_CU(cudaEventCreate(&ev[q]));
  for (int q = 0; q < kStages; q++) ms[q] = 0.0;
  sph_status st = SPH_OK;
  for (int r = 0; r < reps && st == SPH_OK; r++) {
    st = launch_step(ev);
    if (st != SPH_OK) break;
    cudaError_t e = cudaEventSynchronize(ev[kStages]);
    if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); st = SPH_ERR_CUDA; break; }
    for (int q = 0; q < kStages; q++) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      ms[q] += t / reps;
    }
    steps_taken++;
    for (int a : act) meta[a].steps_done++;
  }
  for (int q = 0; q <= kStages; q++) cudaEventDestroy(ev[q]);
  return st;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::capture() {
  if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
  cudaGraph_t g;
  SPH_CU(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  sph_status st = launch_step(nullptr);
  cudaError_t e = cudaStreamEndCapture(stream, &g);
  if (st != SPH_OK) return st;
  SPH_CU(e);
  SPH_CU(cudaGraphInstantiate(&graph, g, 0));
  cudaGraphDestroy(g);
  graph_dirty = false;
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::check_status(int idx, bool* nonfinite) {
  int st[16];
  SPH_CU(cudaMemcpyAsync(st, hs[idx].status, sizeof(st), cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  *nonfinite = st[0] != 0;
  if (st[3] != 0) {
    set_error("inconsistent cell table or particle kinds (scene %d)", idx);
    return SPH_ERR_INVALID;
  }
  if (st[ST_CAPACITY] != 0) {
    set_error("body capacity exceeded by new bodies from solidification (scene %d)", idx);
    return SPH_ERR_CAPACITY;
  }
  if (st[ST_HOOK_TIMEOUT] != 0) {
    set_error("union-find hooking of new bodies gave up after %d retries (scene %d): relabel not applied",
              (int)SPH_RL_HOOK_TRIES, idx);
    return SPH_ERR_TIMEOUT;
  }
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::step(int32_t nsteps, bool sync) {
  if (nsteps < 0) { set_error("nsteps must be >= 0"); return SPH_ERR_INVALID; }
  if (act.empty() || nsteps == 0) return SPH_OK;
  if (graph_dirty) SPH_TRY(capture());
  for (int32_t s = 0; s < nsteps; s++) SPH_CU(cudaGraphLaunch(graph, stream));
  steps_taken += nsteps;
  for (int a : act) meta[a].steps_done += nsteps;
  if (sync) {
    SPH_CU(cudaStreamSynchronize(stream));
    for (int i : act) {
      bool nf = false;
      SPH_TRY(check_status(i, &nf));
      if (nf) { set_error("non-finite velocity in scene %d", i); return SPH_ERR_NONFINITE; }
    }
  }
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::read_fields(int idx, uint32_t mask, void* const* dst, int original_order) {
  if (!dst) { set_error("null destination array"); return SPH_ERR_INVALID; }
  const Scene<R>& S = hs[idx];
  size_t n = (size_t)S.n;
  static const int comps[SPH_F_COUNT] = {3, 3, 3, 1, 1, 1, 1, 1, 1, 3, 3, 1, 1, 3, 1, 1};
  static const int isint[SPH_F_COUNT] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 0, 0, 1, 0, 0, 0, 0};
  size_t bytes = 0;
  for (int f = 0; f < SPH_F_COUNT; f++)
    if (mask & (1u << f)) {
      if (!dst[f]) { set_error("field %d requested with a null destination", f); return SPH_ERR_INVALID; }
      bytes += n * comps[f] * (isint[f] ? 4 : 8);
    }
  if (!bytes) return SPH_OK;
  SPH_TRY(ensure_stage(bytes));
  ExportArgs ea;
  memset(&ea, 0, sizeof(ea));
  ea.original = original_order ? 1 : 0;
  // staged, then copied by the copy engine: a kernel writing page-locked host memory in
  // place measured 3.5x slower than the copy (reading it in place, for sph_write_fields,
  // measured faster)
  char* p = (char*)d_stage;
  for (int f = 0; f < SPH_F_COUNT; f++)
    if (mask & (1u << f)) {
      if (isint[f]) ea.fi[f] = (int*)p; else ea.f[f] = (double*)p;
      p += n * comps[f] * (isint[f] ? 4 : 8);
    }
  k_export<R><<<grid_for((int64_t)n, 256, grid_part), 256, 0, stream>>>(S.self, ea);
  SPH_CU(cudaGetLastError());
  p = (char*)d_stage;
  for (int f = 0; f < SPH_F_COUNT; f++)
    if (mask & (1u << f)) {
      size_t b = n * comps[f] * (isint[f] ? 4 : 8);
      SPH_CU(cudaMemcpyAsync(dst[f], p, b, cudaMemcpyDeviceToHost, stream));
      p += b;
    }
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::interpolate(int idx, int64_t nq, const double* query, int32_t field, uint32_t mask,
                                       double* out) {
  if (field != SPH_F_VEL && field != SPH_F_RHO && field != SPH_F_PRES && field != SPH_F_TEMP && field != SPH_F_CONC) {
    set_error("field %d cannot be interpolated (VEL, RHO, PRES, TEMP or CONC)", field);
    return SPH_ERR_INVALID;
  }
  if (nq < 0 || (nq > 0 && (!query || !out))) { set_error("bad query arguments"); return SPH_ERR_INVALID; }
  if (nq == 0) return SPH_OK;
  if (nq > (1LL << 30)) { set_error("at most 2^30 query points per call"); return SPH_ERR_INVALID; }
  const Scene<R>& S = hs[idx];
  int comps = field == SPH_F_VEL ? 3 : 1;
  SPH_TRY(ensure_stage(sizeof(double) * (size_t)nq * (3 + comps)));
  double* dq = (double*)d_stage;
  double* dout = dq + 3 * nq;
  SPH_CU(cudaMemcpyAsync(dq, query, sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, stream));
  k_interpolate<R, DIM><<<grid_for(nq, 128, grid_part), 128, 0, stream>>>(S.self, (int)nq, dq, field, mask, dout);
  SPH_CU(cudaGetLastError());
  SPH_CU(cudaMemcpyAsync(out, dout, sizeof(double) * comps * nq, cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::write_fields(int idx, uint32_t mask, const void* const* src) {
  const Scene<R>& S = hs[idx];
  size_t n = (size_t)S.n;
  uint32_t ok = (1u << SPH_F_POS) | (1u << SPH_F_VEL) | (1u << SPH_F_TEMP);
  if (!src || (mask & ~ok)) { set_error("write_fields supports POS, VEL and TEMP"); return SPH_ERR_INVALID; }
  for (int f = 0; f < SPH_F_COUNT; f++)
    if ((mask & (1u << f)) && !src[f]) { set_error("field %d written from a null source", f); return SPH_ERR_INVALID; }
  SPH_TRY(ensure_stage(n * 7 * 8));
  double* pos = (double*)d_stage;
  double* vel = pos + 3 * n;
  double* tmp = vel + 3 * n;
  // page-locked host buffers are read by the import kernel in place, others are staged
  struct { int f; double** d; size_t b; } in[] = {{SPH_F_POS, &pos, 24 * n}, {SPH_F_VEL, &vel, 24 * n},
                                                  {SPH_F_TEMP, &tmp, 8 * n}};
  for (auto& x : in)
    if (mask & (1u << x.f)) {
      if (void* v = device_view(src[x.f])) *x.d = (double*)v;
      else SPH_CU(cudaMemcpyAsync(*x.d, src[x.f], x.b, cudaMemcpyHostToDevice, stream));
    }
  k_import_fluid<R><<<grid_for((int64_t)n, 256, grid_part), 256, 0, stream>>>(
      S.self, (mask & (1u << SPH_F_POS)) ? pos : nullptr, (mask & (1u << SPH_F_VEL)) ? vel : nullptr,
      (mask & (1u << SPH_F_TEMP)) ? tmp : nullptr);
  SPH_CU(cudaGetLastError());
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::read_bodies(int idx, const sph_bodies_out* o, int32_t* kout) {
  const Scene<R>& S = hs[idx];
  int K = 0;
  SPH_CU(cudaMemcpyAsync(&K, S.K, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  if (kout) *kout = K;
  if (!o || K == 0) return SPH_OK;
  struct { double* h; const double* d; int c; } f[] = {{o->com, S.br, 3}, {o->quat, S.bq, 4}, {o->vel, S.bu, 3},
      {o->omega, S.bw, 3}, {o->mass, S.bm, 1}, {o->inertia, S.bIw, 9}, {o->force, S.bf, 3}, {o->torque, S.bt, 3}};
  for (auto& x : f)
    if (x.h) SPH_CU(cudaMemcpyAsync(x.h, x.d, sizeof(double) * x.c * K, cudaMemcpyDeviceToHost, stream));
  if (o->alive) SPH_CU(cudaMemcpyAsync(o->alive, S.balive, sizeof(int) * K, cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::diagnostics(int idx, double out[16]) {
  const Scene<R>& S = hs[idx];
  int nblk = grid_for(S.n, 256, 1024);
  SPH_TRY(ensure_stage(sizeof(double) * (NDIAG * nblk + 16)));
  double* part = (double*)d_stage;
  double* res = part + NDIAG * nblk;
  k_diag_part<R><<<nblk, 256, 0, stream>>>(S.self, part);
  k_diag_fin<R><<<1, 32, 0, stream>>>(S.self, part, nblk, res);
  SPH_CU(cudaGetLastError());
  SPH_CU(cudaMemcpyAsync(out, res, sizeof(double) * 16, cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

template <class R, int DIM>
sph_status Engine<R, DIM>::neighbors(int idx, int64_t* counts, int32_t* list, int64_t cap_list, int64_t* total) {
  const Scene<R>& S = hs[idx];
  size_t n = (size_t)S.n;
  int64_t* dcnt = nullptr;
  int64_t* doff = nullptr;
  int32_t* dlist = nullptr;
  SPH_CU(cudaMallocAsync((void**)&dcnt, 8 * (n + 1), stream));
  int gw = grid_for((int64_t)S.ngroups * 32, 128, grid_warp);
  k_neighbors<R, DIM><<<gw, 128, 0, stream>>>(S.self, S.ngroups, dcnt, nullptr, nullptr);
  SPH_CU(cudaGetLastError());
  std::vector<int64_t> hc(n), off(n + 1, 0);
  SPH_CU(cudaMemcpyAsync(hc.data(), dcnt, 8 * n, cudaMemcpyDeviceToHost, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  for (size_t i = 0; i < n; i++) off[i + 1] = off[i] + hc[i];
  if (counts) memcpy(counts, hc.data(), 8 * n);
  if (total) *total = off[n];
  if (list && cap_list >= off[n] && off[n] > 0) {
    SPH_CU(cudaMallocAsync((void**)&doff, 8 * (n + 1), stream));
    SPH_CU(cudaMallocAsync((void**)&dlist, 4 * (size_t)off[n], stream));
    SPH_CU(cudaMemcpyAsync(doff, off.data(), 8 * (n + 1), cudaMemcpyHostToDevice, stream));
    k_neighbors<R, DIM><<<gw, 128, 0, stream>>>(S.self, S.ngroups, dcnt, doff, dlist);
    k_sort_segments<<<grid_for((int64_t)n, 256, grid_part), 256, 0, stream>>>(doff, (int)n, dlist);
    SPH_CU(cudaGetLastError());
    SPH_CU(cudaMemcpyAsync(list, dlist, 4 * (size_t)off[n], cudaMemcpyDeviceToHost, stream));
    SPH_CU(cudaFreeAsync(doff, stream));
    SPH_CU(cudaFreeAsync(dlist, stream));
  }
  SPH_CU(cudaFreeAsync(dcnt, stream));
  SPH_CU(cudaStreamSynchronize(stream));
  return SPH_OK;
}

}  // namespace sph

namespace sph {
// continuous batching: advance every unfinished job; a job that reaches its step total
// leaves the batch tables (its memory stays until released), the others go on
template <class R, int DIM>
sph_status Engine<R, DIM>::advance_jobs(int32_t nsteps) {
  while (nsteps > 0 && !act.empty()) {
    int chunk = nsteps;
    for (int a : act)
      if (meta[a].nsteps_total > 0) chunk = std::min(chunk, meta[a].nsteps_total - meta[a].steps_done);
    if (chunk > 0) {
      SPH_TRY(step(chunk, false));
      nsteps -= chunk;
    }
    bool changed = false;
    for (int a : act)
      if (meta[a].nsteps_total > 0 && meta[a].steps_done >= meta[a].nsteps_total) {
        meta[a].done = true;
        changed = true;
      }
    if (changed) SPH_TRY(upload_tables());
    if (chunk <= 0 && !changed) break;
  }
  return SPH_OK;
}
}  // namespace sph
