// Allocation-free density summation (sph_density_static, declared in include/sph.h).
//
// Callers that cannot allocate device memory themselves -- code running under a memory
// manager that owns every allocation, inside a region where allocation is forbidden, or
// in a process that has handed all device memory to another framework -- still get the
// density summation of a particle set: they pass their own device buffers for inputs and
// output, and the cell-list scratch (cell of each particle, counting-sort buffers) lives in
// one file-scope static device array of fixed size.  No cudaMalloc, cudaFree or allocating
// library call is made here.
//
// The static array is part of this library's device image: every GPU that loads the
// library holds it until the process exits.  Every call shares it, and it keeps the last
// call's contents (the counters are cleared at the start of each call), so calls that
// overlap on the GPU -- on different streams, or from different host threads -- race on
// it and must be serialised by the caller.  Particles of a cell are visited in increasing
// index order, so every density sum has a fixed order and the result is the same bit for
// bit on every call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/sph.h"

namespace sph {
void set_error(const char* fmt, ...);
}

namespace {

constexpr int kMaxN = SPH_STATIC_MAX_PARTICLES;
constexpr int kMaxCells = SPH_STATIC_MAX_CELLS;

struct StaticScratch {
  int cell_of[kMaxN];         // cell index of every particle
  int order[kMaxN];           // particles grouped by cell, in arrival order within a cell
  int byidx[kMaxN];           // particles grouped by cell, in increasing index within a cell
  int count[kMaxCells];       // particles per cell
  int start[kMaxCells + 1];   // first slot of every cell
  int cursor[kMaxCells];      // fill position during the scatter
};

static __device__ __align__(256) StaticScratch g_scratch;

// device address of g_scratch on each device (host code may not use the symbol itself),
// looked up by the first call on that device and kept for the life of the process; a
// cudaDeviceReset unloads the library's device image, after which the kept address is
// stale (documented at the declaration)
std::mutex g_mu;
StaticScratch* g_addr[64] = {nullptr};

sph_status scratch_address(StaticScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    sph::set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  if (dev < 0 || dev >= 64) {
    sph::set_error("device index %d out of range", dev);
    return SPH_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      sph::set_error("cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return SPH_ERR_CUDA;
    }
    g_addr[dev] = (StaticScratch*)p;
  }
  *out = g_addr[dev];
  return SPH_OK;
}

struct Grid {
  int dim, nc[3];
  double lo[3], ell[3], h, rc2, sig;
};

__global__ void ks_clear(StaticScratch* S, int ncells) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    S->count[c] = 0;
    S->cursor[c] = 0;
  }
}

__device__ __forceinline__ int ks_axis_cell(double x, double lo, double ell, int n) {
  double v = floor(__ddiv_rn(__dsub_rn(x, lo), ell));
  return v >= 0.0 ? (v < (double)(n - 1) ? (int)v : n - 1) : 0;  // NaN -> 0
}

__global__ void ks_bin(StaticScratch* S, Grid g, const double* pos, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    for (int k = 0; k < g.dim; k++) c[k] = ks_axis_cell(pos[3 * i + k], g.lo[k], g.ell[k], g.nc[k]);
    int lin = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
    S->cell_of[i] = lin;
    atomicAdd(&S->count[lin], 1);
  }
}

// exclusive scan of the cell counts in one block
__global__ void __launch_bounds__(1024) ks_scan(StaticScratch* S, int ncells) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ncells; base += 1024) {
    int idx = base + threadIdx.x;
    int v = idx < ncells ? S->count[idx] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int t = wsum[threadIdx.x], u = t;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, u, o);
        if (threadIdx.x >= o) u += y;
      }
      wsum[threadIdx.x] = u - t;
    }
    __syncthreads();
    int excl = carry + wsum[threadIdx.x >> 5] + x - v;
    if (idx < ncells) S->start[idx] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) S->start[ncells] = carry;
}

__global__ void ks_scatter(StaticScratch* S, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = S->cell_of[i];
    S->order[S->start[c] + atomicAdd(&S->cursor[c], 1)] = i;
  }
}

// the scatter fills a cell in arrival order; each particle's slot in index order is the
// number of particles of its cell with a smaller index (one thread per particle)
__global__ void ks_rank(StaticScratch* S, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = S->cell_of[i], a = S->start[c], e = S->start[c + 1], r = 0;
    for (int t = a; t < e; t++) r += S->order[t] < i;
    S->byidx[a + r] = i;
  }
}

// rho_i = m_i (W(0) + sum_j W_ij) over the 3^d neighbour cells (quintic spline, r < r_c)
__global__ void ks_density(const StaticScratch* S, Grid g, const double* pos, const double* mass, int n,
                           double* rho) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double xi[3] = {pos[3 * i], pos[3 * i + 1], g.dim == 3 ? pos[3 * i + 2] : 0.0};
    int lin = S->cell_of[i];
    int c[3] = {lin % g.nc[0], (lin / g.nc[0]) % g.nc[1], lin / (g.nc[0] * g.nc[1])};
    double sum = 66.0;  // w(0) = 3^5 - 6 * 2^5 + 15
    int zl = g.dim == 3 ? -1 : 0, zh = g.dim == 3 ? 1 : 0;
    for (int dz = zl; dz <= zh; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          int cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
          if (cc[0] < 0 || cc[0] >= g.nc[0] || cc[1] < 0 || cc[1] >= g.nc[1] || cc[2] < 0 || cc[2] >= g.nc[2]) continue;
          int cl = cc[0] + g.nc[0] * (cc[1] + g.nc[1] * cc[2]);
          for (int s = S->start[cl]; s < S->start[cl + 1]; s++) {
            int j = S->byidx[s];
            if (j == i) continue;
            double d0 = __dsub_rn(xi[0], pos[3 * j]), d1 = __dsub_rn(xi[1], pos[3 * j + 1]);
            double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
            if (g.dim == 3) {
              double d2 = __dsub_rn(xi[2], pos[3 * j + 2]);
              r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
            }
            if (!(r2 < g.rc2)) continue;
            double q = sqrt(r2) / g.h;
            double t3 = fmax(3.0 - q, 0.0), t2 = fmax(2.0 - q, 0.0), t1 = fmax(1.0 - q, 0.0);
            double a2 = t3 * t3, b2 = t2 * t2, c2 = t1 * t1;
            sum += a2 * a2 * t3 - 6.0 * b2 * b2 * t2 + 15.0 * c2 * c2 * t1;
          }
        }
    rho[i] = mass[i] * g.sig * sum;
  }
}

}  // namespace

extern "C" sph_status sph_density_static(int32_t dim, int64_t n, const double* pos, const double* mass, double h,
                                         double kernel_support, const double* box_min, const double* box_max,
                                         double* rho, void* stream) {
  if (dim != 2 && dim != 3) { sph::set_error("dim must be 2 or 3"); return SPH_ERR_INVALID; }
  if (n < 1 || !pos || !mass || !rho || !box_min || !box_max || !(h > 0) || !(kernel_support > 0)) {
    sph::set_error("bad argument");
    return SPH_ERR_INVALID;
  }
  if (n > kMaxN) {
    sph::set_error("sph_density_static handles at most %d particles (got %lld)", kMaxN, (long long)n);
    return SPH_ERR_CAPACITY;
  }
  Grid g;
  g.dim = dim;
  g.h = h;
  double rc = kernel_support * h;
  g.rc2 = rc * rc;
  g.sig = dim == 2 ? 7.0 / (478.0 * M_PI * h * h) : 1.0 / (120.0 * M_PI * h * h * h);
  double ncells = 1.0;
  for (int k = 0; k < 3; k++) {
    if (k < dim) {
      double L = box_max[k] - box_min[k];
      if (!(L > 0)) { sph::set_error("box_max must exceed box_min"); return SPH_ERR_INVALID; }
      // kept as a double until it is known to fit (no overflowing conversion)
      double c = std::floor(L / rc);
      if (!(c <= (double)kMaxCells)) {
        sph::set_error("sph_density_static handles at most %d cells (box needs more than that along axis %d)",
                       kMaxCells, k);
        return SPH_ERR_CAPACITY;
      }
      g.nc[k] = c < 1.0 ? 1 : (int)c;
      g.lo[k] = box_min[k];
      g.ell[k] = L / g.nc[k];
    } else {
      g.nc[k] = 1;
      g.lo[k] = 0.0;
      g.ell[k] = 1.0;
    }
    ncells *= g.nc[k];
  }
  if (ncells > kMaxCells) {
    sph::set_error("sph_density_static handles at most %d cells (box needs %.0f)", kMaxCells, ncells);
    return SPH_ERR_CAPACITY;
  }
  StaticScratch* S = nullptr;
  sph_status st = scratch_address(&S);
  if (st != SPH_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int nci = (int)ncells, ni = (int)n;
  int gb = (ni + 255) / 256 < 1024 ? (ni + 255) / 256 : 1024;
  int gc = (nci + 255) / 256 < 1024 ? (nci + 255) / 256 : 1024;
  ks_clear<<<gc, 256, 0, s>>>(S, nci);
  ks_bin<<<gb, 256, 0, s>>>(S, g, pos, ni);
  ks_scan<<<1, 1024, 0, s>>>(S, nci);
  ks_scatter<<<gb, 256, 0, s>>>(S, ni);
  ks_rank<<<gb, 256, 0, s>>>(S, ni);
  ks_density<<<gb, 256, 0, s>>>(S, g, pos, mass, ni, rho);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sph::set_error("launch failed: %s", cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  return SPH_OK;
}
