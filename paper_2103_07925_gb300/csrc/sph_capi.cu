// C ABI of libsph (declared in include/sph.h).  No exception or C++ type crosses this
// boundary; errors are status codes with a thread-local message.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "sph_iface.h"

namespace sph {
static thread_local char g_err[1024];
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
}  // namespace sph

using namespace sph;

struct sph_scene {
  EngineIface* e;
  int prec, dim;
};

struct sph_batch {
  EngineIface* e[2];  // 2D and 3D scenes
  int prec;
  size_t cap_bytes;
  int cap_scenes;
  cudaStream_t stream;
  bool own_stream;
  int64_t next_id;
};

static EngineIface* make_engine(int prec, int dim) {
  try {
    return prec == 32 ? make_engine_f32(dim) : make_engine_f64(dim);
  } catch (...) {
    return nullptr;
  }
}

static sph_status check_common(const sph_params* p) {
  if (!p) { set_error("null params"); return SPH_ERR_INVALID; }
  if (p->dim != 2 && p->dim != 3) { set_error("dim must be 2 or 3"); return SPH_ERR_INVALID; }
  if (p->precision != 32 && p->precision != 64) { set_error("precision must be 32 or 64"); return SPH_ERR_INVALID; }
  return SPH_OK;
}

extern "C" {

const char* sph_last_error(void) { return g_err; }

sph_status sph_create_scene(const sph_params* params, const sph_particles_in* particles,
                            const sph_bodies_in* bodies, void* stream, sph_scene** out) {
  if (!out) { set_error("null output pointer"); return SPH_ERR_INVALID; }
  *out = nullptr;
  sph_status st = check_common(params);
  if (st != SPH_OK) return st;
  EngineIface* e = make_engine(params->precision, params->dim);
  if (!e) { set_error("out of host memory"); return SPH_ERR_OOM; }
  st = e->init(1, (cudaStream_t)stream);
  if (st == SPH_OK) {
    int idx = -1;
    st = e->add(params, particles, bodies, -1, 0, &idx);
  }
  if (st != SPH_OK) {
    delete e;
    return st;
  }
  sph_scene* s = new (std::nothrow) sph_scene{e, params->precision, params->dim};
  if (!s) { delete e; set_error("out of host memory"); return SPH_ERR_OOM; }
  *out = s;
  return SPH_OK;
}

sph_status sph_step(sph_scene* s, int32_t nsteps) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->step(nsteps, true);
}

sph_status sph_step_async(sph_scene* s, int32_t nsteps) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->step(nsteps, false);
}

sph_status sph_read_fields(sph_scene* s, uint32_t mask, void* const* dst, int32_t original_order) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->read_fields(0, mask, dst, original_order);
}

sph_status sph_write_fields(sph_scene* s, uint32_t mask, const void* const* src) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->write_fields(0, mask, src);
}

sph_status sph_interpolate(sph_scene* s, int64_t nq, const double* query, int32_t field, uint32_t material_mask,
                           double* out) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->interpolate(0, nq, query, field, material_mask, out);
}

sph_status sph_read_bodies(sph_scene* s, const sph_bodies_out* out, int32_t* k_out) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->read_bodies(0, out, k_out);
}

sph_status sph_diagnostics(sph_scene* s, double out[16]) {
  if (!s || !out) { set_error("null argument"); return SPH_ERR_INVALID; }
  return s->e->diagnostics(0, out);
}

sph_status sph_neighbors(sph_scene* s, int64_t* counts, int32_t* list, int64_t cap, int64_t* total) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->neighbors(0, counts, list, cap, total);
}

sph_status sph_info(sph_scene* s, int64_t out[32]) {
  if (!s || !out) { set_error("null argument"); return SPH_ERR_INVALID; }
  return s->e->info(0, out);
}

sph_status sph_set_launch(sph_scene* s, const int32_t* cfg, int32_t n) {
  if (!s || (n > 0 && !cfg)) { set_error("null argument"); return SPH_ERR_INVALID; }
  return s->e->set_launch(cfg, n);
}

sph_status sph_time_steps(sph_scene* s, int32_t nsteps, double* ms) {
  if (!s) { set_error("null scene"); return SPH_ERR_INVALID; }
  return s->e->time_steps(nsteps, ms);
}

sph_status sph_profile(sph_scene* s, int32_t reps, double* ms_per_stage) {
  if (!s || !ms_per_stage || reps < 1) { set_error("bad argument"); return SPH_ERR_INVALID; }
  return s->e->profile(reps, ms_per_stage);
}

const char* sph_profile_stage_name(int32_t i) {
  static const char* const names[] = {"umax", "dt", "body_kick_drift", "kick_drift", "decide", "bin",
                                      "scan_blocks", "scan_top", "scan_cells", "scatter", "rank", "permute",
                                      "flip", "search", "density", "extrap", "force", "body_reduce",
                                      "final", "relabel", "end_step"};
  static_assert(sizeof(names) / sizeof(names[0]) == SPH_PROFILE_STAGES, "one name per profiled stage");
  if (i < 0 || i >= SPH_PROFILE_STAGES) return "";
  return names[i];
}

void sph_destroy_scene(sph_scene* s) {
  if (!s) return;
  delete s->e;
  delete s;
}

// ------------------------------------------------------------------------ batches
sph_status sph_batch_create(int32_t capacity_scenes, size_t hbm_cap_bytes, int32_t precision, void* stream,
                            sph_batch** out) {
  if (!out) { set_error("null output pointer"); return SPH_ERR_INVALID; }
  *out = nullptr;
  if (capacity_scenes < 1 || capacity_scenes > (1 << 20)) { set_error("capacity must be in [1, 2^20]"); return SPH_ERR_INVALID; }
  if (precision != 32 && precision != 64) { set_error("precision must be 32 or 64"); return SPH_ERR_INVALID; }
  sph_batch* b = new (std::nothrow) sph_batch();
  if (!b) { set_error("out of host memory"); return SPH_ERR_OOM; }
  b->prec = precision;
  b->cap_bytes = hbm_cap_bytes;
  b->cap_scenes = capacity_scenes;
  b->next_id = 1;
  b->own_stream = stream == nullptr;
  if (stream) b->stream = (cudaStream_t)stream;
  else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    set_error("cannot create a CUDA stream");
    return SPH_ERR_CUDA;
  }
  for (int d = 0; d < 2; d++) {
    b->e[d] = make_engine(precision, d + 2);
    sph_status st = b->e[d] ? b->e[d]->init(capacity_scenes, b->stream) : SPH_ERR_OOM;
    if (st != SPH_OK) {
      sph_batch_destroy(b);
      return st;
    }
  }
  *out = b;
  return SPH_OK;
}

static sph_status footprint_of(const sph_job_desc* job, int prec, size_t* bytes) {
  if (!job || !job->params || !job->particles) { set_error("incomplete job"); return SPH_ERR_INVALID; }
  const sph_params* p = job->params;
  if (p->dim != 2 && p->dim != 3) { set_error("dim must be 2 or 3"); return SPH_ERR_INVALID; }
  if (!(p->dx > 0.0) || !(p->h > 0.0) || !(p->kernel_support > 0.0) || !std::isfinite(p->dx) ||
      !std::isfinite(p->h * p->kernel_support)) {
    set_error("dx, h and kernel_support must be positive and finite");
    return SPH_ERR_INVALID;
  }
  if (job->particles->n < 1 || job->particles->n > (1LL << 26)) {
    set_error("particle count must be in [1, 2^26]");
    return SPH_ERR_INVALID;
  }
  if (!job->particles->material || !p->materials || p->n_materials < 1) {
    set_error("materials and particle materials are required");
    return SPH_ERR_INVALID;
  }
  for (int64_t i = 0; i < job->particles->n; i++)
    if (job->particles->material[i] < 0 || job->particles->material[i] >= p->n_materials) {
      set_error("particle %lld: material %d out of range", (long long)i, job->particles->material[i]);
      return SPH_ERR_INVALID;
    }
  double rc = p->kernel_support * p->h;
  int64_t nc = 1;
  for (int d = 0; d < p->dim; d++) {
    double L = p->box_max[d] - p->box_min[d];
    int64_t c = (int64_t)std::floor(L / rc);
    nc *= c < 1 ? 1 : c;
  }
  int64_t n = job->particles->n, nr = 0;
  bool trans = false;
  for (int q = 0; q < p->n_materials; q++) trans |= p->materials[q].transitions_to >= 0;
  for (int64_t i = 0; i < n; i++)
    if (p->materials[job->particles->material[i]].kind == SPH_RIGID) nr++;
  int64_t K = job->bodies ? job->bodies->k : 0;
  int64_t kcap = p->body_capacity > K ? p->body_capacity : K + (trans ? 1024 : 0);
  if (trans) nr = n;
  EngineIface* e = make_engine(prec, p->dim);
  if (!e) { set_error("out of host memory"); return SPH_ERR_OOM; }
  double skin = p->skin > 0.0 ? p->skin : 0.0;
  *bytes = e->footprint(n, nc, kcap < 1 ? 1 : kcap, nr < 1 ? 1 : nr, trans, p->p_background > 0.0, rc / p->dx,
                        (rc + skin) / p->dx);
  delete e;
  return SPH_OK;
}

sph_status sph_job_footprint(const sph_job_desc* job, size_t* bytes) {
  if (!bytes) { set_error("null output"); return SPH_ERR_INVALID; }
  int prec = (job && job->params && job->params->precision == 32) ? 32 : 64;
  return footprint_of(job, prec, bytes);
}

sph_status sph_batch_admit(sph_batch* b, const sph_job_desc* job, int64_t* job_id) {
  if (!b || !job || !job->params) { set_error("null argument"); return SPH_ERR_INVALID; }
  sph_params p = *job->params;
  p.precision = b->prec;
  sph_status st = check_common(&p);
  if (st != SPH_OK) return st;
  size_t need = 0;
  sph_job_desc jd = *job;
  jd.params = &p;
  st = footprint_of(&jd, b->prec, &need);
  if (st != SPH_OK) return st;
  size_t used = b->e[0]->bytes_in_use() + b->e[1]->bytes_in_use();
  int resident = b->e[0]->nscenes() + b->e[1]->nscenes();
  if (resident >= b->cap_scenes || used + need > b->cap_bytes) {
    set_error("job does not fit: %d resident, %zu + %zu bytes over the cap %zu", resident, used, need, b->cap_bytes);
    return SPH_ERR_CAPACITY;
  }
  int64_t id = b->next_id++;
  int idx = -1;
  st = b->e[p.dim - 2]->add(&p, job->particles, job->bodies, id, job->nsteps_total, &idx);
  if (st != SPH_OK) return st;
  if (job_id) *job_id = id;
  return SPH_OK;
}

sph_status sph_batch_step(sph_batch* b, int32_t nsteps) {
  if (!b) { set_error("null batch"); return SPH_ERR_INVALID; }
  for (int d = 0; d < 2; d++) {
    sph_status st = b->e[d]->advance(nsteps);
    if (st != SPH_OK) return st;
  }
  return SPH_OK;
}

sph_status sph_batch_poll(sph_batch* b, int64_t* done_ids, int32_t max_done, int32_t* n_done) {
  if (!b || !n_done) { set_error("null argument"); return SPH_ERR_INVALID; }
  *n_done = 0;
  for (int d = 0; d < 2; d++) {
    sph_status st = b->e[d]->sync();
    if (st == SPH_OK) st = b->e[d]->check_failed();
    if (st != SPH_OK) return st;
    for (int i = 0; i < b->e[d]->nscenes() && *n_done < max_done; i++)
      if (b->e[d]->job_done(i) && !b->e[d]->job_reported(i)) {
        if (done_ids) done_ids[*n_done] = b->e[d]->job_id(i);
        (*n_done)++;
        b->e[d]->set_reported(i);
      }
  }
  return SPH_OK;
}

static bool locate(sph_batch* b, int64_t id, int* d, int* idx) {
  for (int q = 0; q < 2; q++) {
    int i = b->e[q]->find_job(id);
    if (i >= 0) { *d = q; *idx = i; return true; }
  }
  set_error("unknown job id %lld", (long long)id);
  return false;
}

sph_status sph_batch_job_state(sph_batch* b, int64_t job_id, int32_t* state) {
  if (!b || !state) { set_error("null argument"); return SPH_ERR_INVALID; }
  int d, i;
  if (!locate(b, job_id, &d, &i)) return SPH_ERR_INVALID;
  *state = b->e[d]->job_failed(i) ? 2 : (b->e[d]->job_done(i) ? 1 : 0);
  return SPH_OK;
}

sph_status sph_batch_read_fields(sph_batch* b, int64_t job_id, uint32_t mask, void* const* dst) {
  if (!b) { set_error("null batch"); return SPH_ERR_INVALID; }
  int d, i;
  if (!locate(b, job_id, &d, &i)) return SPH_ERR_INVALID;
  return b->e[d]->read_fields(i, mask, dst, 1);
}

sph_status sph_batch_job_diagnostics(sph_batch* b, int64_t job_id, double out[16]) {
  if (!b || !out) { set_error("null argument"); return SPH_ERR_INVALID; }
  int d, i;
  if (!locate(b, job_id, &d, &i)) return SPH_ERR_INVALID;
  return b->e[d]->diagnostics(i, out);
}

sph_status sph_batch_release(sph_batch* b, int64_t job_id) {
  if (!b) { set_error("null batch"); return SPH_ERR_INVALID; }
  int d, i;
  if (!locate(b, job_id, &d, &i)) return SPH_ERR_INVALID;
  return b->e[d]->remove(i);
}

sph_status sph_batch_info(sph_batch* b, int64_t out[8]) {
  if (!b || !out) { set_error("null argument"); return SPH_ERR_INVALID; }
  for (int q = 0; q < 8; q++) out[q] = 0;
  for (int d = 0; d < 2; d++) {
    out[0] += b->e[d]->nscenes();
    out[1] += b->e[d]->active_particles();
    out[2] += (int64_t)b->e[d]->bytes_in_use();
    out[3] += b->e[d]->steps_taken();
    out[4] += b->e[d]->nactive();
    out[5] += b->e[d]->kernels_per_step();
    int64_t pc = 0;
    sph_status st = b->e[d]->pairs_total(&pc);
    if (st != SPH_OK) return st;
    out[6] += pc;
  }
  return SPH_OK;
}

sph_status sph_batch_set_launch(sph_batch* b, int32_t dim, const int32_t* cfg, int32_t n) {
  if (!b || (n > 0 && !cfg)) { set_error("null argument"); return SPH_ERR_INVALID; }
  if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return SPH_ERR_INVALID; }
  return b->e[dim - 2]->set_launch(cfg, n);
}

sph_status sph_batch_time_steps(sph_batch* b, int32_t nsteps, double* ms) {
  if (!b || !ms || nsteps < 1) { set_error("time_steps needs a batch, nsteps >= 1 and an output"); return SPH_ERR_INVALID; }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) { set_error("cudaEventCreate failed"); return SPH_ERR_CUDA; }
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); set_error("cudaEventCreate failed"); return SPH_ERR_CUDA; }
  sph_status st = cudaEventRecord(e0, b->stream) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
  for (int d = 0; d < 2 && st == SPH_OK; d++) st = b->e[d]->advance(nsteps);
  if (st == SPH_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) st = SPH_ERR_CUDA;
  if (st == SPH_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SPH_ERR_CUDA;
  float t = 0.f;
  if (st == SPH_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = SPH_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == SPH_ERR_CUDA) set_error("event timing failed");
  *ms = t;
  return st;
}

void sph_batch_destroy(sph_batch* b) {
  if (!b) return;
  for (int d = 0; d < 2; d++) delete b->e[d];
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
