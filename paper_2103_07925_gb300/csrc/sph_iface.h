// Precision- and dimension-independent interface of the engines (host only).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

struct EngineIface {
  virtual ~EngineIface() {}
  virtual sph_status init(int capacity, cudaStream_t s) = 0;
  virtual sph_status add(const sph_params* p, const sph_particles_in* in, const sph_bodies_in* b,
                         int64_t job_id, int32_t nsteps_total, int* idx) = 0;
  virtual sph_status remove(int idx) = 0;
  virtual sph_status step(int32_t n, bool sync) = 0;
  virtual sph_status advance(int32_t n) = 0;
  virtual sph_status read_fields(int idx, uint32_t mask, void* const* dst, int original) = 0;
  virtual sph_status write_fields(int idx, uint32_t mask, const void* const* src) = 0;
  virtual sph_status interpolate(int idx, int64_t nq, const double* q, int32_t field, uint32_t mask, double* out) = 0;
  virtual sph_status read_bodies(int idx, const sph_bodies_out* o, int32_t* k) = 0;
  virtual sph_status diagnostics(int idx, double* out) = 0;
  virtual sph_status neighbors(int idx, int64_t* counts, int32_t* list, int64_t cap, int64_t* total) = 0;
  virtual sph_status info(int idx, int64_t* out) = 0;
  virtual sph_status profile(int32_t reps, double* ms) = 0;
  virtual sph_status sync() = 0;
  virtual int find_job(int64_t id) = 0;
  virtual size_t bytes_in_use() = 0;
  virtual int nscenes() = 0;
  virtual int nactive() = 0;
  virtual int64_t active_particles() = 0;
  virtual bool job_done(int idx) = 0;
  virtual bool job_reported(int idx) = 0;
  virtual bool job_failed(int idx) = 0;
  virtual sph_status check_failed() = 0;
  virtual void set_reported(int idx) = 0;
  virtual int64_t job_id(int idx) = 0;
  virtual int64_t steps_taken() = 0;
  virtual int kernels_per_step() = 0;
  virtual sph_status pairs_total(int64_t* out) = 0;  // force-sweep pairs of all resident scenes
  virtual size_t footprint(int64_t n, int64_t ncells, int64_t kcap, int64_t nrigid, bool trans, bool tvf,
                           double rc_dx, double rl_dx) = 0;
  virtual sph_status set_launch(const int32_t* cfg, int32_t n) = 0;
  virtual void get_launch(int32_t* cfg) = 0;
  virtual sph_status time_steps(int32_t n, double* ms) = 0;
};

EngineIface* make_engine_f64(int dim);
EngineIface* make_engine_f32(int dim);

}  // namespace sph
