// EngineIface implementation over Engine<R, DIM>; included by one translation unit per
// precision so that the two instantiations compile in parallel.
#pragma once
#include "sph_engine.cuh"
#include "sph_iface.h"

namespace sph {

template <class R, int DIM>
struct EngineImpl final : EngineIface {
  Engine<R, DIM> e;
  sph_status init(int capacity, cudaStream_t s) override { return e.init(capacity, s); }
  sph_status add(const sph_params* p, const sph_particles_in* in, const sph_bodies_in* b, int64_t job,
                 int32_t total, int* idx) override {
    return e.add_scene(p, in, b, job, total, idx);
  }
  sph_status remove(int idx) override { return e.remove_scene(idx); }
  sph_status step(int32_t n, bool sync) override { return e.step(n, sync); }
  sph_status advance(int32_t n) override { return e.advance_jobs(n); }
  sph_status read_fields(int idx, uint32_t m, void* const* d, int o) override { return e.read_fields(idx, m, d, o); }
  sph_status write_fields(int idx, uint32_t m, const void* const* s) override { return e.write_fields(idx, m, s); }
  sph_status interpolate(int idx, int64_t nq, const double* q, int32_t f, uint32_t m, double* out) override {
    return e.interpolate(idx, nq, q, f, m, out);
  }
  sph_status read_bodies(int idx, const sph_bodies_out* o, int32_t* k) override { return e.read_bodies(idx, o, k); }
  sph_status diagnostics(int idx, double* out) override { return e.diagnostics(idx, out); }
  sph_status neighbors(int idx, int64_t* c, int32_t* l, int64_t cap, int64_t* t) override {
    return e.neighbors(idx, c, l, cap, t);
  }
  sph_status info(int idx, int64_t* out) override {
    const Scene<R>& S = e.hs[idx];
    const HostScene& M = e.meta[idx];
    for (int q = 0; q < 32; q++) out[q] = 0;
    out[0] = S.n; out[1] = M.nfluid; out[2] = M.nrigid; out[3] = M.nwall; out[4] = M.K0;
    out[5] = S.ncells; out[6] = S.ncell[0]; out[7] = S.ncell[1]; out[8] = S.ncell[2];
    out[9] = M.steps_done; out[10] = e.kernels_per_step; out[11] = (int64_t)M.bytes;
    out[12] = S.ngroups; out[13] = S.G; out[14] = S.key_order;
    unsigned long long pc[2] = {0, 0};
    int st[16] = {0};
    if (cudaMemcpyAsync(pc, S.pairs, sizeof(pc), cudaMemcpyDeviceToHost, e.stream) != cudaSuccess ||
        cudaMemcpyAsync(st, S.status, sizeof(st), cudaMemcpyDeviceToHost, e.stream) != cudaSuccess ||
        cudaStreamSynchronize(e.stream) != cudaSuccess) {
      set_error("cannot read the scene counters");
      return SPH_ERR_CUDA;
    }
    out[15] = (int64_t)pc[1];
    out[16] = st[6];
    out[17] = S.maxnb;
    out[18] = st[9];
    int32_t lc[3];
    e.get_launch(lc);
    out[19] = lc[0]; out[20] = lc[1]; out[21] = lc[2];
    return SPH_OK;
  }
  sph_status set_launch(const int32_t* cfg, int32_t n) override { return e.set_launch(cfg, n); }
  void get_launch(int32_t* cfg) override { e.get_launch(cfg); }
  sph_status time_steps(int32_t n, double* ms) override { return e.time_steps(n, ms); }
  sph_status profile(int32_t reps, double* ms) override { return e.profile(reps, ms); }
  sph_status sync() override {
    cudaError_t err = cudaStreamSynchronize(e.stream);
    if (err != cudaSuccess) { set_error("%s", cudaGetErrorString(err)); return SPH_ERR_CUDA; }
    return SPH_OK;
  }
  int find_job(int64_t id) override { return e.find_job(id); }
  size_t bytes_in_use() override { return e.bytes_in_use(); }
  int nscenes() override { return (int)e.hs.size(); }
  int nactive() override { return (int)e.act.size(); }
  int64_t active_particles() override {
    int64_t t = 0;
    for (int a : e.act) t += e.hs[a].n;
    return t;
  }
  bool job_done(int idx) override { return e.meta[idx].done; }
  bool job_reported(int idx) override { return e.meta[idx].reported; }
  bool job_failed(int idx) override { return e.meta[idx].failed; }
  sph_status check_failed() override { return e.check_failed(); }
  void set_reported(int idx) override { e.meta[idx].reported = true; }
  int64_t job_id(int idx) override { return e.meta[idx].job_id; }
  int64_t steps_taken() override { return e.steps_taken; }
  int kernels_per_step() override { return e.act.empty() ? 0 : e.kernels_per_step; }
  sph_status pairs_total(int64_t* out) override {
    *out = 0;
    for (auto& S : e.hs) {
      unsigned long long pc[2] = {0, 0};
      if (cudaMemcpyAsync(pc, S.pairs, sizeof(pc), cudaMemcpyDeviceToHost, e.stream) != cudaSuccess ||
          cudaStreamSynchronize(e.stream) != cudaSuccess) {
        set_error("cannot read the scene counters");
        return SPH_ERR_CUDA;
      }
      *out += (int64_t)pc[1];
    }
    return SPH_OK;
  }
  size_t footprint(int64_t n, int64_t nc, int64_t kc, int64_t nr, bool trans, bool tvf, double rc_dx,
                   double rl_dx) override {
    return Engine<R, DIM>::footprint(n, nc, kc, nr, trans, tvf, rc_dx, rl_dx);
  }
};

}  // namespace sph
