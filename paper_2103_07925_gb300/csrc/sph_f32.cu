// FP32 instantiation of the engine (2D and 3D): FP32 pair sums on cell-relative
// positions, FP64 bodies and diagnostics.
#include "sph_impl.cuh"

namespace sph {
EngineIface* make_engine_f32(int dim) {
  if (dim == 2) return new EngineImpl<float, 2>();
  return new EngineImpl<float, 3>();
}
}  // namespace sph
