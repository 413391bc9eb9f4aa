// FP64 instantiation of the engine (2D and 3D).
#include "sph_impl.cuh"

namespace sph {
EngineIface* make_engine_f64(int dim) {
  if (dim == 2) return new EngineImpl<double, 2>();
  return new EngineImpl<double, 3>();
}
}  // namespace sph
