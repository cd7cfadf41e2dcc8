// K2 placeholder (replaced by the tcgen05 shapelet contraction).
#include "wn_internal.cuh"
namespace wn {
int launch_shapelets(wn_ctx*, const ObsDev&, const Model*, float2*, int, const PeelArgs&, cudaStream_t) {
  return set_error(WN_EINVAL, "shapelet kernel not built yet");
}
}  // namespace wn
extern "C" int wn_predict_grad(wn_ctx*, const wn_obs*, int, const void*, int, int, const void*, void*,
                               const wn_sky_grad*, double*, void*) {
  return wn::set_error(WN_EINVAL, "adjoint not built yet");
}
