// K3': standalone streaming peel of an already predicted model (Sec. 5.1):
//   resid = data - g[ant1] conj(g[ant2]) model.
// HBM-bound: reads data and model, writes resid (24 bytes per visibility) plus gains that stay in
// L1/L2.  Each thread moves two visibilities per 16-byte vector access; the grid is a multiple of
// the SM count and strides over the array.
#include "wn_internal.cuh"

namespace wn {

__device__ __forceinline__ float2 peel_one(const PeelArgs& p, int n_base, int n_chan, size_t i, float2 d, float2 v,
                                           unsigned* err) {
  const int row = (int)(i / n_chan), f = (int)(i - (size_t)row * n_chan);
  float2 G;
  if (!gain_product(p, row, n_base, f, G)) atomicOr(err, WN_DEVERR_ANTENNA);
  return make_float2(d.x - (G.x * v.x - G.y * v.y), d.y - (G.x * v.y + G.y * v.x));
}

__global__ void __launch_bounds__(256) k3_peel(PeelArgs p, int n_base, int n_chan, size_t n, const float2* model,
                                               float2* resid, unsigned* err) {
  const size_t n2 = n / 2;
  const float4* d4 = reinterpret_cast<const float4*>(p.data);
  const float4* m4 = reinterpret_cast<const float4*>(model);
  float4* r4 = reinterpret_cast<float4*>(resid);
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += (size_t)gridDim.x * blockDim.x) {
    const float4 d = __ldcs(d4 + k);
    const float4 v = __ldcs(m4 + k);
    const float2 a = peel_one(p, n_base, n_chan, 2 * k, make_float2(d.x, d.y), make_float2(v.x, v.y), err);
    const float2 b = peel_one(p, n_base, n_chan, 2 * k + 1, make_float2(d.z, d.w), make_float2(v.z, v.w), err);
    __stcs(r4 + k, make_float4(a.x, a.y, b.x, b.y));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
    const size_t i = n - 1;
    resid[i] = peel_one(p, n_base, n_chan, i, p.data[i], model[i], err);
  }
}

int launch_peel_model(wn_ctx* ctx, const ObsDev& o, const PeelArgs& pa, const float2* model, float2* resid,
                      cudaStream_t st) {
  const size_t n = (size_t)o.n_rows * o.n_chan;
  if (((uintptr_t)pa.data | (uintptr_t)model | (uintptr_t)resid) & 15)
    return set_error(WN_EINVAL, "wn_peel_model: data, model and resid must be 16-byte aligned");
  const size_t want = (n / 2 + 255) / 256;
  const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)ctx->num_sms * 8));
  k3_peel<<<blocks, 256, 0, st>>>(pa, o.n_base, o.n_chan, n, model, resid, ctx->d_err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("peel kernel launch: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
