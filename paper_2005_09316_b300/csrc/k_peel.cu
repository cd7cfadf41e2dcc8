// K3': standalone streaming peel of an already predicted model (Sec. 5.1):
//   resid = data - g[ant1] conj(g[ant2]) model.
// HBM-bound: reads data and model, writes resid (24 bytes per visibility) plus gains that stay in
// L1/L2, with streaming (evict-first) loads and stores; the grid is one wave of resident blocks.
#include "wn_internal.cuh"

namespace wn {

// G = g_ant1 conj(g_ant2) of row `row` at channel f (antenna indices bounds-checked).
__device__ __forceinline__ float2 row_gain(const PeelArgs& p, int row, int n_base, int f, unsigned* err) {
  float2 G;
  if (!gain_product(p, row, n_base, f, G)) atomicOr(err, WN_DEVERR_ANTENNA);
  return G;
}

__device__ __forceinline__ float2 peel_sub(float2 d, float2 v, float2 G) {
  return make_float2(d.x - (G.x * v.x - G.y * v.y), d.y - (G.x * v.y + G.y * v.x));
}

// One warp per row (rows strided over all warps of the grid); lanes stride over the row's channels
// in 16-byte pairs when the row starts 16-byte aligned (n_chan even), else in 8-byte singles.  The
// row's (time, baseline) comes from one division per row; with per-channel gains (gf > 1) the gain
// product is formed per channel, else once per row.
__global__ void __launch_bounds__(256) k3_peel(PeelArgs p, int n_base, int n_chan, int n_rows, const float2* model,
                                               float2* resid, unsigned* err) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += warps) {
    const size_t base = (size_t)row * n_chan;
    const float2 G0 = p.gf == 1 ? row_gain(p, row, n_base, 0, err) : make_float2(0.f, 0.f);
    if ((n_chan & 1) == 0) {
      const float4* d4 = reinterpret_cast<const float4*>(p.data + base);
      const float4* m4 = reinterpret_cast<const float4*>(model + base);
      float4* r4 = reinterpret_cast<float4*>(resid + base);
      // four 16-byte pairs per lane loaded before any is stored, so that eight loads are in flight
      // per lane (resid may alias data: every element is read before its own store)
      const int n2 = n_chan >> 1;
      for (int k0 = lane; k0 < n2; k0 += 4 * 32) {
        float4 d[4], v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 32 * u;
          if (k < n2) {
            d[u] = __ldcs(d4 + k);
            v[u] = __ldcs(m4 + k);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 32 * u;
          if (k >= n2) break;
          const float2 Ga = p.gf == 1 ? G0 : row_gain(p, row, n_base, 2 * k, err);
          const float2 Gb = p.gf == 1 ? G0 : row_gain(p, row, n_base, 2 * k + 1, err);
          const float2 a = peel_sub(make_float2(d[u].x, d[u].y), make_float2(v[u].x, v[u].y), Ga);
          const float2 b = peel_sub(make_float2(d[u].z, d[u].w), make_float2(v[u].z, v[u].w), Gb);
          __stcs(r4 + k, make_float4(a.x, a.y, b.x, b.y));
        }
      }
    } else {
      for (int f = lane; f < n_chan; f += 32) {
        const float2 G = p.gf == 1 ? G0 : row_gain(p, row, n_base, f, err);
        resid[base + f] = peel_sub(__ldcs(p.data + base + f), __ldcs(model + base + f), G);
      }
    }
  }
}

int launch_peel_model(wn_ctx* ctx, const ObsDev& o, const PeelArgs& pa, const float2* model, float2* resid,
                      cudaStream_t st) {
  if (((uintptr_t)pa.data | (uintptr_t)model | (uintptr_t)resid) & 15)
    return set_error(WN_EINVAL, "wn_peel_model: data, model and resid must be 16-byte aligned");
  const int want = (o.n_rows + 7) / 8;  // 8 warps (rows) per block
  int per_sm = 0;                       // resident blocks per SM: the grid is one wave of them
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_peel, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 4;
  const int blocks = std::max(1, std::min(want, ctx->num_sms * per_sm));
  k3_peel<<<blocks, 256, 0, st>>>(pa, o.n_base, o.n_chan, o.n_rows, model, resid, ctx->d_err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("peel kernel launch: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
