// K7: per-antenna complex gain calibration, the linearised least squares of Sec. 5.1 (eq:peeling-iter).
//
// For one (time, channel) the model is M_ij = g_i conj(g_j) I_ij and the data V_ij.  With additive
// errors e on the gains and the e e* term dropped, R = V - M ~ e_i a_ij + conj(e_j) c_ij with
// a_ij = conj(g_j) I_ij and c_ij = g_i I_ij.  The real parameters are Re(e_i), Im(e_i); the
// conjugation shows up as sign flips on Im(e_j).  Each iteration solves the normal equations
// [A^T A] x = A^T b (b = Re, Im of R) and sets g <- g + e.  The overall phase of the gains is free,
// so A^T A as printed is singular; the gauge is fixed by holding Im(e_0) = 0 (its column is dropped),
// leaving n = 2A - 1 parameters.
//
// A^T A has a closed block form that the kernel accumulates directly, without the design matrix:
//   diagonal 2x2 block of antenna i:  (sum over its baselines of |a|^2 or |c|^2) times the identity;
//   off-diagonal block of baseline (p, q):  [[P, Q], [Q, -P]] with P + iQ = conj(a_pq) c_pq;
//   A^T b for antenna i:  conj(a) R as (Re, Im) where i = ant1, and (Re, -Im) of conj(c) R where i = ant2.
//
// One CTA per (time, channel) owns its problem through every iteration: gains and the packed lower
// triangle of [A^T A | A^T b] (the right-hand side as an extra row, so the Cholesky factorisation also
// does the forward substitution) stay in shared memory.  Warp w accumulates antennas w, w + 16, ...
// over their incident baselines in a fixed order (no atomics on the sums), the factorisation is a
// right-looking Cholesky in FP32 over all warps, and warp 0 back-substitutes.  A non-positive pivot
// stops the problem's iterations with the last gains kept and WN_DEVERR_CALIB set.
#include "wn_internal.cuh"

namespace wn {

constexpr int K7_THREADS = 512;
constexpr int K7_WARPS = K7_THREADS / 32;
constexpr int K7_MAX_ANT = 128;

struct K7Args {
  const float2* model;  // I [T][B][F]
  const float2* data;   // V [T][B][F]
  float2* gains;        // [T][F][A], in and out
  const int* ant1;
  const int* ant2;
  const int* inc_off;   // [A + 1] offsets into inc_list
  const int* inc_list;  // (baseline << 1) | role, role 0: antenna is ant1, 1: antenna is ant2
  int n_ant, n_base, n_time, n_chan, n_iter;
  unsigned* err;
};

__device__ __forceinline__ int col_re(int i) { return i == 0 ? 0 : 2 * i - 1; }
__device__ __forceinline__ int col_im(int i) { return 2 * i; }  // antennas i >= 1
__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }  // r >= c

__device__ __forceinline__ float2 cmul(float2 x, float2 y) {
  return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}
__device__ __forceinline__ float2 cconj(float2 x) { return make_float2(x.x, -x.y); }

// Incidence lists: for each antenna its baselines in increasing order, tagged with the antenna's role.
// One block, thread per antenna.  A baseline with an antenna index outside [0, n_ant) or ant1 >= ant2
// is left out of every list (so the solve never indexes with it) and sets WN_DEVERR_ANTENNA.
__device__ __forceinline__ bool k7_valid(int p, int q, int n_ant) { return 0 <= p && p < q && q < n_ant; }

__global__ void k7_incidence(const int* ant1, const int* ant2, int n_base, int n_ant, int* off, int* list,
                             unsigned* err) {
  __shared__ int cnt[K7_MAX_ANT + 1];
  const int i = threadIdx.x;
  if (i < n_ant) {
    int c = 0;
    for (int b = 0; b < n_base; ++b)
      if (k7_valid(ant1[b], ant2[b], n_ant)) c += (ant1[b] == i) + (ant2[b] == i);
    cnt[i] = c;
  }
  if (i == 0) {
    for (int b = 0; b < n_base; ++b)
      if (!k7_valid(ant1[b], ant2[b], n_ant)) atomicOr(err, WN_DEVERR_ANTENNA);
  }
  __syncthreads();
  if (i == 0) {
    int s = 0;
    for (int a = 0; a < n_ant; ++a) {
      off[a] = s;
      s += cnt[a];
    }
    off[n_ant] = s;
  }
  __syncthreads();
  if (i < n_ant) {
    int k = off[i];
    for (int b = 0; b < n_base; ++b) {
      if (!k7_valid(ant1[b], ant2[b], n_ant)) continue;
      if (ant1[b] == i) list[k++] = b << 1;
      else if (ant2[b] == i) list[k++] = (b << 1) | 1;
    }
  }
}

__global__ void __launch_bounds__(K7_THREADS, 1) k7_calib(const K7Args a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int A = a.n_ant, n = 2 * A - 1;
  float* N = reinterpret_cast<float*>(sm);                            // packed lower, (n+1)(n+2)/2
  float* col = N + (n + 1) * (n + 2) / 2;                             // [n + 1]
  float* x = col + n + 1;                                             // [n]
  float2* g = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(x + n + 1) + 7) & ~(uintptr_t)7);  // [A]
  __shared__ float s_rinv;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = blockIdx.x / a.n_chan, f = blockIdx.x % a.n_chan;
  float2* gout = a.gains + ((size_t)t * a.n_chan + f) * A;
  for (int i = tid; i < A; i += K7_THREADS) g[i] = gout[i];
  if (tid == 0) s_bad = 0;
  const int packed = (n + 1) * (n + 2) / 2;
  const size_t plane = (size_t)a.n_base * a.n_chan;

  for (int it = 0; it < a.n_iter; ++it) {
    __syncthreads();
    for (int k = tid; k < packed; k += K7_THREADS) N[k] = 0.f;
    __syncthreads();
    // --- [A^T A | A^T b] at the current gains
    for (int i = warp; i < A; i += K7_WARPS) {
      float d = 0.f, br = 0.f, bi = 0.f;
      for (int k = a.inc_off[i] + lane; k < a.inc_off[i + 1]; k += 32) {
        const int e = a.inc_list[k], b = e >> 1;
        const size_t idx = (size_t)t * plane + (size_t)b * a.n_chan + f;
        const float2 I = a.model[idx], V = a.data[idx];
        const int p = a.ant1[b], q = a.ant2[b];
        const float2 gp = g[p], gq = g[q];
        const float2 M = cmul(cmul(gp, cconj(gq)), I);
        const float2 R = make_float2(V.x - M.x, V.y - M.y);
        if ((e & 1) == 0) {
          const float2 av = cmul(cconj(gq), I), cv = cmul(gp, I);
          d += av.x * av.x + av.y * av.y;
          const float2 aR = cmul(cconj(av), R);
          br += aR.x;
          bi += aR.y;
          // the block of this baseline, rows of q (> p) and columns of p
          const float2 ac = cmul(cconj(av), cv);
          atomicAdd(&N[tri(col_re(q), col_re(p))], ac.x);
          atomicAdd(&N[tri(col_im(q), col_re(p))], ac.y);
          if (p > 0) {
            atomicAdd(&N[tri(col_re(q), col_im(p))], ac.y);
            atomicAdd(&N[tri(col_im(q), col_im(p))], -ac.x);
          }
        } else {
          const float2 cv = cmul(gp, I);
          d += cv.x * cv.x + cv.y * cv.y;
          const float2 cR = cmul(cconj(cv), R);
          br += cR.x;
          bi -= cR.y;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        br += __shfl_xor_sync(0xffffffffu, br, o);
        bi += __shfl_xor_sync(0xffffffffu, bi, o);
      }
      if (lane == 0) {
        N[tri(col_re(i), col_re(i))] = d;
        N[tri(n, col_re(i))] = br;  // right-hand side: row n
        if (i > 0) {
          N[tri(col_im(i), col_im(i))] = d;
          N[tri(n, col_im(i))] = bi;
        }
      }
    }
    // --- Cholesky of the leading n x n block; row n becomes L^{-1} (A^T b)
    for (int k = 0; k < n; ++k) {
      __syncthreads();
      if (tid == 0) {
        float piv = N[tri(k, k)];
        if (!(piv > 0.f) || !isfinite(piv)) {
          s_bad = 1;
          piv = 1.f;
        }
        const float l = sqrtf(piv);
        N[tri(k, k)] = l;
        s_rinv = 1.0f / l;
      }
      __syncthreads();
      const float rinv = s_rinv;
      for (int j = k + 1 + tid; j <= n; j += K7_THREADS) {
        const float v = N[tri(j, k)] * rinv;
        N[tri(j, k)] = v;
        col[j] = v;
      }
      __syncthreads();
      for (int i = k + 1 + warp; i <= n; i += K7_WARPS) {
        const float ci = col[i];
        float* row = N + tri(i, 0);
        const int jmax = min(i, n - 1);
        for (int j = k + 1 + lane; j <= jmax; j += 32) row[j] -= ci * col[j];
      }
    }
    __syncthreads();
    // --- back substitution L^T x = y (warp 0)
    if (warp == 0) {
      for (int k = n - 1; k >= 0; --k) {
        float s = 0.f;
        for (int j = k + 1 + lane; j < n; j += 32) s += N[tri(j, k)] * x[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[k] = (N[tri(n, k)] - s) / N[tri(k, k)];
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_bad) break;
    // --- g <- g + e
    for (int i = tid; i < A; i += K7_THREADS) {
      const float2 gi = g[i];
      g[i] = make_float2(gi.x + x[col_re(i)], gi.y + (i > 0 ? x[col_im(i)] : 0.f));
    }
  }
  __syncthreads();
  if (s_bad && tid == 0) atomicOr(a.err, WN_DEVERR_CALIB);
  for (int i = tid; i < A; i += K7_THREADS) gout[i] = g[i];
}

size_t k7_smem_bytes(int n_ant) {
  const int n = 2 * n_ant - 1;
  return sizeof(float) * ((size_t)(n + 1) * (n + 2) / 2 + (n + 1) + ((n + 1) & ~1) + 1) + sizeof(float2) * n_ant + 16;
}

int launch_calibrate(wn_ctx* ctx, const ObsDev& o, const float2* model, const float2* data, float2* gains, int n_iter,
                     cudaStream_t st) {
  if (o.n_ant > K7_MAX_ANT) return set_error(WN_EINVAL, "wn_calibrate: at most 128 antennas");
  // workspace: incidence offsets and lists (reuses the adjoint workspace)
  const size_t need = ((size_t)(o.n_ant + 1) * 4 + 255 & ~(size_t)255) + (size_t)2 * o.n_base * 4;
  if (ctx->ws2_bytes < need) {
    if (ctx->ws2) {
      cudaStreamSynchronize(st);
      cudaFree(ctx->ws2);
      ctx->ws2 = nullptr;
      ctx->ws2_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws2, need);
    if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("calibration workspace: ") + cudaGetErrorString(e));
    ctx->ws2_bytes = need;
  }
  int* off = static_cast<int*>(ctx->ws2);
  int* list = off + (((size_t)(o.n_ant + 1) * 4 + 255 & ~(size_t)255) / 4);
  k7_incidence<<<1, K7_MAX_ANT, 0, st>>>(o.ant1, o.ant2, o.n_base, o.n_ant, off, list, ctx->d_err);
  K7Args a;
  a.model = model;
  a.data = data;
  a.gains = gains;
  a.ant1 = o.ant1;
  a.ant2 = o.ant2;
  a.inc_off = off;
  a.inc_list = list;
  a.n_ant = o.n_ant;
  a.n_base = o.n_base;
  a.n_time = o.n_time;
  a.n_chan = o.n_chan;
  a.n_iter = n_iter;
  a.err = ctx->d_err;
  const size_t smem = k7_smem_bytes(o.n_ant);
  cudaError_t e = cudaFuncSetAttribute(k7_calib, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    k7_calib<<<o.n_time * o.n_chan, K7_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("calibration kernel: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
