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
// does the forward substitution) stay in shared memory as 32 x 32 tiles.  Warp w accumulates antennas
// w, w + 16, ... over their incident baselines in a fixed order (no atomics on the sums).  The
// factorisation is a tiled right-looking Cholesky in FP32: one warp factors the diagonal tile, a lane
// per row solves the panel below it, and every warp updates trailing tiles with an 8 x 4 register
// block per lane.  Warp 0 back-substitutes.  A non-positive pivot
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

// Storage of the augmented lower triangle [A^T A | A^T b] in 32 x 32 tiles: tile (I, J), J <= I, at
// index I (I + 1) / 2 + J, rows padded to 33 floats so a column of a tile is conflict-free.
constexpr int K7_TS = 36;               // row stride of a tile: 9 float4 (odd), so rows read as float4 without conflicts
constexpr int K7_TILE = 32 * K7_TS;     // floats per tile
__device__ __forceinline__ float* k7_elem(float* T, int r, int c) {
  return T + ((r >> 5) * ((r >> 5) + 1) / 2 + (c >> 5)) * K7_TILE + (r & 31) * K7_TS + (c & 31);
}
__device__ __forceinline__ float* k7_tile(float* T, int I, int J) { return T + (I * (I + 1) / 2 + J) * K7_TILE; }

// One tile row (32 floats, 16-byte aligned) to registers and back, as float4: with the row stride of 9
// float4 the 8 lanes of each quarter-warp hit distinct banks.
__device__ __forceinline__ void k7_row_load(const float* r, float (&v)[32]) {
#pragma unroll
  for (int c = 0; c < 32; c += 4) {
    const float4 q = *reinterpret_cast<const float4*>(r + c);
    v[c] = q.x;
    v[c + 1] = q.y;
    v[c + 2] = q.z;
    v[c + 3] = q.w;
  }
}
__device__ __forceinline__ void k7_row_store(float* r, const float (&v)[32]) {
#pragma unroll
  for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4*>(r + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
}

// Column C of the unblocked factorisation of a 32 x 32 diagonal tile held one row per lane; recursion
// keeps every register index a compile-time constant.  n_here = rows of this tile that are part of the
// system (pivots at or past it belong to the right-hand side row or the padding and are kept positive).
template <int C>
__device__ __forceinline__ void k7_diag_col(float (&row)[32], float* dinv, int lane, int n_here, int* s_bad) {
  float piv = __shfl_sync(0xffffffffu, row[C], C);
  if (!(piv > 0.f) || !isfinite(piv)) {
    if (C < n_here && lane == 0) *s_bad = 1;
    piv = 1.f;
  }
  const float rinv = rsqrtf(piv), l = piv * rinv;
  if (lane == C) {
    row[C] = l;
    dinv[C] = rinv;
  } else if (lane > C) {
    row[C] *= rinv;
  }
  const float lc = row[C];
#pragma unroll
  for (int j = C + 1; j < 32; ++j) {
    const float ljc = __shfl_sync(0xffffffffu, lc, j);  // L[j][C], held by lane j
    if (lane >= j) row[j] -= lc * ljc;
  }
  if constexpr (C + 1 < 32) k7_diag_col<C + 1>(row, dinv, lane, n_here, s_bad);
}

// Factor diagonal tile K in place (warp-wide): lane r holds row r, columns by shuffle; 1 / L_kk to dinv.
__device__ __forceinline__ void k7_factor_diag(float* T, int K, float* dinv, int lane, int n, int* s_bad) {
  float* D = k7_tile(T, K, K);
  float row[32];
  k7_row_load(D + lane * K7_TS, row);
  k7_diag_col<0>(row, dinv + K * 32, lane, n - K * 32, s_bad);
  k7_row_store(D + lane * K7_TS, row);
}

// Trailing update of tile (K + 1 + I, K + 1 + J) by step K's panel: A -= L_IK L_JK^T.  A warp per tile;
// lane (rg, cg) = (lane / 8, lane % 8) holds rows rg + 4i (i < 8) and columns cg + 8j (j < 4), and reads
// both panels four k at a time as float4: the 4 (or 8) distinct rows a load touches are adjacent, at
// distinct banks.
__device__ __forceinline__ void k7_trail_tile(float* T, int K, int I, int J, int lane) {
  const int rg = lane >> 3, cg = lane & 7;
  const float* PI = k7_tile(T, K + 1 + I, K);
  const float* PJ = k7_tile(T, K + 1 + J, K);
  float* C = k7_tile(T, K + 1 + I, K + 1 + J);
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 2
  for (int k = 0; k < 32; k += 4) {
    float4 av[8], bv[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) av[i] = *reinterpret_cast<const float4*>(PI + (rg + 4 * i) * K7_TS + k);
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = *reinterpret_cast<const float4*>(PJ + (cg + 8 * j) * K7_TS + k);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j] = fmaf(av[i].x, bv[j].x, acc[i][j]);
        acc[i][j] = fmaf(av[i].y, bv[j].y, acc[i][j]);
        acc[i][j] = fmaf(av[i].z, bv[j].z, acc[i][j]);
        acc[i][j] = fmaf(av[i].w, bv[j].w, acc[i][j]);
      }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) C[(rg + 4 * i) * K7_TS + cg + 8 * j] -= acc[i][j];
}

__global__ void __launch_bounds__(K7_THREADS, 1) k7_calib(const K7Args a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int A = a.n_ant, n = 2 * A - 1;
  const int NT = (n + 1 + 31) / 32;                                   // tile rows (row n is A^T b)
  float* T = reinterpret_cast<float*>(sm);                            // NT (NT + 1) / 2 tiles
  float* x = T + NT * (NT + 1) / 2 * K7_TILE;                         // [n]
  float* dinv = x + NT * 32;                                          // [NT * 32]: 1 / L_kk
  float2* g = reinterpret_cast<float2*>(dinv + NT * 32);              // [A]
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = blockIdx.x / a.n_chan, f = blockIdx.x % a.n_chan;
  float2* gout = a.gains + ((size_t)t * a.n_chan + f) * A;
  for (int i = tid; i < A; i += K7_THREADS) g[i] = gout[i];
  if (tid == 0) s_bad = 0;
  const int nfl = NT * (NT + 1) / 2 * K7_TILE;
  const size_t plane = (size_t)a.n_base * a.n_chan;

  for (int it = 0; it < a.n_iter; ++it) {
    __syncthreads();
    for (int k = tid; k < nfl; k += K7_THREADS) T[k] = 0.f;
    __syncthreads();
    // rows past the right-hand side row pad the last tile row: unit pivots
    for (int r = n + 1 + tid; r < NT * 32; r += K7_THREADS) *k7_elem(T, r, r) = 1.f;
    // --- [A^T A | A^T b] at the current gains
    for (int i = warp; i < A; i += K7_WARPS) {
      float d = 0.f, br = 0.f, bi = 0.f;
      const int k0 = a.inc_off[i], k1 = a.inc_off[i + 1];
      for (int kb = k0 + lane; kb < k1; kb += 4 * 32) {
        // four gathers in flight per lane; the sums still run over k in increasing order
        int ev[4];
        float2 Iv[4], Vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = kb + 32 * u;
          ev[u] = k < k1 ? a.inc_list[k] : -1;
          if (ev[u] >= 0) {
            const size_t idx = (size_t)t * plane + (size_t)(ev[u] >> 1) * a.n_chan + f;
            Iv[u] = a.model[idx];
            Vv[u] = a.data[idx];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (ev[u] < 0) continue;
          const int e = ev[u], b = e >> 1;
          const float2 I = Iv[u], V = Vv[u];
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
            // the block of this baseline, rows of q (> p) and columns of p: written once, since each
            // antenna pair appears at most once among the baselines
            const float2 ac = cmul(cconj(av), cv);
            *k7_elem(T, col_re(q), col_re(p)) = ac.x;
            *k7_elem(T, col_im(q), col_re(p)) = ac.y;
            if (p > 0) {
              *k7_elem(T, col_re(q), col_im(p)) = ac.y;
              *k7_elem(T, col_im(q), col_im(p)) = -ac.x;
            }
          } else {
            const float2 cv = cmul(gp, I);
            d += cv.x * cv.x + cv.y * cv.y;
            const float2 cR = cmul(cconj(cv), R);
            br += cR.x;
            bi -= cR.y;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        br += __shfl_xor_sync(0xffffffffu, br, o);
        bi += __shfl_xor_sync(0xffffffffu, bi, o);
      }
      if (lane == 0) {
        *k7_elem(T, col_re(i), col_re(i)) = d;
        *k7_elem(T, n, col_re(i)) = br;  // right-hand side: row n
        if (i > 0) {
          *k7_elem(T, col_im(i), col_im(i)) = d;
          *k7_elem(T, n, col_im(i)) = bi;
        }
      }
    }
    // --- tiled right-looking Cholesky of the augmented matrix; row n becomes L^{-1} (A^T b).  Pivots of
    // row n and of the padding rows are not part of the system and are only kept positive.  Look-ahead:
    // while warps 1.. apply step K's trailing update, warp 0 updates the next diagonal tile first and
    // factors it, so no phase runs the diagonal factorisation alone.
    __syncthreads();
    if (warp == 0) k7_factor_diag(T, 0, dinv, lane, n, &s_bad);
    for (int K = 0; K < NT; ++K) {
      __syncthreads();
      // panel: X L_KK^T = A_IK for the tiles below; lane r solves row r of one tile, column by column
      for (int I = K + 1 + warp; I < NT; I += K7_WARPS) {
        float* P = k7_tile(T, I, K);
        const float* D = k7_tile(T, K, K);
        float xr[32];
        k7_row_load(P + lane * K7_TS, xr);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          xr[c] *= dinv[K * 32 + c];
#pragma unroll
          for (int j = c + 1; j < 32; ++j) xr[j] -= xr[c] * D[j * K7_TS + c];
        }
        k7_row_store(P + lane * K7_TS, xr);
      }
      __syncthreads();
      // trailing update A_IJ -= L_IK L_JK^T, K < J <= I: tile q = 0 is the next diagonal tile (warp 0,
      // which then factors it); the others go to warps 1.. in turn
      const int m = NT - K - 1;
      if (warp == 0) {
        if (m > 0) {
          k7_trail_tile(T, K, 0, 0, lane);
          __syncwarp();
          k7_factor_diag(T, K + 1, dinv, lane, n, &s_bad);
        }
      } else {
        for (int q = warp; q < m * (m + 1) / 2; q += K7_WARPS - 1) {
          int I = 0;
          while ((I + 1) * (I + 2) / 2 <= q) ++I;
          k7_trail_tile(T, K, I, q - I * (I + 1) / 2, lane);
        }
      }
    }
    __syncthreads();
    // --- back substitution L^T x = y, by tile rows R = NT-1 .. 0: warp 0 solves the diagonal block
    // (x_k = y_k / L_kk, then y_j -= L_kj x_k for j < k in the block), then warp J subtracts L_RJ^T x_R
    // from y_J for every J < R.  x holds y, and becomes x block by block.
    for (int j = tid; j < NT * 32; j += K7_THREADS) x[j] = j < n ? *k7_elem(T, n, j) : 0.f;
    for (int R = NT - 1; R >= 0; --R) {
      __syncthreads();
      if (warp == 0) {
        const float* D = k7_tile(T, R, R);
        float yv = x[32 * R + lane];
        for (int c = 31; c >= 0; --c) {
          const int k = 32 * R + c;
          const float xk = k < n ? __shfl_sync(0xffffffffu, yv, c) * dinv[k] : 0.f;
          if (lane == c) yv = xk;
          else if (lane < c) yv -= D[c * K7_TS + lane] * xk;  // L_{k, 32R + lane}
        }
        x[32 * R + lane] = yv;
      }
      __syncthreads();
      for (int J = warp; J < R; J += K7_WARPS) {
        const float* P = k7_tile(T, R, J);
        float sum = 0.f;
#pragma unroll 8
        for (int c = 0; c < 32; ++c) sum = fmaf(P[c * K7_TS + lane], x[32 * R + c], sum);  // L_{32R+c, 32J+lane}
        x[32 * J + lane] -= sum;
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
  const int n = 2 * n_ant - 1, NT = (n + 1 + 31) / 32;
  return sizeof(float) * ((size_t)NT * (NT + 1) / 2 * K7_TILE + 2 * NT * 32) + sizeof(float2) * n_ant;
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
    cudaError_t e = dev_malloc(&ctx->ws2, need);
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
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k7_calib));
  if (e == cudaSuccess) {
    k7_calib<<<o.n_time * o.n_chan, K7_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("calibration kernel: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
