// K4, shapelet coefficient gradients on the tensor cores (tcgen05).
//
// The visibilities are linear in the coefficients (eq:shape-env), so the gradient of
// L = sum |D - G V|^2 with respect to C[a][b] is a sum over visibilities v of phi_a(x_v) phi_b(y_v) times
// a weight: with Y_v = conj(W_v) (nu_v / nu_ref)^alpha P_v (W = conj(G) R, P the phasor),
//   dL/dC[a][b] = -2 S_ref Re(Y_v (-i)^(a+b)) phi_a(x_v) phi_b(y_v)  summed over v,
// i.e. -2 S_ref (Re Y, Im Y, -Re Y, -Im Y)[(a+b) mod 4] weighted sums.  Written as one contraction over
// the visibilities (K),
//   D[n][a] = sum_v Bz[v][n] A[v][a],   Bz[v][2b] = phi_b(y_v) Re Y_v,  Bz[v][2b+1] = phi_b(y_v) Im Y_v,
//   A[v][a] = phi_a(x_v),
// the gradient is dL/dC[a][b] = -+2 S_ref D[2b + ((a+b) mod 2)][a].  D has M = 2 (n_max + 1) rows (one
// or two blocks of 128) and N = n_max + 1 columns (padded to k_pad): a tall-skinny GEMM with K = N_vis.
//
// Kernel organisation (persistent, one CTA per SM; tiles of 128 visibilities, two in flight):
//  * producer warpgroups P0, P1 (warps 0-3, 4-7) take the even / odd tiles; thread t forms visibility
//    t's x, y, Y (phasor, spectrum, gains and residual) and the Hermite functions phi_a(x), phi_b(y) by the
//    normalised recurrence, and writes Bz and A as bf16 hi / lo in the MN-major no-swizzle layout: each
//    16-byte core-matrix row holds 8 consecutive n (or a) of its own visibility, so every store is one
//    16-byte vector;
//  * warp 8 allocates TMEM and one of its threads issues, per tile, 8 K steps x 3 products (hi hi, hi lo,
//    lo hi) x the M blocks of tcgen05.mma kind::f16 (M = 128, N = k_pad, K = 16, both operands MN-major)
//    into one FP32 accumulator that sums every tile of the CTA, and commits to the parity's mbarrier;
//  * after the last tile the accumulator is read once (tcgen05.ld), staged in shared memory and
//    gathered into the coefficients' order as this CTA's FP64 partial sums, which a fixed-order
//    reduction adds over CTAs.
// Every wait is bounded; on a timeout the kernel raises WN_DEVERR_TIMEOUT, lets its issued MMAs finish
// and frees TMEM before returning.
#include <algorithm>
#include <cmath>
#include <string>

#include "tc05.cuh"
#include "wn_internal.cuh"

namespace wn {

constexpr int K4M_TV = 128;                 // visibilities per tile: 8 K steps of 16
constexpr int K4M_THREADS = 32 * 9;         // producer warpgroups P0, P1 and the MMA warp
constexpr int K4M_MMA_WARP = 8;

struct K4MArgs {
  const float4* rowinfo;   // per row: (xs, ys, tau hi, tau lo)
  const float4* chaninfo;  // per channel: (nu/c hi, nu/c lo, log2(nu/nu0), nu)
  const float2* resid;     // R = D - G V
  PeelArgs peel;           // gains and antenna indices
  const float2* rowg;      // [n_rows] gain product of frequency-independent gains, or nullptr
  long long n_vis;
  int n_chan, n_base;
  int nmax, k_pad, n_mblk, groups, n_tiles;
  float c_amp, alpha;      // flux-free log2 amplitude at nu0, spectral index
  int nnz;
  const int *n1, *n2;      // this shapelet's triples
  const double* flux;      // device scalar S_ref
  double* part_c;          // [gridDim.x][nnz] this CTA's partial gradient sums
  unsigned* err;
};

// Shared memory per tile parity: Bz hi then lo (n_mblk blocks of 128 rows x 128 visibilities, 32 KB each),
// then A hi then lo (k_pad x 128); after the buffers the recurrence constants and the barriers.
struct K4MLayout {
  int bz_bytes, av_bytes, buf_bytes, coef, bars, total;
};
__host__ __device__ inline K4MLayout k4m_layout(int k_pad, int n_mblk, int groups) {
  K4MLayout L;
  L.bz_bytes = n_mblk * 128 * K4M_TV * 2 * 2;
  L.av_bytes = k_pad * K4M_TV * 2 * 2;
  L.buf_bytes = (L.bz_bytes + L.av_bytes + 1023) & ~1023;
  L.coef = groups * L.buf_bytes;  // a_n, b_n (128 floats each), then {a_n, a_n}, {-b_n, -b_n} (128 float2 each)
  L.bars = L.coef + 2 * (kNmaxLimit + 1) * 4 + 2 * (kNmaxLimit + 1) * 8;
  L.total = L.bars + 64;  // afull[2], mdone[2], dfin, TMEM address slot
  return L;
}

// 8 floats as bf16 hi = RN(v) and lo = RN(v - hi), packed as two 16-byte vectors.
__device__ __forceinline__ void bf16_pack8(const float (&v)[8], uint4& hi, uint4& lo) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h[i]);
    l[i] = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
  }
  hi = *reinterpret_cast<uint4*>(h);
  lo = *reinterpret_cast<uint4*>(l);
}

// phi_0 .. phi_{8 nc - 1}(x) by the normalised recurrence phi_{n+1} = a_n x phi_n - b_n phi_{n-1}, eight
// at a time: emit(c, v) receives values 8c .. 8c + 7.  Where phi_0 = e^{-x^2/2} would underflow FP32
// (|x| > 12.5) the recurrence runs on values scaled by 2^E and scales back on output; beyond xcut every
// value of interest is below 1e-20 and the row is zero.
template <class Emit>
__device__ __forceinline__ void hermite_chunks(float x, bool zero, float xcut, int nc, const float* ca, const float* cb,
                                               Emit emit) {
  zero = zero || !(fabsf(x) <= xcut);
  const float hx = 0.5f * x * x * 1.4426950408889634f;
  const bool fast = zero || fabsf(x) <= 12.5f;
  int E = fast ? 0 : max(0, (int)ceilf(hx) - 100);
  float p = zero ? 0.f : exp2f((float)E - hx), p_prev = 0.f;
  float scale = __int_as_float(max(0, 127 - E) << 23);
  for (int c = 0; c < nc; ++c) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = 8 * c + i;
      v[i] = fast ? p : p * scale;
      const float pn = fmaf(ca[n] * x, p, -cb[n] * p_prev);
      p_prev = p;
      p = pn;
    }
    if (!fast && fabsf(p) > 1.8446744e19f) {  // 2^64: rescale (8 steps grow by at most 2^43)
      p *= 5.421011e-20f;
      p_prev *= 5.421011e-20f;
      E -= 64;
      scale = __int_as_float(max(0, 127 - E) << 23);
    }
    emit(c, v);
  }
}

__global__ void __launch_bounds__(K4M_THREADS, 1) k4_coeff_mma(const K4MArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ng = a.groups;
  const K4MLayout lay = k4m_layout(a.k_pad, a.n_mblk, ng);
  float* ca = reinterpret_cast<float*>(smem + lay.coef);
  float* cb = ca + (kNmaxLimit + 1);
  float2* ca2 = reinterpret_cast<float2*>(cb + (kNmaxLimit + 1));
  float2* cb2 = ca2 + (kNmaxLimit + 1);
  uint64_t* afull = reinterpret_cast<uint64_t*>(smem + lay.bars);  // [parity] producers -> MMA: tile written
  uint64_t* mdone = afull + 2;                                      // [parity] MMA -> producers: tile read
  uint64_t* dfin = mdone + 2;                                       // MMA -> all: every MMA complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(dfin + 1);
  // warp index and TMEM base broadcast from lane 0: warp-uniform values for the tcgen05 operands
  const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0), t = threadIdx.x & 127;
  const int acc_cols = a.n_mblk * a.k_pad;
  const uint32_t ncols = acc_cols <= 32 ? 32 : (acc_cols <= 64 ? 64 : (acc_cols <= 128 ? 128 : 256));
  if (threadIdx.x == 0) {
    for (int g = 0; g < 2; ++g) {
      mbar_init(&afull[g], 128);
      mbar_init(&mdone[g], 1);
    }
    mbar_init(dfin, 1);
    fence_mbar_init();
  }
  if (threadIdx.x <= kNmaxLimit) {  // sqrt(2 / (n + 1)), sqrt(n / (n + 1)), correctly rounded via FP64
    const double np1 = (double)(threadIdx.x + 1);
    const float fa = (float)sqrt(2.0 / np1), fb = (float)sqrt((double)threadIdx.x / np1);
    ca[threadIdx.x] = fa;
    cb[threadIdx.x] = fb;
    ca2[threadIdx.x] = make_float2(fa, fa);
    cb2[threadIdx.x] = make_float2(-fb, -fb);
  }
  if (warp == K4M_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = __shfl_sync(0xffffffffu, *tslot, 0);
  const int n_it = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t skb = (uint32_t)(a.k_pad >> 3) << 7;  // A: bytes between core matrices adjacent in K

  if (warp == K4M_MMA_WARP) {
    // ---------------- MMA issue: every tile into the one accumulator ----------------
    // The whole warp runs the loop (warp-uniform descriptors); the elected lane issues.
    {
      const uint32_t lead = elect_lane();
      const uint32_t idesc = umma_idesc_bf16(a.k_pad, true, true);
      bool ok = true;
      for (int it = 0; ok && it < n_it; ++it) {
        const int sp = it % ng, j = it / ng;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&afull[sp], j & 1, a.err))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = smem_u32(smem + sp * lay.buf_bytes);
        const uint32_t av = base + (uint32_t)lay.bz_bytes, av_lo = av + (uint32_t)(a.k_pad * K4M_TV * 2);
#pragma unroll 1
        for (int bk = 0; bk < a.n_mblk; ++bk) {
          const uint32_t bz = base + (uint32_t)(bk * 128 * K4M_TV * 2), bz_lo = bz + (uint32_t)(a.n_mblk * 128 * K4M_TV * 2);
          const uint32_t d = tmem + (uint32_t)(bk * a.k_pad);
#pragma unroll 1
          for (int p = 0; p < 3; ++p) {  // hi*hi, hi*lo, lo*hi
            const uint32_t aa = p == 2 ? bz_lo : bz, bb = p == 1 ? av_lo : av;
#pragma unroll
            for (int kk = 0; kk < K4M_TV / 16; ++kk) {
              // Bz (MMA A): K cores 2048 B apart, 8-row MN cores 128 B apart; A (MMA B): K cores skb apart
              const uint64_t da = umma_desc(aa + (uint32_t)(2 * kk) * 2048u, 2048u, 128u);
              const uint64_t db = umma_desc(bb + (uint32_t)(2 * kk) * skb, skb, 128u);
              umma_bf16_by(lead, d, da, db, idesc, (it > 0 || p > 0 || kk > 0) ? 1u : 0u);
            }
          }
        }
        umma_commit_by(lead, &mdone[sp]);
      }
      umma_commit_by(lead, dfin);  // completes once every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---------------- producers: tile it of parity sp = warp / 4 ----------------
    const int sp = warp >> 2;
    if (sp < ng) {
      unsigned char* buf = smem + sp * lay.buf_bytes;
      unsigned char* av = buf + lay.bz_bytes;
      unsigned char* av_lo = av + a.k_pad * K4M_TV * 2;
      unsigned char* bz_lo = buf + a.n_mblk * 128 * K4M_TV * 2;
      const float xcut = sqrtf(2.0f * a.nmax + 1.0f) + 10.0f;
      const int nb1 = a.nmax + 1;
      const int nca = a.k_pad >> 3, ncb = (nb1 + 7) >> 3;  // chunks of 8 of phi(x) and of phi(y)
      // this visibility's place in the A and Bz tiles: K core t / 8, core-matrix row t % 8
      const uint32_t a_off = (uint32_t)(t >> 3) * skb + (uint32_t)(t & 7) * 16u;
      const uint32_t z_off = (uint32_t)(t >> 3) * 2048u + (uint32_t)(t & 7) * 16u;
      auto bz_at = [&](int c) { return (uint32_t)(c >> 4) * (128u * K4M_TV * 2u) + z_off + (uint32_t)(c & 15) * 128u; };
      // Bz rows of orders above those present are zero in every tile: written once here
      for (int c = 2 * ncb; c < 16 * a.n_mblk; ++c) {
        *reinterpret_cast<uint4*>(buf + bz_at(c)) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(bz_lo + bz_at(c)) = make_uint4(0, 0, 0, 0);
      }
      auto store_a = [&](int c, const float (&v)[8]) {
        uint4 hi, lo;
        bf16_pack8(v, hi, lo);
        *reinterpret_cast<uint4*>(av + a_off + (uint32_t)c * 128u) = hi;
        *reinterpret_cast<uint4*>(av_lo + a_off + (uint32_t)c * 128u) = lo;
      };
      // chunk c8 of phi(y) (b = 8 c8 ..) fills Bz chunks 2 c8, 2 c8 + 1: rows 2b (Re Y), 2b + 1 (Im Y)
      auto store_b = [&](int c8, const float (&v)[8], float yr, float yi) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * c8 + h;
          float z[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ph = 4 * c + i < nb1 ? v[4 * h + i] : 0.f;
            z[2 * i] = ph * yr;
            z[2 * i + 1] = ph * yi;
          }
          uint4 hi, lo;
          bf16_pack8(z, hi, lo);
          *reinterpret_cast<uint4*>(buf + bz_at(c)) = hi;
          *reinterpret_cast<uint4*>(bz_lo + bz_at(c)) = lo;
        }
      };
      // inputs of one tile's visibility, loaded a tile ahead of their use
      struct In {
        float4 ri, ci;
        float2 R, G;
        bool valid;
      };
      auto load_in = [&](int it) {
        In v;
        const long long vis = (long long)(blockIdx.x + (long long)it * gridDim.x) * K4M_TV + t;
        v.valid = it < n_it && vis < a.n_vis;
        const int row = v.valid ? (int)(vis / a.n_chan) : 0;
        const int f = v.valid ? (int)(vis - (long long)row * a.n_chan) : 0;
        v.ri = __ldg(a.rowinfo + row);
        v.ci = __ldg(a.chaninfo + f);
        v.R = v.valid ? __ldg(a.resid + vis) : make_float2(0.f, 0.f);
        v.G = make_float2(0.f, 0.f);
        if (v.valid) {
          if (a.rowg) v.G = __ldg(a.rowg + row);
          else if (!gain_product(a.peel, row, a.n_base, f, v.G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
        }
        return v;
      };
      In cur = load_in(sp);
      for (int it = sp, j = 0; it < n_it; it += ng, ++j) {
        const In nxt = load_in(it + ng);
        const float x = cur.ri.x * cur.ci.w, y = cur.ri.y * cur.ci.w;
        float yr = 0.f, yi = 0.f;
        if (cur.valid) {
          const float2 W = make_float2(cur.G.x * cur.R.x + cur.G.y * cur.R.y, cur.G.x * cur.R.y - cur.G.y * cur.R.x);
          const float2 P = phasor_fast(reduce_turns(cur.ri.z, cur.ri.w, cur.ci.x, cur.ci.y));
          const float S = ex2_approx(fmaf(a.alpha, cur.ci.z, a.c_amp));
          yr = S * (W.x * P.x + W.y * P.y);  // Y = conj(W) S P
          yi = S * (W.x * P.y - W.y * P.x);
        }
        if (j > 0 && !mbar_wait_bounded(&mdone[sp], (j - 1) & 1, a.err)) break;  // MMA(j-1) has read the buffer
        const bool zx = !cur.valid || !(fabsf(x) <= xcut), zy = !cur.valid || !(fabsf(y) <= xcut);
        if ((zx || fabsf(x) <= 12.5f) && (zy || fabsf(y) <= 12.5f)) {
          // both recurrences unscaled, as one f32x2 recurrence {phi(x), phi(y)}
          const float2 X = make_float2(x, y);
          float2 P = make_float2(zx ? 0.f : exp2f(-0.5f * x * x * 1.4426950408889634f),
                                 zy ? 0.f : exp2f(-0.5f * y * y * 1.4426950408889634f));
          float2 Pp = make_float2(0.f, 0.f);
          const int nc = max(nca, ncb);
          for (int c = 0; c < nc; ++c) {
            float vx[8], vy[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              vx[i] = P.x;
              vy[i] = P.y;
              const float2 Pn = __ffma2_rn(__fmul2_rn(ca2[8 * c + i], X), P, __fmul2_rn(cb2[8 * c + i], Pp));
              Pp = P;
              P = Pn;
            }
            if (c < nca) store_a(c, vx);
            if (c < ncb) store_b(c, vy, yr, yi);
          }
        } else {
          hermite_chunks(x, !cur.valid, xcut, nca, ca, cb, [&](int c, const float (&v)[8]) { store_a(c, v); });
          hermite_chunks(y, !cur.valid, xcut, ncb, ca, cb, [&](int c8, const float (&v)[8]) { store_b(c8, v, yr, yi); });
        }
        fence_async_smem();
        mbar_arrive(&afull[sp]);
        cur = nxt;
      }
    }
  }
  // ---------------- epilogue: the accumulator, once, into this CTA's partial sums ----------------
  // uniform over the CTA (the TMEM loads below are warp-collective): every MMA has completed
  const bool have = __syncthreads_and(n_it > 0 && mbar_wait_bounded(dfin, 0, a.err)) != 0;
  tc_fence_after();  // every producer is done with the buffers, which now hold D
  float* Ds = reinterpret_cast<float*>(smem);  // [n_mblk * 128][k_pad]
  if (warp < 4 && have) {
    for (int bk = 0; bk < a.n_mblk; ++bk)
      for (int c16 = 0; c16 < (a.k_pad >> 4); ++c16) {
        uint32_t r[16];
        tmem_issue16x(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bk * a.k_pad + 16 * c16), r);
        tmem_wait16(r);
        float* dst = Ds + (size_t)(bk * 128 + warp * 32 + (threadIdx.x & 31)) * a.k_pad + 16 * c16;
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[i] = __uint_as_float(r[i]);
      }
  }
  tc_fence_before();
  __syncthreads();
  const double flux = *a.flux;
  for (int k = threadIdx.x; k < a.nnz; k += blockDim.x) {
    const int na = __ldg(a.n1 + k), nb = __ldg(a.n2 + k);
    double v = 0.0;
    if (have) {
      const float d = Ds[(size_t)(2 * nb + ((na + nb) & 1)) * a.k_pad + na];
      v = (double)d * (((na + nb) & 3) >= 2 ? 2.0 : -2.0) * flux;
    }
    a.part_c[(size_t)blockIdx.x * a.nnz + k] = v;
  }
  __syncthreads();
  if (warp == K4M_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Launch for shapelet q of M: coefficient-gradient partial sums [grid][nnz] into part_c (grid returned),
// from the residual and the per-row / per-channel tables the shapelet prep wrote (rowinfo, chaninfo);
// rowg_ws (n_rows float2, or nullptr) receives the per-row gain products when the gains do not depend
// on frequency.
int launch_coeff_mma(wn_ctx* ctx, const ObsDev& o, const Model* M, int q, const PeelArgs& pa, const float2* resid,
                     const float4* rowinfo, const float4* chaninfo, float2* rowg_ws, double* part_c, int* grid_out,
                     cudaStream_t st) {
  const ShapeRec& h = M->sh_host[q];
  K4MArgs a;
  a.rowinfo = rowinfo;
  a.chaninfo = chaninfo;
  a.resid = resid;
  a.peel = pa;
  a.rowg = nullptr;
  if (rowg_ws && pa.gf == 1) {  // frequency-independent gains: one product per row, read without dependent loads
    launch_rowgain(pa, o.n_rows, o.n_base, rowg_ws, ctx->d_err, st);
    a.rowg = rowg_ws;
  }
  a.n_vis = (long long)o.n_rows * o.n_chan;
  a.n_chan = o.n_chan;
  a.n_base = o.n_base;
  a.nmax = h.nmax;
  a.k_pad = (h.nmax + 1 + 15) / 16 * 16;
  a.n_mblk = 2 * (h.nmax + 1) <= 128 ? 1 : 2;
  const double L0 = std::log2(o.nu0);
  a.c_amp = (float)((double)h.alpha * (L0 - h.lref));  // flux-free
  a.alpha = h.alpha;
  a.nnz = M->s_off_host[q + 1] - M->s_off_host[q];
  a.n1 = M->m_n1() + M->s_off_host[q];
  a.n2 = M->m_n2() + M->s_off_host[q];
  a.flux = M->r_flux() + M->n_point + M->n_gauss + q;
  a.part_c = part_c;
  a.err = ctx->d_err;
  a.groups = 2;
  K4MLayout lay = k4m_layout(a.k_pad, a.n_mblk, a.groups);
  if (lay.total > 227 * 1024) {
    a.groups = 1;
    lay = k4m_layout(a.k_pad, a.n_mblk, a.groups);
  }
  if (lay.total > 227 * 1024) return set_error(WN_EINVAL, "adjoint: shapelet coefficient operand does not fit in shared memory");
  a.n_tiles = (int)((a.n_vis + K4M_TV - 1) / K4M_TV);
  const int grid = std::max(1, std::min(a.n_tiles, ctx->num_sms));
  *grid_out = grid;
  if (cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k4_coeff_mma)))
    return set_error(WN_ECUDA, std::string("coefficient adjoint attribute: ") + cudaGetErrorString(e));
  k4_coeff_mma<<<grid, K4M_THREADS, lay.total, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("coefficient adjoint launch: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
