// K2: shapelet envelopes on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// For one shapelet and every visibility (row (t,b), channel f), eq:shape-env with eq:basis_FT gives
//   xi = sum_{n1+n2<=nmax} C[n1,n2] (-i)^(n1+n2) phi_n1(x) phi_n2(y),
//   x = beta1 K (sin pa u' + cos pa v') nu/c,  y = beta2 K (cos pa u' - sin pa v') nu/c   (eq:scale-shape-x/y)
// with (u', v') re-phased to the shapelet centre and phi_n the peak-normalised Hermite functions.
// Writing A[vis, n1] = phi_n1(x) and splitting C (-i)^(n1+n2) into real and imaginary parts gives a
// dense contraction T = A [C_re | C_im] (M = visibilities, K = n1, N = 2 (nmax+1)) followed by a
// per-row dot product xi = sum_n2 T[., n2] phi_n2(y).  The contribution S(nu) xi exp(-2 pi i tau nu/c)
// is then stored, accumulated, or subtracted as G times it for the peel.
//
// Kernel organisation (persistent, one CTA per SM):
//  * warps 0-3 and 4-7 are two producer/epilogue warpgroups; thread i of a group owns row i of a
//    128-visibility tile: it computes phi_n(x) by the normalised Hermite recurrence (FP32, rescaled to
//    stay in range) and writes them as bf16 hi/lo into the canonical K-major shared-memory layout
//    (8x8 core matrices, no swizzle), then, after the MMA, reads its accumulator row from TMEM and
//    forms the epilogue;
//  * warp 8 allocates TMEM, loads the packed coefficient operand with one TMA bulk copy, and one of
//    its threads issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32; three products hi*hi + hi*lo + lo*hi
//    in the split mode) into the group's TMEM accumulator and commits to an mbarrier;
//  * the two groups alternate tiles so that one group's Hermite production and epilogue overlap the
//    other group's MMAs.
// Every wait is bounded; on a timeout the kernel raises WN_DEVERR_TIMEOUT, drains its own commits and
// frees TMEM before returning.
#include "wn_internal.cuh"

namespace wn {

constexpr int K2_M = 128;
constexpr int K2_GROUPS = 2;
constexpr int K2_THREADS = 32 * (4 * K2_GROUPS + 1);
constexpr int K2_SLACK = 32 * 1024;  // spare shared memory behind the operands

// sqrt(2/(n+1)) and sqrt(n/(n+1)) of the normalised Hermite recurrence
//   phi_{n+1} = sqrt(2/(n+1)) x phi_n - sqrt(n/(n+1)) phi_{n-1}.
__constant__ float c_herm_a[kNmaxLimit + 1];
__constant__ float c_herm_b[kNmaxLimit + 1];

struct K2Args {
  const float4* rowinfo;     // [n_rows] (xs, ys, tau_hi, tau_lo): x = xs nu, y = ys nu, tau in metres
  const float4* chaninfo;    // [n_chan] (nu/c hi, nu/c lo, log2(nu/nu0), nu)
  const __nv_bfloat16* bop;  // this shapelet's packed B operand: hi [n_pad][kp], then lo
  int n_pad, nmax, passes, n_chan, n_base, n_tiles, mode, groups;
  long long n_vis;
  float c_amp, alpha, sgn;
  float2* out;
  PeelArgs peel;
  unsigned* err;
};

// ---- tcgen05 helpers (inline PTX) ------------------------------------------------------------

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension byte offset (between
// core matrices adjacent in K), stride byte offset (between 8-row groups), fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(K2_M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool k2_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 32)) {
      atomicOr(err, WN_DEVERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Offset in bytes of element (row, k) in a canonical K-major no-swizzle tile with `rows` rows.
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k, int rows) {
  return (uint32_t)((((k >> 3) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

struct K2Layout {
  int b_bytes, a_bytes, a0, bars, total;
};

__host__ __device__ inline K2Layout k2_layout(int kp, int n_pad, int passes, int groups) {
  K2Layout L;
  const int parts = passes > 1 ? 2 : 1;
  L.b_bytes = parts * kp * n_pad * 2;
  L.a_bytes = parts * kp * K2_M * 2;  // one group's A (hi [+ lo])
  L.a0 = (L.b_bytes + 1023) & ~1023;
  L.bars = L.a0 + groups * L.a_bytes;
  L.total = L.bars + 128 + K2_SLACK;
  return L;
}

// Hermite functions phi_0..phi_{KP-1}(x) (zero beyond nmax), FP32 with a running power-of-two scale
// so the recurrence neither underflows (phi_0 = e^{-x^2/2} is far below FP32 range for |x| > 13)
// nor overflows; written as bf16 hi (and lo) into row `row` of the K-major tile(s).
template <int KP>
__device__ __forceinline__ void produce_row(float x, int nmax, bool valid, unsigned char* a_hi, unsigned char* a_lo,
                                            int row) {
  const float ax = fabsf(x);
  const float xcut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;  // beyond it every phi_n, n <= nmax, is < 1e-20
  const bool zero = !valid || !(ax <= xcut);
  const float hx = 0.5f * x * x * 1.4426950408889634f;  // log2 of 1/phi_0
  int E = zero ? 0 : max(0, (int)ceilf(hx) - 100);       // stored value = phi * 2^E
  float p_prev = 0.f;
  float p = zero ? 0.f : exp2f((float)E - hx);
  float scale = ldexpf(1.0f, -E);
#pragma unroll
  for (int k0 = 0; k0 < KP; k0 += 8) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = k0 + i;
      v[i] = (n <= nmax) ? p * scale : 0.f;
      const float pn = fmaf(c_herm_a[n] * x, p, -c_herm_b[n] * p_prev);
      p_prev = p;
      p = pn;
      if ((i & 3) == 3 && fabsf(p) > 1.8446744e19f) {  // 2^64: rescale by 2^-64
        p *= 5.421011e-20f;
        p_prev *= 5.421011e-20f;
        E -= 64;
        scale = ldexpf(1.0f, -E);
      }
    }
    __nv_bfloat162 h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      const float2 hf = __bfloat1622float2(h[i]);
      l[i] = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    }
    const uint32_t off = kmaj_off(row, k0, K2_M);
    *reinterpret_cast<uint4*>(a_hi + off) = *reinterpret_cast<uint4*>(h);
    if (a_lo) *reinterpret_cast<uint4*>(a_lo + off) = *reinterpret_cast<uint4*>(l);
  }
}

template <int KP>
__global__ void __launch_bounds__(K2_THREADS, 1) k2_shapelet(const K2Args a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const K2Layout lay = k2_layout(KP, a.n_pad, a.passes, a.groups);
  uint64_t* bfull = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* afull = bfull + 1;             // [groups]
  uint64_t* mdone = bfull + 1 + K2_GROUPS;  // [groups]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bfull + 1 + 2 * K2_GROUPS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mma_warp = 4 * K2_GROUPS;
  const uint32_t ncols = a.n_pad * a.groups <= 32 ? 32 : (a.n_pad * a.groups <= 64 ? 64 :
                         (a.n_pad * a.groups <= 128 ? 128 : (a.n_pad * a.groups <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    mbar_init(bfull, 1);
    for (int g = 0; g < K2_GROUPS; ++g) {
      mbar_init(&afull[g], 128);
      mbar_init(&mdone[g], 1);
    }
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == mma_warp) {
    // ---------------- TMA of the coefficient operand, then the MMA issue loop ----------------
    if (lane == 0) {
      mbar_arrive_expect_tx(bfull, (uint32_t)lay.b_bytes);
      tma_bulk_g2s(smem, a.bop, (uint32_t)lay.b_bytes, bfull);
      const uint32_t idesc = umma_idesc_bf16(a.n_pad);
      const uint32_t b_hi = smem_u32(smem), b_lo = b_hi + (uint32_t)(KP * a.n_pad * 2);
      const uint32_t lbo_b = (uint32_t)(a.n_pad >> 3) << 7, lbo_a = (uint32_t)(K2_M >> 3) << 7;
      bool ok = k2_wait(bfull, 0, a.err);
      int issued[K2_GROUPS] = {0, 0};
      for (int it = 0; ok; ++it) {
        const int g = it % a.groups;
        const int tile = blockIdx.x + it * gridDim.x;
        if (tile >= a.n_tiles) break;
        const int kg = issued[g];
        if (!k2_wait(&afull[g], kg & 1, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_hi = smem_u32(smem + lay.a0 + g * lay.a_bytes);
        const uint32_t a_lo = a_hi + (uint32_t)(KP * K2_M * 2);
        const uint32_t d = tmem + (uint32_t)(g * a.n_pad);
#pragma unroll 1
        for (int p = 0; p < a.passes; ++p) {
          const uint32_t aa = (p == 2) ? a_lo : a_hi;  // hi*hi, hi*lo, lo*hi
          const uint32_t bb = (p == 1) ? b_lo : b_hi;
#pragma unroll
          for (int kk = 0; kk < KP / 16; ++kk) {
            const uint64_t da = umma_desc(aa + (uint32_t)(2 * kk) * lbo_a, lbo_a, 128);
            const uint64_t db = umma_desc(bb + (uint32_t)(2 * kk) * lbo_b, lbo_b, 128);
            umma_bf16(d, da, db, idesc, (p > 0 || kk > 0) ? 1u : 0u);
          }
        }
        umma_commit(&mdone[g]);
        issued[g] = kg + 1;
      }
      // drain: wait for the last commit of each group so no MMA is in flight at teardown
      for (int g = 0; g < a.groups; ++g)
        if (issued[g] > 0) k2_wait(&mdone[g], (issued[g] - 1) & 1, a.err);
    }
    __syncwarp();
  } else if (warp < 4 * a.groups) {
    // ---------------- producer / epilogue warpgroups ----------------
    const int g = warp >> 2;
    const int m = threadIdx.x & 127;  // tile row == TMEM lane
    unsigned char* a_hi = smem + lay.a0 + g * lay.a_bytes;
    unsigned char* a_lo = a.passes > 1 ? a_hi + KP * K2_M * 2 : nullptr;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * a.n_pad);
    int kg = 0;
    for (int it = g;; it += a.groups, ++kg) {
      const int tile = blockIdx.x + it * gridDim.x;
      if (tile >= a.n_tiles) break;
      const long long vis = (long long)tile * K2_M + m;
      const bool valid = vis < a.n_vis;
      const int row = valid ? (int)(vis / a.n_chan) : 0;
      const int f = valid ? (int)(vis - (long long)row * a.n_chan) : 0;
      const float4 ri = valid ? __ldg(a.rowinfo + row) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 ci = valid ? __ldg(a.chaninfo + f) : make_float4(0.f, 0.f, 0.f, 1.f);
      const float x = ri.x * ci.w, y = ri.y * ci.w;
      produce_row<KP>(x, a.nmax, valid, a_hi, a_lo, m);
      fence_async_smem();
      mbar_arrive(&afull[g]);
      // phase and amplitude of this visibility while the MMA runs
      const float2 P = phasor_fast(reduce_turns(ri.z, ri.w, ci.x, ci.y));
      const float amp = valid ? a.sgn * ex2_approx(fmaf(a.alpha, ci.z, a.c_amp)) : 0.f;
      // y-direction Hermite functions streamed against the accumulator row
      const float ay = fabsf(y);
      const float ycut = sqrtf(2.0f * a.nmax + 1.0f) + 10.0f;
      const bool yzero = !valid || !(ay <= ycut);
      const float hy = 0.5f * y * y * 1.4426950408889634f;
      int E = yzero ? 0 : max(0, (int)ceilf(hy) - 100);
      float q_prev = 0.f, q = yzero ? 0.f : exp2f((float)E - hy);
      float scale = ldexpf(1.0f, -E);
      if (!k2_wait(&mdone[g], kg & 1, a.err)) break;
      tc_fence_after();
      float xr = 0.f, xi = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < 2 * KP; c0 += 16) {
        if (c0 < a.n_pad) {
          float t[16];
          tmem_ld16(trow + (uint32_t)c0, t);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int n = (c0 >> 1) + i;
            const float ph = q * scale;
            xr = fmaf(t[2 * i], ph, xr);
            xi = fmaf(t[2 * i + 1], ph, xi);
            const float qn = fmaf(c_herm_a[n] * y, q, -c_herm_b[n] * q_prev);
            q_prev = q;
            q = qn;
            if ((i & 3) == 3 && fabsf(q) > 1.8446744e19f) {
              q *= 5.421011e-20f;
              q_prev *= 5.421011e-20f;
              E -= 64;
              scale = ldexpf(1.0f, -E);
            }
          }
        }
      }
      tc_fence_before();
      if (valid) {
        // Z = amp (xr + i xi) P
        const float zr = amp * (xr * P.x - xi * P.y), zi = amp * (xr * P.y + xi * P.x);
        const size_t idx = (size_t)vis;
        if (a.mode == OUT_STORE) {
          a.out[idx] = make_float2(zr, zi);
        } else if (a.mode == OUT_ACCUM) {
          const float2 o = a.out[idx];
          a.out[idx] = make_float2(o.x + zr, o.y + zi);
        } else {
          float2 G;
          if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
          const float2 base = a.mode == OUT_PEEL ? a.peel.data[idx] : a.out[idx];
          a.out[idx] = make_float2(base.x - (G.x * zr - G.y * zi), base.y - (G.x * zi + G.y * zr));
        }
      }
    }
  }
  __syncthreads();
  if (warp == mma_warp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Per-launch prep (FP64, tiny): per-channel constants and, for one shapelet, per-row constants.
__global__ void k2_chaninfo(const double* freq, int n_chan, double nu0, float4* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_chan) return;
  const double nu = freq[f], a = nu / kC;
  const float ah = __double2float_rn(a);
  out[f] = make_float4(ah, __double2float_rn(a - (double)ah), (float)log2(nu / nu0), (float)nu);
}

__global__ void k2_rowinfo(const double* uvw, int n_rows, const ShapeRec* sh, double dec0, float4* out) {
  __shared__ double F[9];
  if (threadIdx.x == 0) shapelet_frame(sh->l, sh->m, dec0, F);
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const double u = uvw[3 * (size_t)r], v = uvw[3 * (size_t)r + 1], w = uvw[3 * (size_t)r + 2];
  const double up = F[0] * u + F[1] * v + F[2] * w, vp = F[3] * u + F[4] * v + F[5] * w;
  const double xs = ((double)sh->kx_u * up + (double)sh->kx_v * vp) / kC;
  const double ys = ((double)sh->ky_u * up + (double)sh->ky_v * vp) / kC;
  const double tau = u * sh->l + v * sh->m + w * sh->nm1;
  const float th = __double2float_rn(tau);
  out[r] = make_float4((float)xs, (float)ys, th, __double2float_rn(tau - (double)th));
}

static int g_consts_ready[64] = {0};

static int k2_setup_constants(int device, cudaStream_t st) {
  if (device >= 0 && device < 64 && g_consts_ready[device]) return WN_OK;
  float ha[kNmaxLimit + 1], hb[kNmaxLimit + 1];
  for (int n = 0; n <= kNmaxLimit; ++n) {
    ha[n] = (float)std::sqrt(2.0 / (n + 1));
    hb[n] = (float)std::sqrt((double)n / (n + 1));
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_herm_a, ha, sizeof(ha), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_herm_b, hb, sizeof(hb), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet constants: ") + cudaGetErrorString(e));
  if (device >= 0 && device < 64) g_consts_ready[device] = 1;
  return WN_OK;
}

template <int KP>
static cudaError_t k2_launch_t(const K2Args& a, int grid, int smem, cudaStream_t st) {
  auto fn = k2_shapelet<KP>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, K2_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

// Workspace: grow-only device buffer owned by the context.
static int ws_reserve(wn_ctx* ctx, size_t bytes, cudaStream_t st) {
  if (ctx->ws_bytes >= bytes) return WN_OK;
  if (ctx->ws) {
    cudaStreamSynchronize(st);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("workspace: ") + cudaGetErrorString(e));
  ctx->ws_bytes = bytes;
  return WN_OK;
}

int launch_shapelets(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                     cudaStream_t st) {
  if (int r = k2_setup_constants(ctx->device, st)) return r;
  const size_t chan_bytes = ((size_t)o.n_chan * sizeof(float4) + 255) & ~(size_t)255;
  if (int r = ws_reserve(ctx, chan_bytes + (size_t)o.n_rows * sizeof(float4), st)) return r;
  float4* chaninfo = static_cast<float4*>(ctx->ws);
  float4* rowinfo = reinterpret_cast<float4*>(static_cast<char*>(ctx->ws) + chan_bytes);
  k2_chaninfo<<<(o.n_chan + 255) / 256, 256, 0, st>>>(o.freq, o.n_chan, o.nu0, chaninfo);
  const long long n_vis = (long long)o.n_rows * o.n_chan;
  const int n_tiles = (int)((n_vis + K2_M - 1) / K2_M);
  const int passes = ctx->shape_mode == WN_SHAPE_BF16X1 ? 1 : 3;
  const double L0 = std::log2(o.nu0);
  for (int q = 0; q < M->n_shape; ++q) {
    const ShapeRec& h = M->sh_host[q];
    k2_rowinfo<<<(o.n_rows + 255) / 256, 256, 0, st>>>(o.uvw, o.n_rows, M->sh + q, o.dec0, rowinfo);
    K2Args a;
    a.rowinfo = rowinfo;
    a.chaninfo = chaninfo;
    a.bop = M->bop + h.b_off;
    a.n_pad = h.n_pad;
    a.nmax = h.nmax;
    a.passes = passes;
    a.n_chan = o.n_chan;
    a.n_base = o.n_base;
    a.n_tiles = n_tiles;
    a.n_vis = n_vis;
    a.c_amp = (float)((double)h.lS + (double)h.alpha * (L0 - h.lref));
    a.alpha = h.alpha;
    a.sgn = h.sgn;
    a.out = out;
    a.peel = pa;
    a.err = ctx->d_err;
    // the first shapelet applies the caller's mode, the rest add (or subtract G times) their part
    a.mode = q == 0 ? mode : (mode == OUT_STORE ? OUT_ACCUM : (mode == OUT_PEEL ? OUT_SUBG : mode));
    a.groups = K2_GROUPS;
    K2Layout lay = k2_layout(h.k_pad, h.n_pad, passes, a.groups);
    if (lay.total > 227 * 1024) {
      a.groups = 1;
      lay = k2_layout(h.k_pad, h.n_pad, passes, 1);
    }
    if (lay.total > 227 * 1024) return set_error(WN_EINVAL, "shapelet operand does not fit in shared memory");
    const int grid = std::min(n_tiles, ctx->num_sms);
    cudaError_t e;
    switch (h.k_pad) {
      case 16: e = k2_launch_t<16>(a, grid, lay.total, st); break;
      case 32: e = k2_launch_t<32>(a, grid, lay.total, st); break;
      case 48: e = k2_launch_t<48>(a, grid, lay.total, st); break;
      case 64: e = k2_launch_t<64>(a, grid, lay.total, st); break;
      case 80: e = k2_launch_t<80>(a, grid, lay.total, st); break;
      case 96: e = k2_launch_t<96>(a, grid, lay.total, st); break;
      case 112: e = k2_launch_t<112>(a, grid, lay.total, st); break;
      default: e = k2_launch_t<128>(a, grid, lay.total, st); break;
    }
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet kernel launch: ") + cudaGetErrorString(e));
  }
  return WN_OK;
}

}  // namespace wn

extern "C" int wn_predict_grad(wn_ctx*, const wn_obs*, int, const void*, int, int, const void*, void*,
                               const wn_sky_grad*, double*, void*) {
  return wn::set_error(WN_EINVAL, "adjoint not built yet");
}
