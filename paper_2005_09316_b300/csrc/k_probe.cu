// Pipe-throughput microbenchmarks: the rates the roofline fractions of the phasor kernels are read
// against.  Each kernel runs eight independent dependency chains per thread (enough to hide the
// pipe latency at 8 CTAs of 256 threads per SM) for a fixed iteration count; the host times the
// launch with CUDA events (best of three) and converts to lane operations per second.
#include "wn_internal.cuh"
#include "k1_loop.cuh"

#include <vector>

namespace wn {

constexpr int KP_CHAINS = 8;

__global__ void kp_ffma(float* out, int iters, float a, float b) {
  float x[KP_CHAINS];
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < KP_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void kp_ffma2(float* out, int iters, float a, float b) {
  float2 x[KP_CHAINS];
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < KP_CHAINS; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) s += x[i].x + x[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void kp_ex2(float* out, int iters, float a) {
  float x[KP_CHAINS];
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) x[i] = threadIdx.x * 1e-6f + i * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < KP_CHAINS; ++i) x[i] = ex2_approx(x[i]) * a;
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void kp_dfma(float* out, int iters, double a, double b) {
  double x[KP_CHAINS];
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < KP_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < KP_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// The point/Gaussian kernel's channel loop by itself (ks_comp_uniform, K = 12, the single-launch
// form): per pass, four groups of 16 points and one of 16 Gaussians (the 4:1 mix of the MWA-like
// workload), their 48-byte records and spectrum values held in shared memory, against two rows x 12
// channels per lane, at the kernel's occupancy of one CTA of 512 threads per SM.  No record building,
// no global memory and no barriers inside the loop: the rate the full kernel approaches.
constexpr int KP_LOOP_K = 12;
constexpr int KP_LOOP_GROUPS = 5;    // groups of 16 components per pass
constexpr int KP_LOOP_THREADS = 512;

__global__ void __launch_bounds__(KP_LOOP_THREADS, 1) kp_loop(float* out, int passes) {
  extern __shared__ __align__(16) unsigned char kp_smem[];
  float4* rec = reinterpret_cast<float4*>(kp_smem);          // [16][3]
  float* tab = reinterpret_cast<float*>(rec + 48);             // [16][384]
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 16) {
    const float ph = 1e-3f * tid;
    rec[3 * tid] = make_float4(1234.5f + tid, 2345.25f + tid, 1e-5f, -1e-5f);
    rec[3 * tid + 1] = make_float4(cosf(ph), cosf(2.f * ph), -sinf(ph), -sinf(2.f * ph));
    rec[3 * tid + 2] = make_float4(-1e-3f * tid, -2e-3f * tid, (tid & 1) ? 3.14159265f : 0.f, 0.f);
  }
  for (int i = tid; i < 16 * 384; i += KP_LOOP_THREADS) tab[i] = 1.0f + 1e-4f * (i & 511);
  __syncthreads();
  float wg[KP_LOOP_K];
  const float a0h = 0.557f + 1e-4f * lane, a0l = 1e-9f;
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) wg[k] = 1e-3f * (k + 1);
  float2 Vre[KP_LOOP_K], Vim[KP_LOOP_K];
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);
  const float* tb = tab + lane * KP_LOOP_K;
  for (int it = 0; it < passes; ++it) {
    for (int t = 0; t < KP_LOOP_GROUPS; ++t) {
      if (t == KP_LOOP_GROUPS - 1) {
#pragma unroll 4
        for (int j = 0; j < 16; ++j)
          ks_comp_uniform<KP_LOOP_K, true>(rec[3 * j], rec[3 * j + 1], rec[3 * j + 2], tb + j * 384, a0h, a0l, wg,
                                           Vre, Vim);
      } else {
#pragma unroll 4
        for (int j = 0; j < 16; ++j)
          ks_comp_uniform<KP_LOOP_K, false>(rec[3 * j], rec[3 * j + 1], rec[3 * j + 2], tb + j * 384, a0h, a0l, wg,
                                            Vre, Vim);
      }
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) sum += Vre[k].x + Vre[k].y + Vim[k].x + Vim[k].y;
  out[blockIdx.x * blockDim.x + tid] = sum;
}

// tcgen05 throughput as the shapelet kernel uses it: kind::f16 MMAs (M = 128, K = 16, bf16 operands,
// FP32 accumulator in TMEM) with both operands K-major in shared memory in the same no-swizzle
// core-matrix layout, issued back to back by one thread per CTA, one CTA per SM.  The operands are zero
// (the timing does not depend on them).  Block 0, warp 0 then times 16-column TMEM loads: one load and
// its wait at a time, and eight loads under one wait.  clk = {MMA issue-to-completion clocks of each
// CTA, then the two load timings}.
constexpr int KP_MMA_REP = 512;  // K = 64 passes (4 MMAs each)

template <bool TF32>
__global__ void __launch_bounds__(128, 1) kp_mma(int n, long long* clk, unsigned* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* a_t = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);  // 128 x 64 bf16
  unsigned char* b_t = a_t + 16384;                                            // n x 64 bf16
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (16384 + n * 128) / 16; i += 128) reinterpret_cast<uint4*>(a_t)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    // kind::f16 with bf16 A and B (formats 1), or kind::tf32 (formats 2); D f32; M = 128, N = n
    const uint32_t fmt = TF32 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t a0 = smem_u32(a_t), b0 = smem_u32(b_t);
    const uint32_t lbo_a = (128u >> 3) << 7, lbo_b = ((uint32_t)n >> 3) << 7;
    auto desc = [](uint32_t addr, uint32_t lbo) {
      return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)(128u >> 4) << 32) |
             (1ull << 46);
    };
    const long long t0 = clock64();
    for (int r = 0; r < KP_MMA_REP; ++r) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = desc(a0 + 2u * kk * lbo_a, lbo_a), db = desc(b0 + 2u * kk * lbo_b, lbo_b);
        const uint32_t acc = (r > 0 || kk > 0) ? 1u : 0u;
        if (TF32)  // K = 8 four-byte elements: the same 32 bytes of each row as K = 16 bf16
          asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                       "l"(da), "l"(db), "r"(idesc), "r"(acc)
                       : "memory");
        else
          asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                       "l"(da), "l"(db), "r"(idesc), "r"(acc)
                       : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    const bool ok = mbar_wait_bounded(&bar, 0, err);
    clk[blockIdx.x] = ok ? (clock64() - t0) : -1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (blockIdx.x == 0 && warp == 0) {
    uint32_t v[8][16];
    float acc = 0.f;
    const long long t0 = clock64();
    for (int rep = 0; rep < 16; ++rep) {
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[0][4]), "=r"(v[0][5]), "=r"(v[0][6]),
                     "=r"(v[0][7]), "=r"(v[0][8]), "=r"(v[0][9]), "=r"(v[0][10]), "=r"(v[0][11]), "=r"(v[0][12]),
                     "=r"(v[0][13]), "=r"(v[0][14]), "=r"(v[0][15])
                   : "r"(tmem + (uint32_t)((rep & 7) * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(v[0][0]), "+r"(v[0][15])::"memory");
      acc += __uint_as_float(v[0][0]) + __uint_as_float(v[0][15]);
    }
    const long long t1 = clock64();
    for (int rep = 0; rep < 2; ++rep) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[c][0]), "=r"(v[c][1]), "=r"(v[c][2]), "=r"(v[c][3]), "=r"(v[c][4]), "=r"(v[c][5]),
                       "=r"(v[c][6]), "=r"(v[c][7]), "=r"(v[c][8]), "=r"(v[c][9]), "=r"(v[c][10]), "=r"(v[c][11]),
                       "=r"(v[c][12]), "=r"(v[c][13]), "=r"(v[c][14]), "=r"(v[c][15])
                     : "r"(tmem + (uint32_t)(c * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 8; ++c) acc += __uint_as_float(v[c][rep]) + __uint_as_float(v[c][15 - rep]);
    }
    const long long t2 = clock64();
    if (tid == 0) {
      clk[gridDim.x] = (t1 - t0) / 16;
      clk[gridDim.x + 1] = (t2 - t1) / 2;
    }
    if (acc != 0.f) atomicOr(err, WN_DEVERR_TIMEOUT);  // zero operands give a zero accumulator
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// The failure path of the kernels' bounded waits: one thread waits on an mbarrier that nothing ever
// arrives at, with the given limit, using the same helper as the kernels.  It must give up, raise
// WN_DEVERR_TIMEOUT and return; nothing faults and the context stays usable.
__global__ void kp_wait_timeout(unsigned* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    (void)mbar_wait_bounded(&bar, 0, err, limit);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace wn

using namespace wn;

extern "C" int wn_selftest_timeout(wn_ctx* ctx, double seconds) {
  if (!ctx) return set_error(WN_EINVAL, "NULL argument");
  if (!(seconds > 0.0 && seconds <= 5.0)) return set_error(WN_EINVAL, "wn_selftest_timeout: seconds must be in (0, 5]");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(ctx->device);
  int khz = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
  const long long limit = (long long)(seconds * 1e3 * (double)(khz > 0 ? khz : 2032000));
  if (e == cudaSuccess) {
    kp_wait_timeout<<<1, 32>>>(ctx->d_err, limit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  return WN_OK;
}

extern "C" int wn_phasor_loop_rate(wn_ctx* ctx, double* evals_per_s) {
  if (!ctx || !evals_per_s) return set_error(WN_EINVAL, "NULL argument");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(ctx->device);
  const int blocks = ctx->num_sms, threads = KP_LOOP_THREADS, passes = 40;
  const int smem = 48 * 16 + 16 * 384 * 4;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * blocks * threads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
    e = cudaEventRecord(e0, st);
    kp_loop<<<blocks, threads, smem, st>>>(out, passes);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  *evals_per_s = (double)blocks * threads * passes * KP_LOOP_GROUPS * 16 * 2 * KP_LOOP_K / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("phasor loop probe: ") + cudaGetErrorString(e));
  return WN_OK;
}

extern "C" int wn_pipe_rates(wn_ctx* ctx, double* rates) {
  if (!ctx || !rates) return set_error(WN_EINVAL, "NULL argument");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(ctx->device);
  const int blocks = ctx->num_sms * 8, threads = 256;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * blocks * threads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int iters[4] = {1 << 14, 1 << 13, 1 << 12, 1 << 9};
  const double per_iter[4] = {KP_CHAINS, 2.0 * KP_CHAINS, KP_CHAINS, KP_CHAINS};  // lane operations
  for (int kind = 0; kind < 4 && e == cudaSuccess; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, st);
      if (kind == 0) kp_ffma<<<blocks, threads, 0, st>>>(out, iters[0], 0.999f, 1e-3f);
      else if (kind == 1) kp_ffma2<<<blocks, threads, 0, st>>>(out, iters[1], 0.999f, 1e-3f);
      else if (kind == 2) kp_ex2<<<blocks, threads, 0, st>>>(out, iters[2], 0.999f);
      else kp_dfma<<<blocks, threads, 0, st>>>(out, iters[3], 0.999, 1e-3);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) best = ms;
    }
    rates[kind] = (double)blocks * threads * iters[kind] * per_iter[kind] / (best * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("pipe-rate probe: ") + cudaGetErrorString(e));
  return WN_OK;
}

// Clocks per MMA at N = 128 and N = 64 (out[0], out[1]) and the two TMEM load timings (out[2], out[3]).
template <bool TF32>
static int mma_rate(wn_ctx* ctx, double* out) {
  if (!ctx || !out) return set_error(WN_EINVAL, "NULL argument");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(ctx->device);
  const int grid = ctx->num_sms;
  long long* clk = nullptr;
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&clk, sizeof(long long) * (grid + 2));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<long long> h(grid + 2);
  const int ns[2] = {128, 64};
  // 64 KB of shared memory per CTA: at most 3 CTAs (384 TMEM columns) share an SM, so no allocation waits
  const int smem = 64 * 1024;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kp_mma<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
      kp_mma<TF32><<<grid, 128, smem, st>>>(ns[i], clk, ctx->d_err);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), clk, sizeof(long long) * (grid + 2), cudaMemcpyDeviceToHost);
    double sum = 0.0;
    int cnt = 0;
    for (int b = 0; b < grid; ++b)
      if (h[b] > 0) {
        sum += (double)h[b];
        ++cnt;
      }
    out[i] = cnt ? sum / cnt / (4.0 * KP_MMA_REP) : -1.0;
    if (i == 0) {
      out[2] = (double)h[grid];
      out[3] = (double)h[grid + 1];
    }
  }
  if (st) cudaStreamDestroy(st);
  cudaFree(clk);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("MMA rate probe: ") + cudaGetErrorString(e));
  return WN_OK;
}

extern "C" int wn_mma_rate(wn_ctx* ctx, double* out) { return mma_rate<false>(ctx, out); }

extern "C" int wn_mma_rate_tf32(wn_ctx* ctx, double* out) {
  if (!out) return set_error(WN_EINVAL, "NULL argument");
  double full[4];
  const int r = mma_rate<true>(ctx, full);
  if (r == WN_OK) {
    out[0] = full[0];
    out[1] = full[1];
  }
  return r;
}
