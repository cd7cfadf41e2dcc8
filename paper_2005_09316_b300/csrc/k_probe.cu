// Pipe-throughput microbenchmarks: the rates the roofline fractions of the phasor kernels are read
// against.  Each kernel runs eight independent dependency chains per thread (enough to hide the
// pipe latency at 8 CTAs of 256 threads per SM) for a fixed iteration count; the host times the
// launch with CUDA events (best of three) and converts to lane operations per second.
#include "wn_internal.cuh"
#include "k1_loop.cuh"

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

// The point/Gaussian kernel's channel loop by itself (k1_comp_uniform, K = 12): per pass, four tiles of
// 32 points and one of 32 Gaussians (the 4:1 mix of the MWA-like workload) read from shared memory
// against two rows x 12 channels per lane, at the kernel's occupancy of 2 CTAs of 256 threads per SM.
// No records, no global memory and no barriers inside the loop: the rate the full kernel approaches.
constexpr int KP_LOOP_K = 12;

__global__ void __launch_bounds__(256, 2) kp_loop(float* out, int passes) {
  __shared__ float4 rec[32 * 3];
  __shared__ float4 cs[32];
  const int tid = threadIdx.x;
  if (tid < 32) {
    const float ph = 1e-3f * tid;
    rec[3 * tid] = make_float4(1234.5f + tid, 1e-5f, 2345.25f + tid, -1e-5f);
    rec[3 * tid + 1] = make_float4(cosf(ph), cosf(2.f * ph), -sinf(ph), -sinf(2.f * ph));
    rec[3 * tid + 2] = make_float4(sinf(ph), sinf(2.f * ph), -1e-3f * tid, -2e-3f * tid);
    cs[tid] = make_float4(-0.01f * tid, -0.8f, (tid & 1) ? 3.14159265f : 0.f, (tid & 1) ? -1.f : 1.f);
  }
  __syncthreads();
  float lam[KP_LOOP_K], wg[KP_LOOP_K];
  const float a0h = 0.557f + 1e-4f * (tid & 31), a0l = 1e-9f;
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) {
    lam[k] = 0.01f * k + 1e-4f * tid;
    wg[k] = 1e-3f * (k + 1);
  }
  float2 Vre[KP_LOOP_K], Vim[KP_LOOP_K];
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);
  for (int it = 0; it < passes; ++it) {
    for (int t = 0; t < 4; ++t)
      for (int j = 0; j < 32; ++j)
        k1_comp_uniform<KP_LOOP_K, false>(cs[j], rec[3 * j], rec[3 * j + 1], rec[3 * j + 2], a0h, a0l, lam, wg, Vre,
                                          Vim);
    for (int j = 0; j < 32; ++j)
      k1_comp_uniform<KP_LOOP_K, true>(cs[j], rec[3 * j], rec[3 * j + 1], rec[3 * j + 2], a0h, a0l, lam, wg, Vre, Vim);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < KP_LOOP_K; ++k) s += Vre[k].x + Vre[k].y + Vim[k].x + Vim[k].y;
  out[blockIdx.x * blockDim.x + tid] = s;
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
  const int blocks = ctx->num_sms * 2, threads = 256, passes = 40;
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
    kp_loop<<<blocks, threads, 0, st>>>(out, passes);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  *evals_per_s = (double)blocks * threads * passes * 5 * 32 * 2 * KP_LOOP_K / (best * 1e-3);
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
