// K1: mixed-precision direct prediction for point and Gaussian components.
//
//   V(t,b,f) = sum_j S_j(nu_f) xi_j exp(-2 pi i tau_j(t,b) nu_f / c),
//   tau_j = u l_j + v m_j + w (n_j - 1)   (metres; eq:measure_eq_discrete, eq:env_visi_def)
//
// Design (one GPU, output-stationary, no atomics):
//  * A CTA owns a tile of rows (t,b) x a block of channels; every output stays in registers while
//    the CTA streams the whole component table through shared memory (TMA bulk copies into a ring
//    of stages, mbarrier-synchronised), then writes each visibility once (predict, accumulate or
//    the fused peel R = D - g1 conj(g2) V of Sec. 5.1).
//  * Within a warp, L lanes share a pair of rows; each lane owns K channels of both rows.
//  * FP64 is used only for the phase argument: tau is formed in FP64 once per (component, row) and
//    split into a float pair; per-channel phases are reduced to [-1/2, 1/2] turns in double-float
//    FP32 arithmetic (no FP64 in the channel loop).
//  * Uniformly spaced channels: the phasor of channel f+1 is the phasor of channel f times
//    Delta = exp(-2 pi i tau dnu / c) (one complex multiply), restarted from an exact phase at the
//    first channel of every lane; Delta itself is formed from an exactly reduced phase with the
//    accurate sincospif.  Arbitrary channel lists reduce and evaluate every channel.
//  * Spectrum and Gaussian envelope share one exp2: amplitude = sgn * 2^(log2|S| + alpha log2(nu/nu_ref)
//    - q (nu/c)^2 E log2 e), q the Gaussian quadratic form in (u, v) metres.
#include "wn_internal.cuh"

namespace wn {

constexpr int K1_WARPS = 8;
constexpr int K1_THREADS = 32 * K1_WARPS;
constexpr int K1_CT = 32;      // components per TMA stage
constexpr int K1_NSTAGE = 4;   // stages in the ring



constexpr int K1_FLUSH = 4;     // tiles (128 components) per register partial sum

struct K1Smem {
  // offsets in bytes into dynamic shared memory
  int stage, bars, uvw, rec, q, cs, acc, total;
};

// acc holds the second-level sums: every K1_FLUSH tiles the register partial sums (at most 128
// components) are added into it, which keeps the FP32 rounding of a 25,000-term sum near 1e-7.
__host__ __device__ inline K1Smem k1_smem_layout(int log2L, int K) {
  int groups = 32 >> log2L;
  int rpw = 2 * groups;  // rows per warp
  K1Smem s;
  s.stage = 0;
  s.bars = s.stage + K1_NSTAGE * K1_CT * (int)sizeof(PGRec);
  s.uvw = s.bars + 2 * K1_NSTAGE * 8;
  s.rec = s.uvw + K1_WARPS * rpw * 3 * 8;
  s.q = s.rec + K1_WARPS * K1_CT * rpw * 16;
  s.cs = s.q + K1_WARPS * K1_CT * rpw * 4;
  s.acc = s.cs + K1_WARPS * K1_CT * 16;
  s.total = s.acc + K1_THREADS * 2 * K * 8;
  return s;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 32)) {  // ~2 s at the B300 clock: something is wrong
      atomicOr(err, WN_DEVERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// One (row tile, channel block) of one observation: the body of the single-launch kernel below and
// of the batched serving kernel.  Re-entrant: it initialises and invalidates its own barriers.
template <int K, bool UNIFORM>
__device__ __forceinline__ void k1_tile(const K1Args& a, const int bx, const int by, unsigned char* smem) {
  const K1Smem lay = k1_smem_layout(a.log2L, K);
  PGRec* stage = reinterpret_cast<PGRec*>(smem + lay.stage);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* empty = full + K1_NSTAGE;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = 1 << a.log2L;
  const int groups = 32 >> a.log2L;
  const int rpw = 2 * groups;
  const int g = lane >> a.log2L, sub = lane & (L - 1);
  const int row_w0 = bx * (K1_WARPS * rpw) + warp * rpw;
  const int f0 = by * a.chan_block + sub * K;

  double* uvw_s = reinterpret_cast<double*>(smem + lay.uvw) + warp * rpw * 3;
  float4* rec = reinterpret_cast<float4*>(smem + lay.rec) + warp * K1_CT * rpw;
  float* qs = reinterpret_cast<float*>(smem + lay.q) + warp * K1_CT * rpw;
  float4* cs = reinterpret_cast<float4*>(smem + lay.cs) + warp * K1_CT;
  float2* acc = reinterpret_cast<float2*>(smem + lay.acc) + threadIdx.x;  // [2K][K1_THREADS]
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i * K1_THREADS] = make_float2(0.f, 0.f);

  const int n_pt_tiles = (a.n_point + K1_CT - 1) / K1_CT;
  const int n_tiles = n_pt_tiles + (a.n_gauss + K1_CT - 1) / K1_CT;
  auto tile_start = [&](int t) { return t < n_pt_tiles ? t * K1_CT : a.n_point + (t - n_pt_tiles) * K1_CT; };
  auto tile_count = [&](int t) {
    return t < n_pt_tiles ? min(K1_CT, a.n_point - t * K1_CT) : min(K1_CT, a.n_gauss - (t - n_pt_tiles) * K1_CT);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < K1_NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], K1_WARPS);
    }
    fence_mbar_init();
  }
  // rows of this warp: (u, v, w) in FP64
  for (int i = lane; i < rpw * 3; i += 32) {
    int r = row_w0 + i / 3;
    uvw_s[i] = r < a.n_rows ? a.uvw[(size_t)r * 3 + i % 3] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 0; t < min(K1_NSTAGE, n_tiles); ++t) {
      uint32_t bytes = tile_count(t) * (uint32_t)sizeof(PGRec);
      mbar_arrive_expect_tx(&full[t], bytes);
      tma_bulk_g2s(stage + t * K1_CT, a.comps + tile_start(t), bytes, &full[t]);
    }
  }

  // Per-lane channel constants: nu/c as float pairs (an FP64 multiply and split), the rest in FP32.
  float lam[K], wg[K];
  float ah[UNIFORM ? 1 : K], al[UNIFORM ? 1 : K];
  const float inv_nu0 = (float)(1.0 / a.nu0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int f = min(f0 + k, a.n_chan - 1);
    const double nu = a.freq[f];
    lam[k] = log2f((float)nu * inv_nu0);
    const float x = (float)(nu * (1.0 / kC));
    wg[k] = (float)(kGaussE * kLog2e) * x * x;
    if (!UNIFORM) split_double(nu * (1.0 / kC), ah[k], al[k]);
  }
  float a0h, a0l;
  split_double(a.freq[min(f0, a.n_chan - 1)] * (1.0 / kC), a0h, a0l);
  const double L0 = log2(a.nu0);

  float2 V0[K], V1[K];
#pragma unroll
  for (int k = 0; k < K; ++k) V0[k] = V1[k] = make_float2(0.f, 0.f);

  bool ok = true;
  for (int t = 0; t < n_tiles && ok; ++t) {
    const int s = t % K1_NSTAGE;
    if (threadIdx.x == 0 && t > 0 && t - 1 + K1_NSTAGE < n_tiles) {
      // refill the stage of tile t-1 once every warp has produced its records from it
      const int sp = (t - 1) % K1_NSTAGE, tn = t - 1 + K1_NSTAGE;
      if (bounded_wait(&empty[sp], ((t - 1) / K1_NSTAGE) & 1, a.err)) {
        uint32_t bytes = tile_count(tn) * (uint32_t)sizeof(PGRec);
        mbar_arrive_expect_tx(&full[sp], bytes);
        tma_bulk_g2s(stage + sp * K1_CT, a.comps + tile_start(tn), bytes, &full[sp]);
      }
    }
    if (!bounded_wait(&full[s], (t / K1_NSTAGE) & 1, a.err)) {
      ok = false;
      break;
    }
    const int cnt = tile_count(t);
    const bool gauss = t >= n_pt_tiles;
    const PGRec* st = stage + s * K1_CT;

    // --- records: FP64 phase argument per (component, row), shared by the L lanes of a row pair
    const int rshift = 6 - a.log2L;  // rpw == 1 << rshift
    for (int idx = lane; idx < (cnt << rshift); idx += 32) {
      const int j = idx >> rshift, rr = idx & (rpw - 1);
      const double u = uvw_s[rr * 3 + 0], v = uvw_s[rr * 3 + 1], w = uvw_s[rr * 3 + 2];
      const double tau = fma(u, st[j].l, fma(v, st[j].m, w * st[j].nm1));
      float th, tl;
      split_double(tau, th, tl);
      float4 r;
      r.x = th;
      r.y = tl;
      if (UNIFORM) {
        float2 D = phasor_accurate(reduce_turns(th, tl, a.dnu_h, a.dnu_l));
        r.z = D.x;
        r.w = D.y;
      } else {
        r.z = r.w = 0.f;
      }
      rec[j * rpw + rr] = r;
      if (gauss) {
        const float uf = (float)u, vf = (float)v;
        qs[j * rpw + rr] = st[j].ga * uf * uf + st[j].gb * uf * vf + st[j].gc * vf * vf;
      }
    }
    for (int j = lane; j < cnt; j += 32)
      cs[j] = make_float4(st[j].lS + st[j].alpha * (float)(L0 - st[j].lref), st[j].alpha, st[j].sgn, 0.f);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);

    // --- channel loop: K channels of two rows per lane
    for (int j = 0; j < cnt; ++j) {
      const float4 c = cs[j];
      const float4 R0 = rec[j * rpw + 2 * g], R1 = rec[j * rpw + 2 * g + 1];
      const float q0 = gauss ? qs[j * rpw + 2 * g] : 0.f;
      const float q1 = gauss ? qs[j * rpw + 2 * g + 1] : 0.f;
      if (UNIFORM) {
        float2 P0 = phasor_fast(reduce_turns(R0.x, R0.y, a0h, a0l));
        float2 P1 = phasor_fast(reduce_turns(R1.x, R1.y, a0h, a0l));
        P0.x *= c.z; P0.y *= c.z;
        P1.x *= c.z; P1.y *= c.z;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          // amplitude: spectrum and (for Gaussians) envelope in one exp2
          const float e = fmaf(c.y, lam[k], c.x);
          const float A0 = ex2_approx(gauss ? fmaf(-q0, wg[k], e) : e);
          const float A1 = gauss ? ex2_approx(fmaf(-q1, wg[k], e)) : A0;
          V0[k].x = fmaf(A0, P0.x, V0[k].x);
          V0[k].y = fmaf(A0, P0.y, V0[k].y);
          V1[k].x = fmaf(A1, P1.x, V1[k].x);
          V1[k].y = fmaf(A1, P1.y, V1[k].y);
          if (k + 1 < K) {
            const float x0 = P0.x * R0.z - P0.y * R0.w, y0 = P0.x * R0.w + P0.y * R0.z;
            const float x1 = P1.x * R1.z - P1.y * R1.w, y1 = P1.x * R1.w + P1.y * R1.z;
            P0 = make_float2(x0, y0);
            P1 = make_float2(x1, y1);
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float2 P0 = phasor_fast(reduce_turns(R0.x, R0.y, ah[k], al[k]));
          const float2 P1 = phasor_fast(reduce_turns(R1.x, R1.y, ah[k], al[k]));
          const float e = fmaf(c.y, lam[k], c.x);
          const float s0 = c.z * ex2_approx(gauss ? fmaf(-q0, wg[k], e) : e);
          const float s1 = gauss ? c.z * ex2_approx(fmaf(-q1, wg[k], e)) : s0;
          V0[k].x = fmaf(s0, P0.x, V0[k].x);
          V0[k].y = fmaf(s0, P0.y, V0[k].y);
          V1[k].x = fmaf(s1, P1.x, V1[k].x);
          V1[k].y = fmaf(s1, P1.y, V1[k].y);
        }
      }
    }
    __syncwarp();
    if ((t + 1) % K1_FLUSH == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 x = acc[k * K1_THREADS], y = acc[(K + k) * K1_THREADS];
        acc[k * K1_THREADS] = make_float2(x.x + V0[k].x, x.y + V0[k].y);
        acc[(K + k) * K1_THREADS] = make_float2(y.x + V1[k].x, y.y + V1[k].y);
        V0[k] = V1[k] = make_float2(0.f, 0.f);
      }
    }
  }

  // --- epilogue: each visibility written once
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int row = row_w0 + 2 * g + rr;
    if (row >= a.n_rows) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int f = f0 + k;
      if (f >= a.n_chan) continue;
      const size_t idx = (size_t)row * a.n_chan + f;
      const float2 p = rr == 0 ? V0[k] : V1[k];
      const float2 q = acc[(rr * K + k) * K1_THREADS];
      float2 v = make_float2(q.x + p.x, q.y + p.y);
      if (!ok) v = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
      if (a.mode == OUT_STORE) {
        a.out[idx] = v;
      } else if (a.mode == OUT_ACCUM) {
        float2 o = a.out[idx];
        a.out[idx] = make_float2(o.x + v.x, o.y + v.y);
      } else {
        float2 G;
        if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
        const float2 d = a.peel.data[idx];
        a.out[idx] = make_float2(d.x - (G.x * v.x - G.y * v.y), d.y - (G.x * v.y + G.y * v.x));
      }
    }
  }
  __syncthreads();  // every warp is past its last barrier wait and shared-memory read
  if (threadIdx.x == 0) {
    for (int s = 0; s < K1_NSTAGE; ++s) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
  }
  __syncthreads();
}

template <int K, bool UNIFORM>
__global__ void __launch_bounds__(K1_THREADS, 2) k1_phasor(const K1Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  k1_tile<K, UNIFORM>(a, blockIdx.x, blockIdx.y, smem);
}

struct K1Choice {
  int log2L, K;
};

// Pick lanes-per-row L and channels-per-lane K: fewest padded channel slots, then the widest channel
// block (each FP64 phase record per (component, row) then serves the most channels), then larger K.
static K1Choice k1_choose(int F) {
  K1Choice best{5, 12};
  long best_slots = -1, best_cb = 0;
  const int Ks[4] = {12, 8, 16, 4};
  for (int li = 2; li <= 5; ++li) {
    for (int K : Ks) {
      long cb = (long)K << li;
      long slots = ((F + cb - 1) / cb) * cb;
      bool better = best_slots < 0 || slots < best_slots || (slots == best_slots && cb > best_cb) ||
                    (slots == best_slots && cb == best_cb && K > best.K && K <= 12);
      if (better) {
        best_slots = slots;
        best_cb = cb;
        best = {li, K};
      }
    }
  }
  return best;
}

template <int K, bool U>
static cudaError_t k1_launch(const K1Args& a, dim3 grid, int smem, cudaStream_t st) {
  auto fn = k1_phasor<K, U>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, K1_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

int launch_phasor_mixed(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        cudaStream_t st) {
  K1Choice ch = k1_choose(o.n_chan);
  K1Args a;
  a.uvw = o.uvw;
  a.freq = o.freq;
  a.n_rows = o.n_rows;
  a.n_chan = o.n_chan;
  a.n_base = o.n_base;
  a.log2L = ch.log2L;
  a.chan_block = ch.K << ch.log2L;
  a.nu0 = o.nu0;
  double dn = o.dnu / kC;
  a.dnu_h = (float)dn;
  a.dnu_l = (float)(dn - (double)a.dnu_h);
  a.comps = M->pg;
  a.n_point = M->n_point;
  a.n_gauss = M->n_gauss;
  a.out = out;
  a.mode = mode;
  a.peel = pa;
  a.err = ctx->d_err;
  const int rows_per_cta = K1_WARPS * 2 * (32 >> ch.log2L);
  dim3 grid((o.n_rows + rows_per_cta - 1) / rows_per_cta, (o.n_chan + a.chan_block - 1) / a.chan_block);
  const int smem = k1_smem_layout(ch.log2L, ch.K).total;
  cudaError_t e;
  switch (ch.K * 2 + (o.uniform ? 1 : 0)) {
    case 4 * 2 + 1: e = k1_launch<4, true>(a, grid, smem, st); break;
    case 4 * 2: e = k1_launch<4, false>(a, grid, smem, st); break;
    case 8 * 2 + 1: e = k1_launch<8, true>(a, grid, smem, st); break;
    case 8 * 2: e = k1_launch<8, false>(a, grid, smem, st); break;
    case 12 * 2 + 1: e = k1_launch<12, true>(a, grid, smem, st); break;
    case 12 * 2: e = k1_launch<12, false>(a, grid, smem, st); break;
    case 16 * 2 + 1: e = k1_launch<16, true>(a, grid, smem, st); break;
    default: e = k1_launch<16, false>(a, grid, smem, st); break;
  }
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("phasor kernel launch: ") + cudaGetErrorString(e));
  return WN_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched persistent form for the serving loop: one launch walks a work table of (request, row
// tile, channel block) entries of many observations; CTA b takes entries b, b + gridDim.x, ...
// Every entry runs the same k1_tile code as a single launch, so a request's visibilities are
// bit-identical whether it is predicted alone or in a batch.
// ------------------------------------------------------------------------------------------------
constexpr int K1B_KMAX = 12;  // channels per lane in the batched form: 8 or 12, chosen per request
constexpr int K1B_MIN_LOG2L = 3;

__global__ void __launch_bounds__(K1_THREADS, 2) k1_batched(const K1Args* reqs, const K1Work* work,
                                                            const int* n_work) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ K1Args args;
  const int n = *n_work;
  for (int e = blockIdx.x; e < n; e += gridDim.x) {
    const K1Work w = work[e];
    if (threadIdx.x == 0) args = reqs[w.req];
    __syncthreads();
    if (args.chan_block == (12 << args.log2L)) k1_tile<12, true>(args, w.bx, w.by, smem);
    else k1_tile<8, true>(args, w.bx, w.by, smem);
  }
}

int k1_batched_smem() { return k1_smem_layout(K1B_MIN_LOG2L, K1B_KMAX).total; }

// Arguments and tile grid of one observation for the batched kernel (uniform channels only).
int k1_batched_args(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                    K1Args* args, int* grid_x, int* grid_y) {
  if (!o.uniform) return set_error(WN_EINVAL, "batched prediction needs uniformly spaced channels");
  // fewest padded channel slots over K in {12, 8} and L in {8, 16, 32}; ties go to the wider block
  int log2L = 5, K = 12;
  long best = -1;
  for (int li = K1B_MIN_LOG2L; li <= 5; ++li)
    for (int kk : {12, 8}) {
      const long cb = (long)kk << li, slots = ((o.n_chan + cb - 1) / cb) * cb;
      if (best < 0 || slots < best || (slots == best && cb > ((long)K << log2L))) {
        best = slots;
        log2L = li;
        K = kk;
      }
    }
  K1Args& a = *args;
  a.uvw = o.uvw;
  a.freq = o.freq;
  a.n_rows = o.n_rows;
  a.n_chan = o.n_chan;
  a.n_base = o.n_base;
  a.log2L = log2L;
  a.chan_block = K << log2L;
  a.nu0 = o.nu0;
  const double dn = o.dnu / kC;
  a.dnu_h = (float)dn;
  a.dnu_l = (float)(dn - (double)a.dnu_h);
  a.comps = M->pg;
  a.n_point = M->n_point;
  a.n_gauss = M->n_gauss;
  a.out = out;
  a.mode = mode;
  a.peel = pa;
  a.err = ctx->d_err;
  const int rows_per_cta = K1_WARPS * 2 * (32 >> log2L);
  *grid_x = (o.n_rows + rows_per_cta - 1) / rows_per_cta;
  *grid_y = (o.n_chan + a.chan_block - 1) / a.chan_block;
  return WN_OK;
}

cudaError_t k1_batched_setup() {
  return cudaFuncSetAttribute(k1_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, k1_batched_smem());
}

cudaError_t k1_batched_launch(const K1Args* reqs, const K1Work* work, const int* n_work, int grid, cudaStream_t st) {
  k1_batched<<<grid, K1_THREADS, k1_batched_smem(), st>>>(reqs, work, n_work);
  return cudaGetLastError();
}

}  // namespace wn
