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
//  * Within a warp, L lanes share a pair of rows; each lane owns K channels of both rows, and the two
//    rows travel together in f32x2 register pairs (one packed FFMA2/FMUL2 does both rows).
//  * No FP64 in the loops: tau is formed once per (component, row) in double-float FP32 from float-pair
//    operands (error-free two-product and two-sum) and per-channel phases are reduced to [-1/2, 1/2]
//    turns in double-float FP32 arithmetic.
//  * Uniformly spaced channels: the phasors follow the three-term recurrence P(f+1) = 2 cos(delta) P(f)
//    - P(f-1), delta = 2 pi tau dnu / c (one packed FMA per component of the complex value), run up and
//    down from an exact phase at the middle channel of every lane (k1_loop.cuh); the one-channel step
//    exp(-i delta) is formed from an exactly reduced phase with the accurate sincospif.  Arbitrary
//    channel lists reduce and evaluate every channel.
//  * Spectrum and Gaussian envelope share one exp2: amplitude = sgn * 2^(log2|S| + alpha log2(nu/nu_ref)
//    - q (nu/c)^2 E log2 e), q the Gaussian quadratic form in (u, v) metres.
#include "wn_internal.cuh"
#include "k1_loop.cuh"

#include <algorithm>
#include <climits>

namespace wn {

constexpr int K1_WARPS = 8;
constexpr int K1_THREADS = 32 * K1_WARPS;
constexpr int K1_CT = 32;      // components per TMA stage
constexpr int K1_NSTAGE = 4;   // stages in the ring



constexpr int K1_FLUSH = 4;     // tiles (128 components) per register partial sum

struct K1Smem {
  // offsets in bytes into dynamic shared memory
  int stage, bars, uvw, rec, cs, acc, total;
};

// Per warp: (u, v, w) of its rows as float pairs, and per (component, row pair) a 48-byte record of
// three float4: {th0, tl0, th1, tl1} (tau pairs), {D0.x, D1.x, D0.y, D1.y} and {-D0.y, -D1.y, -q0, -q1}
// (D the one-channel phasor step, q the Gaussian form), laid out so each pair of the two rows loads
// straight into an f32x2 register pair.  acc holds the second-level sums: every K1_FLUSH tiles the
// register partial sums (at most 128 components) are added into it, which keeps the FP32 rounding of a
// 25,000-term sum near 1e-7.
__host__ __device__ inline K1Smem k1_smem_layout(int log2L, int K) {
  const int groups = 32 >> log2L;  // row pairs per warp
  const int rpw = 2 * groups;      // rows per warp
  K1Smem s;
  s.stage = 0;
  s.bars = s.stage + K1_NSTAGE * K1_CT * (int)sizeof(PGRec);
  s.uvw = s.bars + 2 * K1_NSTAGE * 8;
  s.rec = s.uvw + K1_WARPS * rpw * 6 * 4;
  s.cs = s.rec + K1_WARPS * K1_CT * groups * 48;
  s.acc = s.cs + K1_WARPS * K1_CT * 16;
  s.total = s.acc + K1_THREADS * 2 * K * 8;
  return s;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
  return mbar_wait_bounded(bar, parity, err);
}

// As k1_comp_uniform, for an arbitrary channel list: every channel's phase is reduced and evaluated.
template <int K, bool GAUSS>
__device__ __forceinline__ void k1_comp_list(const float4 c, const float4 Ra, const float4 Rc, const float* ah,
                                             const float* al, const float* lam, const float* wg, float2* Vre,
                                             float2* Vim) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 P0 = phasor_fast(reduce_turns(Ra.x, Ra.y, ah[k], al[k]));
    const float2 P1 = phasor_fast(reduce_turns(Ra.z, Ra.w, ah[k], al[k]));
    const float e = fmaf(c.y, lam[k], c.x);
    float2 A;
    if (GAUSS) {
      A.x = c.w * ex2_approx(fmaf(Rc.z, wg[k], e));
      A.y = c.w * ex2_approx(fmaf(Rc.w, wg[k], e));
    } else {
      A.x = c.w * ex2_approx(e);
      A.y = A.x;
    }
    Vre[k] = __ffma2_rn(make_float2(P0.x, P1.x), A, Vre[k]);
    Vim[k] = __ffma2_rn(make_float2(P0.y, P1.y), A, Vim[k]);
  }
}

// One (row tile, channel block) of one observation over the component tiles t_beg .. t_end-1 (32
// components each, points first): the body of the single-launch kernel below and of the batched
// serving kernel.  With part == nullptr the visibilities are written in the output mode; otherwise the
// raw partial sums go to part (2K x 256 float2, thread fastest) for k1_tail_sum.  Re-entrant: it
// initialises and invalidates its own barriers.
template <int K, bool UNIFORM>
__device__ __forceinline__ void k1_tile(const K1Args& a, const int bx, const int by, int t_beg, int t_end,
                                        float2* part, unsigned char* smem) {
  const K1Smem lay = k1_smem_layout(a.log2L, K);
  PGRec* stage = reinterpret_cast<PGRec*>(smem + lay.stage);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* empty = full + K1_NSTAGE;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = 1 << a.log2L;
  const int gshift = 5 - a.log2L;
  const int groups = 1 << gshift;  // row pairs per warp
  const int rpw = 2 * groups;
  const int g = lane >> a.log2L, sub = lane & (L - 1);
  const int row_w0 = bx * (K1_WARPS * rpw) + warp * rpw;
  const int f0 = by * a.chan_block + sub * K;

  float* uvw_s = reinterpret_cast<float*>(smem + lay.uvw) + warp * rpw * 6;
  float4* rec = reinterpret_cast<float4*>(smem + lay.rec) + warp * K1_CT * groups * 3;
  float4* cs = reinterpret_cast<float4*>(smem + lay.cs) + warp * K1_CT;
  float2* acc = reinterpret_cast<float2*>(smem + lay.acc) + threadIdx.x;  // [2K][K1_THREADS]: re, then im pairs
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i * K1_THREADS] = make_float2(0.f, 0.f);

  const int n_pt_tiles = (a.n_point + K1_CT - 1) / K1_CT;
  t_end = min(t_end, n_pt_tiles + (a.n_gauss + K1_CT - 1) / K1_CT);
  const int n_tiles = max(t_end - t_beg, 0);  // component tiles t_beg .. t_end-1 of this CTA, local index u
  auto tile_start = [&](int u) {
    const int t = t_beg + u;
    return t < n_pt_tiles ? t * K1_CT : a.n_point + (t - n_pt_tiles) * K1_CT;
  };
  auto tile_count = [&](int u) {
    const int t = t_beg + u;
    return t < n_pt_tiles ? min(K1_CT, a.n_point - t * K1_CT) : min(K1_CT, a.n_gauss - (t - n_pt_tiles) * K1_CT);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < K1_NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], K1_WARPS);
    }
    fence_mbar_init();
  }
  // rows of this warp: (u, v, w) split into float pairs
  for (int i = lane; i < rpw * 3; i += 32) {
    const int r = row_w0 + i / 3;
    float h, l;
    split_double(r < a.n_rows ? a.uvw[(size_t)r * 3 + i % 3] : 0.0, h, l);
    uvw_s[2 * i] = h;
    uvw_s[2 * i + 1] = l;
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
  // nu / c of the start channel: the lane's first (channel lists) or middle (uniform, k1_mid) channel
  float a0h, a0l;
  split_double(a.freq[min(f0, a.n_chan - 1)] * (1.0 / kC) +
                   (UNIFORM ? k1_mid(K) * ((double)a.dnu_h + (double)a.dnu_l) : 0.0),
               a0h, a0l);
  const double L0 = log2(a.nu0);

  float2 Vre[K], Vim[K];
#pragma unroll
  for (int k = 0; k < K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);

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
    const bool gauss = t_beg + t >= n_pt_tiles;
    const PGRec* st = stage + s * K1_CT;

    // --- records per (component, row pair), shared by the L lanes of the pair
    for (int idx = lane; idx < (cnt << gshift); idx += 32) {
      const int j = idx >> gshift, gg = idx & (groups - 1);
      const PGRec& c = st[j];
      const float* x0 = uvw_s + 12 * gg;
      const float* x1 = x0 + 6;
      float th0, tl0, th1, tl1;
      tau_df(x0, c, th0, tl0);
      tau_df(x1, c, th1, tl1);
      float4 Rb = make_float4(0.f, 0.f, 0.f, 0.f), Rc = Rb;
      if (UNIFORM) {
        const float2 D0 = phasor_accurate(reduce_turns(th0, tl0, a.dnu_h, a.dnu_l));
        const float2 D1 = phasor_accurate(reduce_turns(th1, tl1, a.dnu_h, a.dnu_l));
        Rb = make_float4(D0.x, D1.x, D0.y, D1.y);
        Rc.x = -D0.y;
        Rc.y = -D1.y;
      }
      if (gauss) {
        const float u0 = x0[0], v0 = x0[2], u1 = x1[0], v1 = x1[2];
        Rc.z = -(c.ga * u0 * u0 + c.gb * u0 * v0 + c.gc * v0 * v0);
        Rc.w = -(c.ga * u1 * u1 + c.gb * u1 * v1 + c.gc * v1 * v1);
      }
      float4* R = rec + 3 * (j * groups + gg);
      R[0] = make_float4(th0, tl0, th1, tl1);
      R[1] = Rb;
      R[2] = Rc;
    }
    // per component: log2 of |flux| at the log-frequency reference (-inf for a zero or rejected
    // component, whose amplitude is then exactly 0), alpha, the sign as a half turn, and the sign
    for (int j = lane; j < cnt; j += 32) {
      const float sg = st[j].sgn;
      cs[j] = make_float4(sg == 0.f ? __int_as_float(0xff800000) : st[j].lS + st[j].alpha * (float)(L0 - st[j].lref), st[j].alpha,
                          sg < 0.f ? 3.14159265358979f : 0.f, sg);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);

    // --- channel loop: K channels of two rows per lane
    const float4* Rg = rec + 3 * g;
    if (UNIFORM) {
      if (gauss) {
        for (int j = 0; j < cnt; ++j)
          k1_comp_uniform<K, true>(cs[j], Rg[3 * groups * j], Rg[3 * groups * j + 1], Rg[3 * groups * j + 2], a0h, a0l,
                                   lam, wg, Vre, Vim);
      } else {
        for (int j = 0; j < cnt; ++j)
          k1_comp_uniform<K, false>(cs[j], Rg[3 * groups * j], Rg[3 * groups * j + 1], Rg[3 * groups * j + 2], a0h,
                                    a0l, lam, wg, Vre, Vim);
      }
    } else {
      if (gauss) {
        for (int j = 0; j < cnt; ++j)
          k1_comp_list<K, true>(cs[j], Rg[3 * groups * j], Rg[3 * groups * j + 2], ah, al, lam, wg, Vre, Vim);
      } else {
        for (int j = 0; j < cnt; ++j)
          k1_comp_list<K, false>(cs[j], Rg[3 * groups * j], Rg[3 * groups * j + 2], ah, al, lam, wg, Vre, Vim);
      }
    }
    __syncwarp();
    if ((t + 1) % K1_FLUSH == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[k * K1_THREADS] = __fadd2_rn(acc[k * K1_THREADS], Vre[k]);
        acc[(K + k) * K1_THREADS] = __fadd2_rn(acc[(K + k) * K1_THREADS], Vim[k]);
        Vre[k] = Vim[k] = make_float2(0.f, 0.f);
      }
    }
  }

  // --- epilogue: each visibility written once (or, for a component-range part of a split tile, the
  // raw partial sums in thread order for k1_tail_sum)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    Vre[k] = __fadd2_rn(acc[k * K1_THREADS], Vre[k]);
    Vim[k] = __fadd2_rn(acc[(K + k) * K1_THREADS], Vim[k]);
    if (UNIFORM && k1_neg(K, k)) {  // the uniform loop's signed sums (k1_comp_uniform)
      Vre[k] = make_float2(-Vre[k].x, -Vre[k].y);
      Vim[k] = make_float2(-Vim[k].x, -Vim[k].y);
    }
  }
  if (part) {
    const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      part[(2 * k) * K1_THREADS + threadIdx.x] = ok ? Vre[k] : nan2;
      part[(2 * k + 1) * K1_THREADS + threadIdx.x] = ok ? Vim[k] : nan2;
    }
  } else {
    k1_store<K>(a, row_w0 + 2 * g, f0, Vre, Vim, ok);
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

// Single launch over a 1-D grid.  CTAs 0 .. n_main-1 are whole tiles in (row tile fastest, channel
// block) order.  When the tile count leaves the last wave of resident CTAs mostly empty, each of the
// remaining tiles is split into tail_parts CTAs over consecutive ranges of tail_ct component tiles,
// so the tail fills that wave; k1_tail_sum then adds their partial sums in part order and writes them.
template <int K, bool UNIFORM>
__global__ void __launch_bounds__(K1_THREADS, 2) k1_phasor(const K1Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  int lin = blockIdx.x, t_beg = 0, t_end = INT_MAX;
  float2* part = nullptr;
  if (lin >= a.n_main) {
    const int j = lin - a.n_main, p = j % a.tail_parts;
    lin = a.n_main + j / a.tail_parts;
    t_beg = p * a.tail_ct;
    t_end = t_beg + a.tail_ct;
    part = a.part + (size_t)j * (2 * K * K1_THREADS);
  }
  k1_tile<K, UNIFORM>(a, lin % a.grid_x, lin / a.grid_x, t_beg, t_end, part, smem);
}

// The split tail tiles: CTA i sums the tail_parts partial sums of tile n_main + i in part order (a
// fixed order, so the result does not depend on scheduling) and writes them in the output mode.  Each
// thread owns the same (rows, channels) as the k1_tile thread of the same index.
template <int K>
__global__ void __launch_bounds__(K1_THREADS) k1_tail_sum(const K1Args a) {
  const int lin = a.n_main + blockIdx.x;
  const int bx = lin % a.grid_x, by = lin / a.grid_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rpw = 2 << (5 - a.log2L);
  const int g = lane >> a.log2L, sub = lane & ((1 << a.log2L) - 1);
  float2 Vre[K], Vim[K];
#pragma unroll
  for (int k = 0; k < K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);
  const float2* src = a.part + (size_t)blockIdx.x * a.tail_parts * (2 * K * K1_THREADS) + threadIdx.x;
  for (int p = 0; p < a.tail_parts; ++p, src += 2 * K * K1_THREADS) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      Vre[k] = __fadd2_rn(Vre[k], src[(2 * k) * K1_THREADS]);
      Vim[k] = __fadd2_rn(Vim[k], src[(2 * k + 1) * K1_THREADS]);
    }
  }
  k1_store<K>(a, bx * (K1_WARPS * rpw) + warp * rpw + 2 * g, by * a.chan_block + sub * K, Vre, Vim, true);
}

struct K1Choice {
  int log2L, K;
};

// Estimated cost of a (lanes per row pair L = 2^log2L, channels per lane K) configuration, in units
// of one component-visibility evaluation: every padded channel slot costs one evaluation plus the
// lane's per-(component, row) start phasor spread over its K channels (about 1.5 evaluations), and
// every (component, row, channel block) one record (about 12).  `waves` > 0 rounds the CTA count up
// to whole waves of that many resident CTAs; configurations that fit only one CTA per SM pay 30%.
static double k1_cost(long rows, int F, int log2L, int K, int waves) {
  const long cb = (long)K << log2L, nblk = (F + cb - 1) / cb;
  const long rpc = (long)K1_WARPS * 2 * (32 >> log2L);
  const long ctas = ((rows + rpc - 1) / rpc) * nblk;
  const double per_cta = (double)rpc * ((double)cb * (1.0 + 1.5 / K) + 12.0);
  const bool two = k1_smem_layout(log2L, K).total <= 113 * 1024;
  double c = per_cta * (waves > 0 ? (double)((ctas + (two ? 2 : 1) * waves - 1) / ((two ? 2 : 1) * waves)) *
                                        (two ? 2 : 1) * waves
                                  : (double)ctas);
  return two ? c : 1.3 * c;
}

// Pick L in {8, 16, 32} and K in {4, 8, 12, 16} by the cost above (ties: the wider block).  The single
// launch splits a partial last wave over component ranges (k1_phasor), so whole waves are not counted
// (waves = 0) unless the model has a single component tile, which cannot be split.
static K1Choice k1_choose(long rows, int F, int num_sms, bool splittable) {
  K1Choice best{5, 12};
  double best_c = -1.0;
  const int Ks[4] = {12, 16, 8, 4};
  for (int li = 5; li >= 3; --li)
    for (int K : Ks) {
      const double c = k1_cost(rows, F, li, K, splittable ? 0 : num_sms);
      if (best_c < 0 || c < best_c * 0.999) {
        best_c = c;
        best = {li, K};
      }
    }
  return best;
}

template <int K, bool U>
static cudaError_t k1_launch(const K1Args& a, int n_tail, int smem, cudaStream_t st) {
  auto fn = k1_phasor<K, U>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(fn));
  if (e != cudaSuccess) return e;
  fn<<<a.n_main + n_tail * a.tail_parts, K1_THREADS, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || n_tail == 0) return e;
  k1_tail_sum<K><<<n_tail, K1_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

// Partial sums of the split tail tiles: room for 4 * num_sms parts of the per-warp form at K = 16 (it uses
// at most 2 * num_sms, one per resident CTA), which the single-launch form's split also draws on.
size_t k1_part_bytes(int num_sms) { return (size_t)4 * num_sms * 2 * 16 * K1_THREADS * sizeof(float2); }

int launch_phasor_mixed(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        cudaStream_t st) {
  const int n_ct_all = (M->n_point + K1_CT - 1) / K1_CT + (M->n_gauss + K1_CT - 1) / K1_CT;
  K1Choice ch = k1_choose(o.n_rows, o.n_chan, ctx->num_sms, n_ct_all >= 2);
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
  a.grid_x = (o.n_rows + rows_per_cta - 1) / rows_per_cta;
  const long n_cta = (long)a.grid_x * ((o.n_chan + a.chan_block - 1) / a.chan_block);
  if (n_cta > INT_MAX / 2) return set_error(WN_EINVAL, "observation too large for one phasor launch");
  const int smem = k1_smem_layout(ch.log2L, ch.K).total;
  // Tail split: the last n_cta mod slots tiles (slots = resident CTAs) would run as a mostly empty
  // wave; split each into parts over component ranges so that they fill it.
  const int slots = ctx->num_sms * (smem <= 113 * 1024 ? 2 : 1);
  const int n_ct = (M->n_point + K1_CT - 1) / K1_CT + (M->n_gauss + K1_CT - 1) / K1_CT;
  const int rem = (int)(n_cta % slots);
  a.n_main = (int)n_cta;
  a.tail_parts = 1;
  a.tail_ct = n_ct;
  a.part = ctx->k1_part;
  int n_tail = 0;
  if (rem > 0 && n_ct >= 2 && ctx->k1_part) {
    int parts = std::min(slots / rem, n_ct);
    if (parts >= 2) {
      a.tail_ct = (n_ct + parts - 1) / parts;
      a.tail_parts = (n_ct + a.tail_ct - 1) / a.tail_ct;  // no empty part
      a.n_main = (int)n_cta - rem;
      n_tail = rem;
    }
  }
  cudaError_t e;
  switch (ch.K * 2 + (o.uniform ? 1 : 0)) {
    case 4 * 2 + 1: e = k1_launch<4, true>(a, n_tail, smem, st); break;
    case 4 * 2: e = k1_launch<4, false>(a, n_tail, smem, st); break;
    case 8 * 2 + 1: e = k1_launch<8, true>(a, n_tail, smem, st); break;
    case 8 * 2: e = k1_launch<8, false>(a, n_tail, smem, st); break;
    case 12 * 2 + 1: e = k1_launch<12, true>(a, n_tail, smem, st); break;
    case 12 * 2: e = k1_launch<12, false>(a, n_tail, smem, st); break;
    case 16 * 2 + 1: e = k1_launch<16, true>(a, n_tail, smem, st); break;
    default: e = k1_launch<16, false>(a, n_tail, smem, st); break;
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
  // raw storage: K1Args has default member initialisers, which a __shared__ variable cannot run
  __shared__ __align__(16) unsigned char args_raw[sizeof(K1Args)];
  K1Args& args = *reinterpret_cast<K1Args*>(args_raw);
  const int n = *n_work;
  for (int e = blockIdx.x; e < n; e += gridDim.x) {
    const K1Work w = work[e];
    if (threadIdx.x == 0) args = reqs[w.req];
    __syncthreads();
    if (args.chan_block == (12 << args.log2L)) k1_tile<12, true>(args, w.bx, w.by, 0, INT_MAX, nullptr, smem);
    else k1_tile<8, true>(args, w.bx, w.by, 0, INT_MAX, nullptr, smem);
    // k1_tile ends with a barrier, so every thread is done with args before the next entry's write
  }
}

int k1_batched_smem() { return k1_smem_layout(K1B_MIN_LOG2L, K1B_KMAX).total; }

// Arguments and tile grid of one observation for the batched kernel (uniform channels only).
int k1_batched_args(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                    K1Args* args, int* grid_x, int* grid_y) {
  if (!o.uniform) return set_error(WN_EINVAL, "batched prediction needs uniformly spaced channels");
  // the cheapest of K in {12, 8} and L in {8, 16, 32} by the single-launch cost model, without waves
  // (the batched kernel is persistent)
  int log2L = 5, K = 12;
  double best = -1.0;
  for (int li = 5; li >= K1B_MIN_LOG2L; --li)
    for (int kk : {12, 8}) {
      const double c = k1_cost(o.n_rows, o.n_chan, li, kk, 0);
      if (best < 0 || c < best * 0.999) {
        best = c;
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
  return allow_max_dynamic_smem(reinterpret_cast<const void*>(k1_batched));
}

cudaError_t k1_batched_launch(const K1Args* reqs, const K1Work* work, const int* n_work, int grid, cudaStream_t st) {
  k1_batched<<<grid, K1_THREADS, k1_batched_smem(), st>>>(reqs, work, n_work);
  return cudaGetLastError();
}

}  // namespace wn
