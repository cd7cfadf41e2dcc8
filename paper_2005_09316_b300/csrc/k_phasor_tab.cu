// K1, single-launch form: the point/Gaussian phasor sum with the spectrum taken from a table.
//
//   V(t,b,f) = sum_j S_j(nu_f) xi_j exp(-2 pi i tau_j(t,b) nu_f / c)     (eq:env_visi_def)
//
// The spectrum S_j(nu_f) = S_ref,j (nu_f / nu_ref,j)^alpha_j (Sec. 4.1) does not depend on the row, so it
// is formed once per launch for every (component, channel) into a table in device memory (38 MB for
// 25,000 components x 384 channels, read from L2), instead of once per (component, channel) in every
// warp that needs it.  A CTA streams the table's slice of each group of 32 components into shared
// memory beside the group's component records, with two TMA bulk copies into one stage of a 2-stage
// mbarrier ring, and all 16 warps of the CTA read it there.
//  * Points: the table holds |S_j(nu_f)| (the exp2 of the old per-warp exponent, bit for bit), so the
//    channel loop spends no FMA and no MUFU on the amplitude.  The sign of S_ref enters as a half turn
//    added to the start phase.
//  * Gaussians: the table holds log2 S_j(nu_f); the lane adds the envelope exponent -q (nu/c)^2 E log2 e
//    of its row and takes one exp2 per row and channel.
//  * One CTA per SM of 16 warps (512 threads), 32 rows x 384 channels for the MWA-like workload: the
//    ring (2 x 50 KB), the per-warp records (24 KB) and the second-level sums (96 KB) fill 221 KB.
//  * Per (component, row pair) a 48-byte record: both rows' tau pairs (laid out for the packed start
//    reduction), the one-channel step D, the Gaussian forms and the sign's half turn.
//  * The start phase of both rows is reduced in f32x2 (one packed instruction per step for two rows),
//    and the rest of the channel loop is the three-term recurrence of k1_loop.cuh.
// The rest (double-float phase argument, recurrence from the middle channel, output modes, split tail,
// second-level sums every 128 components, fixed summation order) is as in k_phasor.cu.
#include "wn_internal.cuh"
#include "k1_loop.cuh"

#include <algorithm>
#include <climits>
#include <cmath>

namespace wn {

constexpr int KS_WARPS = 16;
constexpr int KS_THREADS = 32 * KS_WARPS;
constexpr int KS_GC = 32;      // components per ring stage (one group)
constexpr int KS_NSTAGE = 2;   // stages in the ring
constexpr int KS_FLUSH = 4;    // groups (128 components) per register partial sum

// Arguments: the observation, model and output as for the per-warp form, plus the spectrum table
// [n_cb][n_grp][KS_GC][chan_block] (channel blocks, groups of 32 components: points then Gaussians).
struct KSArgs {
  K1Args k;
  const float* spec;
  int n_grp_pt, n_grp;
};

struct KSSmem {
  int stage, stage_bytes, bars, uvw, rec, acc, total;
};

// Stage s: the group's PGRec records (32 x 64 B) then its spectrum slice (32 x chan_block floats).
// Per warp: its rows' (u, v, w) as float pairs and the 48-byte records of (component, row pair).
__host__ __device__ inline KSSmem ks_smem_layout(int log2L, int K) {
  const int groups = 32 >> log2L, rpw = 2 * groups, cb = K << log2L;
  KSSmem s;
  s.stage = 0;
  s.stage_bytes = KS_GC * (int)sizeof(PGRec) + KS_GC * cb * 4;
  s.bars = s.stage + KS_NSTAGE * s.stage_bytes;
  s.uvw = s.bars + 2 * KS_NSTAGE * 8;
  s.rec = s.uvw + KS_WARPS * rpw * 6 * 4;
  s.acc = s.rec + KS_WARPS * KS_GC * groups * 48;
  s.total = s.acc + KS_THREADS * 2 * K * 8;
  return s;
}

// As ks_comp_uniform for an arbitrary channel list: every channel's phase is reduced and evaluated.
template <int K, bool GAUSS>
__device__ __forceinline__ void ks_comp_list(const float4 R0, const float4 R2, const float* tab, const float* ah,
                                             const float* al, const float* wg, float2* Vre, float2* Vim) {
  const float2 th = make_float2(R0.x, R0.y), tl = make_float2(R0.z, R0.w), nq = make_float2(R2.x, R2.y);
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(tab)[q];
    const float tv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * q + i;
      float2 re, im;
      phasor_pair(reduce_turns_pair(th, tl, ah[k], al[k]), R2.z, re, im);
      const float2 A = ks_amp<GAUSS>(tv[i], nq, GAUSS ? wg[k] : 0.f);
      Vre[k] = __ffma2_rn(re, A, Vre[k]);
      Vim[k] = __ffma2_rn(im, A, Vim[k]);
    }
  }
}

// The spectrum table: entry (channel block cb, group gi, member jj, channel fl) of a point holds
// |S_j(nu_f)| = 2^(log2|S_ref| + alpha log2(nu_f / nu_ref)), of a Gaussian the exponent itself; both
// formed with exactly the FP32 operations of the per-warp kernel (log2 of nu / nu0 in FP32, one FMA,
// one exp2).  Entries past the last component of a group or past the last channel are 0 (points) or
// -inf (Gaussians): they add nothing.
__global__ void ks_spectrum(const PGRec* comps, int n_point, int n_gauss, int n_grp_pt, int n_grp, const double* freq,
                            int n_chan, double nu0, int cb, long long n_entries, float* spec) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_entries) return;
  const int fl = (int)(idx % cb);
  long long rest = idx / cb;
  const int jj = (int)(rest % KS_GC);
  rest /= KS_GC;
  const int gi = (int)(rest % n_grp);
  const int blk = (int)(rest / n_grp);
  const int f = blk * cb + fl;
  const bool gauss = gi >= n_grp_pt;
  const int j = gauss ? n_point + (gi - n_grp_pt) * KS_GC + jj : gi * KS_GC + jj;
  const bool valid = gauss ? (gi - n_grp_pt) * KS_GC + jj < n_gauss : j < n_point;
  if (!valid || f >= n_chan) {
    spec[idx] = gauss ? __int_as_float(0xff800000) : 0.f;
    return;
  }
  const PGRec& c = comps[j];
  const float lam = log2f((float)freq[f] * (float)(1.0 / nu0));
  const float e0 = c.sgn == 0.f ? __int_as_float(0xff800000) : c.lS + c.alpha * (float)(log2(nu0) - c.lref);
  const float e = fmaf(c.alpha, lam, e0);
  spec[idx] = gauss ? e : ex2_approx(e);
}

// One output element in the output mode: store, accumulate, the peel residual D - G V, or subtract
// G V from the output; data and output are streamed past L2 (evict first) so that the spectrum table
// stays resident.
__device__ __forceinline__ float2 ks_out_value(const K1Args& a, int row, int f, float2 v, const float2* out) {
  if (a.mode == OUT_STORE) return v;
  if (a.mode == OUT_ACCUM) {
    const float2 o = __ldcs(out);
    return make_float2(o.x + v.x, o.y + v.y);
  }
  float2 G;
  if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
  const float2 d = a.mode == OUT_SUBG ? __ldcs(out) : __ldcs(a.peel.data + (out - a.out));
  return make_float2(d.x - (G.x * v.x - G.y * v.y), d.y - (G.x * v.y + G.y * v.x));
}

// A warp writes its rpw rows (row0 ..) of one channel block (channels fbase .. fbase + cb - 1) from
// the staged values stg[row][channel]: consecutive lanes take consecutive channel pairs as 16-byte
// vectors, or single channels when a pair could start on an 8-byte boundary (an odd n_chan, or an
// output array that is 8- but not 16-byte aligned).
__device__ __forceinline__ void ks_store_rows(const K1Args& a, int row0, int rpw, int fbase, int cb, const float2* stg,
                                              int lane) {
  const int nf = min(cb, a.n_chan - fbase);
  for (int rr = 0; rr < rpw; ++rr) {
    const int row = row0 + rr;
    if (row >= a.n_rows) break;
    const float2* src = stg + rr * cb;
    float2* dst = a.out + (size_t)row * a.n_chan + fbase;
    if ((a.n_chan & 1) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0) {  // nf is even
      for (int i = lane; 2 * i < nf; i += 32) {
        const float2 v0 = ks_out_value(a, row, fbase + 2 * i, src[2 * i], dst + 2 * i);
        const float2 v1 = ks_out_value(a, row, fbase + 2 * i + 1, src[2 * i + 1], dst + 2 * i + 1);
        __stcs(reinterpret_cast<float4*>(dst + 2 * i), make_float4(v0.x, v0.y, v1.x, v1.y));
      }
    } else {
      for (int i = lane; i < nf; i += 32) __stcs(dst + i, ks_out_value(a, row, fbase + i, src[i], dst + i));
    }
  }
}

// One (row tile, channel block) over component groups g_beg .. g_end-1.  With part == nullptr the
// visibilities are written in the output mode; otherwise the raw partial sums go to part (2K x 512
// float2, thread fastest) for ks_tail_sum.
template <int K, bool UNIFORM>
__device__ __forceinline__ void ks_tile(const KSArgs& A, const int bx, const int by, int g_beg, int g_end, float2* part,
                                        unsigned char* smem) {
  const K1Args& a = A.k;
  const KSSmem lay = ks_smem_layout(a.log2L, K);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* empty = full + KS_NSTAGE;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = 1 << a.log2L;
  const int gshift = 5 - a.log2L;
  const int groups = 1 << gshift;  // row pairs per warp
  const int rpw = 2 * groups;
  const int g = lane >> a.log2L, sub = lane & (L - 1);
  const int cb = a.chan_block;
  const int row_w0 = bx * (KS_WARPS * rpw) + warp * rpw;
  const int f0 = by * cb + sub * K;

  float* uvw_s = reinterpret_cast<float*>(smem + lay.uvw) + warp * rpw * 6;
  float4* rec = reinterpret_cast<float4*>(smem + lay.rec) + warp * KS_GC * groups * 3;
  float2* acc = reinterpret_cast<float2*>(smem + lay.acc) + threadIdx.x;  // [2K][KS_THREADS]
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i * KS_THREADS] = make_float2(0.f, 0.f);

  g_end = min(g_end, A.n_grp);
  const int n_g = max(g_end - g_beg, 0);
  auto grp_first = [&](int u) {
    const int gi = g_beg + u;
    return gi < A.n_grp_pt ? gi * KS_GC : a.n_point + (gi - A.n_grp_pt) * KS_GC;
  };
  auto grp_count = [&](int u) {
    const int gi = g_beg + u;
    return gi < A.n_grp_pt ? min(KS_GC, a.n_point - gi * KS_GC) : min(KS_GC, a.n_gauss - (gi - A.n_grp_pt) * KS_GC);
  };
  const uint32_t spec_bytes = (uint32_t)(KS_GC * cb * 4);
  auto issue = [&](int u, int s) {  // thread 0: the group's records and spectrum slice into stage s
    unsigned char* st = smem + lay.stage + s * lay.stage_bytes;
    const uint32_t rb = (uint32_t)grp_count(u) * (uint32_t)sizeof(PGRec);
    mbar_arrive_expect_tx(&full[s], rb + spec_bytes);
    tma_bulk_g2s(st, a.comps + grp_first(u), rb, &full[s]);
    tma_bulk_g2s(st + KS_GC * sizeof(PGRec), A.spec + ((size_t)by * A.n_grp + (size_t)(g_beg + u)) * KS_GC * cb,
                 spec_bytes, &full[s]);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < KS_NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], KS_WARPS);
    }
    fence_mbar_init();
  }
  for (int i = lane; i < rpw * 3; i += 32) {
    const int r = row_w0 + i / 3;
    float h, l;
    split_double(r < a.n_rows ? a.uvw[(size_t)r * 3 + i % 3] : 0.0, h, l);
    uvw_s[2 * i] = h;
    uvw_s[2 * i + 1] = l;
  }
  __syncthreads();
  int issued = 0;  // groups whose copies thread 0 has issued
  if (threadIdx.x == 0)
    for (; issued < min(KS_NSTAGE, n_g); ++issued) issue(issued, issued);

  // per-lane channel constants: the Gaussian envelope's (nu/c)^2 E log2(e); nu / c as float pairs for
  // channel lists
  float wg[K];
  float ah[UNIFORM ? 1 : K], al[UNIFORM ? 1 : K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int f = min(f0 + k, a.n_chan - 1);
    const double nu = a.freq[f];
    const float x = (float)(nu * (1.0 / kC));
    wg[k] = (float)(kGaussE * kLog2e) * x * x;
    if (!UNIFORM) split_double(nu * (1.0 / kC), ah[k], al[k]);
  }
  float a0h, a0l;
  split_double(a.freq[min(f0, a.n_chan - 1)] * (1.0 / kC) +
                   (UNIFORM ? k1_mid(K) * ((double)a.dnu_h + (double)a.dnu_l) : 0.0),
               a0h, a0l);

  float2 Vre[K], Vim[K];
#pragma unroll
  for (int k = 0; k < K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);

  bool ok = true;
  int done = 0;  // groups this thread has waited for
  for (int u = 0; u < n_g && ok; ++u) {
    const int s = u % KS_NSTAGE;
    if (threadIdx.x == 0 && u > 0 && issued < n_g) {
      // refill the stage of group u-1 once every warp has left it
      const int sp = (u - 1) % KS_NSTAGE;
      if (!mbar_wait_bounded(&empty[sp], ((u - 1) / KS_NSTAGE) & 1, a.err)) {
        ok = false;
        break;
      }
      issue(issued, sp);
      ++issued;
    }
    if (!mbar_wait_bounded(&full[s], (u / KS_NSTAGE) & 1, a.err)) {
      ok = false;
      break;
    }
    done = u + 1;
    const int cnt = grp_count(u);
    const bool gauss = g_beg + u >= A.n_grp_pt;
    const PGRec* st = reinterpret_cast<const PGRec*>(smem + lay.stage + s * lay.stage_bytes);
    const float* spec = reinterpret_cast<const float*>(st + KS_GC);

    // --- records per (component, row pair), shared by the L lanes of the pair
    for (int idx = lane; idx < (cnt << gshift); idx += 32) {
      const int j = idx >> gshift, gg = idx & (groups - 1);
      const PGRec& c = st[j];
      const float* x0 = uvw_s + 12 * gg;
      const float* x1 = x0 + 6;
      float th0, tl0, th1, tl1;
      tau_df(x0, c, th0, tl0);
      tau_df(x1, c, th1, tl1);
      float4 R1 = make_float4(0.f, 0.f, 0.f, 0.f), R2 = R1;
      if (UNIFORM) {
        const float2 D0 = phasor_accurate(reduce_turns(th0, tl0, a.dnu_h, a.dnu_l));
        const float2 D1 = phasor_accurate(reduce_turns(th1, tl1, a.dnu_h, a.dnu_l));
        R1 = make_float4(D0.x, D1.x, D0.y, D1.y);
      }
      if (gauss) {
        const float u0 = x0[0], v0 = x0[2], u1 = x1[0], v1 = x1[2];
        R2.x = -(c.ga * u0 * u0 + c.gb * u0 * v0 + c.gc * v0 * v0);
        R2.y = -(c.ga * u1 * u1 + c.gb * u1 * v1 + c.gc * v1 * v1);
      }
      R2.z = c.sgn < 0.f ? 3.14159265358979f : 0.f;
      float4* R = rec + 3 * (j * groups + gg);
      R[0] = make_float4(th0, th1, tl0, tl1);
      R[1] = R1;
      R[2] = R2;
    }
    __syncwarp();

    // --- channel loop: K channels of two rows per lane
    const float4* Rg = rec + 3 * g;
    const float* tb = spec + sub * K;
    if (UNIFORM) {
      // four components per loop trip: the compiler interleaves one component's start (reduction, MUFU
      // sin/cos) with another's recurrence (measured 1.2 % faster than one per trip)
      if (gauss) {
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
          const float4* R = Rg + 3 * groups * j;
          ks_comp_uniform<K, true>(R[0], R[1], R[2], tb + j * cb, a0h, a0l, wg, Vre, Vim);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
          const float4* R = Rg + 3 * groups * j;
          ks_comp_uniform<K, false>(R[0], R[1], R[2], tb + j * cb, a0h, a0l, wg, Vre, Vim);
        }
      }
    } else {
      if (gauss) {
        for (int j = 0; j < cnt; ++j) {
          const float4* R = Rg + 3 * groups * j;
          ks_comp_list<K, true>(R[0], R[2], tb + j * cb, ah, al, wg, Vre, Vim);
        }
      } else {
        for (int j = 0; j < cnt; ++j) {
          const float4* R = Rg + 3 * groups * j;
          ks_comp_list<K, false>(R[0], R[2], tb + j * cb, ah, al, wg, Vre, Vim);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if ((u + 1) % KS_FLUSH == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[k * KS_THREADS] = __fadd2_rn(acc[k * KS_THREADS], Vre[k]);
        acc[(K + k) * KS_THREADS] = __fadd2_rn(acc[(K + k) * KS_THREADS], Vim[k]);
        Vre[k] = Vim[k] = make_float2(0.f, 0.f);
      }
    }
  }

  // --- epilogue: each visibility written once (or the raw partial sums of a component-range part)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    Vre[k] = __fadd2_rn(acc[k * KS_THREADS], Vre[k]);
    Vim[k] = __fadd2_rn(acc[(K + k) * KS_THREADS], Vim[k]);
    if (UNIFORM && k1_neg(K, k)) {  // the recurrence's signed sums
      Vre[k] = make_float2(-Vre[k].x, -Vre[k].y);
      Vim[k] = make_float2(-Vim[k].x, -Vim[k].y);
    }
  }
  if (part) {
    const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      part[(2 * k) * KS_THREADS + threadIdx.x] = ok ? Vre[k] : nan2;
      part[(2 * k + 1) * KS_THREADS + threadIdx.x] = ok ? Vim[k] : nan2;
    }
  } else {
    // stage the warp's rows in the freed second-level-sum area as [row][channel], then write them with
    // warp-coalesced 16-byte accesses
    __syncthreads();  // every thread has read its second-level sums
    float2* stg = reinterpret_cast<float2*>(smem + lay.acc) + (size_t)warp * rpw * cb;
    const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      stg[(2 * g) * cb + sub * K + k] = ok ? make_float2(Vre[k].x, Vim[k].x) : nan2;
      stg[(2 * g + 1) * cb + sub * K + k] = ok ? make_float2(Vre[k].y, Vim[k].y) : nan2;
    }
    __syncwarp();
    ks_store_rows(a, row_w0, rpw, by * cb, cb, stg, lane);
  }
  __syncthreads();  // every warp is past its last barrier wait and shared-memory read
  if (threadIdx.x == 0) {
    // after an expired wait: let the copies still in flight land (bounded) before the CTA exits
    for (int u = done; u < issued; ++u) (void)mbar_wait_bounded(&full[u % KS_NSTAGE], (u / KS_NSTAGE) & 1, nullptr, 1ll << 24);
    for (int s = 0; s < KS_NSTAGE; ++s) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
  }
  __syncthreads();
}

// Single launch over a 1-D grid: CTAs 0 .. n_main-1 are whole tiles (row tile fastest); each tile after
// them is split into tail_parts CTAs over consecutive ranges of tail_ct groups, summed by ks_tail_sum.
template <int K, bool UNIFORM>
__global__ void __launch_bounds__(KS_THREADS, 1) ks_phasor(const KSArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  const K1Args& a = A.k;
  int lin = blockIdx.x, g_beg = 0, g_end = INT_MAX;
  float2* part = nullptr;
  if (lin >= a.n_main) {
    const int j = lin - a.n_main, p = j % a.tail_parts;
    lin = a.n_main + j / a.tail_parts;
    g_beg = p * a.tail_ct;
    g_end = g_beg + a.tail_ct;
    part = a.part + (size_t)j * (2 * K * KS_THREADS);
  }
  ks_tile<K, UNIFORM>(A, lin % a.grid_x, lin / a.grid_x, g_beg, g_end, part, smem);
}

// The split tail tiles: CTA i adds the tail_parts partial sums of tile n_main + i in part order and
// writes them in the output mode; each thread owns the (rows, channels) of the ks_tile thread of the
// same index.
template <int K>
__global__ void __launch_bounds__(KS_THREADS) ks_tail_sum(const K1Args a) {
  const int lin = a.n_main + blockIdx.x;
  const int bx = lin % a.grid_x, by = lin / a.grid_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rpw = 2 << (5 - a.log2L);
  const int g = lane >> a.log2L, sub = lane & ((1 << a.log2L) - 1);
  float2 Vre[K], Vim[K];
#pragma unroll
  for (int k = 0; k < K; ++k) Vre[k] = Vim[k] = make_float2(0.f, 0.f);
  const float2* src = a.part + (size_t)blockIdx.x * a.tail_parts * (2 * K * KS_THREADS) + threadIdx.x;
  for (int p = 0; p < a.tail_parts; ++p, src += 2 * K * KS_THREADS) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      Vre[k] = __fadd2_rn(Vre[k], src[(2 * k) * KS_THREADS]);
      Vim[k] = __fadd2_rn(Vim[k], src[(2 * k + 1) * KS_THREADS]);
    }
  }
  k1_store<K>(a, bx * (KS_WARPS * rpw) + warp * rpw + 2 * g, by * a.chan_block + sub * K, Vre, Vim, true);
}

template <int K, bool U>
static cudaError_t ks_launch(const KSArgs& A, int n_tail, int smem, cudaStream_t st) {
  auto fn = ks_phasor<K, U>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(fn));
  if (e != cudaSuccess) return e;
  fn<<<A.k.n_main + n_tail * A.k.tail_parts, KS_THREADS, smem, st>>>(A);
  e = cudaGetLastError();
  if (e != cudaSuccess || n_tail == 0) return e;
  ks_tail_sum<K><<<n_tail, KS_THREADS, 0, st>>>(A.k);
  return cudaGetLastError();
}

// Estimated cost of (L = 2^log2L lanes per row pair, K channels per lane), in component-visibility
// evaluations: every padded channel slot, the per-(component, row) start spread over K channels (about
// 1.3 evaluations), and one record per (component, row pair, channel block) (about 12 per row).
static double ks_cost(long rows, int F, int log2L, int K) {
  const long cb = (long)K << log2L, nblk = (F + cb - 1) / cb;
  const long rpc = (long)KS_WARPS * 2 * (32 >> log2L);
  const long ctas = ((rows + rpc - 1) / rpc) * nblk;
  return (double)ctas * (double)rpc * ((double)cb * (1.0 + 1.3 / K) + 12.0);
}

// Launch shape (L = 2^log2L lanes per row pair, K channels per lane) of the cheapest estimated cost.
static void ks_choose(const ObsDev& o, int& log2L, int& K) {
  log2L = 5;
  K = 12;
  double best = -1.0;
  for (int li = 5; li >= 3; --li)
    for (int kk : {12, 8, 4}) {
      const double c = ks_cost(o.n_rows, o.n_chan, li, kk);
      if (best < 0 || c < best * 0.999) {
        best = c;
        log2L = li;
        K = kk;
      }
    }
}

size_t phasor_table_spec_bytes(const ObsDev& o, const Model* M) {
  int log2L, K;
  ks_choose(o, log2L, K);
  const int cb = K << log2L, n_cb = (o.n_chan + cb - 1) / cb;
  const long long n_grp = (M->n_point + KS_GC - 1) / KS_GC + (M->n_gauss + KS_GC - 1) / KS_GC;
  return (size_t)n_cb * n_grp * KS_GC * cb * sizeof(float);
}

int launch_phasor_table(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        cudaStream_t st) {
  if (M->n_point + M->n_gauss == 0) return launch_phasor_mixed(ctx, o, M, out, mode, pa, st);
  // the spectrum table, in the context's grow-only workspace
  const size_t bytes = phasor_table_spec_bytes(o, M);
  if (ctx->ws_spec_bytes < bytes) {
    if (ctx->ws_spec) {
      cudaStreamSynchronize(st);
      cudaFree(ctx->ws_spec);
      ctx->ws_spec = nullptr;
      ctx->ws_spec_bytes = 0;
    }
    cudaError_t e = dev_malloc(&ctx->ws_spec, bytes);
    if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("spectrum table workspace: ") + cudaGetErrorString(e));
    ctx->ws_spec_bytes = bytes;
  }
  KsWork w;
  w.spec = ctx->ws_spec;
  w.spec_bytes = ctx->ws_spec_bytes;
  w.part = ctx->k1_part;
  return launch_phasor_table_ws(ctx, o, M, out, mode, pa, w, st);
}

int launch_phasor_table_ws(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                           KsWork& w, cudaStream_t st) {
  if (M->n_point + M->n_gauss == 0) return launch_phasor_mixed(ctx, o, M, out, mode, pa, st);
  int log2L, K;
  ks_choose(o, log2L, K);
  KSArgs A;
  K1Args& a = A.k;
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
  A.n_grp_pt = (M->n_point + KS_GC - 1) / KS_GC;
  A.n_grp = A.n_grp_pt + (M->n_gauss + KS_GC - 1) / KS_GC;
  const int cb = a.chan_block;
  const int n_cb = (o.n_chan + cb - 1) / cb;
  const int rows_per_cta = KS_WARPS * 2 * (32 >> log2L);
  a.grid_x = (o.n_rows + rows_per_cta - 1) / rows_per_cta;
  const long n_cta = (long)a.grid_x * n_cb;
  if (n_cta > INT_MAX / 2) return set_error(WN_EINVAL, "observation too large for one phasor launch");

  // the spectrum table: built here unless w already holds this model's table for this channel block
  const long long n_entries = (long long)n_cb * A.n_grp * KS_GC * cb;
  const size_t bytes = (size_t)n_entries * sizeof(float);
  if (!w.spec || w.spec_bytes < bytes) return set_error(WN_EINVAL, "spectrum table workspace too small");
  A.spec = w.spec;
  if (!(w.spec_model == M && w.spec_cb == cb)) {
    ks_spectrum<<<(unsigned)((n_entries + 255) / 256), 256, 0, st>>>(M->pg, M->n_point, M->n_gauss, A.n_grp_pt, A.n_grp,
                                                                    o.freq, o.n_chan, o.nu0, cb, n_entries, w.spec);
    w.spec_model = M;
    w.spec_cb = cb;
  }

  // tail split: the last n_cta mod slots tiles (one resident CTA per SM) are split into parts over
  // group ranges so that they fill the last wave.  The part count p minimises the tail's estimated
  // time in tiles, ceil(rem p / slots) (1 / p + h), within the partial-sum workspace, where h is a
  // part's fixed cost (its start, its partial sums written and summed again: taken as 5e5
  // evaluations, about 15 us of an SM) over a tile's evaluations.  With rem = 80 of 148 slots and long
  // tiles, 3 parts (two waves of thirds) take 0.67 of a tile instead of 1; short tiles split less.
  const int smem = ks_smem_layout(log2L, K).total;
  const int slots = ctx->num_sms;
  const int rem = (int)(n_cta % slots);
  a.n_main = (int)n_cta;
  a.tail_parts = 1;
  a.tail_ct = A.n_grp;
  a.part = w.part;
  int n_tail = 0;
  if (rem > 0 && A.n_grp >= 2 && w.part) {
    const long cap = (long)(k1_part_bytes(slots) / ((size_t)2 * K * KS_THREADS * sizeof(float2)));
    const double tile_evals = (double)rows_per_cta * cb * (double)(M->n_point + M->n_gauss);
    const double h = 5.0e5 / std::max(tile_evals, 1.0);
    int parts = 1;
    double best = 1.0;
    for (int p = 2; p <= A.n_grp && (long)rem * p <= cap; ++p) {
      const double t = (double)((rem * p + slots - 1) / slots) * (1.0 / p + h);
      if (t < best - 1e-9) {
        best = t;
        parts = p;
      }
    }
    if (parts >= 2) {
      a.tail_ct = (A.n_grp + parts - 1) / parts;
      a.tail_parts = (A.n_grp + a.tail_ct - 1) / a.tail_ct;  // no empty part
      a.n_main = (int)n_cta - rem;
      n_tail = rem;
    }
  }
  cudaError_t e;
  switch (K * 2 + (o.uniform ? 1 : 0)) {
    case 4 * 2 + 1: e = ks_launch<4, true>(A, n_tail, smem, st); break;
    case 4 * 2: e = ks_launch<4, false>(A, n_tail, smem, st); break;
    case 8 * 2 + 1: e = ks_launch<8, true>(A, n_tail, smem, st); break;
    case 8 * 2: e = ks_launch<8, false>(A, n_tail, smem, st); break;
    case 12 * 2 + 1: e = ks_launch<12, true>(A, n_tail, smem, st); break;
    default: e = ks_launch<12, false>(A, n_tail, smem, st); break;
  }
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("phasor kernel launch: ") + cudaGetErrorString(e));
  return WN_OK;
}

}  // namespace wn
