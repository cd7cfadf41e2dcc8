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
// Kernel organisation (persistent, one CTA per SM; tiles of 128 R visibilities, two in flight):
//  * producer warpgroups P0, P1 (warps 0-3, 4-7) take the even / odd tiles: thread i computes
//    phi_n(x) of rows i, i + 128, ... (R of them, interleaved so the serial recurrences overlap) by the
//    normalised Hermite recurrence (FP32, rescaled to stay in range) and writes them as bf16 hi/lo into
//    that parity's A buffer (one 128-row block per r) in the canonical K-major shared-memory layout
//    (8x8 core matrices, no swizzle);
//  * warp 16 allocates TMEM, loads the packed coefficient operand with one TMA bulk copy, and one of
//    its threads issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32; three products hi*hi + hi*lo + lo*hi
//    in the split mode; one M = 128 block per r) into the parity's TMEM accumulators and commits to an
//    mbarrier;
//  * epilogue warpgroups E0, E1 (warps 8-11, 12-15) read their accumulator rows from TMEM (warp w
//    reaches lanes 32 (w % 4) ..), stream phi_n(y) against them (R rows per thread, interleaved),
//    release TMEM, and write the output.
//  R = 2 when two parities of the doubled A buffers and 4 n_pad TMEM columns fit (n_pad <= 128),
//  else R = 1.
//  Per parity: P(k+2) waits for MMA(k) to finish reading A, MMA(k+2) for E(k) to release TMEM.
// Every wait is bounded; on a timeout the kernel raises WN_DEVERR_TIMEOUT, drains its own commits and
// frees TMEM before returning.
#include <cmath>
#include <mutex>

#include "wn_internal.cuh"
#include "tc05.cuh"

namespace wn {

constexpr int K2_M = 128;
constexpr int K2_GROUPS = 2;                     // tile parities in flight
constexpr int K2_THREADS = 32 * (8 * K2_GROUPS + 1);
constexpr int K2_MMA_WARP = 8 * K2_GROUPS;
// Rows per thread whose output the epilogue forms itself (the rest go to the producers): half of them.
#define K2_RE(R) ((R) / 2)

// sqrt(2/(n+1)) and sqrt(n/(n+1)) of the normalised Hermite recurrence
//   phi_{n+1} = sqrt(2/(n+1)) x phi_n - sqrt(n/(n+1)) phi_{n-1}.

// Lookup-table form of the basis (the 1-D tables of Sec. 3.2): phi_0..phi_127 at x_i = -K2_LUT_X + i / K2_LUT_D,
// row i of 128 floats, interpolated linearly.  |x| beyond sqrt(2 * 127 + 1) + 10 < K2_LUT_X is zero.
constexpr float K2_LUT_X = 26.0f;
constexpr int K2_LUT_D = 256;                                   // samples per unit of x
constexpr int K2_LUT_N = 2 * 26 * K2_LUT_D + 2;                 // samples
constexpr int K2_LUT_W = 128;                                   // orders per sample

struct K2Args {
  const float4* rowinfo;     // [n_rows] (xs, ys, tau_hi, tau_lo): x = xs nu, y = ys nu, tau in metres
  const float4* chaninfo;    // [n_chan] (nu/c hi, nu/c lo, log2(nu/nu0), nu)
  const __nv_bfloat16* bop;  // this shapelet's packed B operand: hi [n_pad][kp], then lo
  const float* lut;          // basis table (lookup-table mode only)
  int n_pad, nmax, passes, n_chan, n_base, n_tiles, mode, groups;
  long long n_vis;
  float c_amp, alpha, sgn;
  float2* out;
  PeelArgs peel;
  const float2* rowg;  // [n_rows] gain product g[ant1] conj(g[ant2]) of a peel whose gains do not depend on
                       // frequency (else nullptr: the epilogue forms it from the gains)
  unsigned* err;
};

__device__ __forceinline__ bool k2_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
  return mbar_wait_bounded(bar, parity, err);
}

// Offset in bytes of element (row, k) in a canonical K-major no-swizzle tile with `rows` rows.
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k, int rows) {
  return (uint32_t)((((k >> 3) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// The same for 4-byte (tf32) elements: core matrices of 8 rows x 4 elements.
__host__ __device__ __forceinline__ uint32_t kmaj_off32(int row, int k, int rows) {
  return (uint32_t)((((k >> 2) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

struct K2Layout {
  int b_bytes, a_bytes, a0, coef, bars, xfer, total;
};

__host__ __device__ inline K2Layout k2_layout(int kp, int n_pad, int passes, int groups, int R, bool tf32 = false) {
  K2Layout L;
  // 2-byte units per element: bf16 (1), bf16 hi + lo or one tf32 (2), tf32 hi + lo (4)
  const int parts = tf32 ? (passes > 1 ? 4 : 2) : (passes > 1 ? 2 : 1);
  L.b_bytes = parts * kp * n_pad * 2;
  L.a_bytes = R * parts * kp * K2_M * 2;  // one group's A: R blocks of 128 rows (hi [+ lo])
  L.a0 = (L.b_bytes + 1023) & ~1023;
  L.coef = L.a0 + groups * L.a_bytes;  // recurrence coefficients a_n, b_n: 2 x 128 floats, then the
                                       // pairs {a_n, a_n}, {-b_n, -b_n} for two rows at once: 2 x 128 float2
  L.bars = L.coef + 2 * (kNmaxLimit + 1) * 4 + 2 * (kNmaxLimit + 1) * 8;
  L.xfer = L.bars + 128;  // barriers (1 + 5 per parity) and the TMEM address slot
  // the epilogue's dot products (xr, xi) per visibility of a tile, handed to the producers for the output
  L.total = L.xfer + groups * R * K2_M * 8;
  return L;
}

// Hermite functions phi_0..phi_{KP-1}(x) by the normalised recurrence, written as bf16 hi (and lo)
// into row `row` of the K-major tile(s).  Values past nmax meet zero rows of the coefficient operand;
// they only need to be finite.  For |x| <= 12.5 every value stays in the normal FP32 range
// (phi_0 >= e^-78, |phi_n| <~ 1) and no scaling is needed.  Beyond that phi_0 = e^{-x^2/2} underflows
// FP32: the recurrence runs on values scaled by 2^E (E lowered by 64 whenever they pass 2^64) and is
// scaled back on output.  Beyond xcut every phi_n, n <= nmax, is below 1e-20 and the row is zero.
// Coefficients come from shared memory, four at a time.
__device__ __forceinline__ void store_bf16_split(float (&v)[8], unsigned char* a_hi, unsigned char* a_lo, uint32_t off) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h[i]);
    l[i] = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
  }
  *reinterpret_cast<uint4*>(a_hi + off) = *reinterpret_cast<uint4*>(h);
  if (a_lo) *reinterpret_cast<uint4*>(a_lo + off) = *reinterpret_cast<uint4*>(l);
}

// Columns k0 .. k0 + 7 of one row as tf32 (rounded to nearest) into a K-major tile of 4-byte elements:
// two core matrices, 16 row groups x 128 B apart.  With a_lo, the remainders v - hi (exact in FP32),
// rounded to tf32, go to the same place in a second tile (the split operand of WN_SHAPE_TF32X3).
__device__ __forceinline__ void store_tf32(const float (&v)[8], unsigned char* a, unsigned char* a_lo, int row, int k0) {
  const uint32_t off = kmaj_off32(row, k0, K2_M);
  float h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = to_tf32(v[i]);
  *reinterpret_cast<float4*>(a + off) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(a + off + (K2_M >> 3) * 128) = make_float4(h[4], h[5], h[6], h[7]);
  if (a_lo) {
    float l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) l[i] = to_tf32(v[i] - h[i]);
    *reinterpret_cast<float4*>(a_lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    *reinterpret_cast<float4*>(a_lo + off + (K2_M >> 3) * 128) = make_float4(l[4], l[5], l[6], l[7]);
  }
}

template <int KP, int R, bool SCALED, bool TF32>
__device__ __forceinline__ void produce_rows_run(const float (&x)[R], float (&p)[R], float (&p_prev)[R], float (&scale)[R],
                                                 int (&E)[R], unsigned char* a_base, int blk, bool split, int row,
                                                 const float4* ca, const float4* cb, const float2* ca2,
                                                 const float2* cb2) {
  if constexpr (R == 2 && !SCALED) {
    // two rows as one f32x2 recurrence: {p_r0, p_r1}' = {a,a} {x0,x1} {p_r0,p_r1} + {-b,-b} {p'_r0,p'_r1}
    float2 P = make_float2(p[0], p[1]), Pp = make_float2(p_prev[0], p_prev[1]);
    const float2 X = make_float2(x[0], x[1]);
#pragma unroll 1
    for (int k0 = 0; k0 < KP; k0 += 8) {
      float v[2][8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v[0][i] = P.x;
        v[1][i] = P.y;
        const float2 Pn = __ffma2_rn(__fmul2_rn(ca2[k0 + i], X), P, __fmul2_rn(cb2[k0 + i], Pp));
        Pp = P;
        P = Pn;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        unsigned char* hi = a_base + r * blk;
        if constexpr (TF32) store_tf32(v[r], hi, split ? hi + KP * K2_M * 4 : nullptr, row, k0);
        else store_bf16_split(v[r], hi, split ? hi + KP * K2_M * 2 : nullptr, kmaj_off(row, k0, K2_M));
      }
    }
    return;
  }
#pragma unroll 1
  for (int k0 = 0; k0 < KP; k0 += 8) {
    const float4 A0 = ca[k0 >> 2], A1 = ca[(k0 >> 2) + 1], B0 = cb[k0 >> 2], B1 = cb[(k0 >> 2) + 1];
    const float av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
    const float bv[8] = {B0.x, B0.y, B0.z, B0.w, B1.x, B1.y, B1.z, B1.w};
    float v[R][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
      for (int r = 0; r < R; ++r) {  // R independent recurrences, interleaved
        v[r][i] = SCALED ? p[r] * scale[r] : p[r];
        const float pn = fmaf(av[i] * x[r], p[r], -bv[i] * p_prev[r]);
        p_prev[r] = p[r];
        p[r] = pn;
      }
    }
    if (SCALED) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (fabsf(p[r]) > 1.8446744e19f) {  // 2^64: rescale (8 steps grow by at most 2^43)
          p[r] *= 5.421011e-20f;
          p_prev[r] *= 5.421011e-20f;
          E[r] -= 64;
          scale[r] = __int_as_float(max(0, 127 - E[r]) << 23);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      unsigned char* hi = a_base + r * blk;
      if constexpr (TF32) store_tf32(v[r], hi, split ? hi + KP * K2_M * 4 : nullptr, row, k0);
      else store_bf16_split(v[r], hi, split ? hi + KP * K2_M * 2 : nullptr, kmaj_off(row, k0, K2_M));
    }
  }
}

// Rows r of this thread go to row `row` of block r (a_base + r * blk).  The scaled form is taken for
// all R rows when any of them needs it (it is exact for every x).
// Table position of x: sample index i (rows i, i + 1 interpolated with weight t), or -1 for a zero row.
__device__ __forceinline__ int lut_pos(float x, bool valid, float xcut, float& t) {
  if (!valid || !(fabsf(x) <= xcut)) {
    t = 0.f;
    return -1;
  }
  const float u = (x + K2_LUT_X) * (float)K2_LUT_D;
  const int i = min(max((int)floorf(u), 0), K2_LUT_N - 2);
  t = u - (float)i;
  return i;
}

template <int KP, int R>
__device__ __forceinline__ void produce_rows_lut(const float (&x)[R], int nmax, const bool (&valid)[R],
                                                 unsigned char* a_base, int blk, bool split, int row, const float* lut) {
  const float xcut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;
  int ip[R];
  float tw[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ip[r] = lut_pos(x[r], valid[r], xcut, tw[r]);
#pragma unroll 1
  for (int k0 = 0; k0 < KP; k0 += 8) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float v[8];
      if (ip[r] < 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      } else {
        const float4* a = reinterpret_cast<const float4*>(lut + (size_t)ip[r] * K2_LUT_W + k0);
        const float4* b = reinterpret_cast<const float4*>(lut + (size_t)(ip[r] + 1) * K2_LUT_W + k0);
        const float4 a0 = __ldg(a), a1 = __ldg(a + 1), b0 = __ldg(b), b1 = __ldg(b + 1);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fmaf(tw[r], bv[i] - av[i], av[i]);
      }
      unsigned char* hi = a_base + r * blk;
      store_bf16_split(v, hi, split ? hi + KP * K2_M * 2 : nullptr, kmaj_off(row, k0, K2_M));
    }
  }
}

template <int KP, int R, bool TF32>
__device__ __forceinline__ void produce_rows(const float (&x)[R], int nmax, const bool (&valid)[R], unsigned char* a_base,
                                             int blk, bool split, int row, const float4* ca, const float4* cb,
                                             const float2* ca2, const float2* cb2) {
  const float xcut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;
  bool zero[R], fast = true;
  float hx[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float ax = fabsf(x[r]);
    zero[r] = !valid[r] || !(ax <= xcut);
    hx[r] = 0.5f * x[r] * x[r] * 1.4426950408889634f;  // log2 of 1/phi_0
    fast = fast && (zero[r] || ax <= 12.5f);
  }
  float p[R], p_prev[R], scale[R];
  int E[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    p_prev[r] = 0.f;
    E[r] = fast ? 0 : max(0, (int)ceilf(hx[r]) - 100);  // stored value = phi * 2^E
    p[r] = zero[r] ? 0.f : exp2f((float)E[r] - hx[r]);
    scale[r] = __int_as_float(max(0, 127 - E[r]) << 23);  // 2^-E (0 below 2^-126)
  }
  if (fast) produce_rows_run<KP, R, false, TF32>(x, p, p_prev, scale, E, a_base, blk, split, row, ca, cb, ca2, cb2);
  else produce_rows_run<KP, R, true, TF32>(x, p, p_prev, scale, E, a_base, blk, split, row, ca, cb, ca2, cb2);
}

// Epilogue dot product of one accumulator chunk (16 n2 values: columns 2 n2, 2 n2 + 1 = Re, Im) with
// phi_n2(y), advancing the y recurrence.  SCALED: values carry 2^E as in produce_row.
template <bool SCALED, int G4 = 2>
__device__ __forceinline__ void epi_chunk(const uint32_t* t, const float4* ca, const float4* cb, int n0, float y,
                                          float& q, float& q_prev, float& xr, float& xi, int& E, float& scale) {
#pragma unroll
  for (int g4 = 0; g4 < G4; ++g4) {
    const float4 A = ca[(n0 >> 2) + g4], B = cb[(n0 >> 2) + g4];
    const float av[4] = {A.x, A.y, A.z, A.w};
    const float bv[4] = {B.x, B.y, B.z, B.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * g4 + u;
      const float ph = SCALED ? q * scale : q;
      xr = fmaf(__uint_as_float(t[2 * i]), ph, xr);
      xi = fmaf(__uint_as_float(t[2 * i + 1]), ph, xi);
      const float qn = fmaf(av[u] * y, q, -bv[u] * q_prev);
      q_prev = q;
      q = qn;
    }
    if (SCALED && g4 == G4 - 1 && fabsf(q) > 1.8446744e19f) {
      q *= 5.421011e-20f;
      q_prev *= 5.421011e-20f;
      E -= 64;
      scale = __int_as_float(max(0, 127 - E) << 23);
    }
  }
}

// Epilogue of two rows at once (no scaling): their y recurrences as one f32x2 recurrence, each row's
// accumulator chunk (16 columns, 8 n2) against its half of the pair.
__device__ __forceinline__ void epi_chunk2(const uint32_t* t0, const uint32_t* t1, const float2* ca2, const float2* cb2,
                                           int n0, float2 Y, float2& Q, float2& Qp, float (&xr)[2], float (&xi)[2]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    xr[0] = fmaf(__uint_as_float(t0[2 * i]), Q.x, xr[0]);
    xi[0] = fmaf(__uint_as_float(t0[2 * i + 1]), Q.x, xi[0]);
    xr[1] = fmaf(__uint_as_float(t1[2 * i]), Q.y, xr[1]);
    xi[1] = fmaf(__uint_as_float(t1[2 * i + 1]), Q.y, xi[1]);
    const float2 Qn = __ffma2_rn(__fmul2_rn(ca2[n0 + i], Y), Q, __fmul2_rn(cb2[n0 + i], Qp));
    Qp = Q;
    Q = Qn;
  }
}

// Epilogue dot product of one 16-column chunk with table-interpolated phi_n2(y), n2 = n0 .. n0 + 7.
__device__ __forceinline__ void epi_chunk_lut(const uint32_t* t, const float* lut, int iy, float ty, int n0, float& xr,
                                              float& xi) {
  if (iy < 0) return;
  const float4* a = reinterpret_cast<const float4*>(lut + (size_t)iy * K2_LUT_W + n0);
  const float4* b = reinterpret_cast<const float4*>(lut + (size_t)(iy + 1) * K2_LUT_W + n0);
  const float4 a0 = __ldg(a), a1 = __ldg(a + 1), b0 = __ldg(b), b1 = __ldg(b + 1);
  const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float ph = fmaf(ty, bv[i] - av[i], av[i]);
    xr = fmaf(__uint_as_float(t[2 * i]), ph, xr);
    xi = fmaf(__uint_as_float(t[2 * i + 1]), ph, xi);
  }
}

// The output of one visibility of a shapelet launch: S(nu) xi e^{-2 pi i tau nu / c} (eq:shape-env,
// eq:measure_eq_discrete) from the dot product xi = xr + i xi_i, stored, added to the output, or
// subtracted as G times it from the data or the output (Sec. 5.1).  k2_out_load issues the loads of
// its inputs; k2_out_store forms and writes it once xi is known.
struct K2OutIn {
  float4 ri, ci;  // (., ., tau hi, tau lo), (nu/c hi, nu/c lo, log2(nu/nu0), .)
  float2 base, G;
};

__device__ __forceinline__ void k2_out_load(const K2Args& a, long long vis, K2OutIn& o) {
  const bool ok = vis < a.n_vis;
  const int row = ok ? (int)(vis / a.n_chan) : 0;
  const int f = ok ? (int)(vis - (long long)row * a.n_chan) : 0;
  o.ri = ok ? __ldg(a.rowinfo + row) : make_float4(0.f, 0.f, 0.f, 0.f);
  o.ci = ok ? __ldg(a.chaninfo + f) : make_float4(0.f, 0.f, 0.f, 1.f);
  o.base = make_float2(0.f, 0.f);
  o.G = make_float2(0.f, 0.f);
  if (ok && a.mode != OUT_STORE) o.base = a.mode == OUT_PEEL ? a.peel.data[vis] : a.out[vis];
  if (ok && a.mode >= OUT_PEEL) {
    if (a.rowg) o.G = __ldg(a.rowg + row);
    else if (!gain_product(a.peel, row, a.n_base, f, o.G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
  }
}

__device__ __forceinline__ void k2_out_store(const K2Args& a, long long vis, const K2OutIn& o, float xr, float xi) {
  if (vis >= a.n_vis) return;
  const float2 P = phasor_fast(reduce_turns(o.ri.z, o.ri.w, o.ci.x, o.ci.y));
  const float amp = a.sgn * ex2_approx(fmaf(a.alpha, o.ci.z, a.c_amp));
  const float zr = amp * (xr * P.x - xi * P.y), zi = amp * (xr * P.y + xi * P.x);  // amp (xr + i xi) P
  const size_t idx = (size_t)vis;
  if (a.mode == OUT_STORE) a.out[idx] = make_float2(zr, zi);
  else if (a.mode == OUT_ACCUM) a.out[idx] = make_float2(o.base.x + zr, o.base.y + zi);
  else a.out[idx] = make_float2(o.base.x - (o.G.x * zr - o.G.y * zi), o.base.y - (o.G.x * zi + o.G.y * zr));
}

// FORM: 0 = bf16 operands, basis by the recurrence; 1 = bf16, basis from the lookup table; 2 = tf32.
template <int KP, int R, int FORM>
__global__ void __launch_bounds__(K2_THREADS, 1) k2_shapelet(const K2Args a) {
  constexpr bool LUT = FORM == 1, TF32 = FORM == 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ng = a.groups;  // tile parities in flight (2, or 1 when two A buffers do not fit)
  const K2Layout lay = k2_layout(KP, a.n_pad, a.passes, ng, R, TF32);
  const int blk = lay.a_bytes / R;  // one 128-row block of A (hi [+ lo])
  uint64_t* bfull = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* afull = bfull + 1;                // [parity] producer -> MMA: A written
  uint64_t* mdone = afull + K2_GROUPS;        // [parity] MMA -> producer/epilogue: MMA complete
  uint64_t* tfree = mdone + K2_GROUPS;        // [parity] epilogue -> MMA: TMEM read
  uint64_t* xfull = tfree + K2_GROUPS;        // [parity] epilogue -> producers: dot products written
  uint64_t* xempty = xfull + K2_GROUPS;       // [parity] producers -> epilogue: dot products read
  uint32_t* tslot = reinterpret_cast<uint32_t*>(xempty + K2_GROUPS);
  const int warp = threadIdx.x >> 5;
  const int acc_cols = a.n_pad * ng * R;
  const uint32_t ncols = acc_cols <= 32 ? 32 : (acc_cols <= 64 ? 64 : (acc_cols <= 128 ? 128 : (acc_cols <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    mbar_init(bfull, 1);
    for (int g = 0; g < K2_GROUPS; ++g) {
      mbar_init(&afull[g], 128);
      mbar_init(&mdone[g], 1);
      mbar_init(&tfree[g], 128);
      mbar_init(&xfull[g], 128);
      mbar_init(&xempty[g], 128);
    }
    fence_mbar_init();
  }
  if (threadIdx.x <= kNmaxLimit) {
    // the normalised recurrence's constants sqrt(2 / (n + 1)) and sqrt(n / (n + 1)), correctly rounded in
    // FP64 and then to FP32 (the device's FP64 division and square root round to nearest), formed here in
    // every CTA so that no upload has to be ordered with the launches of other streams
    const double np1 = (double)(threadIdx.x + 1);
    const float ha = (float)sqrt(2.0 / np1), hb = (float)sqrt((double)threadIdx.x / np1);
    float* cf = reinterpret_cast<float*>(smem + lay.coef);
    cf[threadIdx.x] = ha;
    cf[kNmaxLimit + 1 + threadIdx.x] = hb;
    float2* cp = reinterpret_cast<float2*>(cf + 2 * (kNmaxLimit + 1));
    cp[threadIdx.x] = make_float2(ha, ha);
    cp[kNmaxLimit + 1 + threadIdx.x] = make_float2(-hb, -hb);
  }
  if (warp == K2_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const float4* ca = reinterpret_cast<const float4*>(smem + lay.coef);
  const float4* cb = ca + (kNmaxLimit + 1) / 4;
  const float2* ca2 = reinterpret_cast<const float2*>(cb + (kNmaxLimit + 1) / 4);  // {a_n, a_n}
  const float2* cb2 = ca2 + (kNmaxLimit + 1);                                      // {-b_n, -b_n}
  // tiles of this CTA: it = 0, 1, 2, ... -> tile blockIdx.x + it * gridDim.x; parity s = it % ng, j = it / ng
  const int n_it = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == K2_MMA_WARP) {
    // ---------------- TMA of the coefficient operand, then the MMA issue loop ----------------
    if ((threadIdx.x & 31) == 0) {
      mbar_arrive_expect_tx(bfull, (uint32_t)lay.b_bytes);
      tma_bulk_g2s(smem, a.bop, (uint32_t)lay.b_bytes, bfull);
      const uint32_t idesc = umma_idesc_bf16(a.n_pad), idesc32 = umma_idesc_tf32(a.n_pad);
      // the lo halves follow the hi ones: 2-byte bf16 or 4-byte tf32 elements
      const uint32_t b_hi = smem_u32(smem), b_lo = b_hi + (uint32_t)(KP * a.n_pad * (TF32 ? 4 : 2));
      const uint32_t lbo_b = (uint32_t)(a.n_pad >> 3) << 7, lbo_a = (uint32_t)(K2_M >> 3) << 7;
      bool ok = k2_wait(bfull, 0, a.err);
      int done = 0;
      for (int it = 0; ok && it < n_it; ++it) {
        const int sp = it % ng, j = it / ng;
        if (!k2_wait(&afull[sp], j & 1, a.err)) break;
        if (j > 0 && !k2_wait(&tfree[sp], (j - 1) & 1, a.err)) break;
        tc_fence_after();
#pragma unroll
        for (int r = 0; r < R; ++r) {  // block r of the tile into accumulator sp * R + r
          const uint32_t a_hi = smem_u32(smem + lay.a0 + sp * lay.a_bytes + r * blk);
          const uint32_t a_lo = a_hi + (uint32_t)(KP * K2_M * (TF32 ? 4 : 2));
          const uint32_t d = tmem + (uint32_t)((sp * R + r) * a.n_pad);
          if constexpr (TF32) {  // K = 8 per instruction: two core matrices of 4-byte elements
#pragma unroll 1
            for (int p = 0; p < a.passes; ++p) {  // one product, or hi*hi, hi*lo, lo*hi
              const uint32_t aa = (p == 2) ? a_lo : a_hi;
              const uint32_t bb = (p == 1) ? b_lo : b_hi;
#pragma unroll
              for (int kk = 0; kk < KP / 8; ++kk) {
                const uint64_t da = umma_desc(aa + (uint32_t)(2 * kk) * lbo_a, lbo_a, 128);
                const uint64_t db = umma_desc(bb + (uint32_t)(2 * kk) * lbo_b, lbo_b, 128);
                umma_tf32(d, da, db, idesc32, (p > 0 || kk > 0) ? 1u : 0u);
              }
            }
            continue;
          }
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
        }
        umma_commit(&mdone[sp]);
        done = it + 1;
      }
      // drain: the last commit of each parity has landed before teardown
      for (int sp = 0; sp < ng; ++sp) {
        const int cnt = done > sp ? (done - 1 - sp) / ng + 1 : 0;  // commits issued on this parity
        if (cnt > 0) k2_wait(&mdone[sp], (cnt - 1) & 1, a.err);
      }
    }
    __syncwarp();
  } else if (warp < 4 * K2_GROUPS) {
    // ---------------- producers: phi_n(x) into the parity's A buffer ----------------
    const int sp = warp >> 2;
    if (sp >= ng) goto done;
    const int m = threadIdx.x & 127;
    unsigned char* a_base = smem + lay.a0 + sp * lay.a_bytes;
    // the next tile's (xs, nu) are loaded one tile ahead and multiplied only when used
    auto load_x = [&](int it, bool (&valid)[R], float (&xs)[R], float (&nu)[R]) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long vis = (long long)(blockIdx.x + it * gridDim.x) * (K2_M * R) + r * K2_M + m;
        valid[r] = it < n_it && vis < a.n_vis;
        xs[r] = 0.f;
        nu[r] = 0.f;
        if (valid[r]) {
          const int row = (int)(vis / a.n_chan);
          const int f = (int)(vis - (long long)row * a.n_chan);
          xs[r] = __ldg(&a.rowinfo[row].x);
          nu[r] = __ldg(&a.chaninfo[f].w);
        }
      }
    };
    bool valid[R];
    float xs[R], nu[R];
    load_x(sp, valid, xs, nu);
    const float2* xfer = reinterpret_cast<const float2*>(smem + lay.xfer) + sp * R * K2_M + m;
    // The output of rows RE .. R-1 of this parity's tile jo (tile index ito); the epilogue forms rows
    // 0 .. RE-1 itself.  The inputs' loads are issued first and arrive while the epilogue finishes.
    auto out_tile = [&](int ito, int jo) -> bool {
      K2OutIn o[R];
#pragma unroll
      for (int r = K2_RE(R); r < R; ++r)
        k2_out_load(a, (long long)(blockIdx.x + ito * gridDim.x) * (K2_M * R) + r * K2_M + m, o[r]);
      if (!k2_wait(&xfull[sp], jo & 1, a.err)) return false;
#pragma unroll
      for (int r = K2_RE(R); r < R; ++r) {
        const float2 d = xfer[r * K2_M];
        k2_out_store(a, (long long)(blockIdx.x + ito * gridDim.x) * (K2_M * R) + r * K2_M + m, o[r], d.x, d.y);
      }
      mbar_arrive(&xempty[sp]);
      return true;
    };
    int last = -1;  // this parity's last tile produced whose output is still to be formed
    for (int it = sp, j = 0; it < n_it; it += ng, ++j) {
      float x[R];
      bool v0[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        x[r] = xs[r] * nu[r];
        v0[r] = valid[r];
      }
      load_x(it + ng, valid, xs, nu);
      if (j > 0 && !k2_wait(&mdone[sp], (j - 1) & 1, a.err)) break;  // MMA(j-1) has read A
      if (LUT) produce_rows_lut<KP, R>(x, a.nmax, v0, a_base, blk, a.passes > 1, m, a.lut);
      else produce_rows<KP, R, TF32>(x, a.nmax, v0, a_base, blk, a.passes > 1, m, ca, cb, ca2, cb2);
      fence_async_smem();
      mbar_arrive(&afull[sp]);
      // the previous tile's output, while the MMA of this one runs
      if (j > 0 && !out_tile(it - ng, j - 1)) {
        last = -1;
        break;
      }
      last = j;
    }
    if (last >= 0) out_tile(sp + last * ng, last);
  } else {
    // ---------------- epilogues: xi = sum_n2 T[., n2] phi_n2(y), handed to the producers ----------------
    const int sp = (warp - 4 * K2_GROUPS) >> 2;
    if (sp >= ng) goto done;
    const int m = threadIdx.x & 127;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(sp * R * a.n_pad);
    const float ycut = sqrtf(2.0f * a.nmax + 1.0f) + 10.0f;
    float2* xfer = reinterpret_cast<float2*>(smem + lay.xfer) + sp * R * K2_M + m;
    struct EpiIn {
      float ys, nu;  // y = ys nu
    };
    auto vis_of = [&](int it, int r) { return (long long)(blockIdx.x + it * gridDim.x) * (K2_M * R) + r * K2_M + m; };
    auto valid_of = [&](int it, long long vis) { return it < n_it && vis < a.n_vis; };
    auto load_epi = [&](int it, int r) {
      EpiIn e;
      const long long vis = vis_of(it, r);
      const bool valid = valid_of(it, vis);
      const int row = valid ? (int)(vis / a.n_chan) : 0;
      const int f = valid ? (int)(vis - (long long)row * a.n_chan) : 0;
      e.ys = valid ? __ldg(&a.rowinfo[row].y) : 0.f;
      e.nu = valid ? __ldg(&a.chaninfo[f].w) : 1.f;
      return e;
    };
    EpiIn nxt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) nxt[r] = load_epi(sp, r);
    for (int it = sp, j = 0; it < n_it; it += ng, ++j) {
      EpiIn cur[R];
#pragma unroll
      for (int r = 0; r < R; ++r) cur[r] = nxt[r];
      long long vis[R];
      bool valid[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        vis[r] = vis_of(it, r);
        valid[r] = valid_of(it, vis[r]);
      }
      K2OutIn eo[R];  // the inputs of this thread's own outputs, in flight during the wait
#pragma unroll
      for (int r = 0; r < K2_RE(R); ++r) k2_out_load(a, valid[r] ? vis[r] : a.n_vis, eo[r]);
      if (!k2_wait(&mdone[sp], j & 1, a.err)) break;
#pragma unroll
      for (int r = 0; r < R; ++r) nxt[r] = load_epi(it + ng, r);  // next tile's constants in flight
      tc_fence_after();
      float y[R], q[R], q_prev[R], scale[R], xr[R], xi[R];
      int E[R];
      bool yfast = true;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        y[r] = cur[r].ys * cur[r].nu;
        const bool yzero = !valid[r] || !(fabsf(y[r]) <= ycut);
        yfast = yfast && (yzero || fabsf(y[r]) <= 12.5f);
        q[r] = yzero ? 0.f : 1.f;  // marks zero rows until the seed below
        xr[r] = xi[r] = 0.f;
        q_prev[r] = 0.f;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float hy = 0.5f * y[r] * y[r] * 1.4426950408889634f;
        E[r] = yfast ? 0 : max(0, (int)ceilf(hy) - 100);
        q[r] = q[r] == 0.f ? 0.f : exp2f((float)E[r] - hy);
        scale[r] = __int_as_float(max(0, 127 - E[r]) << 23);
      }
      // accumulator rows in chunks of 16 columns (8 n2).  Once the last chunk's loads have completed the
      // accumulator is released to the MMA warp (tfree), before that chunk is used.
      const int nch = a.n_pad >> 4;
      bool released = false;
      auto release = [&]() {
        tc_fence_before();
        mbar_arrive(&tfree[sp]);
        released = true;
      };
      if (LUT) {  // table-interpolated phi_n2(y): one chunk of every row at a time
        int iy[R];
        float ty[R];
#pragma unroll
        for (int r = 0; r < R; ++r) iy[r] = lut_pos(y[r], valid[r], ycut, ty[r]);
        uint32_t tb[R][16];
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
#pragma unroll
          for (int r = 0; r < R; ++r) tmem_issue16x(trow + (uint32_t)(r * a.n_pad + (c << 4)), tb[r]);
#pragma unroll
          for (int r = 0; r < R; ++r) tmem_wait16(tb[r]);
          if (c == nch - 1) release();
#pragma unroll
          for (int r = 0; r < R; ++r) epi_chunk_lut(tb[r], a.lut, iy[r], ty[r], c << 3, xr[r], xi[r]);
        }
      } else if (R == 1) {  // one row: the next chunk's load in flight while one is used
        uint32_t tb0[16], tb1[16];
        tmem_issue16x(trow, tb0);
        tmem_wait16(tb0);
#pragma unroll 1
        for (int c = 0; c < nch; c += 2) {
          if (c + 1 < nch) tmem_issue16x(trow + (uint32_t)((c + 1) << 4), tb1);
          if (yfast) epi_chunk<false>(tb0, ca, cb, c << 3, y[0], q[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
          else epi_chunk<true>(tb0, ca, cb, c << 3, y[0], q[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
          tmem_wait16(tb1);
          if (c + 1 < nch) {
            if (c + 2 < nch) tmem_issue16x(trow + (uint32_t)((c + 2) << 4), tb0);
            if (yfast) epi_chunk<false>(tb1, ca, cb, (c + 1) << 3, y[0], q[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
            else epi_chunk<true>(tb1, ca, cb, (c + 1) << 3, y[0], q[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
            tmem_wait16(tb0);
          }
        }
      } else {  // R rows: a 16-column chunk of every row in flight, their recurrences interleaved
        uint32_t tb[R][16];
        if constexpr (R == 2) {
          // The TMEM loads are warp-collective (.sync.aligned): every thread issues them in the same
          // order whatever its rows need; only the arithmetic below depends on the thread.
          float2 Q = make_float2(q[0], q[1]), Qp = make_float2(q_prev[0], q_prev[1]);
          const float2 Y = make_float2(y[0], y[1]);
#pragma unroll 1
          for (int c = 0; c < nch; ++c) {
            tmem_issue16x(trow + (uint32_t)(c << 4), tb[0]);
            tmem_issue16x(trow + (uint32_t)(a.n_pad + (c << 4)), tb[1]);
            tmem_wait16(tb[0]);
            tmem_wait16(tb[1]);
            if (c == nch - 1) release();
            if (yfast) {  // both rows unscaled: one f32x2 recurrence
              epi_chunk2(tb[0], tb[1], ca2, cb2, c << 3, Y, Q, Qp, xr, xi);
            } else {
#pragma unroll
              for (int r = 0; r < R; ++r)
                epi_chunk<true>(tb[r], ca, cb, c << 3, y[r], q[r], q_prev[r], xr[r], xi[r], E[r], scale[r]);
            }
          }
        }
      }
      if (!released) release();
      if (j > 0 && !k2_wait(&xempty[sp], (j - 1) & 1, a.err)) break;  // the producers have read tile j-1's
#pragma unroll
      for (int r = K2_RE(R); r < R; ++r) xfer[r * K2_M] = valid[r] ? make_float2(xr[r], xi[r]) : make_float2(0.f, 0.f);
      mbar_arrive(&xfull[sp]);
#pragma unroll
      for (int r = 0; r < K2_RE(R); ++r) k2_out_store(a, valid[r] ? vis[r] : a.n_vis, eo[r], xr[r], xi[r]);
    }
  }
done:
  __syncthreads();
  if (warp == K2_MMA_WARP) {
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

__global__ void k2_rowinfo(const double* uvw, int n_rows, const ShapeRec* sh, double sd0, double cd0, float4* out) {
  __shared__ double F[9];
  if (threadIdx.x == 0) shapelet_frame(sh->l, sh->m, sd0, cd0, F);
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

// Per-row gain product of a peel with frequency-independent gains: G[row] = g[tg][0][ant1] conj(g[tg][0][ant2]),
// NaN (and the antenna flag) for an antenna index out of range, as the epilogue would form it.
__global__ void k2_rowgain(PeelArgs p, int n_rows, int n_base, float2* out, unsigned* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  float2 G;
  if (!gain_product(p, r, n_base, 0, G)) atomicOr(err, WN_DEVERR_ANTENNA);
  out[r] = G;
}

void launch_rowgain(const PeelArgs& pa, int n_rows, int n_base, float2* out, unsigned* err, cudaStream_t st) {
  k2_rowgain<<<(n_rows + 255) / 256, 256, 0, st>>>(pa, n_rows, n_base, out, err);
}

template <int KP, int R, int FORM>
static cudaError_t k2_launch_t(const K2Args& a, int grid, int smem, cudaStream_t st) {
  auto fn = k2_shapelet<KP, R, FORM>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(fn));
  if (e != cudaSuccess) return e;
  fn<<<grid, K2_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <int FORM>
static cudaError_t k2_dispatch_t(const K2Args& a, int k_pad, int R, int grid, int smem, cudaStream_t st) {
  if (R == 2) {
    switch (k_pad) {
      case 16: return k2_launch_t<16, 2, FORM>(a, grid, smem, st);
      case 32: return k2_launch_t<32, 2, FORM>(a, grid, smem, st);
      case 48: return k2_launch_t<48, 2, FORM>(a, grid, smem, st);
      default: return k2_launch_t<64, 2, FORM>(a, grid, smem, st);
    }
  }
  switch (k_pad) {
    case 16: return k2_launch_t<16, 1, FORM>(a, grid, smem, st);
    case 32: return k2_launch_t<32, 1, FORM>(a, grid, smem, st);
    case 48: return k2_launch_t<48, 1, FORM>(a, grid, smem, st);
    case 64: return k2_launch_t<64, 1, FORM>(a, grid, smem, st);
    case 80: return k2_launch_t<80, 1, FORM>(a, grid, smem, st);
    case 96: return k2_launch_t<96, 1, FORM>(a, grid, smem, st);
    case 112: return k2_launch_t<112, 1, FORM>(a, grid, smem, st);
    default: return k2_launch_t<128, 1, FORM>(a, grid, smem, st);
  }
}

static cudaError_t k2_dispatch(const K2Args& a, int k_pad, int R, int form, int grid, int smem, cudaStream_t st) {
  if (form == 1) return k2_dispatch_t<1>(a, k_pad, R, grid, smem, st);
  if (form == 2) return k2_dispatch_t<2>(a, k_pad, R, grid, smem, st);
  return k2_dispatch_t<0>(a, k_pad, R, grid, smem, st);
}

// The basis table of the lookup-table mode: phi_0..phi_127 in FP64 by the normalised recurrence at every
// sample, stored in FP32.  Built once per context.
__global__ void k2_lut_build(float* lut) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K2_LUT_N) return;
  const double x = -(double)K2_LUT_X + (double)i / K2_LUT_D;
  double p_prev = 0.0, p = exp(-0.5 * x * x);
  for (int n = 0; n < K2_LUT_W; ++n) {
    lut[(size_t)i * K2_LUT_W + n] = (float)p;
    const double pn = sqrt(2.0 / (n + 1)) * x * p - sqrt((double)n / (n + 1)) * p_prev;
    p_prev = p;
    p = pn;
  }
}

static int k2_lut(wn_ctx* ctx, cudaStream_t st, const float** out) {
  if (!ctx->lut) {
    cudaError_t e = dev_malloc(&ctx->lut, sizeof(float) * (size_t)K2_LUT_N * K2_LUT_W);
    if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("basis table: ") + cudaGetErrorString(e));
    k2_lut_build<<<(K2_LUT_N + 127) / 128, 128, 0, st>>>(ctx->lut);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("basis table: ") + cudaGetErrorString(e));
  }
  *out = ctx->lut;
  return WN_OK;
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
  cudaError_t e = dev_malloc(&ctx->ws, bytes);
  if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("workspace: ") + cudaGetErrorString(e));
  ctx->ws_bytes = bytes;
  return WN_OK;
}

// Shapelet launches with caller-supplied tables: per-channel (n_chan float4) and per-row (n_rows float4).
int launch_shapelets_ws(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        float4* chaninfo, float4* rowinfo, cudaStream_t st, float2* rowg) {
  k2_chaninfo<<<(o.n_chan + 255) / 256, 256, 0, st>>>(o.freq, o.n_chan, o.nu0, chaninfo);
  const long long n_vis = (long long)o.n_rows * o.n_chan;
  const bool tf32 = ctx->shape_mode == WN_SHAPE_TF32 || ctx->shape_mode == WN_SHAPE_TF32X3;
  const int passes = ctx->shape_mode == WN_SHAPE_BF16X1 || ctx->shape_mode == WN_SHAPE_TF32 ? 1 : 3;
  const float* lut = nullptr;
  if (ctx->shape_mode == WN_SHAPE_LUT_BF16X3)
    if (int r = k2_lut(ctx, st, &lut)) return r;
  const double L0 = std::log2(o.nu0);
  const bool peeling = mode == OUT_PEEL || mode == OUT_SUBG;
  if (rowg && (!peeling || pa.gf != 1)) rowg = nullptr;
  if (rowg) k2_rowgain<<<(o.n_rows + 255) / 256, 256, 0, st>>>(pa, o.n_rows, o.n_base, rowg, ctx->d_err);
  for (int q = 0; q < M->n_shape; ++q) {
    const ShapeRec& h = M->sh_host[q];
    k2_rowinfo<<<(o.n_rows + 255) / 256, 256, 0, st>>>(o.uvw, o.n_rows, M->sh + q, std::sin(o.dec0), std::cos(o.dec0), rowinfo);
    K2Args a;
    a.rowinfo = rowinfo;
    a.chaninfo = chaninfo;
    a.bop = tf32 ? reinterpret_cast<const __nv_bfloat16*>(M->bop32 + h.b_off) : M->bop + h.b_off;
    a.lut = lut;
    a.n_pad = h.n_pad;
    a.nmax = h.nmax;
    a.passes = passes;
    a.n_chan = o.n_chan;
    a.n_base = o.n_base;
    a.n_vis = n_vis;
    a.c_amp = (float)((double)h.lS + (double)h.alpha * (L0 - h.lref));
    a.alpha = h.alpha;
    a.sgn = h.sgn;
    a.out = out;
    a.peel = pa;
    a.rowg = rowg;
    a.err = ctx->d_err;
    // the first shapelet applies the caller's mode, the rest add (or subtract G times) their part
    a.mode = q == 0 ? mode : (mode == OUT_STORE ? OUT_ACCUM : (mode == OUT_PEEL ? OUT_SUBG : mode));
    // two rows per producer / epilogue thread when both parities' doubled A buffers and 4 n_pad TMEM
    // columns fit; else one
    a.groups = K2_GROUPS;
    int R = 2;
    K2Layout lay = k2_layout(h.k_pad, h.n_pad, passes, a.groups, R, tf32);
    if (h.n_pad > 128 || lay.total > 227 * 1024) {
      R = 1;
      lay = k2_layout(h.k_pad, h.n_pad, passes, a.groups, R, tf32);
    }
    if (lay.total > 227 * 1024) {  // large n_max in the split mode: one tile in flight
      a.groups = 1;
      lay = k2_layout(h.k_pad, h.n_pad, passes, 1, R, tf32);
    }
    if (lay.total > 227 * 1024)
      return set_error(WN_EINVAL, "shapelet operand of orders up to " + std::to_string(h.nmax) + " (k_pad " +
                                      std::to_string(h.k_pad) + ", n_pad " + std::to_string(h.n_pad) +
                                      ") does not fit in shared memory in this shapelet mode");
    const int n_tiles = (int)((n_vis + K2_M * R - 1) / (K2_M * R));
    a.n_tiles = n_tiles;
    const int grid = std::min(n_tiles, ctx->num_sms);
    cudaError_t e = k2_dispatch(a, h.k_pad, R, lut != nullptr ? 1 : (tf32 ? 2 : 0), grid, lay.total, st);
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet kernel launch: ") + cudaGetErrorString(e));
  }
  return WN_OK;
}

int launch_shapelets(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                     cudaStream_t st) {
  const size_t chan_bytes = ((size_t)o.n_chan * sizeof(float4) + 255) & ~(size_t)255;
  const size_t row_bytes = ((size_t)o.n_rows * sizeof(float4) + 255) & ~(size_t)255;
  if (int r = ws_reserve(ctx, chan_bytes + row_bytes + (size_t)o.n_rows * sizeof(float2), st)) return r;
  float4* chaninfo = static_cast<float4*>(ctx->ws);
  float4* rowinfo = reinterpret_cast<float4*>(static_cast<char*>(ctx->ws) + chan_bytes);
  float2* rowg = reinterpret_cast<float2*>(static_cast<char*>(ctx->ws) + chan_bytes + row_bytes);
  return launch_shapelets_ws(ctx, o, M, out, mode, pa, chaninfo, rowinfo, st, rowg);
}

}  // namespace wn



// ------------------------------------------------------------------------------------------------
// Allocation-free shapelet launches (wn_predict_static).  The per-channel and per-row constants
// that launch_shapelets keeps in the context's growable workspace live here in a fixed device array
// instead, so the call never allocates.  Every GPU that loads the library holds its own copy of the
// array until the process exits.  The copy is shared by every call on that device and keeps the last
// call's contents; both tables are fully rewritten by the prep kernels before the main kernel reads
// them, so nothing needs clearing, but calls whose work overlaps on the same device race on it.
// ------------------------------------------------------------------------------------------------
namespace wn {

constexpr size_t kStaticScratchEntries = size_t(1) << 18;  // float4 entries (4 MiB): n_chan (padded to 16) + n_rows
static __device__ __align__(256) float4 g_static_scratch[kStaticScratchEntries];

// Set-up at context creation (wn_create), with the context's device current: in host code the array's
// name is only a host-side stand-in, so its device address is looked up here and kept in the context.
// A context created after a device reset looks it up again.
int static_scratch_setup(wn_ctx* ctx) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
  ctx->static_scratch = static_cast<float4*>(p);
  return WN_OK;
}

size_t static_scratch_entries() { return kStaticScratchEntries; }

int launch_shapelets_static(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                            cudaStream_t st) {
  const size_t chan_entries = ((size_t)o.n_chan + 15) & ~(size_t)15;
  if (chan_entries + (size_t)o.n_rows > kStaticScratchEntries)
    return set_error(WN_EINVAL, "wn_predict_static: n_chan (rounded up to 16) + n_time * n_base = " +
                                    std::to_string(chan_entries + (size_t)o.n_rows) + " exceeds the static scratch of " +
                                    std::to_string(kStaticScratchEntries) + " entries");
  float4* base = ctx->static_scratch;
  if (!base) return set_error(WN_ECUDA, "wn_predict_static: the static scratch address was not found at set-up");
  return launch_shapelets_ws(ctx, o, M, out, mode, pa, base, base + chan_entries, st, nullptr);
}

}  // namespace wn

namespace wn {
// Per-channel and per-row tables of shapelet q for the adjoint (same definitions as the prediction).
int launch_shapelet_prep(wn_ctx* ctx, const ObsDev& o, const Model* M, int q, float4* chaninfo, float4* rowinfo,
                         bool chan, cudaStream_t st) {
  (void)ctx;
  if (chan) k2_chaninfo<<<(o.n_chan + 255) / 256, 256, 0, st>>>(o.freq, o.n_chan, o.nu0, chaninfo);
  k2_rowinfo<<<(o.n_rows + 255) / 256, 256, 0, st>>>(o.uvw, o.n_rows, M->sh + q, std::sin(o.dec0), std::cos(o.dec0), rowinfo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet prep: ") + cudaGetErrorString(e));
  return WN_OK;
}
}  // namespace wn
