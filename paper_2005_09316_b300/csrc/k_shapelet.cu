// K2: shapelet envelopes on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// For one shapelet and every visibility (row (t,b), channel f), eq:shape-env with eq:basis_FT gives
//   xi = sum_{n1+n2<=nmax} C[n1,n2] (-i)^(n1+n2) phi_n1(x) phi_n2(y),
//   x = beta1 K (sin pa u' + cos pa v') nu/c,  y = beta2 K (cos pa u' - sin pa v') nu/c   (eq:scale-shape-x/y)
// with (u', v') re-phased to the shapelet centre and phi_n the peak-normalised Hermite functions.
// With the rescaled functions g_n = k_n phi_n (herm_k), writing A[vis, n1] = g_n1(x) and splitting
// C (-i)^(n1+n2) / (k_n1 k_n2) into real and imaginary parts gives a dense contraction
// T = A [C_re | C_im] (M = visibilities, K = n1, N = 2 (nmax+1)) followed by a per-row dot product
// xi = sum_n2 T[., n2] g_n2(y).  Each shapelet's contribution is
// S(nu) xi exp(-2 pi i tau nu/c); a launch sums those of up to K2_MAXS shapelets per visibility and
// writes the output once: stored, added, or subtracted as G times the sum for the peel (Sec. 5.1).
//
// Kernel organisation (persistent, one CTA per SM; tiles of 128 R visibilities, two in flight).  The
// unit of work is an item, one (tile, shapelet) pair; the items of a tile follow each other on the same
// parity, and the output of a tile is written after its last item.
//  * producer warpgroups P0, P1 (warps 0-3, 4-7) take the items of the even / odd tiles: thread i
//    computes g_n(x) of rows i, i + 128, ... (R of them, their recurrences run as one f32x2
//    recurrence when R = 2) by the two-operation recurrence (FP32, scaled by powers of two to stay in
//    range) and
//    writes them as bf16 hi/lo into that parity's A buffer (one 128-row block per r) in the canonical
//    K-major shared-memory layout (8x8 core matrices, no swizzle);
//  * warp 16 allocates TMEM, loads the packed coefficient operands of all the launch's shapelets with
//    TMA bulk copies, and one of its threads issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32; three
//    products hi*hi + hi*lo + lo*hi in the split mode; one M = 128 block per r) into the parity's TMEM
//    accumulators and commits to an mbarrier, alternating the parities item by item;
//  * epilogue warpgroups E0, E1 (warps 8-11, 12-15) read their accumulator rows from TMEM (warp w
//    reaches lanes 32 (w % 4) ..), stream g_n(y) against them, release TMEM and hand the dot products
//    to the producers through shared memory;
//  * the producers, while the next item's MMA runs, weight the dot products by the shapelet's spectrum
//    and phasor, sum them over the tile's items and write the tile's output after its last item.
//  R = 2 when two parities of the doubled A buffers and 4 n_pad TMEM columns fit (n_pad <= 128),
//  else R = 1.
//  Per parity: P(k+1) waits for MMA(k) to finish reading A, MMA(k+1) for E(k) to release TMEM.
// Every wait is bounded; on a timeout the kernel raises WN_DEVERR_TIMEOUT, drains its own commits and
// frees TMEM before returning.
#include <cmath>
#include <mutex>

#include "wn_internal.cuh"
#include "tc05.cuh"

namespace wn {

// e_n = sqrt(2/(n+1)) k_(n+1)/k_n of the rescaled Hermite recurrence (herm_k), uploaded at context creation
__constant__ float c_k2e[kNmaxLimit + 1];

constexpr int K2_M = 128;
constexpr int K2_GROUPS = 2;                     // tile parities in flight
constexpr int K2_THREADS = 32 * (8 * K2_GROUPS + 1);
constexpr int K2_MMA_WARP = 8 * K2_GROUPS;
constexpr int K2_MAXS = 8;                       // shapelets summed in one launch

// The normalised Hermite recurrence phi_{n+1} = a_n x phi_n - b_n phi_{n-1}, a_n = sqrt(2/(n+1)),
// b_n = sqrt(n/(n+1)), becomes g_{n+1} = e_n x g_n - g_{n-1} for g_n = k_n phi_n (herm_k), with
// e_n = a_n k_{n+1}/k_n (c_k2e).

// Lookup-table form of the basis (the 1-D tables of Sec. 3.2): g_0..g_127 at x_i = -K2_LUT_X + i / K2_LUT_D,
// row i of 128 floats, interpolated linearly.  |x| beyond sqrt(2 * 127 + 1) + 10 < K2_LUT_X is zero.
constexpr float K2_LUT_X = 26.0f;
constexpr int K2_LUT_D = 256;                                   // samples per unit of x
constexpr int K2_LUT_N = 2 * 26 * K2_LUT_D + 2;                 // samples
constexpr int K2_LUT_W = 128;                                   // orders per sample

// One shapelet of a launch.
struct K2Shape {
  const void* bop;      // its packed B operand in global memory: bf16 hi [n_pad][k_pad] then lo, or the tf32 pair
  int b_smem, b_bytes;  // byte offset and size of its copy in shared memory
  int k_pad, n_pad, nmax;
  float c_amp, alpha, sgn;  // S(nu) = sgn 2^(alpha log2(nu/nu0) + c_amp)
  int pad0, pad1;
};
static_assert(sizeof(K2Shape) == 48, "K2Shape layout");

struct K2Args {
  const float4* rowinfo;   // [n_shape][n_rows] (xs, ys, tau_hi, tau_lo): x = xs nu, y = ys nu, tau in metres
  const float4* chaninfo;  // [n_chan] (nu/c hi, nu/c lo, log2(nu/nu0), nu)
  const float* lut;        // basis table (lookup-table mode only)
  K2Shape sh[K2_MAXS];
  int n_shape;             // shapelets of this launch
  int kp_max, np_max;      // the A buffers' K extent and the accumulator columns per block
  int b_total;             // bytes of shared memory holding the B operands
  int passes, n_chan, n_rows, n_base, n_tiles, mode, groups;
  int step_row, step_f;    // a thread's move from one of its tiles to its next, as whole rows and channels
  long long n_vis;
  float2* out;
  PeelArgs peel;
  const float2* rowg;  // [n_rows] gain product g[ant1] conj(g[ant2]) of a peel whose gains do not depend on
                       // frequency (else nullptr: the output step forms it from the gains)
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
  int a_bytes, a0, coef, shp, bars, xfer, total;
};

// 2-byte units per element: bf16 (1), bf16 hi + lo or one tf32 (2), tf32 hi + lo (4)
__host__ __device__ inline int k2_parts(int passes, bool tf32) { return tf32 ? (passes > 1 ? 4 : 2) : (passes > 1 ? 2 : 1); }

// B operand bytes of one shapelet and its shared-memory footprint (rounded up to 1 KB).
__host__ __device__ inline int k2_b_bytes(int kp, int n_pad, int passes, bool tf32) { return k2_parts(passes, tf32) * kp * n_pad * 2; }

__host__ __device__ inline K2Layout k2_layout(int b_total, int kp, int passes, int groups, int R, bool tf32 = false) {
  K2Layout L;
  L.a_bytes = R * k2_parts(passes, tf32) * kp * K2_M * 2;  // one group's A: R blocks of 128 rows (hi [+ lo])
  L.a0 = (b_total + 1023) & ~1023;
  L.coef = L.a0 + groups * L.a_bytes;  // recurrence constants e_n (128 floats, then 128 unused), then
                                       // the quadruples {e_n, e_n, 0, 0} for two rows at once
  L.shp = L.coef + 2 * (kNmaxLimit + 1) * 4 + (kNmaxLimit + 1) * 16;
  L.bars = L.shp + K2_MAXS * (int)sizeof(K2Shape);
  L.xfer = L.bars + 128;  // barriers (1 + 5 per parity) and the TMEM address slot
  // the epilogue's dot products (xr, xi) per visibility of an item, handed to the producers
  L.total = L.xfer + groups * R * K2_M * 8;
  return L;
}

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

// One row's 8 values into the A block(s): bf16 hi (+ lo) or tf32 hi (+ lo).
template <bool TF32>
__device__ __forceinline__ void store_row8(float (&v)[8], unsigned char* hi, int lo_off, bool split, int row, int k0) {
  if constexpr (TF32) store_tf32(v, hi, split ? hi + lo_off : nullptr, row, k0);
  else store_bf16_split(v, hi, split ? hi + lo_off : nullptr, kmaj_off(row, k0, K2_M));
}

// Rescaled Hermite functions g_n = k_n phi_n, n = 0..kp-1 (herm_k: k_n in [1, 4]; the coefficient operand
// carries 1/(k_n1 k_n2)), by the two-operation recurrence g_(n+1) = e_n x g_n - g_(n-1) from g_0 = phi_0,
// written as bf16 hi (and lo) or tf32 into row `row` of the K-major tile(s).  Values past nmax meet zero
// rows of the coefficient operand; they only need to be finite.  For |x| <= 12.5 every value stays in
// the normal FP32 range (phi_0 >= e^-78, |g_n| <~ 4) and no scaling is needed.  Beyond that
// phi_0 = e^{-x^2/2} underflows FP32: the recurrence runs on values scaled by 2^E (E lowered by 64
// whenever they pass 2^64) and is scaled back on output.  Beyond xcut every phi_n, n <= nmax, is below
// 1e-20 and the row is zero.

// Seed of one row: p = phi_0 2^E (E = 0 on the unscaled path), sc = 2^-E (0 below 2^-126).
__device__ __forceinline__ void herm_seed(float x, bool zero, bool fast, float& p, int& E, float& sc) {
  const float hx = 0.5f * x * x * 1.4426950408889634f;  // log2 of 1/phi_0
  E = fast ? 0 : max(0, (int)ceilf(hx) - 100);
  p = zero ? 0.f : exp2f((float)E - hx);
  sc = __int_as_float(max(0, 127 - E) << 23);
}

// Rescale of one scaled recurrence after a chunk of 8 steps (8 steps grow it by at most 2^43 for
// |x| <= xcut, so it stays far below the FP32 limit).
__device__ __forceinline__ void herm_rescale(float& p, float& pp, int& E, float& sc) {
  if (fabsf(p) > 1.8446744e19f) {  // 2^64
    p *= 5.421011e-20f;
    pp *= 5.421011e-20f;
    E -= 64;
    sc = __int_as_float(max(0, 127 - E) << 23);
  }
}

// Two rows as one f32x2 recurrence: {g_r0, g_r1}' = {e,e} {x0,x1} {g_r0,g_r1} - {g'_r0,g'_r1}.
template <bool SCALED, bool TF32>
__device__ __forceinline__ void produce2_run(float2 X, float2 P, float2 Sc, int E0, int E1, int kp, unsigned char* a_base,
                                             int blk, int lo_off, bool split, int row, const float4* cab) {
  float2 Pp = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int k0 = 0; k0 < kp; k0 += 8) {
    float v[2][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 w = SCALED ? __fmul2_rn(P, Sc) : P;
      v[0][i] = w.x;
      v[1][i] = w.y;
      const float4 c = cab[k0 + i];
      const float2 Pn = __ffma2_rn(__fmul2_rn(make_float2(c.x, c.y), X), P, make_float2(-Pp.x, -Pp.y));
      Pp = P;
      P = Pn;
    }
    if (SCALED) {
      herm_rescale(P.x, Pp.x, E0, Sc.x);
      herm_rescale(P.y, Pp.y, E1, Sc.y);
    }
    store_row8<TF32>(v[0], a_base, lo_off, split, row, k0);
    store_row8<TF32>(v[1], a_base + blk, lo_off, split, row, k0);
  }
}

// One row, scalar recurrence (the constants e_n four at a time from shared memory).
template <bool SCALED, bool TF32>
__device__ __forceinline__ void produce1_run(float x, float p, float sc, int E, int kp, unsigned char* a_base, int lo_off,
                                             bool split, int row, const float4* ca) {
  float pp = 0.f;
#pragma unroll 1
  for (int k0 = 0; k0 < kp; k0 += 8) {
    const float4 A0 = ca[k0 >> 2], A1 = ca[(k0 >> 2) + 1];
    const float av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v[i] = SCALED ? p * sc : p;
      const float pn = fmaf(av[i] * x, p, -pp);
      pp = p;
      p = pn;
    }
    if (SCALED) herm_rescale(p, pp, E, sc);
    store_row8<TF32>(v, a_base, lo_off, split, row, k0);
  }
}

// Rows r of this thread go to row `row` of block r (a_base + r * blk).  The scaled form is taken for
// both rows when either needs it (it is exact for every x).
template <int R, bool TF32>
__device__ __forceinline__ void produce_rows(const float (&x)[R], int nmax, int kp, const bool (&valid)[R],
                                             unsigned char* a_base, int blk, int lo_off, bool split, int row,
                                             const float4* ca, const float4* cab) {
  const float xcut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;
  bool zero[R], fast = true;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float ax = fabsf(x[r]);
    zero[r] = !valid[r] || !(ax <= xcut);
    fast = fast && (zero[r] || ax <= 12.5f);
  }
  float p[R], sc[R];
  int E[R];
#pragma unroll
  for (int r = 0; r < R; ++r) herm_seed(x[r], zero[r], fast, p[r], E[r], sc[r]);
  if constexpr (R == 2) {
    const float2 X = make_float2(x[0], x[1]), P = make_float2(p[0], p[1]), Sc = make_float2(sc[0], sc[1]);
    if (fast) produce2_run<false, TF32>(X, P, Sc, E[0], E[1], kp, a_base, blk, lo_off, split, row, cab);
    else produce2_run<true, TF32>(X, P, Sc, E[0], E[1], kp, a_base, blk, lo_off, split, row, cab);
  } else {
    if (fast) produce1_run<false, TF32>(x[0], p[0], sc[0], E[0], kp, a_base, lo_off, split, row, ca);
    else produce1_run<true, TF32>(x[0], p[0], sc[0], E[0], kp, a_base, lo_off, split, row, ca);
  }
}

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

template <int R>
__device__ __forceinline__ void produce_rows_lut(const float (&x)[R], int nmax, int kp, const bool (&valid)[R],
                                                 unsigned char* a_base, int blk, int lo_off, bool split, int row,
                                                 const float* lut) {
  const float xcut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;
  int ip[R];
  float tw[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ip[r] = lut_pos(x[r], valid[r], xcut, tw[r]);
#pragma unroll 1
  for (int k0 = 0; k0 < kp; k0 += 8) {
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
      store_row8<false>(v, a_base + r * blk, lo_off, split, row, k0);
    }
  }
}

// Epilogue dot product of one accumulator chunk (16 columns: 2 n2, 2 n2 + 1 = Re, Im for 8 n2) with
// g_n2(y), advancing the y recurrence.  SCALED: values carry 2^E as in the producers.
template <bool SCALED>
__device__ __forceinline__ void epi_chunk(const uint32_t* t, const float4* ca, int n0, float y,
                                          float& q, float& q_prev, float& xr, float& xi, int& E, float& scale) {
#pragma unroll
  for (int g4 = 0; g4 < 2; ++g4) {
    const float4 A = ca[(n0 >> 2) + g4];
    const float av[4] = {A.x, A.y, A.z, A.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * g4 + u;
      const float ph = SCALED ? q * scale : q;
      xr = fmaf(__uint_as_float(t[2 * i]), ph, xr);
      xi = fmaf(__uint_as_float(t[2 * i + 1]), ph, xi);
      const float qn = fmaf(av[u] * y, q, -q_prev);
      q_prev = q;
      q = qn;
    }
  }
  if (SCALED) herm_rescale(q, q_prev, E, scale);
}

// Epilogue of two rows at once: their y recurrences as one f32x2 recurrence (scaled per lane when
// SCALED), each row's accumulator chunk against its half of the pair.
template <bool SCALED>
__device__ __forceinline__ void epi_chunk2(const uint32_t* t0, const uint32_t* t1, const float4* cab, int n0, float2 Y,
                                           float2& Q, float2& Qp, float2& Sc, int& E0, int& E1, float (&xr)[2],
                                           float (&xi)[2]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 w = SCALED ? __fmul2_rn(Q, Sc) : Q;
    xr[0] = fmaf(__uint_as_float(t0[2 * i]), w.x, xr[0]);
    xi[0] = fmaf(__uint_as_float(t0[2 * i + 1]), w.x, xi[0]);
    xr[1] = fmaf(__uint_as_float(t1[2 * i]), w.y, xr[1]);
    xi[1] = fmaf(__uint_as_float(t1[2 * i + 1]), w.y, xi[1]);
    const float4 c = cab[n0 + i];
    const float2 Qn = __ffma2_rn(__fmul2_rn(make_float2(c.x, c.y), Y), Q, make_float2(-Qp.x, -Qp.y));
    Qp = Q;
    Q = Qn;
  }
  if (SCALED) {
    herm_rescale(Q.x, Qp.x, E0, Sc.x);
    herm_rescale(Q.y, Qp.y, E1, Sc.y);
  }
}

// Epilogue dot product of one 16-column chunk with table-interpolated g_n2(y), n2 = n0 .. n0 + 7.
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

// A thread's position in the visibility array, as (row, channel): visibility row * n_chan + f.  It exists
// (is below n_vis) exactly when row < n_rows.  Moving to the thread's next tile adds a fixed number of
// rows and channels, so no per-visibility division is needed.
struct VisCur {
  int row, f;
};

__device__ __forceinline__ VisCur vc_start(long long vis, int n_chan) {
  VisCur c;
  const long long row = vis / n_chan;
  c.row = (int)min(row, (long long)0x7fffffff);
  c.f = (int)(vis - row * n_chan);
  return c;
}

__device__ __forceinline__ void vc_next(VisCur& c, const K2Args& a) {
  c.row += a.step_row;
  c.f += a.step_f;
  if (c.f >= a.n_chan) {
    c.f -= a.n_chan;
    ++c.row;
  }
}

// Weight of an item's dot product at one visibility, S(nu) e^{-2 pi i tau nu / c} (eq:shape-env,
// eq:measure_eq_discrete): the shapelet's spectrum and the phasor of its centre.
__device__ __forceinline__ float2 k2_weight(const K2Shape& s, float tau_h, float tau_l, const float4& ci) {
  const float2 P = phasor_fast(reduce_turns(tau_h, tau_l, ci.x, ci.y));
  const float amp = s.sgn * ex2_approx(fmaf(s.alpha, ci.z, s.c_amp));
  return make_float2(amp * P.x, amp * P.y);
}

// z (+)= (xr + i xi) W
__device__ __forceinline__ float2 k2_sum(float2 z, bool first, float2 W, float xr, float xi) {
  const float zr = xr * W.x - xi * W.y, zi = xr * W.y + xi * W.x;
  return first ? make_float2(zr, zi) : make_float2(z.x + zr, z.y + zi);
}

// The output of one visibility from the sum z of its shapelets' contributions: stored, added to the
// output, or subtracted as G z from the data or the output (Sec. 5.1).  k2_base_load issues the loads
// (existing output or data, gain product), k2_store forms and writes it.
struct K2Base {
  float2 base, G;
};

__device__ __forceinline__ void k2_base_load(const K2Args& a, VisCur c, K2Base& b) {
  b.base = make_float2(0.f, 0.f);
  b.G = make_float2(0.f, 0.f);
  if (c.row >= a.n_rows) return;
  const size_t vis = (size_t)c.row * a.n_chan + c.f;
  if (a.mode != OUT_STORE) b.base = a.mode == OUT_PEEL ? a.peel.data[vis] : a.out[vis];
  if (a.mode >= OUT_PEEL) {
    if (a.rowg) b.G = __ldg(a.rowg + c.row);
    else if (!gain_product(a.peel, c.row, a.n_base, c.f, b.G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
  }
}

__device__ __forceinline__ void k2_store(const K2Args& a, VisCur c, const K2Base& b, float2 z) {
  if (c.row >= a.n_rows) return;
  const size_t vis = (size_t)c.row * a.n_chan + c.f;
  if (a.mode == OUT_STORE) a.out[vis] = z;
  else if (a.mode == OUT_ACCUM) a.out[vis] = make_float2(b.base.x + z.x, b.base.y + z.y);
  else a.out[vis] = make_float2(b.base.x - (b.G.x * z.x - b.G.y * z.y), b.base.y - (b.G.x * z.y + b.G.y * z.x));
}

// The K steps of one product into accumulator d: ks MMAs, the first overwriting d when `first`.
template <bool TF32, int KS>
__device__ __forceinline__ void k2_mma_run(uint32_t lead, uint32_t d, uint64_t da, uint64_t db, uint64_t sa, uint64_t sb,
                                           uint32_t idesc, bool first) {
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
    if constexpr (TF32) umma_tf32_by(lead, d, da + kk * sa, db + kk * sb, idesc, acc);
    else umma_bf16_by(lead, d, da + kk * sa, db + kk * sb, idesc, acc);
  }
}

template <bool TF32>
__device__ __forceinline__ void k2_mma_ksteps(uint32_t lead, uint32_t d, uint64_t da, uint64_t db, uint64_t sa, uint64_t sb,
                                              uint32_t idesc, int ks, bool first) {
  switch (ks) {  // k_pad / 16 (bf16) or k_pad / 8 (tf32), k_pad a multiple of 16 up to 128
    case 1: return k2_mma_run<TF32, 1>(lead, d, da, db, sa, sb, idesc, first);
    case 2: return k2_mma_run<TF32, 2>(lead, d, da, db, sa, sb, idesc, first);
    case 3: return k2_mma_run<TF32, 3>(lead, d, da, db, sa, sb, idesc, first);
    case 4: return k2_mma_run<TF32, 4>(lead, d, da, db, sa, sb, idesc, first);
    case 5: return k2_mma_run<TF32, 5>(lead, d, da, db, sa, sb, idesc, first);
    case 6: return k2_mma_run<TF32, 6>(lead, d, da, db, sa, sb, idesc, first);
    case 7: return k2_mma_run<TF32, 7>(lead, d, da, db, sa, sb, idesc, first);
    case 8: return k2_mma_run<TF32, 8>(lead, d, da, db, sa, sb, idesc, first);
    default:
      for (int kk = 0; kk < ks; ++kk) {
        const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
        if constexpr (TF32) umma_tf32_by(lead, d, da + kk * sa, db + kk * sb, idesc, acc);
        else umma_bf16_by(lead, d, da + kk * sa, db + kk * sb, idesc, acc);
      }
  }
}

// FORM: 0 = bf16 operands, basis by the recurrence; 1 = bf16, basis from the lookup table; 2 = tf32.
template <int R, int FORM>
__global__ void __launch_bounds__(K2_THREADS, 1) k2_shapelet(const K2Args a) {
  constexpr bool LUT = FORM == 1, TF32 = FORM == 2;
  constexpr int TV = K2_M * R;  // visibilities per tile
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ng = a.groups;  // tile parities in flight (2, or 1 when two A buffers do not fit)
  const int S = a.n_shape;
  const K2Layout lay = k2_layout(a.b_total, a.kp_max, a.passes, ng, R, TF32);
  const int blk = lay.a_bytes / R;                      // one 128-row block of A (hi [+ lo])
  const int lo_off = a.kp_max * K2_M * (TF32 ? 4 : 2);  // its lo tile follows its hi tile
  uint64_t* bfull = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* afull = bfull + 1;                // [parity] producer -> MMA: A written
  uint64_t* mdone = afull + K2_GROUPS;        // [parity] MMA -> producer/epilogue: MMA complete
  uint64_t* tfree = mdone + K2_GROUPS;        // [parity] epilogue -> MMA: TMEM read
  uint64_t* xfull = tfree + K2_GROUPS;        // [parity] epilogue -> producers: dot products written
  uint64_t* xempty = xfull + K2_GROUPS;       // [parity] producers -> epilogue: dot products read
  uint32_t* tslot = reinterpret_cast<uint32_t*>(xempty + K2_GROUPS);
  K2Shape* shs = reinterpret_cast<K2Shape*>(smem + lay.shp);
  // warp index and TMEM base broadcast from lane 0, so that the compiler sees them as warp-uniform (they feed
  // the operands of the warp's tcgen05 instructions)
  const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
  const int acc_cols = a.np_max * ng * R;
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
    // the rescaled recurrence's constants e_n (uploaded synchronously at context creation, so every launch
    // on any stream reads them complete): singly for the one-row path, as {e, e} pairs for the f32x2 path
    const float e = c_k2e[threadIdx.x];
    float* cf = reinterpret_cast<float*>(smem + lay.coef);
    cf[threadIdx.x] = e;
    cf[kNmaxLimit + 1 + threadIdx.x] = 0.f;
    reinterpret_cast<float4*>(cf + 2 * (kNmaxLimit + 1))[threadIdx.x] = make_float4(e, e, 0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < K2_MAXS; ++q)
    if (threadIdx.x == 160 + q && q < S) shs[q] = a.sh[q];
  if (warp == K2_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = __shfl_sync(0xffffffffu, *tslot, 0);
  const float4* ca = reinterpret_cast<const float4*>(smem + lay.coef);
  const float4* cab = ca + 2 * ((kNmaxLimit + 1) / 4);  // {e_n, e_n, 0, 0}
  // Tiles of this CTA: i = 0, 1, 2, ... -> tile blockIdx.x + i * gridDim.x, on parity i % ng.  A parity's
  // items are its tiles' (tile, shapelet) pairs in order: item jj is shapelet jj % S of its tile jj / S.
  const int n_it = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto n_items = [&](int sp) { return (n_it > sp ? (n_it - 1 - sp) / ng + 1 : 0) * S; };
  auto first_vis = [&](int sp, int r) {
    return (long long)(blockIdx.x + sp * gridDim.x) * TV + r * K2_M + (threadIdx.x & 127);
  };

  if (warp == K2_MMA_WARP) {
    // ---------------- TMA of the coefficient operands, then the MMA issue loop ----------------
    // The whole warp runs the loop (warp-uniform descriptors); the elected lane issues.
    const uint32_t lead = elect_lane();
    if (lead) {
      uint32_t tx = 0;
      for (int q = 0; q < S; ++q) tx += (uint32_t)shs[q].b_bytes;
      mbar_arrive_expect_tx(bfull, tx);
      for (int q = 0; q < S; ++q) tma_bulk_g2s(smem + shs[q].b_smem, shs[q].bop, (uint32_t)shs[q].b_bytes, bfull);
    }
    __syncwarp();
    const uint32_t lbo_a = (uint32_t)(K2_M >> 3) << 7;
    bool ok = __all_sync(0xffffffffu, k2_wait(bfull, 0, a.err));
    const int len0 = n_items(0), len1 = ng > 1 ? n_items(1) : 0;
    int done0 = 0, done1 = 0;  // items issued per parity
    // the parities alternate item by item, so that one parity's MMA runs while the other's epilogue reads
    for (int jj = 0; ok && jj < max(len0, len1); ++jj) {
      for (int sp = 0; sp < ng; ++sp) {
        if (jj >= (sp ? len1 : len0)) continue;
        const K2Shape& sh = shs[jj % S];
        const int b_smem = __shfl_sync(0xffffffffu, sh.b_smem, 0), k_pad = __shfl_sync(0xffffffffu, sh.k_pad, 0);
        const int n_pad = __shfl_sync(0xffffffffu, sh.n_pad, 0);
        ok = __all_sync(0xffffffffu, k2_wait(&afull[sp], jj & 1, a.err) &&
                                         (jj == 0 || k2_wait(&tfree[sp], (jj - 1) & 1, a.err)));
        if (!ok) break;
        tc_fence_after();
        const uint32_t b_hi = smem_u32(smem + b_smem);
        const uint32_t b_lo = b_hi + (uint32_t)(k_pad * n_pad * (TF32 ? 4 : 2));  // lo follows hi
        const uint32_t lbo_b = (uint32_t)(n_pad >> 3) << 7;
        const uint32_t idesc = TF32 ? umma_idesc_tf32(n_pad) : umma_idesc_bf16(n_pad);
        const int ksteps = k_pad / (TF32 ? 8 : 16);
        // A K step (16 bf16 or 8 tf32: two core matrices) moves an operand's start address by 2 LBO; the
        // descriptors hold it in 16-byte units in their low bits, which stay below 2^14 (shared memory is
        // under 256 KB), so a step is an addition to the descriptor
        const uint64_t db_hi = umma_desc(b_hi, lbo_b, 128), db_lo = umma_desc(b_lo, lbo_b, 128);
        const uint64_t sa = (2 * lbo_a) >> 4, sb = (2 * lbo_b) >> 4;
#pragma unroll
        for (int r = 0; r < R; ++r) {  // block r of the tile into accumulator sp * R + r
          const uint32_t a_hi = smem_u32(smem + lay.a0 + sp * lay.a_bytes + r * blk);
          const uint64_t da_hi = umma_desc(a_hi, lbo_a, 128), da_lo = umma_desc(a_hi + (uint32_t)lo_off, lbo_a, 128);
          const uint32_t d = tmem + (uint32_t)((sp * R + r) * a.np_max);
#pragma unroll 1
          for (int p = 0; p < a.passes; ++p)  // one product, or hi*hi, hi*lo, lo*hi
            k2_mma_ksteps<TF32>(lead, d, p == 2 ? da_lo : da_hi, p == 1 ? db_lo : db_hi, sa, sb, idesc, ksteps, p == 0);
        }
        umma_commit_by(lead, &mdone[sp]);
        (sp ? done1 : done0) = jj + 1;
      }
    }
    // drain: the last commit of each parity has landed before teardown
    if (done0 > 0) k2_wait(&mdone[0], (done0 - 1) & 1, a.err);
    if (done1 > 0) k2_wait(&mdone[1], (done1 - 1) & 1, a.err);
    __syncwarp();
  } else if (warp < 4 * K2_GROUPS) {
    // ---------------- producers: g_n(x) into the parity's A buffer ----------------
    const int sp = warp >> 2;
    if (sp >= ng) goto done;
    const int m = threadIdx.x & 127;
    unsigned char* a_base = smem + lay.a0 + sp * lay.a_bytes;
    const int len = n_items(sp);
    const float2* xfer = reinterpret_cast<const float2*>(smem + lay.xfer) + sp * R * K2_M + m;
    VisCur cur[R];  // the tile of the item being produced
#pragma unroll
    for (int r = 0; r < R; ++r) cur[r] = vc_start(first_vis(sp, r), a.n_chan);
    // this item's (xs, nu), loaded one item ahead
    auto load_x = [&](const VisCur (&c)[R], int q, float (&xs)[R], float (&nu)[R]) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const bool v = c[r].row < a.n_rows;
        xs[r] = v ? __ldg(&a.rowinfo[(size_t)q * a.n_rows + c[r].row].x) : 0.f;
        nu[r] = v ? __ldg(&a.chaninfo[c[r].f].w) : 0.f;
      }
    };
    float xs[R], nu[R];
    load_x(cur, 0, xs, nu);
    // The output step of an item: its weight times the epilogue's dot products, summed over the tile's
    // items; the tile's output once its last item is in.  The loads are issued first and arrive while
    // the epilogue finishes.
    float2 z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) z[r] = make_float2(0.f, 0.f);
    auto out_item = [&](const VisCur (&c)[R], int q, int jo) -> bool {
      const bool last = q == S - 1;
      float4 ri[R], ci[R];
      K2Base b[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const bool v = c[r].row < a.n_rows;
        ri[r] = v ? __ldg(a.rowinfo + (size_t)q * a.n_rows + c[r].row) : make_float4(0.f, 0.f, 0.f, 0.f);
        ci[r] = v ? __ldg(a.chaninfo + c[r].f) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (last) k2_base_load(a, c[r], b[r]);
      }
      if (!k2_wait(&xfull[sp], jo & 1, a.err)) return false;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 d = xfer[r * K2_M];
        z[r] = k2_sum(z[r], q == 0, k2_weight(shs[q], ri[r].z, ri[r].w, ci[r]), d.x, d.y);
      }
      mbar_arrive(&xempty[sp]);
      if (last) {
#pragma unroll
        for (int r = 0; r < R; ++r) k2_store(a, c[r], b[r], z[r]);
      }
      return true;
    };
    VisCur pc[R];  // the tile of the item whose output is pending
    int q = 0, pq = -1;
    for (int jj = 0; jj < len; ++jj) {
      float x[R];
      bool v0[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        x[r] = xs[r] * nu[r];
        v0[r] = cur[r].row < a.n_rows;
      }
      const int kp = shs[q].k_pad, nmax = shs[q].nmax;
      // the next item: the next shapelet of this tile, or the first of the parity's next tile
      VisCur nc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) nc[r] = cur[r];
      int nq = q + 1;
      if (nq == S) {
        nq = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) vc_next(nc[r], a);
      }
      if (jj + 1 < len) load_x(nc, nq, xs, nu);
      if (jj > 0 && !k2_wait(&mdone[sp], (jj - 1) & 1, a.err)) break;  // MMA(jj-1) has read A
      if (LUT) produce_rows_lut<R>(x, nmax, kp, v0, a_base, blk, lo_off, a.passes > 1, m, a.lut);
      else produce_rows<R, TF32>(x, nmax, kp, v0, a_base, blk, lo_off, a.passes > 1, m, ca, cab);
      fence_async_smem();
      mbar_arrive(&afull[sp]);
      // the previous item's output, while the MMA of this one runs
      if (jj > 0 && !out_item(pc, pq, jj - 1)) {
        pq = -1;
        break;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        pc[r] = cur[r];
        cur[r] = nc[r];
      }
      pq = q;
      q = nq;
    }
    if (pq >= 0 && len > 0) out_item(pc, pq, len - 1);
  } else {
    // ---------------- epilogues: xi = sum_n2 T[., n2] g_n2(y), handed to the producers ----------------
    const int sp = (warp - 4 * K2_GROUPS) >> 2;
    if (sp >= ng) goto done;
    const int m = threadIdx.x & 127;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(sp * R * a.np_max);
    float2* xfer = reinterpret_cast<float2*>(smem + lay.xfer) + sp * R * K2_M + m;
    const int len = n_items(sp);
    VisCur cur[R];
#pragma unroll
    for (int r = 0; r < R; ++r) cur[r] = vc_start(first_vis(sp, r), a.n_chan);
    // per item: the row table's ys and the channel's nu, loaded one item ahead
    auto load_y = [&](const VisCur (&c)[R], int q, float (&ys)[R], float (&nu)[R]) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const bool v = c[r].row < a.n_rows;
        ys[r] = v ? __ldg(&a.rowinfo[(size_t)q * a.n_rows + c[r].row].y) : 0.f;
        nu[r] = v ? __ldg(&a.chaninfo[c[r].f].w) : 1.f;
      }
    };
    float ys[R], nu[R];
    load_y(cur, 0, ys, nu);
    int q = 0;
    for (int jj = 0; jj < len; ++jj) {
      bool valid[R];
      float y[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        valid[r] = cur[r].row < a.n_rows;
        y[r] = ys[r] * nu[r];
      }
      const int n_pad = __shfl_sync(0xffffffffu, shs[q].n_pad, 0), nmax = shs[q].nmax;
      VisCur nc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) nc[r] = cur[r];
      int nq = q + 1;
      if (nq == S) {
        nq = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) vc_next(nc[r], a);
      }
      if (!k2_wait(&mdone[sp], jj & 1, a.err)) break;
      if (jj + 1 < len) load_y(nc, nq, ys, nu);  // the next item's entries in flight
      tc_fence_after();
      const float ycut = sqrtf(2.0f * nmax + 1.0f) + 10.0f;
      float qv[R], q_prev[R], scale[R], xr[R], xi[R];
      int E[R];
      bool yfast = true, yzero[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        yzero[r] = !valid[r] || !(fabsf(y[r]) <= ycut);
        yfast = yfast && (yzero[r] || fabsf(y[r]) <= 12.5f);
        xr[r] = xi[r] = 0.f;
        q_prev[r] = 0.f;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) herm_seed(y[r], yzero[r], yfast, qv[r], E[r], scale[r]);
      // accumulator rows in chunks of 16 columns (8 n2).  Once the last chunk's loads have completed the
      // accumulator is released to the MMA warp (tfree), before that chunk is used.
      const int nch = n_pad >> 4;
      bool released = false;
      auto release = [&]() {
        tc_fence_before();
        mbar_arrive(&tfree[sp]);
        released = true;
      };
      if (LUT) {  // table-interpolated g_n2(y): one chunk of every row at a time
        int iy[R];
        float ty[R];
#pragma unroll
        for (int r = 0; r < R; ++r) iy[r] = lut_pos(y[r], valid[r], ycut, ty[r]);
        uint32_t tb[R][16];
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
#pragma unroll
          for (int r = 0; r < R; ++r) tmem_issue16x(trow + (uint32_t)(r * a.np_max + (c << 4)), tb[r]);
#pragma unroll
          for (int r = 0; r < R; ++r) tmem_wait16(tb[r]);
          if (c == nch - 1) release();
#pragma unroll
          for (int r = 0; r < R; ++r) epi_chunk_lut(tb[r], a.lut, iy[r], ty[r], c << 3, xr[r], xi[r]);
        }
      } else if constexpr (R == 1) {  // one row: the next chunk's load in flight while one is used
        uint32_t tb0[16], tb1[16];
        tmem_issue16x(trow, tb0);
        tmem_wait16(tb0);
#pragma unroll 1
        for (int c = 0; c < nch; c += 2) {
          if (c + 1 < nch) tmem_issue16x(trow + (uint32_t)((c + 1) << 4), tb1);
          if (yfast) epi_chunk<false>(tb0, ca, c << 3, y[0], qv[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
          else epi_chunk<true>(tb0, ca, c << 3, y[0], qv[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
          tmem_wait16(tb1);
          if (c + 1 < nch) {
            if (c + 2 < nch) tmem_issue16x(trow + (uint32_t)((c + 2) << 4), tb0);
            if (yfast) epi_chunk<false>(tb1, ca, (c + 1) << 3, y[0], qv[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
            else epi_chunk<true>(tb1, ca, (c + 1) << 3, y[0], qv[0], q_prev[0], xr[0], xi[0], E[0], scale[0]);
            tmem_wait16(tb0);
          }
        }
      } else {
        // Two rows: a 16-column chunk of each in flight, their y recurrences as one f32x2 recurrence.  The
        // TMEM loads are warp-collective (.sync.aligned): every thread issues them in the same order
        // whatever its rows need; only the arithmetic below depends on the thread.
        uint32_t tb[2][16];
        float2 Q = make_float2(qv[0], qv[1]), Qp = make_float2(0.f, 0.f), Sc = make_float2(scale[0], scale[1]);
        const float2 Y = make_float2(y[0], y[1]);
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
          tmem_issue16x(trow + (uint32_t)(c << 4), tb[0]);
          tmem_issue16x(trow + (uint32_t)(a.np_max + (c << 4)), tb[1]);
          tmem_wait16(tb[0]);
          tmem_wait16(tb[1]);
          if (c == nch - 1) release();
          if (yfast) epi_chunk2<false>(tb[0], tb[1], cab, c << 3, Y, Q, Qp, Sc, E[0], E[1], xr, xi);
          else epi_chunk2<true>(tb[0], tb[1], cab, c << 3, Y, Q, Qp, Sc, E[0], E[1], xr, xi);
        }
      }
      if (!released) release();
      if (jj > 0 && !k2_wait(&xempty[sp], (jj - 1) & 1, a.err)) break;  // the producers have read item jj-1's
#pragma unroll
      for (int r = 0; r < R; ++r) xfer[r * K2_M] = valid[r] ? make_float2(xr[r], xi[r]) : make_float2(0.f, 0.f);
      mbar_arrive(&xfull[sp]);
#pragma unroll
      for (int r = 0; r < R; ++r) cur[r] = nc[r];
      q = nq;
    }
  }
done:
  __syncthreads();
  if (warp == K2_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Per-launch prep (FP64, tiny): per-channel constants and, for a run of shapelets, per-row constants.
__global__ void k2_chaninfo(const double* freq, int n_chan, double nu0, float4* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_chan) return;
  const double nu = freq[f], a = nu / kC;
  const float ah = __double2float_rn(a);
  out[f] = make_float4(ah, __double2float_rn(a - (double)ah), (float)log2(nu / nu0), (float)nu);
}

// Row table of shapelet sh[blockIdx.y], written at out + blockIdx.y * n_rows.
__global__ void k2_rowinfo(const double* uvw, int n_rows, const ShapeRec* sh, double sd0, double cd0, float4* out) {
  __shared__ double F[9];
  const ShapeRec* s = sh + blockIdx.y;
  if (threadIdx.x == 0) shapelet_frame(s->l, s->m, sd0, cd0, F);
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const double u = uvw[3 * (size_t)r], v = uvw[3 * (size_t)r + 1], w = uvw[3 * (size_t)r + 2];
  const double up = F[0] * u + F[1] * v + F[2] * w, vp = F[3] * u + F[4] * v + F[5] * w;
  const double xs = ((double)s->kx_u * up + (double)s->kx_v * vp) / kC;
  const double ys = ((double)s->ky_u * up + (double)s->ky_v * vp) / kC;
  const double tau = u * s->l + v * s->m + w * s->nm1;
  const float th = __double2float_rn(tau);
  out[(size_t)blockIdx.y * n_rows + r] = make_float4((float)xs, (float)ys, th, __double2float_rn(tau - (double)th));
}

// Per-row gain product of a peel with frequency-independent gains: G[row] = g[tg][0][ant1] conj(g[tg][0][ant2]),
// NaN (and the antenna flag) for an antenna index out of range, as the output step would form it.
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

template <int R, int FORM>
static cudaError_t k2_launch_t(const K2Args& a, int grid, int smem, cudaStream_t st) {
  auto fn = k2_shapelet<R, FORM>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(fn));
  if (e != cudaSuccess) return e;
  fn<<<grid, K2_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t k2_dispatch(const K2Args& a, int R, int form, int grid, int smem, cudaStream_t st) {
  if (R == 2) {
    if (form == 1) return k2_launch_t<2, 1>(a, grid, smem, st);
    if (form == 2) return k2_launch_t<2, 2>(a, grid, smem, st);
    return k2_launch_t<2, 0>(a, grid, smem, st);
  }
  if (form == 1) return k2_launch_t<1, 1>(a, grid, smem, st);
  if (form == 2) return k2_launch_t<1, 2>(a, grid, smem, st);
  return k2_launch_t<1, 0>(a, grid, smem, st);
}

// The basis table of the lookup-table mode: g_n = k_n phi_n, n = 0..127 (herm_k), with phi_n in FP64 by
// the normalised recurrence at every sample, stored in FP32.  Built once per context.
__global__ void k2_lut_build(float* lut) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K2_LUT_N) return;
  const double x = -(double)K2_LUT_X + (double)i / K2_LUT_D;
  double p_prev = 0.0, p = exp(-0.5 * x * x);
  for (int n = 0; n < K2_LUT_W; ++n) {
    lut[(size_t)i * K2_LUT_W + n] = (float)(p * herm_k(n));
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

// Launch shape of a run of shapelets whose operands take b_total bytes: two rows per thread and two tile
// parities when both parities' doubled A buffers and 4 n_pad TMEM columns fit, else one row, else one
// parity.
struct K2Plan {
  int R = 0, groups = 0, smem = 0;
};

static bool k2_plan(int b_total, int kp_max, int np_max, int passes, bool tf32, K2Plan& p) {
  const int opts[3][2] = {{2, K2_GROUPS}, {1, K2_GROUPS}, {1, 1}};
  for (const auto& o : opts) {
    if (o[0] == 2 && np_max > 128) continue;
    const K2Layout L = k2_layout(b_total, kp_max, passes, o[1], o[0], tf32);
    if (L.total <= 227 * 1024) {
      p.R = o[0];
      p.groups = o[1];
      p.smem = L.total;
      return true;
    }
  }
  return false;
}

// Shapelet launches with caller-supplied tables: per-channel (n_chan float4) and per-row (rowinfo_cap
// float4, at least n_rows).  The model's shapelets are summed in runs: a run grows while its operands
// fit in shared memory beside the same launch shape, its row tables fit in rowinfo, and it has at most
// K2_MAXS shapelets.  Each run is one launch that writes the output once; the first applies the caller's
// mode and the later ones add (or subtract G times) their sums.
int launch_shapelets_ws(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        float4* chaninfo, float4* rowinfo, size_t rowinfo_cap, cudaStream_t st, float2* rowg) {
  if (M->n_shape == 0) return WN_OK;
  if (rowinfo_cap < (size_t)o.n_rows)
    return set_error(WN_EINVAL, "shapelet row tables: room for " + std::to_string(rowinfo_cap) + " rows, " +
                                    std::to_string(o.n_rows) + " needed");
  k2_chaninfo<<<(o.n_chan + 255) / 256, 256, 0, st>>>(o.freq, o.n_chan, o.nu0, chaninfo);
  const long long n_vis = (long long)o.n_rows * o.n_chan;
  const bool tf32 = ctx->shape_mode == WN_SHAPE_TF32 || ctx->shape_mode == WN_SHAPE_TF32X3;
  const int passes = ctx->shape_mode == WN_SHAPE_BF16X1 || ctx->shape_mode == WN_SHAPE_TF32 ? 1 : 3;
  const int form = ctx->shape_mode == WN_SHAPE_LUT_BF16X3 ? 1 : (tf32 ? 2 : 0);
  const float* lut = nullptr;
  if (form == 1)
    if (int r = k2_lut(ctx, st, &lut)) return r;
  const double L0 = std::log2(o.nu0);
  const bool peeling = mode == OUT_PEEL || mode == OUT_SUBG;
  if (rowg && (!peeling || pa.gf != 1)) rowg = nullptr;
  if (rowg) k2_rowgain<<<(o.n_rows + 255) / 256, 256, 0, st>>>(pa, o.n_rows, o.n_base, rowg, ctx->d_err);
  const int max_run = (int)std::min<size_t>(K2_MAXS, rowinfo_cap / (size_t)o.n_rows);
  auto b_smem_bytes = [&](const ShapeRec& h) { return (k2_b_bytes(h.k_pad, h.n_pad, passes, tf32) + 1023) & ~1023; };
  int run = 0;
  for (int q0 = 0; q0 < M->n_shape; q0 += run) {  // the run starting at q0
    const ShapeRec& h0 = M->sh_host[q0];
    int b_total = b_smem_bytes(h0), kp = h0.k_pad, np = h0.n_pad;
    K2Plan plan;
    if (!k2_plan(b_total, kp, np, passes, tf32, plan))
      return set_error(WN_EINVAL, "shapelet operand of orders up to " + std::to_string(h0.nmax) + " (k_pad " +
                                      std::to_string(h0.k_pad) + ", n_pad " + std::to_string(h0.n_pad) +
                                      ") does not fit in shared memory in this shapelet mode");
    run = 1;
    while (q0 + run < M->n_shape && run < max_run) {
      const ShapeRec& h = M->sh_host[q0 + run];
      K2Plan p2;
      const int bt = b_total + b_smem_bytes(h), kp2 = std::max(kp, h.k_pad), np2 = std::max(np, h.n_pad);
      if (!k2_plan(bt, kp2, np2, passes, tf32, p2) || p2.R != plan.R || p2.groups != plan.groups) break;
      b_total = bt;
      kp = kp2;
      np = np2;
      plan = p2;
      ++run;
    }
    k2_rowinfo<<<dim3((o.n_rows + 255) / 256, run), 256, 0, st>>>(o.uvw, o.n_rows, M->sh + q0, std::sin(o.dec0),
                                                                  std::cos(o.dec0), rowinfo);
    K2Args a;
    a.rowinfo = rowinfo;
    a.chaninfo = chaninfo;
    a.lut = lut;
    a.n_shape = run;
    a.kp_max = kp;
    a.np_max = np;
    a.b_total = b_total;
    int off = 0;
    for (int i = 0; i < K2_MAXS; ++i) {
      K2Shape& s = a.sh[i];
      s = K2Shape{};
      if (i >= run) continue;
      const ShapeRec& h = M->sh_host[q0 + i];
      s.bop = tf32 ? static_cast<const void*>(M->bop32 + h.b_off) : static_cast<const void*>(M->bop + h.b_off);
      s.b_smem = off;
      s.b_bytes = k2_b_bytes(h.k_pad, h.n_pad, passes, tf32);
      off += b_smem_bytes(h);
      s.k_pad = h.k_pad;
      s.n_pad = h.n_pad;
      s.nmax = h.nmax;
      s.c_amp = (float)((double)h.lS + (double)h.alpha * (L0 - h.lref));
      s.alpha = h.alpha;
      s.sgn = h.sgn;
    }
    a.passes = passes;
    a.n_chan = o.n_chan;
    a.n_rows = o.n_rows;
    a.n_base = o.n_base;
    a.n_vis = n_vis;
    a.out = out;
    a.peel = pa;
    a.rowg = rowg;
    a.err = ctx->d_err;
    // the first run applies the caller's mode, the rest add (or subtract G times) their sums
    a.mode = q0 == 0 ? mode : (mode == OUT_STORE ? OUT_ACCUM : (mode == OUT_PEEL ? OUT_SUBG : mode));
    a.groups = plan.groups;
    const int tv = K2_M * plan.R;
    const long long n_tiles = (n_vis + tv - 1) / tv;
    if (n_tiles > 0x7fffffffLL) return set_error(WN_EINVAL, "shapelet launch: too many visibilities");
    a.n_tiles = (int)n_tiles;
    const int grid = (int)std::min<long long>(n_tiles, ctx->num_sms);
    if (grid == 0) continue;
    const long long step = (long long)plan.groups * grid * tv;  // a thread's move between its tiles
    a.step_row = (int)(step / o.n_chan);
    a.step_f = (int)(step % o.n_chan);
    cudaError_t e = k2_dispatch(a, plan.R, form, grid, plan.smem, st);
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet kernel launch: ") + cudaGetErrorString(e));
  }
  return WN_OK;
}

int launch_shapelets(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                     cudaStream_t st) {
  const size_t chan_bytes = ((size_t)o.n_chan * sizeof(float4) + 255) & ~(size_t)255;
  const size_t n_tab = (size_t)std::max(1, std::min(M->n_shape, K2_MAXS));
  const size_t row_bytes = ((size_t)o.n_rows * n_tab * sizeof(float4) + 255) & ~(size_t)255;
  if (int r = ws_reserve(ctx, chan_bytes + row_bytes + (size_t)o.n_rows * sizeof(float2), st)) return r;
  float4* chaninfo = static_cast<float4*>(ctx->ws);
  float4* rowinfo = reinterpret_cast<float4*>(static_cast<char*>(ctx->ws) + chan_bytes);
  float2* rowg = reinterpret_cast<float2*>(static_cast<char*>(ctx->ws) + chan_bytes + row_bytes);
  return launch_shapelets_ws(ctx, o, M, out, mode, pa, chaninfo, rowinfo, (size_t)o.n_rows * n_tab, st, rowg);
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

constexpr size_t kStaticScratchEntries = size_t(1) << 18;  // float4 entries (4 MiB): n_chan (padded to 16) + row tables
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

// The row tables take what the channel table leaves: as many shapelets per launch as fit, at least one.
int launch_shapelets_static(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                            cudaStream_t st) {
  const size_t chan_entries = ((size_t)o.n_chan + 15) & ~(size_t)15;
  if (chan_entries + (size_t)o.n_rows > kStaticScratchEntries)
    return set_error(WN_EINVAL, "wn_predict_static: n_chan (rounded up to 16) + n_time * n_base = " +
                                    std::to_string(chan_entries + (size_t)o.n_rows) + " exceeds the static scratch of " +
                                    std::to_string(kStaticScratchEntries) + " entries");
  float4* base = ctx->static_scratch;
  if (!base) return set_error(WN_ECUDA, "wn_predict_static: the static scratch address was not found at set-up");
  return launch_shapelets_ws(ctx, o, M, out, mode, pa, base, base + chan_entries, kStaticScratchEntries - chan_entries,
                             st, nullptr);
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

namespace wn {
// The constants e_n = sqrt(2/(n+1)) k_(n+1)/k_n of the shapelet kernel's rescaled Hermite recurrence,
// formed in FP64 on the host and uploaded synchronously at context creation (wn_create, the context's
// device current), so that every later launch on any stream reads them complete.
int k2_constants_setup() {
  float e[kNmaxLimit + 1];
  for (int n = 0; n <= kNmaxLimit; ++n) e[n] = (float)(std::sqrt(2.0 / (n + 1)) * herm_k(n + 1) / herm_k(n));
  const cudaError_t err = cudaMemcpyToSymbol(c_k2e, e, sizeof(e));
  if (err != cudaSuccess) return set_error(WN_ECUDA, std::string("shapelet constants: ") + cudaGetErrorString(err));
  return WN_OK;
}
}  // namespace wn
