// K4: adjoint of the fused predict + peel.  For L = sum_vis |D - G V|^2 with G = g_ant1 conj(g_ant2),
//   dL/dp = -2 sum_vis Re( conj(W) dV/dp ),   W = conj(G) R,   R = D - G V.
// The paper fits in image space and gives no derivatives; they follow term by term from
// eq:env_visi_def, eq:gauss-env and eq:shape-env (V_j = S_j xi_j e^{-2 pi i tau_j nu / c}):
//   dV_j/dS_ref = V_j / S_ref,  dV_j/dalpha = ln(nu / nu_ref) V_j,
//   dV_j/dl = -2 pi i (nu/c) (u - w l / n) V_j (likewise m), plus for a shapelet S P (dxi/dx dx/dl +
//             dxi/dy dy/dl): its (u', v') are re-phased to its own centre (Sec. 3.2), so x and y move with it,
//   Gaussian: dxi/dmaj = -2E (nu/c)^2 maj kx^2 xi, dxi/dmin = -2E (nu/c)^2 min ky^2 xi,
//             dxi/dpa = -2E (nu/c)^2 (maj^2 - min^2) kx ky xi   (kx, ky in metres, E = pi^2 / (4 ln 2)),
//   Shapelet: x = beta1 kx, y = beta2 ky;  phi_n' = sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1};
//             dxi/dbeta1 = sum c s phi_a'(x) (x / beta1) phi_b(y),  dxi/dbeta2 = sum c s phi_a(x) phi_b'(y) (y / beta2),
//             dxi/dpa = sum c s [phi_a'(x) beta1 (y / beta2) phi_b(y) - phi_a(x) phi_b'(y) beta2 (x / beta1)],
//             dxi/dc_k = s_k phi_a(x) phi_b(y),  s = (-i)^(a+b).
// Phasors are recomputed, never stored.  Every sum is reduced in a fixed order (per-lane, warp
// butterfly, per-warp slots, per-CTA partials, then FP64 over CTAs), so results are reproducible.
#include <cmath>

#include "wn_internal.cuh"

namespace wn {

constexpr int K4_CT = 32;     // components per CTA: lane j forms comp j's phase argument and sums
constexpr int K4_WARPS = 8;
constexpr int K4_KMAX = 16;   // most channels per lane per pass (strided by 32): 512 channels per pass
constexpr int K4_NG = 7;      // gradient components per point/Gaussian: flux, alpha, l, m, maj, min, pa
constexpr int K4_FLUSH = 32;  // rows per FP32 partial before it is added to the FP64 sum

struct K4Args {
  const float* uvw_pairs;     // [n_rows][6]: (u, v, w) metres as float pairs hi, lo
  const double* freq;
  int n_rows, n_chan, n_base;
  int f_lo, f_cnt;            // channel pass
  double nu0;
  float dnu_h, dnu_l;         // channel spacing / c as a float pair (uniform channels)
  const PGRec* comps;
  const double *flux, *nuref, *gmaj, *gmin, *gpa;  // raw FP64 tables (all components / Gaussians)
  int n_point, n_gauss;
  const float2* resid;
  PeelArgs peel;              // gains and antenna indices (data unused)
  int rows_per_chunk;
  double* partials;           // [chunks][n_pg][K4_NG]
  unsigned* err;
};

// Point / Gaussian gradients.  grid = (component tiles of 32, row chunks); warp w takes rows
// r0 + w, r0 + w + 8, ...; lane l takes channels f_lo + l + 32 k of each row.
template <int KM>
__global__ void __launch_bounds__(K4_WARPS * 32) k4_grad_pg(const K4Args a) {
  __shared__ PGRec comps[K4_CT];
  __shared__ float cjs[K4_CT];  // alpha log2(nu0 / nu_ref): the flux-free log2 amplitude at nu0
  __shared__ double gsum[K4_WARPS][K4_CT][K4_NG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_pg = a.n_point + a.n_gauss;
  const int c0 = blockIdx.x * K4_CT;
  const int ncomp = min(K4_CT, n_pg - c0);
  if (threadIdx.x < ncomp) {
    const PGRec c = a.comps[c0 + threadIdx.x];
    comps[threadIdx.x] = c;
    cjs[threadIdx.x] = c.alpha * (float)(log2(a.nu0) - c.lref);
  }
  __syncthreads();

  // per-lane channel constants: nu/c as a float pair (one FP64 multiply and split), the rest in FP32
  float ah[KM], al[KM], lam[KM], nuc[KM], wg[KM];
  int fch[KM];
  const float inv_nu0 = (float)(1.0 / a.nu0);
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int fi = lane + 32 * k;
    fch[k] = fi < a.f_cnt ? a.f_lo + fi : -1;
    const double nu = a.freq[fch[k] >= 0 ? fch[k] : a.f_lo];
    split_double(nu * (1.0 / kC), ah[k], al[k]);
    lam[k] = log2f((float)nu * inv_nu0);
    nuc[k] = ah[k];
    wg[k] = (float)(kGaussE * kLog2e) * nuc[k] * nuc[k];
  }
  const double L0 = log2(a.nu0);

  // this lane's component (lane j <-> component c0 + j)
  const bool mine = lane < ncomp;
  const int jc = c0 + (mine ? lane : 0);
  const PGRec& me = comps[mine ? lane : 0];
  const bool my_gauss = mine && jc >= a.n_point;
  const double me_l = (double)me.lh + me.ll, me_m = (double)me.mh + me.ml, me_nm1 = (double)me.nh + me.nl;
  const double my_n = 1.0 + me_nm1;
  const float my_ln = (float)(me_l / my_n), my_mn = (float)(me_m / my_n);  // l / n, m / n
  const float my_lnref = (float)((L0 - me.lref) * 0.6931471805599453);  // ln(nu0 / nu_ref)
  const float my_S = mine ? (float)a.flux[jc] : 0.f;
  float my_pa = 0.f, my_maj = 0.f, my_min = 0.f;
  if (my_gauss) {
    const int g = jc - a.n_point;
    my_maj = (float)a.gmaj[g];
    my_min = (float)a.gmin[g];
    my_pa = (float)a.gpa[g];
  }
  const float sp = sinf(my_pa), cp = cosf(my_pa);

  float acc32[K4_NG];
  double acc64[K4_NG];
#pragma unroll
  for (int i = 0; i < K4_NG; ++i) {
    acc32[i] = 0.f;
    acc64[i] = 0.0;
  }

  const int r_lo = blockIdx.y * a.rows_per_chunk;
  const int r_hi = min(a.n_rows, r_lo + a.rows_per_chunk);
  int nrow = 0;
  for (int row = r_lo + warp; row < r_hi; row += K4_WARPS) {
    float xuvw[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) xuvw[i] = __ldg(a.uvw_pairs + 6 * (size_t)row + i);
    // W = conj(G) R for this lane's channels
    float2 W[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      W[k] = make_float2(0.f, 0.f);
      if (fch[k] >= 0) {
        float2 G;
        if (!gain_product(a.peel, row, a.n_base, fch[k], G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
        const float2 R = a.resid[(size_t)row * a.n_chan + fch[k]];
        W[k] = make_float2(G.x * R.x + G.y * R.y, G.x * R.y - G.y * R.x);
      }
    }
    // this lane's component: phase argument (double-float FP32), Gaussian form and the per-row factors
    float th = 0.f, tl = 0.f, q = 0.f, fl = 0.f, fm = 0.f, fmaj = 0.f, fmin = 0.f, fpa = 0.f;
    if (mine) {
      tau_df(xuvw, me, th, tl);
      const float uf = xuvw[0], vf = xuvw[2], wf = xuvw[4];
      fl = -4.0f * (float)kPi * (uf - wf * my_ln);
      fm = -4.0f * (float)kPi * (vf - wf * my_mn);
      if (my_gauss) {
        q = me.ga * uf * uf + me.gb * uf * vf + me.gc * vf * vf;
        const float kx = sp * uf + cp * vf, ky = cp * uf - sp * vf;
        fmaj = 4.0f * (float)kGaussE * my_maj * kx * kx;
        fmin = 4.0f * (float)kGaussE * my_min * ky * ky;
        fpa = 4.0f * (float)kGaussE * (my_maj * my_maj - my_min * my_min) * kx * ky;
      }
    }
    for (int j = 0; j < ncomp; ++j) {
      const float tj = __shfl_sync(0xffffffffu, th, j), tlj = __shfl_sync(0xffffffffu, tl, j);
      const float qj = __shfl_sync(0xffffffffu, q, j);
      const PGRec& c = comps[j];
      // channel sums use the amplitude without the flux: dV/dS_ref = V / S_ref holds for S_ref = 0 too
      const float cj = cjs[j];
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        if (fch[k] < 0) continue;
        const float2 P = phasor_fast(reduce_turns(tj, tlj, ah[k], al[k]));
        const float A = ex2_approx(fmaf(c.alpha, lam[k], cj) - qj * wg[k]);
        const float vr = A * P.x, vi = A * P.y;
        // z = conj(W) V
        const float zr = W[k].x * vr + W[k].y * vi, zi = W[k].x * vi - W[k].y * vr;
        s0 += zr;
        s1 = fmaf(lam[k], zr, s1);
        s2 = fmaf(nuc[k], zi, s2);
        s3 = fmaf(nuc[k] * nuc[k], zr, s3);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if (lane == j) {
        // s1 holds sum log2(nu/nu0) Re z: ln(nu/nu_ref) = ln2 log2(nu/nu0) + ln(nu0/nu_ref)
        acc32[0] += -2.0f * s0;
        acc32[1] += -2.0f * my_S * (0.6931471805599453f * s1 + my_lnref * s0);
        acc32[2] += my_S * fl * s2;
        acc32[3] += my_S * fm * s2;
        acc32[4] += my_S * fmaj * s3;
        acc32[5] += my_S * fmin * s3;
        acc32[6] += my_S * fpa * s3;
      }
    }
    if (++nrow == K4_FLUSH) {
#pragma unroll
      for (int i = 0; i < K4_NG; ++i) {
        acc64[i] += (double)acc32[i];
        acc32[i] = 0.f;
      }
      nrow = 0;
    }
  }
#pragma unroll
  for (int i = 0; i < K4_NG; ++i) gsum[warp][lane][i] = acc64[i] + (double)acc32[i];
  __syncthreads();
  for (int t = threadIdx.x; t < ncomp * K4_NG; t += blockDim.x) {
    const int j = t / K4_NG, i = t % K4_NG;
    double s = 0.0;
    for (int ww = 0; ww < K4_WARPS; ++ww) s += gsum[ww][j][i];
    a.partials[((size_t)blockIdx.y * n_pg + c0 + j) * K4_NG + i] = s;
  }
}

// Point / Gaussian gradients for uniformly spaced channels.  grid = (component tiles of 32, row
// chunks); warp w takes rows r0 + w, r0 + w + 8, ...; lane j owns component j of the tile and runs over
// every channel of the pass itself, so its sums need no cross-lane reduction.  Per row, the warp first
// writes W = conj(G) R of every channel to shared memory (read back by broadcast); the phasor advances
// by the one-channel step D (accurate) and restarts from an exactly reduced phase every K4U_RS channels.
constexpr int K4U_RS = 16;

struct K4USmem {
  int comps, cjs, cc, nh, wb, total;
};
__host__ __device__ inline K4USmem k4u_layout(int f_cnt) {
  K4USmem L;
  L.comps = 0;
  L.cjs = L.comps + K4_CT * (int)sizeof(PGRec);
  L.cc = L.cjs + K4_CT * 4;
  L.nh = L.cc + f_cnt * 16;
  L.wb = L.nh + f_cnt * 8;
  const int wbytes = K4_WARPS * f_cnt * 8, gbytes = K4_WARPS * K4_CT * K4_NG * 8;
  L.total = L.wb + (wbytes > gbytes ? wbytes : gbytes);
  return L;
}

// The channel sums of one (component, row): s0 = sum Re z, s1 = sum log2(nu/nu0) Re z,
// s2 = sum (nu/c) Im z, s3 = sum (nu/c)^2 Re z with z = conj(W) V / S_ref.  GAUSS = false (a tile of
// points only) leaves out the Gaussian envelope's exponent term and s3, which only Gaussians use.
template <bool GAUSS>
__device__ __forceinline__ void k4u_channel(const float4 c, const float2 W, float q, float alpha, float cj, float2 D,
                                            float2& P, float& s0, float& s1, float& s2, float& s3) {
  // channel sums use the amplitude without the flux: dV/dS_ref = V / S_ref holds for S_ref = 0 too
  const float e = fmaf(alpha, c.x, cj);
  const float A = ex2_approx(GAUSS ? fmaf(-q, c.y, e) : e);
  const float vr = A * P.x, vi = A * P.y;
  const float zr = W.x * vr + W.y * vi, zi = W.x * vi - W.y * vr;  // z = conj(W) V
  s0 += zr;
  s1 = fmaf(c.x, zr, s1);
  s2 = fmaf(c.z, zi, s2);
  if (GAUSS) s3 = fmaf(c.w, zr, s3);
  P = make_float2(P.x * D.x - P.y * D.y, P.x * D.y + P.y * D.x);
}

template <bool GAUSS>
__device__ __forceinline__ void k4u_channels(int F, float th, float tl, float q, float alpha, float cj, float2 D,
                                             const float2* nh, const float4* cc, const float2* myw, float& s0,
                                             float& s1, float& s2, float& s3) {
  for (int fb = 0; fb < F; fb += K4U_RS) {
    float2 P = phasor_fast(reduce_turns(th, tl, nh[fb].x, nh[fb].y));
    if (fb + K4U_RS <= F) {  // a whole block: unrolled, constant offsets
#pragma unroll
      for (int i = 0; i < K4U_RS; ++i) k4u_channel<GAUSS>(cc[fb + i], myw[fb + i], q, alpha, cj, D, P, s0, s1, s2, s3);
    } else {
      for (int f = fb; f < F; ++f) k4u_channel<GAUSS>(cc[f], myw[f], q, alpha, cj, D, P, s0, s1, s2, s3);
    }
  }
}

__global__ void __launch_bounds__(K4_WARPS * 32, 3) k4_grad_pg_u(const K4Args a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int F = a.f_cnt;
  const K4USmem L = k4u_layout(F);
  PGRec* comps = reinterpret_cast<PGRec*>(sm + L.comps);
  float* cjs = reinterpret_cast<float*>(sm + L.cjs);
  float4* cc = reinterpret_cast<float4*>(sm + L.cc);   // per channel: log2(nu/nu0), Gaussian weight, nu/c, (nu/c)^2
  float2* nh = reinterpret_cast<float2*>(sm + L.nh);   // per channel: nu/c as a float pair
  float2* wb = reinterpret_cast<float2*>(sm + L.wb);   // [warp][F] W of the current row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_pg = a.n_point + a.n_gauss;
  const int c0 = blockIdx.x * K4_CT;
  const int ncomp = min(K4_CT, n_pg - c0);
  const double L0 = log2(a.nu0);
  if (threadIdx.x < ncomp) {
    const PGRec c = a.comps[c0 + threadIdx.x];
    comps[threadIdx.x] = c;
    cjs[threadIdx.x] = c.alpha * (float)(L0 - c.lref);
  }
  const float inv_nu0 = (float)(1.0 / a.nu0);
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    const double nu = a.freq[a.f_lo + f];
    float h, l;
    split_double(nu * (1.0 / kC), h, l);
    cc[f] = make_float4(log2f((float)nu * inv_nu0), (float)(kGaussE * kLog2e) * h * h, h, h * h);
    nh[f] = make_float2(h, l);
  }
  __syncthreads();

  // this lane's component
  const bool mine = lane < ncomp;
  const int jc = c0 + (mine ? lane : 0);
  const PGRec& me = comps[mine ? lane : 0];
  const bool my_gauss = mine && jc >= a.n_point;
  const bool tile_gauss = c0 + ncomp > a.n_point;  // the tile holds a Gaussian (uniform over the CTA)
  const double me_l = (double)me.lh + me.ll, me_m = (double)me.mh + me.ml, me_nm1 = (double)me.nh + me.nl;
  const double my_n = 1.0 + me_nm1;
  const float my_ln = (float)(me_l / my_n), my_mn = (float)(me_m / my_n);
  const float my_lnref = (float)((L0 - me.lref) * 0.6931471805599453);
  const float my_S = mine ? (float)a.flux[jc] : 0.f;
  const float my_alpha = me.alpha, my_cj = cjs[mine ? lane : 0];
  float my_pa = 0.f, my_maj = 0.f, my_min = 0.f;
  if (my_gauss) {
    const int g = jc - a.n_point;
    my_maj = (float)a.gmaj[g];
    my_min = (float)a.gmin[g];
    my_pa = (float)a.gpa[g];
  }
  const float sp = sinf(my_pa), cp = cosf(my_pa);

  float acc32[K4_NG];
  double acc64[K4_NG];
#pragma unroll
  for (int i = 0; i < K4_NG; ++i) {
    acc32[i] = 0.f;
    acc64[i] = 0.0;
  }
  float2* myw = wb + warp * F;
  const int r_lo = blockIdx.y * a.rows_per_chunk;
  const int r_hi = min(a.n_rows, r_lo + a.rows_per_chunk);
  int nrow = 0;
  for (int row = r_lo + warp; row < r_hi; row += K4_WARPS) {
    __syncwarp();  // the previous row's W is no longer read
    for (int f = lane; f < F; f += 32) {
      float2 G;
      if (!gain_product(a.peel, row, a.n_base, a.f_lo + f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
      const float2 R = a.resid[(size_t)row * a.n_chan + a.f_lo + f];
      myw[f] = make_float2(G.x * R.x + G.y * R.y, G.x * R.y - G.y * R.x);
    }
    __syncwarp();
    if (mine) {
      float xuvw[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) xuvw[i] = __ldg(a.uvw_pairs + 6 * (size_t)row + i);
      float th, tl;
      tau_df(xuvw, me, th, tl);
      const float uf = xuvw[0], vf = xuvw[2], wf = xuvw[4];
      const float fl = -4.0f * (float)kPi * (uf - wf * my_ln);
      const float fm = -4.0f * (float)kPi * (vf - wf * my_mn);
      float q = 0.f, fmaj = 0.f, fmin = 0.f, fpa = 0.f;
      if (my_gauss) {
        q = me.ga * uf * uf + me.gb * uf * vf + me.gc * vf * vf;
        const float kx = sp * uf + cp * vf, ky = cp * uf - sp * vf;
        fmaj = 4.0f * (float)kGaussE * my_maj * kx * kx;
        fmin = 4.0f * (float)kGaussE * my_min * ky * ky;
        fpa = 4.0f * (float)kGaussE * (my_maj * my_maj - my_min * my_min) * kx * ky;
      }
      const float2 D = phasor_accurate(reduce_turns(th, tl, a.dnu_h, a.dnu_l));
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      if (tile_gauss) {
        k4u_channels<true>(F, th, tl, q, my_alpha, my_cj, D, nh, cc, myw, s0, s1, s2, s3);
      } else {
        k4u_channels<false>(F, th, tl, q, my_alpha, my_cj, D, nh, cc, myw, s0, s1, s2, s3);
      }
      // s1 holds sum log2(nu/nu0) Re z: ln(nu/nu_ref) = ln2 log2(nu/nu0) + ln(nu0/nu_ref)
      acc32[0] += -2.0f * s0;
      acc32[1] += -2.0f * my_S * (0.6931471805599453f * s1 + my_lnref * s0);
      acc32[2] += my_S * fl * s2;
      acc32[3] += my_S * fm * s2;
      acc32[4] += my_S * fmaj * s3;
      acc32[5] += my_S * fmin * s3;
      acc32[6] += my_S * fpa * s3;
    }
    if (++nrow == K4_FLUSH) {
#pragma unroll
      for (int i = 0; i < K4_NG; ++i) {
        acc64[i] += (double)acc32[i];
        acc32[i] = 0.f;
      }
      nrow = 0;
    }
  }
  __syncthreads();  // every warp is done with its W buffer: the area now holds the per-warp sums
  double* gsum = reinterpret_cast<double*>(wb);  // [warp][K4_CT][K4_NG]
#pragma unroll
  for (int i = 0; i < K4_NG; ++i) gsum[(warp * K4_CT + lane) * K4_NG + i] = acc64[i] + (double)acc32[i];
  __syncthreads();
  for (int t = threadIdx.x; t < ncomp * K4_NG; t += blockDim.x) {
    const int j = t / K4_NG, i = t % K4_NG;
    double sum = 0.0;
    for (int ww = 0; ww < K4_WARPS; ++ww) sum += gsum[(ww * K4_CT + j) * K4_NG + i];
    a.partials[((size_t)blockIdx.y * n_pg + c0 + j) * K4_NG + i] = sum;
  }
}

// Sum the per-chunk partials in fixed order and scatter them into the gradient arrays.  Channel
// passes accumulate (first pass writes).
// One warp per component: lane l adds chunks l, l + 32, ..., then a fixed butterfly (deterministic).
__global__ void k4_reduce_pg(const double* partials, int chunks, int n_point, int n_gauss, int first, double* gflux,
                             double* galpha, double* gl, double* gm, double* gmaj, double* gmin, double* gpa) {
  const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int n_pg = n_point + n_gauss;
  if (j >= n_pg) return;  // uniform per warp
  double s[K4_NG] = {0, 0, 0, 0, 0, 0, 0};
  for (int c = lane; c < chunks; c += 32)
    for (int i = 0; i < K4_NG; ++i) s[i] += partials[((size_t)c * n_pg + j) * K4_NG + i];
#pragma unroll
  for (int i = 0; i < K4_NG; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
  if (lane != 0) return;
  auto put = [&](double* p, int idx, double v) {
    if (p) p[idx] = first ? v : p[idx] + v;
  };
  put(gflux, j, s[0]);
  put(galpha, j, s[1]);
  put(gl, j, s[2]);
  put(gm, j, s[3]);
  if (j >= n_point) {
    put(gmaj, j - n_point, s[4]);
    put(gmin, j - n_point, s[5]);
    put(gpa, j - n_point, s[6]);
  }
}

// ---------------------------------------------------------------------------------------------
// Shapelets: one launch per shapelet; persistent CTAs of 128 threads, one visibility per thread per
// tile.  With f_ab = C_ab times the sign of (-i)^(a+b) (real part for even a+b, imaginary for odd),
//   xi      = sum_a phi_a(x)  T_a,   T_a  = sum_b f_ab phi_b(y),
//   dxi/dx  = sum_a phi_a'(x) T_a,
//   dxi/dy  = sum_a phi_a(x)  T'_a,  T'_a = sum_b g_ab phi_b(y),
// where g_ab = sqrt((b+1)/2) f_a,b+1 - sqrt(b/2) f_a,b-1 is the y-derivative folded into the
// coefficients (phi_b' = sqrt(b/2) phi_b-1 - sqrt((b+1)/2) phi_b+1), so both sums run over the same
// phi_b(y) and T'_a takes the opposite real/imaginary part.  Each thread keeps its phi_n(x), phi_n(y)
// rows in shared memory (rows of an odd count of 16-byte quarters: float4 reads conflict-free) and runs
// the sums over K4S_RA rows a at once.  The coefficient gradients
// sum_vis w phi_a(x) phi_b(y) (w = Re or Im of conj(W) S P by the parity of a+b) are a contraction over
// the visibilities and run on the tensor cores (k4_coeff_mma, k_grad_mma.cu).
// ---------------------------------------------------------------------------------------------
constexpr int K4S_T = 128;
constexpr int K4S_NS = 7;  // flux, alpha, l, m, beta1, beta2, pa

// sqrt(n/2) and sqrt((n+1)/2) (derivative phi_n' = sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1}) and the
// recurrence coefficients sqrt(2/(n+1)), sqrt(n/(n+1)), for n <= 128.
__constant__ float c_dn_lo[kNmaxLimit + 2], c_dn_hi[kNmaxLimit + 2], c_ra[kNmaxLimit + 2], c_rb[kNmaxLimit + 2];

struct K4SArgs {
  const float4* rowinfo;   // per row: (xs, ys, tau hi, tau lo)
  const float4* chaninfo;  // per channel: (nu/c hi, nu/c lo, log2(nu/nu0), nu)
  const float* uvw_pairs;  // [n_rows][6]
  int n_rows, n_chan, n_base;
  long long n_vis;
  int nmax, nnz;
  const int *n1, *n2;
  const double* coeff;
  float l_over_n, m_over_n, lnref_nu0_f;   // l / n, m / n, ln(nu0 / nu_ref)
  const double *flux, *beta1, *beta2;      // device scalars of this shapelet (raw FP64 tables)
  float c_amp, alpha;
  const float2* resid;
  const float4* rowframe;  // per row: (dx/dl, dy/dl, dx/dm, dy/dm) / nu, the frame's share of the position gradient
  PeelArgs peel;
  double* part_s;   // [grid][K4S_NS]
  unsigned* err;
};

__device__ void hermite_scaled_row(float x, int nmax1, float* out) {
  // phi_0..phi_nmax1(x) in FP32, running on values scaled by 2^E where phi_0 underflows
  const float hx = 0.5f * x * x * 1.4426950408889634f;
  int E = fabsf(x) <= 12.5f ? 0 : max(0, (int)ceilf(hx) - 100);
  float p_prev = 0.f, p = exp2f((float)E - hx);
  float scale = __int_as_float(max(0, 127 - E) << 23);
  for (int n = 0; n <= nmax1; ++n) {
    out[n] = p * scale;
    const float pn = c_ra[n] * x * p - c_rb[n] * p_prev;
    p_prev = p;
    p = pn;
    if (fabsf(p) > 1.8446744e19f) {
      p *= 5.421011e-20f;
      p_prev *= 5.421011e-20f;
      E -= 64;
      scale = __int_as_float(max(0, 127 - E) << 23);
    }
  }
}

// The factorised sums run over K4S_RA rows a of the folded triangle at once, so each thread's phi(y)
// entries are read once per group of rows instead of once per row.
constexpr int K4S_RA = 4;
// Rows of the folded triangle with the zero rows that complete the last group.
__host__ __device__ inline int k4s_rows(int nmax) { return (nmax + K4S_RA) / K4S_RA * K4S_RA; }
// Folded triangle: row a holds b = 0 .. n - a + 1 and is padded to an even length at least that of the
// first row of its group (b = 0 .. n - a0 + 1, zeros past its own end), so every row starts on a 16-byte
// boundary, two (f, g) pairs load as one float4, and the rows of a group share one b range.  Row offset
// and total entries (rows 0 .. k4s_rows(n) - 1).
__host__ __device__ inline int k4s_row_off(int nmax, int a) {
  int o = 0;
  for (int i = 0; i < a; ++i) o += (nmax - (i - i % K4S_RA) + 2 + 1) & ~1;
  return o;
}
__host__ __device__ inline int k4s_nfg(int nmax) { return k4s_row_off(nmax, k4s_rows(nmax)); }

// Shared-memory layout of k4_grad_shape (bytes): basis rows (a multiple of 4 floats with an odd count of
// 16-byte quarters, so per-thread rows read as float4 without bank conflicts), folded coefficient pairs
// (f, g) per triangle row a (b = 0..n-a+1) and the row offsets.  At the end the second basis-row area holds
// the scalar reduction.
struct K4SSmem {
  int ld, phx, phy, fg, toff, total;
};
__host__ __device__ inline K4SSmem k4s_layout(int nmax, int T) {
  K4SSmem s;
  // entries 0 .. n + 3 (the sums read up to b = n + 1, and float4 reads one past); at least 20, so that
  // one thread's row of the second area holds its K4S_NS doubles of the final reduction
  s.ld = max((nmax + 4 + 3) & ~3, 20);
  if (((s.ld >> 2) & 1) == 0) s.ld += 4;
  const int nfg = k4s_nfg(nmax);
  s.phx = 0;
  s.phy = s.phx + T * s.ld * 4;
  s.fg = (s.phy + T * s.ld * 4 + 15) & ~15;
  s.toff = s.fg + nfg * 8;
  s.total = s.toff + (k4s_rows(nmax) + 1) * 4;
  return s;
}

__global__ void __launch_bounds__(K4S_T) k4_grad_shape(const K4SArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int n = a.nmax;
  const int T = blockDim.x;  // 128, or 64 for the largest n_max
  const K4SSmem lay = k4s_layout(n, T);
  const int ld = lay.ld;
  float* phx = reinterpret_cast<float*>(sm + lay.phx);
  float* phy = reinterpret_cast<float*>(sm + lay.phy);
  float2* fg = reinterpret_cast<float2*>(sm + lay.fg);
  int* toff = reinterpret_cast<int*>(sm + lay.toff);
  const int t = threadIdx.x;
  const double flux = *a.flux, beta1 = *a.beta1, beta2 = *a.beta2;

  // folded coefficients: row a holds (f_ab, g_ab) for b = 0..n-a+1 (f is zero past the triangle)
  const int n_rows_fg = k4s_rows(n);
  for (int aa = t; aa <= n_rows_fg; aa += T) toff[aa] = k4s_row_off(n, aa);
  const int nfg = k4s_nfg(n);
  for (int i = t; i < nfg; i += T) fg[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int k = t; k < a.nnz; k += T) {
    const int na = __ldg(a.n1 + k), nb = __ldg(a.n2 + k);
    const int ph = (na + nb) & 3;  // (-i)^k = 1, -i, -1, i: signs +, -, -, + on the real / imaginary part
    fg[toff[na] + nb].x = (ph == 1 || ph == 2 ? -1.0f : 1.0f) * (float)__ldg(a.coeff + k);
  }
  __syncthreads();
  for (int aa = t; aa <= n; aa += T) {
    float2* row = fg + toff[aa];
    const int nb = n - aa;
    for (int b = 0; b <= nb + 1; ++b) {
      const float up = b + 1 <= nb ? row[b + 1].x : 0.f;   // f_a,b+1
      const float dn = b >= 1 && b - 1 <= nb ? row[b - 1].x : 0.f;  // f_a,b-1
      row[b].y = c_dn_hi[b] * up - c_dn_lo[b] * dn;
    }
  }
  __syncthreads();

  double accs[K4S_NS] = {0, 0, 0, 0, 0, 0, 0};
  float acc32[K4S_NS] = {0, 0, 0, 0, 0, 0, 0};
  int nacc = 0;
  const float rb = (float)(beta1 / beta2), rb2 = (float)(beta2 / beta1);
  const float ib1 = (float)(1.0 / beta1), ib2 = (float)(1.0 / beta2);
  const long long n_tiles = (a.n_vis + T - 1) / T;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long vis = tile * T + t;
    const bool valid = vis < a.n_vis;
    const int row = valid ? (int)(vis / a.n_chan) : 0;
    const int f = valid ? (int)(vis - (long long)row * a.n_chan) : 0;
    const float4 ri = a.rowinfo[row], ci = a.chaninfo[f];
    const float x = ri.x * ci.w, y = ri.y * ci.w;
    float* px = phx + t * ld;
    float* py = phy + t * ld;
    hermite_scaled_row(x, n + 1, px);
    hermite_scaled_row(y, n + 1, py);
    px[n + 2] = px[n + 3] = 0.f;
    py[n + 2] = py[n + 3] = 0.f;
    // W = conj(G) R, amplitude and phasor
    float2 W = make_float2(0.f, 0.f);
    if (valid) {
      float2 G;
      if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
      const float2 R = a.resid[vis];
      W = make_float2(G.x * R.x + G.y * R.y, G.x * R.y - G.y * R.x);
    }
    const float2 P = phasor_fast(reduce_turns(ri.z, ri.w, ci.x, ci.y));
    // Y = conj(W) S' P with S' = (nu / nu_ref)^alpha (the flux multiplies every term below but the
    // flux derivative); contributions are -2 S_ref Re(Y * dxi)
    const float S = valid ? ex2_approx(fmaf(a.alpha, ci.z, a.c_amp)) : 0.f;
    const float yr = S * (W.x * P.x + W.y * P.y), yi = S * (W.x * P.y - W.y * P.x);
    // xi, dxi/dx, dxi/dy by the factorised sums
    float xr = 0.f, xi = 0.f, dxr = 0.f, dxi = 0.f, dyr = 0.f, dyi = 0.f;
    {
      // phi_a(x) for a = 0 .. n + 1 (entries n + 2, n + 3 are zero; rows past n + 1 read entry n + 3)
      auto phx_at = [&](int aa) { return px[min(aa, n + 3)]; };
      float pa_prev = 0.f, pa_cur = px[0];
      for (int a0 = 0; a0 <= n; a0 += K4S_RA) {
        const int nb = n - a0 + 1;  // b = 0..nb for every row of the group (g reaches one past the triangle)
        const float2* r[K4S_RA];
        float te[K4S_RA], to[K4S_RA], ge[K4S_RA], go[K4S_RA];  // f and g sums over even / odd b
  #pragma unroll
        for (int i = 0; i < K4S_RA; ++i) {
          r[i] = fg + toff[a0 + i];
          te[i] = to[i] = ge[i] = go[i] = 0.f;
        }
        int b = 0;
        for (; b + 3 <= nb; b += 4) {
          const float4 p = *reinterpret_cast<const float4*>(py + b);
  #pragma unroll
          for (int i = 0; i < K4S_RA; ++i) {
            const float4 c01 = *reinterpret_cast<const float4*>(r[i] + b);  // f_b, g_b, f_b+1, g_b+1
            const float4 c23 = *reinterpret_cast<const float4*>(r[i] + b + 2);
            te[i] = fmaf(c01.x, p.x, te[i]);
            ge[i] = fmaf(c01.y, p.x, ge[i]);
            to[i] = fmaf(c01.z, p.y, to[i]);
            go[i] = fmaf(c01.w, p.y, go[i]);
            te[i] = fmaf(c23.x, p.z, te[i]);
            ge[i] = fmaf(c23.y, p.z, ge[i]);
            to[i] = fmaf(c23.z, p.w, to[i]);
            go[i] = fmaf(c23.w, p.w, go[i]);
          }
        }
        for (; b + 1 <= nb; b += 2) {
          const float p0 = py[b], p1 = py[b + 1];
  #pragma unroll
          for (int i = 0; i < K4S_RA; ++i) {
            const float4 c = *reinterpret_cast<const float4*>(r[i] + b);
            te[i] = fmaf(c.x, p0, te[i]);
            ge[i] = fmaf(c.y, p0, ge[i]);
            to[i] = fmaf(c.z, p1, to[i]);
            go[i] = fmaf(c.w, p1, go[i]);
          }
        }
        if (b <= nb) {
          const float p0 = py[b];
  #pragma unroll
          for (int i = 0; i < K4S_RA; ++i) {
            const float2 c0 = r[i][b];
            te[i] = fmaf(c0.x, p0, te[i]);
            ge[i] = fmaf(c0.y, p0, ge[i]);
          }
        }
  #pragma unroll
        for (int i = 0; i < K4S_RA; ++i) {
          const int aa = a0 + i;  // rows past n hold zeros: their terms vanish
          const float pa_next = phx_at(aa + 1);
          const int ac = min(aa, n + 1);
          const float dpa = c_dn_lo[ac] * pa_prev - c_dn_hi[ac] * pa_next;  // phi_a'(x)
          // f terms with a+b even are real; g terms take the opposite part (a0 is a multiple of K4S_RA,
          // so the parity of a is that of i)
          const bool odd = i & 1;
          const float Tr = odd ? to[i] : te[i], Ti = odd ? te[i] : to[i];
          const float Dr = odd ? ge[i] : go[i], Di = odd ? go[i] : ge[i];
          xr = fmaf(pa_cur, Tr, xr);
          xi = fmaf(pa_cur, Ti, xi);
          dxr = fmaf(dpa, Tr, dxr);
          dxi = fmaf(dpa, Ti, dxi);
          dyr = fmaf(pa_cur, Dr, dyr);
          dyi = fmaf(pa_cur, Di, dyi);
          pa_prev = pa_cur;
          pa_cur = pa_next;
        }
      }
    }
    if (valid) {
      // Re(Y * (pr + i pi)) = yr pr - yi pi
      const float re_xi = yr * xr - yi * xi;  // Re(conj(W) V) / S_ref
      const float im_xi = yr * xi + yi * xr;  // Im(conj(W) V) / S_ref
      const float re_dx = yr * dxr - yi * dxi, re_dy = yr * dyr - yi * dyi;
      const float nuc = ci.x;                 // nu / c
      const float* xu = a.uvw_pairs + 6 * (size_t)row;
      const float u = __ldg(xu), v = __ldg(xu + 2), w = __ldg(xu + 4);
      acc32[0] += -2.0f * re_xi;
      acc32[1] += -2.0f * re_xi * fmaf(ci.z, 0.6931471805599453f, a.lnref_nu0_f);
      // the position moves the phase centre of the term and the shapelet's re-phasing frame
      const float4 rf = __ldg(a.rowframe + row);
      acc32[2] += -4.0f * (float)kPi * nuc * (u - w * a.l_over_n) * im_xi - 2.0f * ci.w * (re_dx * rf.x + re_dy * rf.y);
      acc32[3] += -4.0f * (float)kPi * nuc * (v - w * a.m_over_n) * im_xi - 2.0f * ci.w * (re_dx * rf.z + re_dy * rf.w);
      acc32[4] += -2.0f * re_dx * x * ib1;
      acc32[5] += -2.0f * re_dy * y * ib2;
      acc32[6] += -2.0f * (re_dx * rb * y - re_dy * rb2 * x);
    }
    if (++nacc == 16) {
#pragma unroll
      for (int i = 0; i < K4S_NS; ++i) {
        accs[i] += (double)acc32[i];
        acc32[i] = 0.f;
      }
      nacc = 0;
    }
  }
  // per-CTA partials of the scalar groups (the flux factor of every group but the flux one is applied
  // here, in FP64); every thread is past its basis rows before the reduction reuses them
  __syncthreads();
  double* red = reinterpret_cast<double*>(sm + lay.phy);  // [T][K4S_NS], in the second basis-row area
  for (int i = 0; i < K4S_NS; ++i) red[t * K4S_NS + i] = (accs[i] + (double)acc32[i]) * (i == 0 ? 1.0 : flux);
  __syncthreads();
  if (t < K4S_NS) {
    double s = 0.0;
    for (int q = 0; q < T; ++q) s += red[q * K4S_NS + t];
    a.part_s[(size_t)blockIdx.x * K4S_NS + t] = s;
  }
}

// One warp per output (coefficient or scalar group): lanes add strided per-CTA partials, then a fixed
// butterfly; deterministic.
__global__ void k4_reduce_shape(const double* part_s, const double* part_c, int grid, int grid_c, int nnz, int j, int q,
                                double* gflux, double* galpha, double* gl, double* gm, double* gb1, double* gb2,
                                double* gpa, double* gcoeff, int coeff_off, int first) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= nnz + K4S_NS) return;
  auto put = [&](double* p, int idx, double v) {
    if (p) p[idx] = first ? v : p[idx] + v;
  };
  double s = 0.0;
  if (t < nnz) {
    for (int c = lane; c < grid_c; c += 32) s += part_c[(size_t)c * nnz + t];
  } else {
    for (int c = lane; c < grid; c += 32) s += part_s[(size_t)c * K4S_NS + (t - nnz)];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  if (t < nnz) {
    put(gcoeff, coeff_off + t, s);
    return;
  }
  switch (t - nnz) {
    case 0: put(gflux, j, s); break;
    case 1: put(galpha, j, s); break;
    case 2: put(gl, j, s); break;
    case 3: put(gm, j, s); break;
    case 4: put(gb1, q, s); break;
    case 5: put(gb2, q, s); break;
    default: put(gpa, q, s); break;
  }
}

// (u, v, w) of every row split into float pairs for the double-float phase arguments.
__global__ void k4_split_uvw(const double* uvw, int n_rows, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_rows) return;
  float h, l;
  split_double(uvw[i], h, l);
  out[2 * i] = h;
  out[2 * i + 1] = l;
}

// L = sum |R|^2: FP32 per thread over a grid-stride run, FP64 from there on, fixed order.
__global__ void k4_loss_partial(const float2* r, size_t n, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  float f = 0.f;
  int cnt = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = r[i];
    f = fmaf(v.x, v.x, fmaf(v.y, v.y, f));
    if (++cnt == 64) {
      s += f;
      f = 0.f;
      cnt = 0;
    }
  }
  red[threadIdx.x] = s + f;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// One warp: lane l adds partials l, l + 32, ..., then a fixed butterfly (deterministic).
__global__ void k4_loss_final(const double* part, int n, double* out) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0 && blockIdx.x == 0) *out = s;
}

// Derivatives of rows 0 and 1 of the re-phasing frame (shapelet_frame) with respect to the shapelet's l and
// m.  The frame's entries are algebraic in (l, m): with n = sqrt(1 - l^2 - m^2), sin dec_j = m cos dec0 +
// n sin dec0, y = n cos dec0 - m sin dec0, cos dec_j = sqrt(l^2 + y^2), sin H_j = -l / cos dec_j and
// cos H_j = y / cos dec_j; each is differentiated in turn.  Zero when the centre sits on the frame's pole.
__device__ void shapelet_frame_dlm(double l, double m, double sd0, double cd0, double Fl[6], double Fm[6]) {
  const double n = sqrt(1.0 - l * l - m * m);
  const double sdj = m * cd0 + n * sd0, y = n * cd0 - m * sd0;
  const double cdj = sqrt(l * l + y * y);
  for (int i = 0; i < 6; ++i) Fl[i] = Fm[i] = 0.0;
  if (!(cdj > 0.0)) return;
  const double shj = -l / cdj, chj = y / cdj;
  const double r0[9] = {0.0, 1.0, 0.0, -sd0, 0.0, cd0, cd0, 0.0, sd0};
  for (int which = 0; which < 2; ++which) {  // 0: d/dl, 1: d/dm
    const double dn = which == 0 ? -l / n : -m / n;
    const double dsdj = which == 0 ? dn * sd0 : cd0 + dn * sd0;
    const double dy = which == 0 ? dn * cd0 : dn * cd0 - sd0;
    const double dcdj = ((which == 0 ? l : 0.0) + y * dy) / cdj;
    const double dshj = which == 0 ? (-cdj + l * dcdj) / (cdj * cdj) : l * dcdj / (cdj * cdj);
    const double dchj = (dy * cdj - y * dcdj) / (cdj * cdj);
    const double d0[3] = {dshj, dchj, 0.0};
    const double d1[3] = {-(dsdj * chj + sdj * dchj), dsdj * shj + sdj * dshj, dcdj};
    double* out = which == 0 ? Fl : Fm;
    for (int b = 0; b < 3; ++b) {
      out[b] = d0[0] * r0[3 * b] + d0[1] * r0[3 * b + 1] + d0[2] * r0[3 * b + 2];
      out[3 + b] = d1[0] * r0[3 * b] + d1[1] * r0[3 * b + 1] + d1[2] * r0[3 * b + 2];
    }
  }
}

// Per row of shapelet sh: (dx/dl, dy/dl, dx/dm, dy/dm) per unit frequency, x = (kx_u u' + kx_v v') nu/c and
// y likewise, through the frame's derivatives (FP64, stored as float).
__global__ void k4_rowframe(const double* uvw, int n_rows, const ShapeRec* sh, double sd0, double cd0, float4* out) {
  __shared__ double D[12];
  if (threadIdx.x == 0) shapelet_frame_dlm(sh->l, sh->m, sd0, cd0, D, D + 6);
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const double u = uvw[3 * (size_t)r], v = uvw[3 * (size_t)r + 1], w = uvw[3 * (size_t)r + 2];
  double o[4];
  for (int which = 0; which < 2; ++which) {
    const double* F = D + 6 * which;
    const double dup = F[0] * u + F[1] * v + F[2] * w, dvp = F[3] * u + F[4] * v + F[5] * w;
    o[2 * which] = ((double)sh->kx_u * dup + (double)sh->kx_v * dvp) / kC;
    o[2 * which + 1] = ((double)sh->ky_u * dup + (double)sh->ky_v * dvp) / kC;
  }
  out[r] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
}

int launch_shapelet_prep(wn_ctx* ctx, const ObsDev& o, const Model* M, int q, float4* chaninfo, float4* rowinfo,
                         bool chan, cudaStream_t st);

static int cuda_err(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return WN_OK;
}

int run_model_peel(wn_ctx* ctx, const ObsDev& d, const Model* M, float2* out, const PeelArgs& pa, cudaStream_t st);

// The Hermite derivative and recurrence constants of the shapelet adjoint, uploaded synchronously at
// context creation (wn_create, the context's device current), so that every later launch, on any
// stream, reads them complete; a context created after a device reset uploads them again.
int grad_constants_setup(wn_ctx* ctx) {
  (void)ctx;
  float lo[kNmaxLimit + 2], hi[kNmaxLimit + 2], ra[kNmaxLimit + 2], rb[kNmaxLimit + 2];
  for (int n = 0; n <= kNmaxLimit + 1; ++n) {
    lo[n] = (float)std::sqrt(0.5 * n);
    hi[n] = (float)std::sqrt(0.5 * (n + 1));
    ra[n] = (float)std::sqrt(2.0 / (n + 1));
    rb[n] = (float)std::sqrt((double)n / (n + 1));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_dn_lo, lo, sizeof(lo));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dn_hi, hi, sizeof(hi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ra, ra, sizeof(ra));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rb, rb, sizeof(rb));
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("adjoint constants: ") + cudaGetErrorString(e));
  return WN_OK;
}

int launch_grad(wn_ctx* ctx, const ObsDev& o, const Model* M, const PeelArgs& pa, float2* resid,
                const wn_sky_grad* g, double* loss, cudaStream_t st) {
  // 1. forward: resid = data - G V
  if (int r = run_model_peel(ctx, o, M, resid, pa, st)) return r;
  // workspace: loss partials, point/Gaussian partials, shapelet tables and partials
  const int n_pg = M->n_point + M->n_gauss;
  const int loss_blocks = ctx->num_sms * 2;
  const int comp_tiles = (n_pg + K4_CT - 1) / K4_CT;
  int chunks = 1;
  if (n_pg > 0) {
    // enough CTAs for ~4 waves, bounded so the partials stay small
    chunks = std::max(1, std::min(o.n_rows / 16, (ctx->num_sms * 8 + comp_tiles - 1) / std::max(1, comp_tiles)));
  }
  const int rows_per_chunk = (o.n_rows + chunks - 1) / chunks;
  int max_nnz = 0;
  for (int q = 0; q < M->n_shape; ++q) max_nnz = std::max(max_nnz, M->s_off_host[q + 1] - M->s_off_host[q]);
  const int sgrid = ctx->num_sms * 4;
  const size_t chan_bytes = ((size_t)o.n_chan * sizeof(float4) + 255) & ~(size_t)255;
  const size_t row_bytes = ((size_t)o.n_rows * sizeof(float4) + 255) & ~(size_t)255;
  const size_t uvp_bytes = ((size_t)o.n_rows * 6 * sizeof(float) + 255) & ~(size_t)255;
  const size_t loss_bytes = ((size_t)loss_blocks * 8 + 255) & ~(size_t)255;
  const size_t pg_bytes = ((size_t)chunks * n_pg * K4_NG * 8 + 255) & ~(size_t)255;
  const size_t sh_bytes = M->n_shape ? (((size_t)sgrid * (K4S_NS + max_nnz) * 8 + 255) & ~(size_t)255) : 0;
  const size_t rowg_bytes = ((size_t)o.n_rows * sizeof(float2) + 255) & ~(size_t)255;
  const size_t frame_bytes = M->n_shape ? row_bytes : 0;
  const size_t need = chan_bytes + row_bytes + uvp_bytes + loss_bytes + pg_bytes + sh_bytes + rowg_bytes + frame_bytes;
  if (ctx->ws2_bytes < need) {
    if (ctx->ws2) {
      cudaStreamSynchronize(st);
      cudaFree(ctx->ws2);
      ctx->ws2 = nullptr;
      ctx->ws2_bytes = 0;
    }
    cudaError_t e = dev_malloc(&ctx->ws2, need);
    if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("adjoint workspace: ") + cudaGetErrorString(e));
    ctx->ws2_bytes = need;
  }
  char* ws = static_cast<char*>(ctx->ws2);
  float4* chaninfo = reinterpret_cast<float4*>(ws);
  float4* rowinfo = reinterpret_cast<float4*>(ws + chan_bytes);
  float* uvp = reinterpret_cast<float*>(ws + chan_bytes + row_bytes);
  double* lpart = reinterpret_cast<double*>(ws + chan_bytes + row_bytes + uvp_bytes);
  double* pgpart = reinterpret_cast<double*>(ws + chan_bytes + row_bytes + uvp_bytes + loss_bytes);
  double* shpart = reinterpret_cast<double*>(ws + chan_bytes + row_bytes + uvp_bytes + loss_bytes + pg_bytes);
  float2* rowg = reinterpret_cast<float2*>(ws + chan_bytes + row_bytes + uvp_bytes + loss_bytes + pg_bytes + sh_bytes);
  float4* rowframe =
      reinterpret_cast<float4*>(ws + chan_bytes + row_bytes + uvp_bytes + loss_bytes + pg_bytes + sh_bytes + rowg_bytes);
  k4_split_uvw<<<(3 * o.n_rows + 255) / 256, 256, 0, st>>>(o.uvw, o.n_rows, uvp);
  if (int r = cuda_err("uvw split")) return r;

  // 2. loss
  const size_t n_vis = (size_t)o.n_rows * o.n_chan;
  if (loss) {
    k4_loss_partial<<<loss_blocks, 256, 0, st>>>(resid, n_vis, lpart);
    k4_loss_final<<<1, 32, 0, st>>>(lpart, loss_blocks, loss);
    if (int r = cuda_err("loss kernels")) return r;
  }
  // 3. points and Gaussians, one pass per 512 channels
  if (n_pg > 0) {
    const int npass = (o.n_chan + 32 * K4_KMAX - 1) / (32 * K4_KMAX);
    for (int p = 0; p < npass; ++p) {
      K4Args a;
      a.uvw_pairs = uvp;
      a.freq = o.freq;
      a.n_rows = o.n_rows;
      a.n_chan = o.n_chan;
      a.n_base = o.n_base;
      a.f_lo = p * 32 * K4_KMAX;
      a.f_cnt = std::min(32 * K4_KMAX, o.n_chan - a.f_lo);
      a.nu0 = o.nu0;
      {
        const double dn = o.dnu / kC;
        a.dnu_h = (float)dn;
        a.dnu_l = (float)(dn - (double)a.dnu_h);
      }
      a.comps = M->pg;
      a.flux = M->r_flux();
      a.nuref = M->r_nuref();
      a.gmaj = M->r_gmaj();
      a.gmin = M->r_gmin();
      a.gpa = M->r_gpa();
      a.n_point = M->n_point;
      a.n_gauss = M->n_gauss;
      a.resid = resid;
      a.peel = pa;
      a.rows_per_chunk = rows_per_chunk;
      a.partials = pgpart;
      a.err = ctx->d_err;
      const dim3 grid(comp_tiles, chunks);
      const int km = (a.f_cnt + 31) / 32;
      if (o.uniform) {
        if (cudaError_t ea = allow_max_dynamic_smem(reinterpret_cast<const void*>(k4_grad_pg_u)))
          return set_error(WN_ECUDA, std::string("adjoint attribute: ") + cudaGetErrorString(ea));
        k4_grad_pg_u<<<grid, K4_WARPS * 32, k4u_layout(a.f_cnt).total, st>>>(a);
      } else if (km <= 2) k4_grad_pg<2><<<grid, K4_WARPS * 32, 0, st>>>(a);
      else if (km <= 4) k4_grad_pg<4><<<grid, K4_WARPS * 32, 0, st>>>(a);
      else if (km <= 8) k4_grad_pg<8><<<grid, K4_WARPS * 32, 0, st>>>(a);
      else if (km <= 12) k4_grad_pg<12><<<grid, K4_WARPS * 32, 0, st>>>(a);
      else k4_grad_pg<16><<<grid, K4_WARPS * 32, 0, st>>>(a);
      k4_reduce_pg<<<(n_pg * 32 + 255) / 256, 256, 0, st>>>(pgpart, chunks, M->n_point, M->n_gauss, p == 0, g->flux,
                                                       g->alpha, g->l, g->m, g->g_maj, g->g_min, g->g_pa);
      if (int r = cuda_err("point/Gaussian adjoint")) return r;
    }
  }
  // 4. shapelets
  const double L0 = std::log2(o.nu0);
  for (int q = 0; q < M->n_shape; ++q) {
    if (int r = launch_shapelet_prep(ctx, o, M, q, chaninfo, rowinfo, q == 0, st)) return r;
    k4_rowframe<<<(o.n_rows + 255) / 256, 256, 0, st>>>(o.uvw, o.n_rows, M->sh + q, std::sin(o.dec0), std::cos(o.dec0),
                                                        rowframe);
    const ShapeRec& h = M->sh_host[q];
    const int j = n_pg + q;
    K4SArgs a;
    a.rowinfo = rowinfo;
    a.chaninfo = chaninfo;
    a.uvw_pairs = uvp;
    a.n_rows = o.n_rows;
    a.n_chan = o.n_chan;
    a.n_base = o.n_base;
    a.n_vis = (long long)n_vis;
    a.nmax = h.nmax;
    a.nnz = M->s_off_host[q + 1] - M->s_off_host[q];
    a.n1 = M->m_n1() + M->s_off_host[q];
    a.n2 = M->m_n2() + M->s_off_host[q];
    a.coeff = M->s_coeff + M->s_off_host[q];
    a.lnref_nu0_f = (float)((L0 - h.lref) * 0.6931471805599453);
    a.l_over_n = (float)(h.l / (1.0 + h.nm1));
    a.m_over_n = (float)(h.m / (1.0 + h.nm1));
    a.c_amp = (float)((double)h.alpha * (L0 - h.lref));  // flux-free
    a.alpha = h.alpha;
    a.flux = M->r_flux() + j;
    a.beta1 = M->r_sb1() + q;
    a.beta2 = M->r_sb2() + q;
    a.resid = resid;
    a.rowframe = rowframe;
    a.peel = pa;
    a.part_s = shpart;
    a.err = ctx->d_err;
    double* part_c = shpart + (size_t)sgrid * K4S_NS;  // the tensor-core kernel's coefficient partials
    const size_t smax = 227 * 1024;
    int T = K4S_T;
    size_t smem = (size_t)k4s_layout(h.nmax, T).total;
    if (smem > smax) {
      T = K4S_T / 2;
      smem = (size_t)k4s_layout(h.nmax, T).total;
    }
    if (smem > smax) return set_error(WN_EINVAL, "adjoint: shapelet too large for the shared-memory reduction");
    if (cudaError_t ea = allow_max_dynamic_smem(reinterpret_cast<const void*>(k4_grad_shape)))
      return set_error(WN_ECUDA, std::string("adjoint attribute: ") + cudaGetErrorString(ea));
    k4_grad_shape<<<sgrid, T, smem, st>>>(a);
    if (int r = cuda_err("shapelet adjoint")) return r;
    int cgrid = 0;
    if (int r = launch_coeff_mma(ctx, o, M, q, pa, resid, rowinfo, chaninfo, rowg, part_c, &cgrid, st)) return r;
    const int nout = a.nnz + K4S_NS;
    k4_reduce_shape<<<(nout * 32 + 255) / 256, 256, 0, st>>>(shpart, part_c, sgrid, cgrid, a.nnz, j, q, g->flux,
                                                            g->alpha, g->l, g->m, g->s_beta1, g->s_beta2, g->s_pa,
                                                            g->s_coeff, M->s_off_host[q], 1);
    if (int r = cuda_err("shapelet adjoint reduction")) return r;
  }
  return WN_OK;
}

// Coefficient gradients only, for a residual the caller provides: gcoeff[k] = dL/dC_k of
// L = sum |R - G V|^2 with respect to every shapelet coefficient of M (triple order), evaluated as
// -2 Re sum conj(conj(G) R) dV/dC_k.  It is linear in R and does not depend on the coefficients, so
// -gcoeff / 2 is the adjoint of the linear map C -> G V_shapelets(C) applied to R.
int launch_grad_shape_coeff(wn_ctx* ctx, const ObsDev& o, const Model* M, const PeelArgs& pa, const float2* resid,
                            double* gcoeff, cudaStream_t st) {
  int max_nnz = 0;
  for (int q = 0; q < M->n_shape; ++q) max_nnz = std::max(max_nnz, M->s_off_host[q + 1] - M->s_off_host[q]);
  const int sgrid = ctx->num_sms * 4;
  const size_t chan_bytes = ((size_t)o.n_chan * sizeof(float4) + 255) & ~(size_t)255;
  const size_t row_bytes = ((size_t)o.n_rows * sizeof(float4) + 255) & ~(size_t)255;
  const size_t sh_bytes = (((size_t)sgrid * (K4S_NS + max_nnz) * 8 + 255) & ~(size_t)255);
  const size_t rowg_bytes = ((size_t)o.n_rows * sizeof(float2) + 255) & ~(size_t)255;
  const size_t need = chan_bytes + row_bytes + sh_bytes + rowg_bytes;
  if (ctx->ws2_bytes < need) {
    if (ctx->ws2) {
      cudaStreamSynchronize(st);
      cudaFree(ctx->ws2);
      ctx->ws2 = nullptr;
      ctx->ws2_bytes = 0;
    }
    cudaError_t e = dev_malloc(&ctx->ws2, need);
    if (e != cudaSuccess) return set_error(WN_ENOMEM, std::string("adjoint workspace: ") + cudaGetErrorString(e));
    ctx->ws2_bytes = need;
  }
  char* ws = static_cast<char*>(ctx->ws2);
  float4* chaninfo = reinterpret_cast<float4*>(ws);
  float4* rowinfo = reinterpret_cast<float4*>(ws + chan_bytes);
  double* shpart = reinterpret_cast<double*>(ws + chan_bytes + row_bytes);
  float2* rowg = reinterpret_cast<float2*>(ws + chan_bytes + row_bytes + sh_bytes);
  const int n_pg = M->n_point + M->n_gauss;
  for (int q = 0; q < M->n_shape; ++q) {
    if (int r = launch_shapelet_prep(ctx, o, M, q, chaninfo, rowinfo, q == 0, st)) return r;
    const int nnz = M->s_off_host[q + 1] - M->s_off_host[q];
    double* part_c = shpart + (size_t)sgrid * K4S_NS;
    int cgrid = 0;
    if (int r = launch_coeff_mma(ctx, o, M, q, pa, resid, rowinfo, chaninfo, rowg, part_c, &cgrid, st)) return r;
    k4_reduce_shape<<<(nnz * 32 + 255) / 256, 256, 0, st>>>(shpart, part_c, sgrid, cgrid, nnz, n_pg + q, q, nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, gcoeff,
                                                           M->s_off_host[q], 1);
    if (int r = cuda_err("shapelet coefficient adjoint")) return r;
  }
  return WN_OK;
}

}  // namespace wn
