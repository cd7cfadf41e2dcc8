// The channel loop of the point/Gaussian phasor kernel (K1), shared by the kernel and by the
// microbenchmark that measures the rate the loop sustains on its own (wn_phasor_loop_rate): the per-warp
// form's loop (k_phasor.cu), the spectrum-table form's loop (k_phasor_tab.cu), and the output store that
// both forms use.
#pragma once
#include "wn_internal.cuh"

namespace wn {

// exp(-2 pi i r), negated when hpi = pi: a negative flux enters as a half turn added to the MUFU
// argument (one FFMA in place of the FMUL by 2 pi), so the start phasor needs no sign multiply.  The
// argument stays within [-pi, 2 pi].
__device__ __forceinline__ float2 phasor_fast_turned(float r, float hpi) {
  float s, c;
  const float x = fmaf(r, 6.283185307179586f, hpi);
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
  return make_float2(c, -s);
}

// Channel of the uniform loop's start phasor: the middle of the lane's K channels, so that the
// three-term recurrence below runs at most K / 2 + 1 steps from it in either direction.
__host__ __device__ constexpr int k1_mid(int K) { return K / 2 - 1; }

// Sign e_k of the uniform loop's sums: it accumulates W_k = e_k V_k, with e_k = +1 when (k - mid) mod 4
// is 0 or 1 and -1 when it is 2 or 3.
__host__ __device__ constexpr bool k1_neg(int K, int k) { return ((k - k1_mid(K)) % 4 + 4) % 4 >= 2; }

// One component against the K channels of this lane's two rows, uniform channels.  The two rows
// travel together in f32x2 pairs (x: row 0, y: row 1).  The phasors P_k = exp(-2 pi i (theta_m + (k -
// m) delta)) of channels k = 0 .. K-1 satisfy the three-term recurrence P_(k+1) + P_(k-1) = c P_k with
// c = 2 cos(delta), in both directions from the start channel m = k1_mid(K).  In the signed form
// X_k = e_k P_k (k1_neg) it reads X_(k+1) = (+-c) X_k + X_(k-1), and likewise downwards, so each step
// is one packed FMA per component of the complex value and every sum V += A P is one more; the signs
// e_k are applied once, when the sums are written.  P_m comes from the exactly reduced phase at the
// start channel, P_(m+1) = P_m D with D = exp(-2 pi i delta).  The amplitude of both rows is one exp2 for
// points, one per row for Gaussians (the envelope depends on (u, v)).
// c = {log2 |S| at the reference, alpha, sign as a half turn, sign}; Ra = the two rows' tau pairs;
// Rb, Rc = the one-channel step D of both rows and the Gaussian forms (the 48-byte record);
// (a0h, a0l) = nu / c at the start channel m.
template <int K, bool GAUSS>
__device__ __forceinline__ void k1_comp_uniform(const float4 c, const float4 Ra, const float4 Rb, const float4 Rc,
                                                const float a0h, const float a0l, const float* lam, const float* wg,
                                                float2* Vre, float2* Vim) {
  constexpr int M = k1_mid(K);
  const float2 P0 = phasor_fast_turned(reduce_turns(Ra.x, Ra.y, a0h, a0l), c.z);
  const float2 P1 = phasor_fast_turned(reduce_turns(Ra.z, Ra.w, a0h, a0l), c.z);
  const float2 Dre = make_float2(Rb.x, Rb.y), Dim = make_float2(Rb.z, Rb.w), nDim = make_float2(Rc.x, Rc.y);
  const float2 Xre = make_float2(P0.x, P1.x), Xim = make_float2(P0.y, P1.y);  // X_m = P_m
  const float2 Yre = __ffma2_rn(Xre, Dre, __fmul2_rn(Xim, nDim));             // X_(m+1) = P_m D
  const float2 Yim = __ffma2_rn(Xre, Dim, __fmul2_rn(Xim, Dre));
  const float2 Cp = __fadd2_rn(Dre, Dre), Cn = __fmul2_rn(Dre, make_float2(-2.f, -2.f));
  auto add = [&](int k, float2 re, float2 im) {
    const float e = fmaf(c.y, lam[k], c.x);
    float2 A;
    if (GAUSS) {
      A.x = ex2_approx(fmaf(Rc.z, wg[k], e));
      A.y = ex2_approx(fmaf(Rc.w, wg[k], e));
    } else {
      A.x = ex2_approx(e);
      A.y = A.x;
    }
    // the phasor in the first operand slot, as in the recurrence: this order keeps the packed pipe
    // busier (measured), the operand being reused from one instruction to the next
    Vre[k] = __ffma2_rn(re, A, Vre[k]);
    Vim[k] = __ffma2_rn(im, A, Vim[k]);
  };
  add(M, Xre, Xim);
  add(M + 1, Yre, Yim);
  // upwards: X_(k+1) = c' X_k + X_(k-1), c' = +c when k - m is even, -c when odd
  float2 Pre = Xre, Pim = Xim, Qre = Yre, Qim = Yim;
#pragma unroll
  for (int k = M + 1; k + 1 < K; ++k) {
    const float2 A = ((k - M) & 1) ? Cn : Cp;
    const float2 nre = __ffma2_rn(A, Qre, Pre), nim = __ffma2_rn(A, Qim, Pim);
    Pre = Qre;
    Pim = Qim;
    Qre = nre;
    Qim = nim;
    add(k + 1, Qre, Qim);
  }
  // downwards: X_(k-1) = c' X_k + X_(k+1), c' = +c when k - m is odd, -c when even
  Pre = Yre;
  Pim = Yim;
  Qre = Xre;
  Qim = Xim;
#pragma unroll
  for (int k = M; k > 0; --k) {
    const float2 A = ((M - k) & 1) ? Cp : Cn;
    const float2 nre = __ffma2_rn(A, Qre, Pre), nim = __ffma2_rn(A, Qim, Pim);
    Pre = Qre;
    Pim = Qim;
    Qre = nre;
    Qim = nim;
    add(k - 1, Qre, Qim);
  }
}

// ---- the loop of the single-launch form (k_phasor_tab.cu): amplitudes from the spectrum table, a
// 48-byte record per (component, row pair), packed start reduction

// Both rows' start phases theta = tau nu / c reduced to [-1/2, 1/2] turns at once (th, tl: the rows'
// tau pairs), each step as reduce_turns does it for one row.
__device__ __forceinline__ float2 reduce_turns_pair(float2 th, float2 tl, float ah, float al) {
  const float2 A = make_float2(ah, ah), Al = make_float2(al, al);
  const float2 p = __fmul2_rn(th, A);
  float2 e = __ffma2_rn(th, A, make_float2(-p.x, -p.y));
  e = __ffma2_rn(th, Al, e);
  e = __ffma2_rn(tl, A, e);
  const float2 S = make_float2(12582912.0f, 12582912.0f);
  const float2 q = __fadd2_rn(p, S);
  const float2 n = __fadd2_rn(q, make_float2(-S.x, -S.y));
  return __fadd2_rn(__fadd2_rn(p, make_float2(-n.x, -n.y)), e);
}

// exp(-2 pi i r) of both rows, each turned by the sign's half turn hpi.
__device__ __forceinline__ void phasor_pair(const float2 r, const float hpi, float2& re, float2& im) {
  const float2 x = __ffma2_rn(r, make_float2(6.283185307179586f, 6.283185307179586f), make_float2(hpi, hpi));
  float s0, c0, s1, c1;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s0) : "f"(x.x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c0) : "f"(x.x));
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s1) : "f"(x.y));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c1) : "f"(x.y));
  re = make_float2(c0, c1);
  im = make_float2(-s0, -s1);
}

// Amplitude of both rows at channel k: the table value for points; exp2(table + envelope exponent)
// for Gaussians (nq: the rows' -q; wg: E log2(e) (nu_k / c)^2).
template <bool GAUSS>
__device__ __forceinline__ float2 ks_amp(const float t, const float2 nq, const float wgk) {
  if (GAUSS) return make_float2(ex2_approx(fmaf(nq.x, wgk, t)), ex2_approx(fmaf(nq.y, wgk, t)));
  return make_float2(t, t);
}

// One component against the K uniform channels of this lane's two rows (the recurrence of
// k1_comp_uniform: from the middle channel m up and down, signed form X_k = e_k P_k).  The 48-byte
// record: R0 = both rows' tau pairs {th0, th1, tl0, tl1}, R1 = the one-channel step D = exp(-2 pi i delta)
// of both rows {D0.x, D1.x, D0.y, D1.y}, R2 = {-q0, -q1, the sign's half turn, 0} with q the rows'
// Gaussian forms; tab: the lane's K spectrum values of this component.
template <int K, bool GAUSS>
__device__ __forceinline__ void ks_comp_uniform(const float4 R0, const float4 R1, const float4 R2, const float* tab,
                                                const float a0h, const float a0l, const float* wg, float2* Vre,
                                                float2* Vim) {
  constexpr int M = k1_mid(K);
  float t[K];
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(tab)[q];
    t[4 * q] = v.x;
    t[4 * q + 1] = v.y;
    t[4 * q + 2] = v.z;
    t[4 * q + 3] = v.w;
  }
  float2 Xre, Xim;
  phasor_pair(reduce_turns_pair(make_float2(R0.x, R0.y), make_float2(R0.z, R0.w), a0h, a0l), R2.z, Xre, Xim);
  const float2 Dre = make_float2(R1.x, R1.y), Dim = make_float2(R1.z, R1.w), nDim = make_float2(-R1.z, -R1.w);
  const float2 nq = make_float2(R2.x, R2.y);
  const float2 Yre = __ffma2_rn(Xre, Dre, __fmul2_rn(Xim, nDim));  // X_(m+1) = P_m D
  const float2 Yim = __ffma2_rn(Xre, Dim, __fmul2_rn(Xim, Dre));
  const float2 Cp = __fadd2_rn(Dre, Dre), Cn = make_float2(-Cp.x, -Cp.y);  // +-2 cos(delta)
  auto add = [&](int k, float2 re, float2 im) {
    const float2 A = ks_amp<GAUSS>(t[k], nq, GAUSS ? wg[k] : 0.f);
    Vre[k] = __ffma2_rn(re, A, Vre[k]);
    Vim[k] = __ffma2_rn(im, A, Vim[k]);
  };
  add(M, Xre, Xim);
  add(M + 1, Yre, Yim);
  float2 Pre = Xre, Pim = Xim, Qre = Yre, Qim = Yim;
#pragma unroll
  for (int k = M + 1; k + 1 < K; ++k) {
    const float2 A = ((k - M) & 1) ? Cn : Cp;
    const float2 nre = __ffma2_rn(A, Qre, Pre), nim = __ffma2_rn(A, Qim, Pim);
    Pre = Qre;
    Pim = Qim;
    Qre = nre;
    Qim = nim;
    add(k + 1, Qre, Qim);
  }
  Pre = Yre;
  Pim = Yim;
  Qre = Xre;
  Qim = Xim;
#pragma unroll
  for (int k = M; k > 0; --k) {
    const float2 A = ((M - k) & 1) ? Cp : Cn;
    const float2 nre = __ffma2_rn(A, Qre, Pre), nim = __ffma2_rn(A, Qim, Pim);
    Pre = Qre;
    Pim = Qim;
    Qre = nre;
    Qim = nim;
    add(k - 1, Qre, Qim);
  }
}

// Write a lane's K channels of its two rows (rows row0, row0 + 1; channels f0 ..) in the output mode:
// store, accumulate, the peel residual D - G V, or subtract G V from the output.
template <int K>
__device__ __forceinline__ void k1_store(const K1Args& a, const int row0, const int f0, const float2* Vre,
                                         const float2* Vim, const bool ok) {
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int row = row0 + rr;
    if (row >= a.n_rows) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int f = f0 + k;
      if (f >= a.n_chan) continue;
      const size_t idx = (size_t)row * a.n_chan + f;
      float2 v = rr == 0 ? make_float2(Vre[k].x, Vim[k].x) : make_float2(Vre[k].y, Vim[k].y);
      if (!ok) v = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
      // data and output stream past L2 (evict first): each element is touched once
      if (a.mode == OUT_STORE) {
        __stcs(a.out + idx, v);
      } else if (a.mode == OUT_ACCUM) {
        const float2 o = __ldcs(a.out + idx);
        __stcs(a.out + idx, make_float2(o.x + v.x, o.y + v.y));
      } else {
        float2 G;
        if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
        const float2 d = a.mode == OUT_SUBG ? __ldcs(a.out + idx) : __ldcs(a.peel.data + idx);
        __stcs(a.out + idx, make_float2(d.x - (G.x * v.x - G.y * v.y), d.y - (G.x * v.y + G.y * v.x)));
      }
    }
  }
}

}  // namespace wn
