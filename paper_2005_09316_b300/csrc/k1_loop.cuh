// The channel loop of the point/Gaussian phasor kernel (K1), shared by the kernel and by the
// microbenchmark that measures the rate this loop sustains on its own (wn_phasor_loop_rate).
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

}  // namespace wn
