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

// One component against the K channels of this lane's two rows, uniform channels.  The two rows
// travel together in f32x2 pairs (x: row 0, y: row 1), so the phasor step P <- P D and the sum
// V += A P each take one packed instruction per component of the complex value.  Start phasors
// come from the exactly reduced phase at the lane's first channel; the amplitude of both rows is one
// exp2 for points, one per row for Gaussians (the envelope depends on (u, v)).
// c = {log2 |S| at the reference, alpha, sign as a half turn, sign}; Ra = the two rows' tau pairs;
// Rb, Rc = the one-channel step D of both rows and the Gaussian forms (the 48-byte record).
template <int K, bool GAUSS>
__device__ __forceinline__ void k1_comp_uniform(const float4 c, const float4 Ra, const float4 Rb, const float4 Rc,
                                                const float a0h, const float a0l, const float* lam, const float* wg,
                                                float2* Vre, float2* Vim) {
  const float2 P0 = phasor_fast_turned(reduce_turns(Ra.x, Ra.y, a0h, a0l), c.z);
  const float2 P1 = phasor_fast_turned(reduce_turns(Ra.z, Ra.w, a0h, a0l), c.z);
  float2 Pre = make_float2(P0.x, P1.x);
  float2 Pim = make_float2(P0.y, P1.y);
  const float2 Dre = make_float2(Rb.x, Rb.y), Dim = make_float2(Rb.z, Rb.w), nDim = make_float2(Rc.x, Rc.y);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float e = fmaf(c.y, lam[k], c.x);
    float2 A;
    if (GAUSS) {
      A.x = ex2_approx(fmaf(Rc.z, wg[k], e));
      A.y = ex2_approx(fmaf(Rc.w, wg[k], e));
    } else {
      A.x = ex2_approx(e);
      A.y = A.x;
    }
    // the phasor in the first operand slot, as in the rotation below: this order keeps the packed
    // pipe about 8 % busier (measured), the operand being reused from one instruction to the next
    Vre[k] = __ffma2_rn(Pre, A, Vre[k]);
    Vim[k] = __ffma2_rn(Pim, A, Vim[k]);
    if (k + 1 < K) {
      const float2 nre = __ffma2_rn(Pre, Dre, __fmul2_rn(Pim, nDim));
      Pim = __ffma2_rn(Pre, Dim, __fmul2_rn(Pim, Dre));
      Pre = nre;
    }
  }
}

}  // namespace wn
