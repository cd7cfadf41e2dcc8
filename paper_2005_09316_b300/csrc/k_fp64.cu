// K5: the prediction with every step in FP64, one thread per visibility and a straight loop over every
// component (eq:env_visi_def with eq:gauss-env and eq:shape-env).  It is the speedup denominator of
// the mixed-precision path and is checked against the oracle like every other kernel.
//
// Two forms:
//  * k5_fp64 (WN_PREC_FP64): the per-component work that does not depend on the visibility is done
//    once per component per CTA, as the mixed-precision kernels do it once per component: n - 1, the
//    log-flux with the spectral index folded in (log2|S| - alpha log2 nu_ref), the Gaussian quadratic
//    form in (u, v) from the axes and position angle, and each shapelet's frame, scales and
//    position-angle terms.  Each component-visibility evaluation is then the phase (3 FMAs), one FP64
//    sincospi, one FP64 exp2 of log-flux + alpha log2 nu (minus the Gaussian form) and the accumulate.
//  * k5_fp64_untuned (WN_PREC_FP64_UNTUNED): the formulas as printed, evaluated per visibility
//    (pow for the spectrum, the position angle's cos and sin per evaluation); kept for comparison.
#include "wn_internal.cuh"

namespace wn {

struct K5Args {
  const double* uvw;
  const double* freq;
  int n_rows, n_chan, n_base, n_point, n_gauss, n_shape;
  const double *l, *m, *flux, *alpha, *nuref, *gmaj, *gmin, *gpa, *sb1, *sb2, *spa, *coeff;
  const int *nmax, *off, *n1, *n2;
  double dec0;
  float2* out;
  int mode;
  PeelArgs peel;
  unsigned* err;
};

constexpr int K5_MAX_SHAPE_SMEM = 64;  // shapelet frames staged in shared memory per launch chunk

__global__ void __launch_bounds__(128) k5_fp64_untuned(const K5Args a, int shape_lo, int shape_hi, int first_chunk) {
  __shared__ double frames[K5_MAX_SHAPE_SMEM * 9];
  const int ns = shape_hi - shape_lo;
  if (threadIdx.x < ns) {
    const int j = a.n_point + a.n_gauss + shape_lo + threadIdx.x;
    shapelet_frame(a.l[j], a.m[j], sin(a.dec0), cos(a.dec0), frames + 9 * threadIdx.x);
  }
  __syncthreads();
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)a.n_rows * a.n_chan) return;
  const int row = (int)(idx / a.n_chan), f = (int)(idx % a.n_chan);
  const double nu = a.freq[f];
  const double u = a.uvw[3 * (size_t)row] * nu / kC, v = a.uvw[3 * (size_t)row + 1] * nu / kC,
               w = a.uvw[3 * (size_t)row + 2] * nu / kC;
  double sr = 0.0, si = 0.0;
  if (first_chunk) {
    for (int j = 0; j < a.n_point + a.n_gauss; ++j) {
      const double l = a.l[j], m = a.m[j], r2 = l * l + m * m;
      const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
      double s, c;
      sincospi(2.0 * (u * l + v * m + w * nm1), &s, &c);
      double amp = a.flux[j] * pow(nu / a.nuref[j], a.alpha[j]);
      if (j >= a.n_point) {
        const int g = j - a.n_point;
        const double kx = cos(a.gpa[g]) * v + sin(a.gpa[g]) * u, ky = -sin(a.gpa[g]) * v + cos(a.gpa[g]) * u;
        amp *= exp(-kGaussE * (kx * kx * a.gmaj[g] * a.gmaj[g] + ky * ky * a.gmin[g] * a.gmin[g]));
      }
      sr += amp * c;
      si -= amp * s;
    }
  }
  for (int q = shape_lo; q < shape_hi; ++q) {
    const int j = a.n_point + a.n_gauss + q;
    const double* F = frames + 9 * (q - shape_lo);
    const double up = F[0] * u + F[1] * v + F[2] * w, vp = F[3] * u + F[4] * v + F[5] * w;
    const double pa = a.spa[q];
    const double x = a.sb1[q] * kShapeK * (cos(pa) * vp + sin(pa) * up);
    const double y = a.sb2[q] * kShapeK * (-sin(pa) * vp + cos(pa) * up);
    double px[kNmaxLimit + 1], py[kNmaxLimit + 1];
    const int nmax = a.nmax[q];
    px[0] = exp(-0.5 * x * x);
    py[0] = exp(-0.5 * y * y);
    if (nmax >= 1) {
      px[1] = sqrt(2.0) * x * px[0];
      py[1] = sqrt(2.0) * y * py[0];
    }
    for (int n = 1; n < nmax; ++n) {
      px[n + 1] = sqrt(2.0 / (n + 1)) * x * px[n] - sqrt((double)n / (n + 1)) * px[n - 1];
      py[n + 1] = sqrt(2.0 / (n + 1)) * y * py[n] - sqrt((double)n / (n + 1)) * py[n - 1];
    }
    double xr = 0.0, xi = 0.0;
    for (int k = a.off[q]; k < a.off[q + 1]; ++k) {
      const double t = a.coeff[k] * px[a.n1[k]] * py[a.n2[k]];
      switch ((a.n1[k] + a.n2[k]) & 3) {  // (-i)^(n1+n2)
        case 0: xr += t; break;
        case 1: xi -= t; break;
        case 2: xr -= t; break;
        default: xi += t; break;
      }
    }
    const double l = a.l[j], m = a.m[j], r2 = l * l + m * m;
    const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
    double s, c;
    sincospi(2.0 * (u * l + v * m + w * nm1), &s, &c);
    const double amp = a.flux[j] * pow(nu / a.nuref[j], a.alpha[j]);
    // amp * (xr + i xi) * (c - i s)
    sr += amp * (xr * c + xi * s);
    si += amp * (xi * c - xr * s);
  }
  const float2 vv = make_float2((float)sr, (float)si);
  // the first launch applies the output mode; later shapelet chunks add their part (or, for the
  // peel, subtract G times their part) to what the earlier launches wrote
  if (a.mode == OUT_PEEL) {
    float2 G;
    if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
    const float2 base = first_chunk ? a.peel.data[idx] : a.out[idx];
    a.out[idx] = make_float2(base.x - (G.x * vv.x - G.y * vv.y), base.y - (G.x * vv.y + G.y * vv.x));
  } else if (a.mode == OUT_STORE && first_chunk) {
    a.out[idx] = vv;
  } else {
    const float2 o = a.out[idx];
    a.out[idx] = make_float2(o.x + vv.x, o.y + vv.y);
  }
}

// Components per shared-memory tile of the hoisted form.
constexpr int K5_TILE = 128;

// The hoisted FP64 form.  Per tile of points or Gaussians, each thread forms one component's constants
// into shared memory; then every thread runs its visibility over the tile.  Shapelets (at most
// K5_MAX_SHAPE_SMEM per launch) keep their frame, axis scales and amplitude terms in shared memory, with
// the Hermite recurrence constants in a shared table.
__global__ void __launch_bounds__(K5_TILE) k5_fp64(const K5Args a, int shape_lo, int shape_hi, int first_chunk) {
  __shared__ double c_l[K5_TILE], c_m[K5_TILE], c_n[K5_TILE], c_ls[K5_TILE], c_al[K5_TILE], c_sg[K5_TILE];
  __shared__ double c_ga[K5_TILE], c_gb[K5_TILE], c_gc[K5_TILE];
  __shared__ double s_fr[K5_MAX_SHAPE_SMEM * 9], s_k[K5_MAX_SHAPE_SMEM * 4], s_ph[K5_MAX_SHAPE_SMEM * 6];
  __shared__ double h_a[kNmaxLimit + 1], h_b[kNmaxLimit + 1];
  const int ns = shape_hi - shape_lo;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int q = shape_lo + i, j = a.n_point + a.n_gauss + q;
    shapelet_frame(a.l[j], a.m[j], sin(a.dec0), cos(a.dec0), s_fr + 9 * i);
    double sp, cp;
    sincos(a.spa[q], &sp, &cp);
    const double b1 = a.sb1[q] * kShapeK, b2 = a.sb2[q] * kShapeK;
    s_k[4 * i] = b1 * sp;    // x = b1 (cos pa v' + sin pa u')
    s_k[4 * i + 1] = b1 * cp;
    s_k[4 * i + 2] = b2 * cp;  // y = b2 (-sin pa v' + cos pa u')
    s_k[4 * i + 3] = -b2 * sp;
    const double l = a.l[j], m = a.m[j], r2 = l * l + m * m, S = a.flux[j];
    s_ph[6 * i] = l;
    s_ph[6 * i + 1] = m;
    s_ph[6 * i + 2] = -r2 / (1.0 + sqrt(1.0 - r2));
    s_ph[6 * i + 3] = (S == 0.0 ? -INFINITY : log2(fabs(S))) - a.alpha[j] * log2(a.nuref[j]);
    s_ph[6 * i + 4] = a.alpha[j];
    s_ph[6 * i + 5] = S < 0.0 ? -1.0 : 1.0;
  }
  for (int n = threadIdx.x; n <= kNmaxLimit; n += blockDim.x) {
    h_a[n] = sqrt(2.0 / (n + 1));
    h_b[n] = sqrt((double)n / (n + 1));
  }
  __syncthreads();
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < (size_t)a.n_rows * a.n_chan;
  const int row = live ? (int)(idx / a.n_chan) : 0, f = live ? (int)(idx % a.n_chan) : 0;
  const double nu = a.freq[f], lnu = log2(nu);
  const double u = a.uvw[3 * (size_t)row] * nu / kC, v = a.uvw[3 * (size_t)row + 1] * nu / kC,
               w = a.uvw[3 * (size_t)row + 2] * nu / kC;
  double sr = 0.0, si = 0.0;
  if (first_chunk) {
    const int n_pg = a.n_point + a.n_gauss;
    for (int t0 = 0; t0 < n_pg;) {
      // tiles do not mix points and Gaussians, so the envelope test below is uniform over the CTA
      const bool gauss = t0 >= a.n_point;
      const int cnt = min(K5_TILE, (gauss ? n_pg : a.n_point) - t0);
      __syncthreads();
      if (threadIdx.x < cnt) {
        const int j = t0 + threadIdx.x;
        const double l = a.l[j], m = a.m[j], r2 = l * l + m * m, S = a.flux[j];
        c_l[threadIdx.x] = l;
        c_m[threadIdx.x] = m;
        c_n[threadIdx.x] = -r2 / (1.0 + sqrt(1.0 - r2));
        c_ls[threadIdx.x] = (S == 0.0 ? -INFINITY : log2(fabs(S))) - a.alpha[j] * log2(a.nuref[j]);
        c_al[threadIdx.x] = a.alpha[j];
        c_sg[threadIdx.x] = S < 0.0 ? -1.0 : 1.0;
        if (gauss) {
          // log2 xi = -(E log2 e) (kx^2 maj^2 + ky^2 min^2), kx = cos pa v + sin pa u, ky = -sin pa v + cos pa u,
          // as the quadratic form ga u^2 + gb u v + gc v^2
          const int g = j - a.n_point;
          double sp, cp;
          sincos(a.gpa[g], &sp, &cp);
          const double M2 = a.gmaj[g] * a.gmaj[g], m2 = a.gmin[g] * a.gmin[g], E = kGaussE * kLog2e;
          c_ga[threadIdx.x] = E * (sp * sp * M2 + cp * cp * m2);
          c_gb[threadIdx.x] = E * 2.0 * sp * cp * (M2 - m2);
          c_gc[threadIdx.x] = E * (cp * cp * M2 + sp * sp * m2);
        }
      }
      __syncthreads();
      if (live) {
        if (gauss) {
          const double uu = u * u, uv = u * v, vv = v * v;
          for (int k = 0; k < cnt; ++k) {
            double s, c;
            sincospi(2.0 * fma(w, c_n[k], fma(v, c_m[k], u * c_l[k])), &s, &c);
            const double amp =
                c_sg[k] * exp2(fma(c_al[k], lnu, c_ls[k]) - fma(c_ga[k], uu, fma(c_gb[k], uv, c_gc[k] * vv)));
            sr = fma(amp, c, sr);
            si = fma(-amp, s, si);
          }
        } else {
          for (int k = 0; k < cnt; ++k) {
            double s, c;
            sincospi(2.0 * fma(w, c_n[k], fma(v, c_m[k], u * c_l[k])), &s, &c);
            const double amp = c_sg[k] * exp2(fma(c_al[k], lnu, c_ls[k]));
            sr = fma(amp, c, sr);
            si = fma(-amp, s, si);
          }
        }
      }
      t0 += cnt;
    }
  }
  if (!live) return;
  for (int q = shape_lo; q < shape_hi; ++q) {
    const int i = q - shape_lo;
    const double* F = s_fr + 9 * i;
    const double up = F[0] * u + F[1] * v + F[2] * w, vp = F[3] * u + F[4] * v + F[5] * w;
    const double x = s_k[4 * i] * up + s_k[4 * i + 1] * vp, y = s_k[4 * i + 2] * up + s_k[4 * i + 3] * vp;
    double px[kNmaxLimit + 1], py[kNmaxLimit + 1];
    const int nmax = a.nmax[q];
    px[0] = exp(-0.5 * x * x);
    py[0] = exp(-0.5 * y * y);
    for (int n = 0; n < nmax; ++n) {
      px[n + 1] = h_a[n] * x * px[n] - (n ? h_b[n] * px[n - 1] : 0.0);
      py[n + 1] = h_a[n] * y * py[n] - (n ? h_b[n] * py[n - 1] : 0.0);
    }
    double xr = 0.0, xi = 0.0;
    for (int k = a.off[q]; k < a.off[q + 1]; ++k) {
      const double t = a.coeff[k] * px[a.n1[k]] * py[a.n2[k]];
      switch ((a.n1[k] + a.n2[k]) & 3) {  // (-i)^(n1+n2)
        case 0: xr += t; break;
        case 1: xi -= t; break;
        case 2: xr -= t; break;
        default: xi += t; break;
      }
    }
    const double* P = s_ph + 6 * i;
    double s, c;
    sincospi(2.0 * fma(w, P[2], fma(v, P[1], u * P[0])), &s, &c);
    const double amp = P[5] * exp2(fma(P[4], lnu, P[3]));
    sr += amp * (xr * c + xi * s);
    si += amp * (xi * c - xr * s);
  }
  const float2 vv = make_float2((float)sr, (float)si);
  if (a.mode == OUT_PEEL) {
    float2 G;
    if (!gain_product(a.peel, row, a.n_base, f, G)) atomicOr(a.err, WN_DEVERR_ANTENNA);
    const float2 base = first_chunk ? a.peel.data[idx] : a.out[idx];
    a.out[idx] = make_float2(base.x - (G.x * vv.x - G.y * vv.y), base.y - (G.x * vv.y + G.y * vv.x));
  } else if (a.mode == OUT_STORE && first_chunk) {
    a.out[idx] = vv;
  } else {
    const float2 o = a.out[idx];
    a.out[idx] = make_float2(o.x + vv.x, o.y + vv.y);
  }
}

int launch_phasor_fp64(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                       bool include_shapelets, cudaStream_t st) {
  K5Args a;
  a.uvw = o.uvw;
  a.freq = o.freq;
  a.n_rows = o.n_rows;
  a.n_chan = o.n_chan;
  a.n_base = o.n_base;
  a.n_point = M->n_point;
  a.n_gauss = M->n_gauss;
  a.n_shape = M->n_shape;
  a.l = M->r_l();
  a.m = M->r_m();
  a.flux = M->r_flux();
  a.alpha = M->r_alpha();
  a.nuref = M->r_nuref();
  a.gmaj = M->r_gmaj();
  a.gmin = M->r_gmin();
  a.gpa = M->r_gpa();
  a.sb1 = M->r_sb1();
  a.sb2 = M->r_sb2();
  a.spa = M->r_spa();
  a.coeff = M->s_coeff;
  a.nmax = M->m_nmax();
  a.off = M->m_off();
  a.n1 = M->m_n1();
  a.n2 = M->m_n2();
  a.dec0 = o.dec0;
  a.out = out;
  a.mode = mode;
  a.peel = pa;
  a.err = ctx->d_err;
  const size_t n = (size_t)o.n_rows * o.n_chan;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  const int ns = include_shapelets ? M->n_shape : 0;
  int lo = 0;
  bool first = true;
  do {
    const int hi = std::min(ns, lo + K5_MAX_SHAPE_SMEM);
    if (ctx->precision == WN_PREC_FP64_UNTUNED)
      k5_fp64_untuned<<<blocks, 128, 0, st>>>(a, lo, hi, first ? 1 : 0);
    else
      k5_fp64<<<blocks, K5_TILE, 0, st>>>(a, lo, hi, first ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("fp64 kernel launch: ") + cudaGetErrorString(e));
    first = false;
    lo = hi;
  } while (lo < ns);
  return WN_OK;
}

}  // namespace wn
