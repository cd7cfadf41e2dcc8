// K5: the plain all-FP64 form of the prediction, one thread per visibility and a straight loop over
// every component (eq:env_visi_def with eq:gauss-env and eq:shape-env).  It is the speedup
// denominator of the mixed-precision path and is checked against the oracle like every other
// kernel; nothing in it is tuned.
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

__global__ void __launch_bounds__(128) k5_fp64(const K5Args a, int shape_lo, int shape_hi, int first_chunk) {
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
    k5_fp64<<<blocks, 128, 0, st>>>(a, lo, hi, first ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("fp64 kernel launch: ") + cudaGetErrorString(e));
    first = false;
    lo = hi;
  } while (lo < ns);
  return WN_OK;
}

}  // namespace wn
