// Sky packing kernels: turn the caller's component tables into the resident device records the
// prediction kernels read.  Runs once per model (wn_sky_upload).
#include "wn_internal.cuh"

#include <vector>

namespace wn {

// Point / Gaussian records (one thread per component).  n - 1 is formed without cancellation as
// -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)) (Sec. 3.1, below eq:measure_eq).  The Gaussian envelope
// (eq:gauss-env with eq:scale-gauss-x/y) is expanded into a quadratic form in (u, v):
//   maj^2 (sin pa u + cos pa v)^2 + min^2 (cos pa u - sin pa v)^2 = ga u^2 + gb u v + gc v^2.
__global__ void k_pack_pg(wn_sky s, PGRec* out, unsigned* err) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int n = s.n_point + s.n_gauss;
  if (j >= n) return;
  double l = s.l[j], m = s.m[j], r2 = l * l + m * m;
  double flux = s.flux[j], nuref = s.nu_ref[j];
  PGRec r;
  bool bad = !(r2 < 1.0) || !(nuref > 0.0) || !isfinite(flux) || !isfinite(s.alpha[j]);
  split_double(l, r.lh, r.ll);
  split_double(m, r.mh, r.ml);
  split_double(bad ? 0.0 : -r2 / (1.0 + sqrt(1.0 - r2)), r.nh, r.nl);
  r.lref = bad ? 0.0 : log2(nuref);
  r.lS = flux == 0.0 ? 0.0f : (float)log2(fabs(flux));
  r.alpha = (float)s.alpha[j];
  r.sgn = bad ? 0.0f : (flux > 0.0 ? 1.0f : (flux < 0.0 ? -1.0f : 0.0f));
  r.ga = r.gb = r.gc = 0.0f;
  if (j >= s.n_point) {
    int g = j - s.n_point;
    double mj = s.g_maj[g], mn = s.g_min[g], pa = s.g_pa[g];
    if (!(mj >= 0.0) || !(mn >= 0.0) || !isfinite(pa)) bad = true;
    double sp = sin(pa), cp = cos(pa), a2 = mj * mj, b2 = mn * mn;
    r.ga = (float)(a2 * sp * sp + b2 * cp * cp);
    r.gb = (float)(2.0 * sp * cp * (a2 - b2));
    r.gc = (float)(a2 * cp * cp + b2 * sp * sp);
  }
  r.pad0 = r.pad1 = 0.0f;
  out[j] = r;
  if (bad) atomicOr(err, WN_DEVERR_SKY);
}

// Shapelet headers (one thread per shapelet): n - 1, log-flux and the beta/PA-scaled axes of
// eq:scale-shape-x/y, x = beta1 K (sin pa u' + cos pa v'), y = beta2 K (cos pa u' - sin pa v'), K = pi/sqrt(2 ln 2).
__global__ void k_pack_shape(wn_sky s, const int* b_off, const int* k_pad, const int* n_pad,
                             ShapeRec* out, unsigned* err) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= s.n_shape) return;
  int j = s.n_point + s.n_gauss + q;
  double l = s.l[j], m = s.m[j], r2 = l * l + m * m;
  double flux = s.flux[j], nuref = s.nu_ref[j];
  bool bad = !(r2 < 1.0) || !(nuref > 0.0) || !isfinite(flux);
  ShapeRec r;
  r.l = l;
  r.m = m;
  double n = bad ? 1.0 : sqrt(1.0 - r2);
  r.nm1 = bad ? 0.0 : -r2 / (1.0 + n);
  r.lref = bad ? 0.0 : log2(nuref);
  r.lS = flux == 0.0 ? 0.0f : (float)log2(fabs(flux));
  r.alpha = (float)s.alpha[j];
  r.sgn = bad ? 0.0f : (flux > 0.0 ? 1.0f : (flux < 0.0 ? -1.0f : 0.0f));
  double b1 = s.s_beta1[q], b2 = s.s_beta2[q], pa = s.s_pa[q];
  r.kx_u = (float)(b1 * kShapeK * sin(pa));
  r.kx_v = (float)(b1 * kShapeK * cos(pa));
  r.ky_u = (float)(b2 * kShapeK * cos(pa));
  r.ky_v = (float)(-b2 * kShapeK * sin(pa));
  r.nmax = s.s_nmax[q];
  r.k_pad = k_pad[q];
  r.n_pad = n_pad[q];
  r.b_off = b_off[q];
  out[q] = r;
  if (bad) atomicOr(err, WN_DEVERR_SKY);
}

// Dense B operand of the shapelet contraction: column n = 2*n2 + {0: real, 1: imaginary} of
// C[n1,n2] (-i)^(n1+n2) / (k_n1 k_n2) (eq:shape-env with the phase of eq:basis_FT; k_n = herm_k, the
// scale of the rescaled Hermite functions the contraction runs on), row k = n1, stored as bf16
// hi = RN(float(C')), lo = RN(float(C') - hi) in the tcgen05 canonical K-major layout without swizzle:
// 8x8 core matrices, element (n, k) at ((k/8) * (n_pad/8) + n/8) * 64 + (n%8) * 8 + k%8.  A tf32 copy goes
// to bop32 in the same layout with 8x4 core matrices of 4-byte elements, element (n, k) at
// ((k/4) * (n_pad/8) + n/8) * 32 + (n%8) * 4 + k%4: hi = RN_tf32(float(C')) at the shapelet's b_off, then
// lo = RN_tf32(float(C') - hi) (the difference is exact in FP32) k_pad * n_pad elements further.
// k_n (herm_k) for n = 0..kNmaxLimit, formed on the host in FP64 and uploaded at context creation.
__constant__ double c_herm_k[kNmaxLimit + 1];

__global__ void k_pack_coeff(int nnz_total, const int* n1, const int* n2, const double* c, const int* s_off,
                             const int* s_nmax, int n_shape, const int* b_off, const int* k_pad, const int* n_pad,
                             __nv_bfloat16* bop, float* bop32, unsigned* err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz_total) return;
  int q = 0;  // shapelet owning triple t (s_off is validated monotone on the host)
  while (q + 1 < n_shape && s_off[q + 1] <= t) ++q;
  int a = n1[t], b = n2[t], nmax = s_nmax[q];
  if (a < 0 || b < 0 || a + b > nmax) {
    atomicOr(err, WN_DEVERR_SKY);
    return;
  }
  int kk = (a + b) & 3;
  const float v = (float)(c[t] / (c_herm_k[a] * c_herm_k[b]));
  float re = kk == 0 ? v : (kk == 2 ? -v : 0.0f);
  float im = kk == 1 ? -v : (kk == 3 ? v : 0.0f);
  int np = n_pad[q], kp = k_pad[q];
  __nv_bfloat16* hi = bop + b_off[q];
  __nv_bfloat16* lo = hi + (size_t)np * kp;
  auto at = [&](int n, int k) { return ((k >> 3) * (np >> 3) + (n >> 3)) * 64 + (n & 7) * 8 + (k & 7); };
  // each (n1, n2) appears once per shapelet: duplicates are summed on the host check, so plain stores
  __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
  hi[at(2 * b, a)] = rh;
  lo[at(2 * b, a)] = __float2bfloat16_rn(re - __bfloat162float(rh));
  hi[at(2 * b + 1, a)] = ih;
  lo[at(2 * b + 1, a)] = __float2bfloat16_rn(im - __bfloat162float(ih));
  // tf32 copy: core matrices of 8 rows x 4 elements (16 B), same order; values rounded to nearest tf32,
  // hi then lo
  float* f = bop32 + b_off[q];
  float* fl = f + (size_t)np * kp;
  auto at32 = [&](int n, int k) { return ((k >> 2) * (np >> 3) + (n >> 3)) * 32 + (n & 7) * 4 + (k & 3); };
  const float rt = to_tf32(re), it = to_tf32(im);
  f[at32(2 * b, a)] = rt;
  fl[at32(2 * b, a)] = to_tf32(re - rt);
  f[at32(2 * b + 1, a)] = it;
  fl[at32(2 * b + 1, a)] = to_tf32(im - it);
}

static int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return WN_OK;
  return set_error(WN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The scales k_n of the packer, uploaded synchronously at context creation (wn_create, the context's
// device current), so that every later upload, on any stream, reads them complete.
int pack_constants_setup() {
  double k[kNmaxLimit + 1];
  for (int n = 0; n <= kNmaxLimit; ++n) k[n] = herm_k(n);
  return cuda_check(cudaMemcpyToSymbol(c_herm_k, k, sizeof(k)), "packer constants");
}

// Pack a new model: its records, shapelet headers and dense coefficient operands.  M->dmeta (device) and
// M->sh_host (sizes) are set up by the caller; the per-shapelet offsets and sizes are copied into dmeta.
int launch_pack(wn_ctx* ctx, const wn_sky* s, Model* M, cudaStream_t st) {
  if (s->n_shape > 0) {
    std::vector<int> meta(3 * (size_t)s->n_shape);
    for (int q = 0; q < s->n_shape; ++q) {
      meta[q] = M->sh_host[q].b_off;
      meta[s->n_shape + q] = M->sh_host[q].k_pad;
      meta[2 * s->n_shape + q] = M->sh_host[q].n_pad;
    }
    if (int r = cuda_check(cudaMemcpyAsync(M->dmeta, meta.data(), sizeof(int) * meta.size(), cudaMemcpyHostToDevice, st),
                           "pack metadata"))
      return r;
  }
  return launch_repack(ctx, s, M, st);
}

// Re-pack from the parameter values in s (device arrays; the shapelet structure, s_nmax and the triples,
// is read from the model): records, shapelet headers and dense operands.  Kernels and device-to-device
// copies only, asynchronous on st, no allocation.
int launch_repack(wn_ctx* ctx, const wn_sky* s, Model* M, cudaStream_t st) {
  const int npg = s->n_point + s->n_gauss;
  if (npg > 0) {
    k_pack_pg<<<(npg + 127) / 128, 128, 0, st>>>(*s, M->pg, ctx->d_err);
    if (int r = cuda_check(cudaGetLastError(), "pack points")) return r;
  }
  if (s->n_shape > 0) {
    const int* dm = M->dmeta;
    k_pack_shape<<<(s->n_shape + 63) / 64, 64, 0, st>>>(*s, dm, dm + s->n_shape, dm + 2 * s->n_shape, M->sh, ctx->d_err);
    cudaMemsetAsync(M->bop, 0, M->bop_elems * sizeof(__nv_bfloat16), st);
    cudaMemsetAsync(M->bop32, 0, M->bop_elems * sizeof(float), st);
    if (M->nnz > 0)
      k_pack_coeff<<<(M->nnz + 255) / 256, 256, 0, st>>>(M->nnz, s->s_n1, s->s_n2, s->s_coeff, s->s_off, s->s_nmax,
                                                         s->n_shape, dm, dm + s->n_shape, dm + 2 * s->n_shape, M->bop,
                                                         M->bop32, ctx->d_err);
    if (int r = cuda_check(cudaGetLastError(), "pack shapelets")) return r;
  }
  return WN_OK;
}

}  // namespace wn

namespace wn {

// Re-pack the dense coefficient operand of a resident model from a new coefficient vector (device,
// FP64, the model's triple order); dmeta holds the per-shapelet b_off, k_pad, n_pad (device ints).
int launch_pack_coeff(wn_ctx* ctx, Model* M, const double* coeff, const int* dmeta, cudaStream_t st) {
  if (M->n_shape == 0 || M->nnz == 0) return WN_OK;
  cudaMemsetAsync(M->bop, 0, M->bop_elems * sizeof(__nv_bfloat16), st);
  cudaMemsetAsync(M->bop32, 0, M->bop_elems * sizeof(float), st);
  k_pack_coeff<<<(M->nnz + 255) / 256, 256, 0, st>>>(M->nnz, M->m_n1(), M->m_n2(), coeff, M->m_off(), M->m_nmax(),
                                                     M->n_shape, dmeta, dmeta + M->n_shape, dmeta + 2 * M->n_shape,
                                                     M->bop, M->bop32, ctx->d_err);
  return cuda_check(cudaGetLastError(), "pack coefficients");
}

}  // namespace wn
