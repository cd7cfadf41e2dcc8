// K8: visibility-space fitting of shapelet coefficients.  The visibilities are linear in the shapelet
// coefficients C (eq:shape-env): V = V_fixed + A C, where (A C)(vis) = G sum_k C_k S(nu) (-i)^(n1+n2)
// phi_n1(x) phi_n2(y) e^{-2 pi i tau nu / c} and V_fixed holds the model's points and Gaussians.  The
// least-squares C of |D - V|^2 over all visibilities solves A^T A C = A^T (D - V_fixed); this is the
// visibility-space counterpart of the image-space fit of Sec. 2.2.  It is solved by CGLS (conjugate
// gradients on the normal equations) without forming A^T A.
//  - A p is one shapelet contraction (K2) of the model re-packed with coefficients p, subtracted as G V
//    from a zero buffer.
//  - A^T r is the coefficient part of the adjoint (K4) for residual r, times -1/2.
//  - Vector updates and norms are small kernels here; norms are reduced in FP64 in a fixed order.
// Positions, scales and position angles stay fixed.
#include <cmath>
#include <vector>

#include "wn_internal.cuh"

namespace wn {

int launch_grad_shape_coeff(wn_ctx* ctx, const ObsDev& o, const Model* M, const PeelArgs& pa, const float2* resid,
                            double* gcoeff, cudaStream_t st);
int launch_pack_coeff(wn_ctx* ctx, Model* M, const double* coeff, const int* dmeta, cudaStream_t st);
int run_model_peel(wn_ctx* ctx, const ObsDev& d, const Model* M, float2* out, const PeelArgs& pa, cudaStream_t st);

constexpr int K8_T = 256;

__global__ void k8_norm2_c64(const float2* v, size_t n, double* part) {
  __shared__ double red[K8_T];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * K8_T + threadIdx.x; i < n; i += (size_t)gridDim.x * K8_T) {
    const float2 x = v[i];
    s += (double)x.x * x.x + (double)x.y * x.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = K8_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k8_norm2_f64(const double* v, int n, double* part) {
  __shared__ double red[K8_T];
  double s = 0.0;
  for (int i = blockIdx.x * K8_T + threadIdx.x; i < n; i += gridDim.x * K8_T) s += v[i] * v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = K8_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k8_sum(const double* part, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

__global__ void k8_axpy_c64(float2* y, const float2* x, size_t n, float a) {  // y += a x
  for (size_t i = (size_t)blockIdx.x * K8_T + threadIdx.x; i < n; i += (size_t)gridDim.x * K8_T) {
    const float2 u = y[i], v = x[i];
    y[i] = make_float2(fmaf(a, v.x, u.x), fmaf(a, v.y, u.y));
  }
}

__global__ void k8_vec_f64(double* y, const double* x, int n, double a, double b) {  // y = a x + b y
  for (int i = blockIdx.x * K8_T + threadIdx.x; i < n; i += gridDim.x * K8_T) y[i] = a * x[i] + b * y[i];
}

// The CGLS scalars stay on the device (no host round trip per iteration): sc = {gam0, gam, qq, gnew,
// stop, iterations done}.  Once stop is set every update below leaves the state as it is, so the
// iterations the host launches before it sees the flag change nothing.
enum { SC_GAM0 = 0, SC_GAM = 1, SC_QQ = 2, SC_GNEW = 3, SC_STOP = 4, SC_IT = 5 };

__global__ void k8_cg_qq(double* sc) {  // breakdown: |A p|^2 not positive
  if (threadIdx.x == 0 && sc[SC_STOP] == 0.0 && !(sc[SC_QQ] > 0.0)) sc[SC_STOP] = 1.0;
}

// x += alpha p and r += alpha q (q = -A p), alpha = gam / qq
__global__ void k8_cg_step(double* x, const double* p, int nnz, float2* r, const float2* q, size_t n_vis,
                           const double* sc) {
  if (sc[SC_STOP] != 0.0) return;
  const double alpha = sc[SC_GAM] / sc[SC_QQ];
  const float af = (float)alpha;
  const size_t stride = (size_t)gridDim.x * K8_T;
  for (size_t i = (size_t)blockIdx.x * K8_T + threadIdx.x; i < (size_t)nnz; i += stride) x[i] = alpha * p[i] + x[i];
  for (size_t i = (size_t)blockIdx.x * K8_T + threadIdx.x; i < n_vis; i += stride) {
    const float2 u = r[i], v = q[i];
    r[i] = make_float2(fmaf(af, v.x, u.x), fmaf(af, v.y, u.y));
  }
}

// p = s + beta p, beta = gnew / gam
__global__ void k8_cg_dir(double* p, const double* s, int nnz, const double* sc) {
  if (sc[SC_STOP] != 0.0) return;
  const double beta = sc[SC_GNEW] / sc[SC_GAM];
  for (int i = blockIdx.x * K8_T + threadIdx.x; i < nnz; i += gridDim.x * K8_T) p[i] = 1.0 * s[i] + beta * p[i];
}

// gam = gnew, one more iteration done; stop once gam <= tol^2 gam0 (or is not positive)
__global__ void k8_cg_finish(double* sc, double tol2) {
  if (threadIdx.x != 0 || sc[SC_STOP] != 0.0) return;
  sc[SC_GAM] = sc[SC_GNEW];
  sc[SC_IT] += 1.0;
  if (!(sc[SC_GAM] > tol2 * sc[SC_GAM0] && sc[SC_GAM] > 0.0)) sc[SC_STOP] = 1.0;
}

int launch_fit_shapelets(wn_ctx* ctx, const ObsDev& o, Model* M, const PeelArgs& pa, int n_iter, double tol,
                         double* coeff, double* info, cudaStream_t st) {
  const size_t n_vis = (size_t)o.n_rows * o.n_chan;
  const int nnz = M->nnz, S = M->n_shape;
  const int vgrid = ctx->num_sms * 2, cgrid = std::max(1, std::min(ctx->num_sms, (nnz + K8_T - 1) / K8_T));
  // scratch: r, q (visibilities), s, p, g (coefficients), meta (b_off, k_pad, n_pad), partials, scalar
  float2 *r = nullptr, *q = nullptr;
  double *sv = nullptr, *pv = nullptr, *gv = nullptr, *part = nullptr, *scal = nullptr;
  int* meta = nullptr;
  cudaError_t e = dev_malloc(&r, n_vis * sizeof(float2));
  if (e == cudaSuccess) e = dev_malloc(&q, n_vis * sizeof(float2));
  if (e == cudaSuccess) e = dev_malloc(&sv, 3 * (size_t)nnz * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc(&part, (vgrid + 8) * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc(&meta, 3 * (size_t)S * sizeof(int));
  auto release = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(r);
    cudaFree(q);
    cudaFree(sv);
    cudaFree(part);
    cudaFree(meta);
  };
  if (e != cudaSuccess) {
    release();
    return set_error(WN_ENOMEM, std::string("fit workspace: ") + cudaGetErrorString(e));
  }
  pv = sv + nnz;
  gv = pv + nnz;
  scal = part + vgrid;
  cudaMemsetAsync(sv, 0, 3 * (size_t)nnz * sizeof(double), st);
  {
    std::vector<int> h(3 * S);
    for (int k = 0; k < S; ++k) {
      h[k] = M->sh_host[k].b_off;
      h[S + k] = M->sh_host[k].k_pad;
      h[2 * S + k] = M->sh_host[k].n_pad;
    }
    cudaMemcpyAsync(meta, h.data(), sizeof(int) * 3 * S, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  auto norm2_vis = [&](const float2* v, double* out_host) {
    k8_norm2_c64<<<vgrid, K8_T, 0, st>>>(v, n_vis, part);
    k8_sum<<<1, 32, 0, st>>>(part, vgrid, scal);
    cudaMemcpyAsync(out_host, scal, sizeof(double), cudaMemcpyDeviceToHost, st);
  };
  auto norm2_coef = [&](const double* v, double* out_host) {
    k8_norm2_f64<<<cgrid, K8_T, 0, st>>>(v, nnz, part);
    k8_sum<<<1, 32, 0, st>>>(part, cgrid, scal);
    cudaMemcpyAsync(out_host, scal, sizeof(double), cudaMemcpyDeviceToHost, st);
  };
  // s = A^T r = -1/2 dL/dC
  auto atr = [&](const float2* res) -> int {
    if (int rc = launch_grad_shape_coeff(ctx, o, M, pa, res, gv, st)) return rc;
    k8_vec_f64<<<cgrid, K8_T, 0, st>>>(sv, gv, nnz, -0.5, 0.0);
    return WN_OK;
  };
  int rc = WN_OK;
  double rr0 = 0, rr = 0, gam0 = 0, gam = 0;
  int it = 0;
  double* sc = scal;  // device CGLS scalars (SC_*)
  // r0 = D - G (V_fixed + A x0)
  if (!rc) rc = launch_pack_coeff(ctx, M, coeff, meta, st);
  if (!rc) rc = run_model_peel(ctx, o, M, r, pa, st);
  if (!rc) norm2_vis(r, &rr0);
  if (!rc) rc = atr(r);
  if (!rc) {
    cudaMemcpyAsync(pv, sv, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
    norm2_coef(sv, &gam0);
    cudaStreamSynchronize(st);
    gam = gam0;
    rr = rr0;
    const double h[6] = {gam0, gam0, 0.0, 0.0, (n_iter > 0 && gam0 > 0.0 && tol < 1.0) ? 0.0 : 1.0, 0.0};
    cudaMemcpyAsync(sc, h, sizeof(h), cudaMemcpyHostToDevice, st);
  }
  const double tol2 = tol * tol;
  const int kCheck = 8;  // iterations between looks at the device's stop flag
  bool stopped = rc != WN_OK || !(n_iter > 0 && gam0 > 0.0 && tol < 1.0);
  // One CGLS iteration's launches on stream s, with no host synchronisation.
  auto iteration = [&](cudaStream_t s) -> int {
    // q = -A p
    if (int r2 = launch_pack_coeff(ctx, M, pv, meta, s)) return r2;
    cudaMemsetAsync(q, 0, n_vis * sizeof(float2), s);
    if (int r2 = launch_shapelets(ctx, o, M, q, OUT_SUBG, pa, s)) return r2;
    k8_norm2_c64<<<vgrid, K8_T, 0, s>>>(q, n_vis, part);
    k8_sum<<<1, 32, 0, s>>>(part, vgrid, sc + SC_QQ);
    k8_cg_qq<<<1, 32, 0, s>>>(sc);
    k8_cg_step<<<vgrid, K8_T, 0, s>>>(coeff, pv, nnz, r, q, n_vis, sc);  // x += alpha p, r -= alpha A p
    // s = A^T r = -1/2 dL/dC
    if (int r2 = launch_grad_shape_coeff(ctx, o, M, pa, r, gv, s)) return r2;
    k8_vec_f64<<<cgrid, K8_T, 0, s>>>(sv, gv, nnz, -0.5, 0.0);
    k8_norm2_f64<<<cgrid, K8_T, 0, s>>>(sv, nnz, part);
    k8_sum<<<1, 32, 0, s>>>(part, cgrid, sc + SC_GNEW);
    k8_cg_dir<<<cgrid, K8_T, 0, s>>>(pv, sv, nnz, sc);  // p = s + beta p
    k8_cg_finish<<<1, 32, 0, s>>>(sc, tol2);
    return WN_OK;
  };
  // The iterations run on a private stream (a graph cannot be captured on the legacy stream): the first
  // as plain launches, which also sizes the workspaces, the rest as replays of a CUDA graph of one
  // iteration, which removes the per-launch gaps.  If the capture fails they stay plain launches.
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  if (!stopped) {
    cudaError_t es = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventRecord(ev, st);
    if (es == cudaSuccess) es = cudaStreamWaitEvent(cs, ev, 0);
    if (es != cudaSuccess) rc = set_error(WN_ECUDA, std::string("fit stream: ") + cudaGetErrorString(es));
  }
  for (int launched = 0; !rc && !stopped && launched < n_iter; ++launched) {
    if (gexec) {
      const cudaError_t eg = cudaGraphLaunch(gexec, cs);
      if (eg != cudaSuccess) rc = set_error(WN_ECUDA, std::string("fit graph launch: ") + cudaGetErrorString(eg));
    } else {
      rc = iteration(cs);
    }
    if (rc) break;
    if (launched == 0 && n_iter > 1 &&
        cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rcap = iteration(cs);  // recorded, not run
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (rcap != WN_OK || ec != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) gexec = nullptr;
      cudaGetLastError();  // a failed capture leaves plain launches, not an error
    }
    if ((launched + 1) % kCheck == 0 || launched + 1 == n_iter) {
      double h[6];
      cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, cs);
      cudaStreamSynchronize(cs);
      stopped = h[SC_STOP] != 0.0;
    }
  }
  if (cs) {
    cudaEventRecord(ev, cs);
    cudaStreamWaitEvent(st, ev, 0);
    cudaStreamSynchronize(cs);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaEventDestroy(ev);
  }
  if (!rc) {
    double h[6];
    cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    gam = h[SC_GAM];
    it = (int)h[SC_IT];
  }
  // the model keeps the fitted coefficients: dense operand and the FP64 copy
  if (!rc) rc = launch_pack_coeff(ctx, M, coeff, meta, st);
  if (!rc) {
    cudaMemcpyAsync(M->s_coeff, coeff, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
    norm2_vis(r, &rr);
    cudaStreamSynchronize(st);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = set_error(WN_ECUDA, std::string("fit: ") + cudaGetErrorString(e));
  }
  if (info) {
    info[0] = it;
    info[1] = gam0 > 0 ? std::sqrt(gam / gam0) : 0.0;
    info[2] = rr;
    info[3] = rr0;
  }
  release();
  return rc;
}

}  // namespace wn
