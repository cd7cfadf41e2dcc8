// C ABI of libwoden_b300: context, resident sky models, argument validation and dispatch to the
// prediction, peel and adjoint kernels.  Every step of the hot path runs in this library's kernels;
// the host only validates, plans launches and packs sizes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <mutex>
#include <set>

#include "wn_internal.cuh"

namespace wn {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

cudaError_t allow_max_dynamic_smem(const void* kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  int mx = 0;
  cudaFuncAttributes fa;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  // the limit excludes the kernel's own static shared memory
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}

static int ok() {
  g_last_error.clear();
  return WN_OK;
}

static int cuda_fail(cudaError_t e, const char* what) {
  return set_error(WN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Scoped device switch: every entry point runs on the context's device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

static int check_obs(const wn_obs* o, ObsDev& d) {
  if (!o) return set_error(WN_EINVAL, "obs is NULL");
  if (o->n_ant < 2 || o->n_base < 1 || o->n_time < 1 || o->n_chan < 1)
    return set_error(WN_EINVAL, "obs sizes must satisfy n_ant >= 2, n_base, n_time, n_chan >= 1");
  if ((long long)o->n_base * o->n_time > (1ll << 30) || (long long)o->n_base * o->n_time * o->n_chan > (1ll << 40))
    return set_error(WN_EINVAL, "obs too large");
  if ((long long)o->n_base > (long long)o->n_ant * (o->n_ant - 1) / 2)
    return set_error(WN_EINVAL, "n_base exceeds n_ant (n_ant - 1) / 2");
  if (!o->uvw || !o->freq_hz || !o->ant1 || !o->ant2) return set_error(WN_EINVAL, "obs has a NULL array");
  if (!(o->freq0_hz > 0.0) || !std::isfinite(o->freq0_hz)) return set_error(WN_EINVAL, "freq0_hz must be > 0");
  if (!(o->chan_spacing_hz >= 0.0) || !std::isfinite(o->chan_spacing_hz))
    return set_error(WN_EINVAL, "chan_spacing_hz must be >= 0 (0 = arbitrary channel list)");
  if (!std::isfinite(o->dec0) || std::fabs(o->dec0) > 0.5 * kPi) return set_error(WN_EINVAL, "dec0 out of range");
  d.n_ant = o->n_ant;
  d.n_base = o->n_base;
  d.n_time = o->n_time;
  d.n_chan = o->n_chan;
  d.n_rows = o->n_base * o->n_time;
  d.uvw = o->uvw;
  d.freq = o->freq_hz;
  d.ant1 = o->ant1;
  d.ant2 = o->ant2;
  d.dec0 = o->dec0;
  d.nu0 = o->freq0_hz;
  d.dnu = o->chan_spacing_hz;
  d.uniform = o->chan_spacing_hz > 0.0 || o->n_chan == 1;
  return WN_OK;
}

static int check_gains(const ObsDev& d, const void* gains, int gt, int gf, const void* data, PeelArgs& pa) {
  if (!gains || !data) return set_error(WN_EINVAL, "gains and data must not be NULL");
  if (!(gt == 1 || gt == d.n_time) || !(gf == 1 || gf == d.n_chan))
    return set_error(WN_EINVAL, "gains_t must be 1 or n_time and gains_f 1 or n_chan");
  pa.data = static_cast<const float2*>(data);
  pa.gains = static_cast<const float2*>(gains);
  pa.ant1 = d.ant1;
  pa.ant2 = d.ant2;
  pa.gt = gt;
  pa.gf = gf;
  pa.n_ant = d.n_ant;
  return WN_OK;
}

static Model* find_model(wn_ctx* ctx, int id) {
  auto it = ctx->models.find(id);
  return it == ctx->models.end() ? nullptr : it->second;
}

static void free_model(Model* M) {
  if (!M) return;
  cudaFree(M->pg);
  cudaFree(M->sh);
  cudaFree(M->bop);
  cudaFree(M->bop32);
  cudaFree(M->raw);
  cudaFree(M->s_meta);
  cudaFree(M->s_coeff);
  cudaFree(M->dmeta);
  delete M;
}

template <class T>
static cudaError_t dalloc(T** p, size_t n, size_t& total) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  total += n * sizeof(T);
  return dev_malloc(p, n * sizeof(T));
}

// Predict (mode STORE / ACCUM) or peel of one resident model on one observation.
static int run_model(wn_ctx* ctx, const ObsDev& d, const Model* M, float2* out, int mode, const PeelArgs& pa,
                     cudaStream_t st) {
  if (ctx->precision != WN_PREC_MIXED) return launch_phasor_fp64(ctx, d, M, out, mode, pa, true, st);
  int r = WN_OK;
  const bool have_pg = M->n_point + M->n_gauss > 0;
  if (have_pg || M->n_shape == 0) r = launch_phasor_table(ctx, d, M, out, mode, pa, st);
  if (r != WN_OK) return r;
  if (M->n_shape > 0) {
    // with points/Gaussians already written the shapelet pass adds (or subtracts G times) its part;
    // otherwise it applies the caller's mode itself
    const int smode = have_pg ? (mode == OUT_PEEL ? OUT_SUBG : OUT_ACCUM) : mode;
    r = launch_shapelets(ctx, d, M, out, smode, pa, st);
  }
  return r;
}

int run_model_peel(wn_ctx* ctx, const ObsDev& d, const Model* M, float2* out, const PeelArgs& pa, cudaStream_t st) {
  return run_model(ctx, d, M, out, OUT_PEEL, pa, st);
}

}  // namespace wn

using namespace wn;

namespace wn {
std::atomic<int> g_fail_allocs{0};
}

extern "C" {

const char* wn_last_error(void) { return g_last_error.c_str(); }

const char* wn_version(void) { return "woden_b300 0.1 (sm_103a)"; }

int wn_create(wn_ctx** out, int device) {
  if (!out) return set_error(WN_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return set_error(WN_EINVAL, "device index out of range");
  DeviceGuard g(device);
  wn_ctx* c = new wn_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  if (major != 10 || minor != 3) {
    delete c;
    return set_error(WN_EINVAL, "woden_b300 is built for sm_103a (B300); device reports sm_" + std::to_string(major) +
                                    std::to_string(minor));
  }
  e = dev_malloc(&c->d_err, sizeof(unsigned));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(error word)");
  }
  cudaMemset(c->d_err, 0, sizeof(unsigned));
  e = dev_malloc(&c->k1_part, k1_part_bytes(c->num_sms));
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "cudaMalloc(phasor tail partial sums)");
  }
  int r = static_scratch_setup(c);  // device address of wn_predict_static's array, this device current
  if (r == WN_OK) r = grad_constants_setup(c);  // the shapelet adjoint's constants
  if (r == WN_OK) r = k2_constants_setup();      // the shapelet contraction's recurrence constants
  if (r == WN_OK) r = pack_constants_setup();    // the coefficient packer's scales
  if (r != WN_OK) {
    cudaFree(c->k1_part);
    cudaFree(c->d_err);
    delete c;
    return r;
  }
  cudaDeviceSynchronize();
  *out = c;
  return ok();
}

void wn_destroy(wn_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->models) free_model(kv.second);
  cudaFree(ctx->d_err);
  cudaFree(ctx->k1_part);
  cudaFree(ctx->ws);
  cudaFree(ctx->ws2);
  cudaFree(ctx->lut);
  cudaFree(ctx->ws_spec);
  delete ctx;
}

int wn_set_precision(wn_ctx* ctx, int precision, int shape_mode) {
  if (!ctx) return set_error(WN_EINVAL, "ctx is NULL");
  if (precision != WN_PREC_MIXED && precision != WN_PREC_FP64 && precision != WN_PREC_FP64_UNTUNED)
    return set_error(WN_EINVAL, "unknown precision");
  if (shape_mode != WN_SHAPE_BF16X3 && shape_mode != WN_SHAPE_BF16X1 && shape_mode != WN_SHAPE_LUT_BF16X3 &&
      shape_mode != WN_SHAPE_TF32 && shape_mode != WN_SHAPE_TF32X3)
    return set_error(WN_EINVAL, "unknown shape mode");
  ctx->precision = precision;
  ctx->shape_mode = shape_mode;
  return ok();
}

int wn_debug_fail_allocs(int n) {
  if (n < 0) return set_error(WN_EINVAL, "wn_debug_fail_allocs: n must be >= 0");
  wn::g_fail_allocs.store(n);
  return ok();
}

int wn_set_trace(wn_ctx* ctx, int on) {
  if (!ctx) return set_error(WN_EINVAL, "ctx is NULL");
  ctx->trace = on ? 1 : 0;
  return ok();
}

int wn_device_errors(wn_ctx* ctx, uint32_t* flags_out) {
  if (!ctx || !flags_out) return set_error(WN_EINVAL, "NULL argument");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  unsigned v = 0;
  e = cudaMemcpy(&v, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read error word");
  cudaMemset(ctx->d_err, 0, sizeof(unsigned));
  *flags_out = v;
  return ok();
}

int wn_sky_upload(wn_ctx* ctx, const wn_sky* s, int* model_id, void* stream) {
  TraceRange trace_range(ctx, "wn_sky_upload");
  if (!ctx || !s || !model_id) return set_error(WN_EINVAL, "NULL argument");
  *model_id = 0;
  if (s->n_point < 0 || s->n_gauss < 0 || s->n_shape < 0) return set_error(WN_EINVAL, "negative component count");
  const long long n_comp = (long long)s->n_point + s->n_gauss + s->n_shape;
  if (n_comp > (1ll << 28)) return set_error(WN_EINVAL, "too many components");
  if (n_comp > 0 && (!s->l || !s->m || !s->flux || !s->alpha || !s->nu_ref))
    return set_error(WN_EINVAL, "sky has a NULL per-component array");
  if (s->n_gauss > 0 && (!s->g_maj || !s->g_min || !s->g_pa)) return set_error(WN_EINVAL, "sky has a NULL Gaussian array");
  if (s->n_shape > 0 && (!s->s_beta1 || !s->s_beta2 || !s->s_pa || !s->s_nmax || !s->s_off))
    return set_error(WN_EINVAL, "sky has a NULL shapelet array");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Model* M = new Model();
  M->n_point = s->n_point;
  M->n_gauss = s->n_gauss;
  M->n_shape = s->n_shape;
  // shapelet sizes back on the host (synchronous by contract)
  std::vector<int> nmax(s->n_shape), off(s->n_shape + 1, 0);
  if (s->n_shape > 0) {
    cudaError_t e = cudaMemcpyAsync(nmax.data(), s->s_nmax, sizeof(int) * s->n_shape, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(off.data(), s->s_off, sizeof(int) * (s->n_shape + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      delete M;
      return cuda_fail(e, "read shapelet sizes");
    }
    if (off[0] != 0) {
      delete M;
      return set_error(WN_EINVAL, "s_off[0] must be 0");
    }
    for (int q = 0; q < s->n_shape; ++q) {
      if (nmax[q] < 0 || nmax[q] > kNmaxLimit) {
        delete M;
        return set_error(WN_EINVAL, "shapelet n_max must lie in [0, 127]");
      }
      if (off[q + 1] < off[q] || off[q + 1] - off[q] > (nmax[q] + 1) * (nmax[q] + 2) / 2) {
        delete M;
        return set_error(WN_EINVAL, "s_off must be non-decreasing with at most p_tot triples per shapelet");
      }
    }
    M->nnz = off[s->n_shape];
    if (M->nnz > 0 && (!s->s_n1 || !s->s_n2 || !s->s_coeff)) {
      delete M;
      return set_error(WN_EINVAL, "sky has NULL coefficient triples");
    }
    // duplicate / range check of the triples on the host (upload is synchronous anyway)
    std::vector<int> n1(M->nnz), n2(M->nnz);
    if (M->nnz > 0) {
      cudaMemcpy(n1.data(), s->s_n1, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost);
      cudaMemcpy(n2.data(), s->s_n2, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost);
    }
    for (int q = 0; q < s->n_shape; ++q) {
      std::vector<char> seen((size_t)(nmax[q] + 1) * (nmax[q] + 1), 0);
      for (int k = off[q]; k < off[q + 1]; ++k) {
        if (n1[k] < 0 || n2[k] < 0 || n1[k] + n2[k] > nmax[q]) {
          delete M;
          return set_error(WN_EINVAL, "coefficient triple outside the triangle n1 + n2 <= n_max");
        }
        char& c = seen[(size_t)n1[k] * (nmax[q] + 1) + n2[k]];
        if (c) {
          delete M;
          return set_error(WN_EINVAL, "duplicate coefficient (n1, n2) in one shapelet");
        }
        c = 1;
      }
    }
    // Each shapelet is sized by the highest order its coefficients reach (n1 + n2), not the declared
    // n_max: the basis functions above it have zero coefficients and contribute nothing, so the
    // envelope is the same and the dense contraction carries no empty orders.
    for (int q = 0; q < s->n_shape; ++q) {
      int hi = 0;
      for (int k = off[q]; k < off[q + 1]; ++k) hi = std::max(hi, n1[k] + n2[k]);
      nmax[q] = hi;
    }
    M->sh_host.resize(s->n_shape);
    size_t b = 0;
    for (int q = 0; q < s->n_shape; ++q) {
      ShapeRec& r = M->sh_host[q];
      std::memset(&r, 0, sizeof(r));
      r.nmax = nmax[q];
      r.k_pad = (nmax[q] + 1 + 15) / 16 * 16;
      r.n_pad = (2 * (nmax[q] + 1) + 15) / 16 * 16;
      r.b_off = (int)b;
      b += 2 * (size_t)r.k_pad * r.n_pad;  // hi and lo operands
    }
    M->bop_elems = b;
  }
  M->s_off_host = off;
  M->s_nmax_host = nmax;
  size_t total = 0;
  const size_t n_raw = 5 * (size_t)n_comp + 3 * s->n_gauss + 3 * s->n_shape;
  cudaError_t e = dalloc(&M->pg, (size_t)s->n_point + s->n_gauss, total);
  if (e == cudaSuccess) e = dalloc(&M->sh, (size_t)s->n_shape, total);
  if (e == cudaSuccess) e = dalloc(&M->bop, M->bop_elems, total);
  if (e == cudaSuccess) e = dalloc(&M->bop32, M->bop_elems, total);  // tf32 hi and lo per shapelet
  if (e == cudaSuccess) e = dalloc(&M->raw, std::max<size_t>(n_raw, 1), total);
  if (e == cudaSuccess) e = dalloc(&M->s_meta, 2 * (size_t)s->n_shape + 1 + 2 * (size_t)M->nnz, total);
  if (e == cudaSuccess) e = dalloc(&M->s_coeff, (size_t)M->nnz, total);
  if (e == cudaSuccess) e = dalloc(&M->dmeta, 3 * (size_t)s->n_shape, total);
  if (e != cudaSuccess) {
    free_model(M);
    return set_error(WN_ENOMEM, std::string("model allocation: ") + cudaGetErrorString(e));
  }
  M->bytes = total;
  // raw FP64 copies (the FP64 form and the adjoint read these)
  auto cp = [&](double* dst, const double* src, size_t n) {
    if (n) cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  };
  cp(M->raw, s->l, n_comp);
  cp(M->raw + n_comp, s->m, n_comp);
  cp(M->raw + 2 * n_comp, s->flux, n_comp);
  cp(M->raw + 3 * n_comp, s->alpha, n_comp);
  cp(M->raw + 4 * n_comp, s->nu_ref, n_comp);
  cp(M->raw + 5 * n_comp, s->g_maj, s->n_gauss);
  cp(M->raw + 5 * n_comp + s->n_gauss, s->g_min, s->n_gauss);
  cp(M->raw + 5 * n_comp + 2 * s->n_gauss, s->g_pa, s->n_gauss);
  cp(M->raw + 5 * n_comp + 3 * s->n_gauss, s->s_beta1, s->n_shape);
  cp(M->raw + 5 * n_comp + 3 * s->n_gauss + s->n_shape, s->s_beta2, s->n_shape);
  cp(M->raw + 5 * n_comp + 3 * s->n_gauss + 2 * s->n_shape, s->s_pa, s->n_shape);
  if (s->n_shape > 0) {
    cudaMemcpyAsync(M->s_meta, nmax.data(), sizeof(int) * s->n_shape, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(M->s_meta + s->n_shape, off.data(), sizeof(int) * (s->n_shape + 1), cudaMemcpyHostToDevice, st);
    if (M->nnz > 0) {
      cudaMemcpyAsync(M->s_meta + 2 * s->n_shape + 1, s->s_n1, sizeof(int) * M->nnz, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(M->s_meta + 2 * s->n_shape + 1 + M->nnz, s->s_n2, sizeof(int) * M->nnz,
                      cudaMemcpyDeviceToDevice, st);
      cp(M->s_coeff, s->s_coeff, M->nnz);
    }
  }
  unsigned zero = 0;
  cudaMemcpyAsync(ctx->d_err, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, st);
  // the packers read each shapelet's order from the model's own (effective) n_max table
  wn_sky sp = *s;
  if (s->n_shape > 0) sp.s_nmax = M->s_meta;
  int r = launch_pack(ctx, &sp, M, st);
  if (r != WN_OK) {
    free_model(M);
    return r;
  }
  unsigned flags = 0;
  e = cudaMemcpyAsync(&flags, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_model(M);
    return cuda_fail(e, "sky upload");
  }
  if (flags & WN_DEVERR_SKY) {
    cudaMemset(ctx->d_err, 0, sizeof(unsigned));
    free_model(M);
    return set_error(WN_EINVAL, "sky rejected: l^2 + m^2 >= 1, nu_ref <= 0, a negative width or a non-finite value");
  }
  // host copy of the shapelet headers (read back: sizes and offsets are needed to plan launches)
  if (s->n_shape > 0) {
    e = cudaMemcpy(M->sh_host.data(), M->sh, sizeof(ShapeRec) * s->n_shape, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      free_model(M);
      return cuda_fail(e, "read shapelet headers");
    }
  }
  const int id = ctx->next_id++;
  ctx->models[id] = M;
  *model_id = id;
  return ok();
}

int wn_sky_update(wn_ctx* ctx, int model_id, const wn_sky* s, void* stream) {
  TraceRange trace_range(ctx, "wn_sky_update");
  if (!ctx || !s) return set_error(WN_EINVAL, "NULL argument");
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (s->n_point != M->n_point || s->n_gauss != M->n_gauss || s->n_shape != M->n_shape)
    return set_error(WN_EINVAL, "wn_sky_update: component counts differ from the resident model's");
  const long long n_comp = (long long)M->n_comp();
  if (n_comp > 0 && (!s->l || !s->m || !s->flux || !s->alpha || !s->nu_ref))
    return set_error(WN_EINVAL, "sky has a NULL per-component array");
  if (M->n_gauss > 0 && (!s->g_maj || !s->g_min || !s->g_pa)) return set_error(WN_EINVAL, "sky has a NULL Gaussian array");
  if (M->n_shape > 0 && (!s->s_beta1 || !s->s_beta2 || !s->s_pa)) return set_error(WN_EINVAL, "sky has a NULL shapelet array");
  if (M->nnz > 0 && !s->s_coeff) return set_error(WN_EINVAL, "sky has NULL shapelet coefficients");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto cp = [&](double* dst, const double* src, size_t n) {
    if (n) cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  };
  // the raw FP64 tables (the FP64 form and the adjoint read these) and the coefficients
  cp(M->raw, s->l, n_comp);
  cp(M->raw + n_comp, s->m, n_comp);
  cp(M->raw + 2 * n_comp, s->flux, n_comp);
  cp(M->raw + 3 * n_comp, s->alpha, n_comp);
  cp(M->raw + 4 * n_comp, s->nu_ref, n_comp);
  cp(M->raw + 5 * n_comp, s->g_maj, M->n_gauss);
  cp(M->raw + 5 * n_comp + M->n_gauss, s->g_min, M->n_gauss);
  cp(M->raw + 5 * n_comp + 2 * M->n_gauss, s->g_pa, M->n_gauss);
  cp(M->raw + 5 * n_comp + 3 * M->n_gauss, s->s_beta1, M->n_shape);
  cp(M->raw + 5 * n_comp + 3 * M->n_gauss + M->n_shape, s->s_beta2, M->n_shape);
  cp(M->raw + 5 * n_comp + 3 * M->n_gauss + 2 * M->n_shape, s->s_pa, M->n_shape);
  cp(M->s_coeff, s->s_coeff, M->nnz);
  // re-pack with the model's own shapelet structure (effective orders, offsets, triples)
  wn_sky sp = *s;
  if (M->n_shape > 0) {
    sp.s_nmax = M->m_nmax();
    sp.s_off = M->m_off();
    sp.s_n1 = M->m_n1();
    sp.s_n2 = M->m_n2();
    sp.s_coeff = M->s_coeff;
  }
  if (int r = launch_repack(ctx, &sp, M, st)) return r;
  if (M->n_shape > 0) {
    // the launch planning reads each shapelet's amplitude terms from the host copy of its header
    cudaError_t e = cudaMemcpyAsync(M->sh_host.data(), M->sh, sizeof(ShapeRec) * M->n_shape, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "read shapelet headers");
  }
  return ok();
}

int wn_sky_free(wn_ctx* ctx, int model_id) {
  if (!ctx) return set_error(WN_EINVAL, "ctx is NULL");
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  free_model(M);
  ctx->models.erase(model_id);
  return ok();
}

int wn_sky_bytes(wn_ctx* ctx, int model_id, size_t* bytes_out) {
  if (!ctx || !bytes_out) return set_error(WN_EINVAL, "NULL argument");
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  *bytes_out = M->bytes;
  return ok();
}

int wn_sky_shapelet_operand(wn_ctx* ctx, int model_id, int q, void* host_out, size_t bytes, int* k_pad, int* n_pad) {
  if (!ctx || !k_pad || !n_pad) return set_error(WN_EINVAL, "NULL argument");
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (q < 0 || q >= M->n_shape) return set_error(WN_EINVAL, "shapelet index out of range");
  const ShapeRec& h = M->sh_host[q];
  *k_pad = h.k_pad;
  *n_pad = h.n_pad;
  if (!host_out) return ok();
  const size_t need = (size_t)4 * h.k_pad * h.n_pad;
  if (bytes < need) return set_error(WN_EINVAL, "wn_sky_shapelet_operand: buffer shorter than 4 k_pad n_pad bytes");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaMemcpy(host_out, M->bop + h.b_off, need, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "wn_sky_shapelet_operand copy");
  return ok();
}

int wn_sky_shapelet_operand_tf32(wn_ctx* ctx, int model_id, int q, void* host_out, size_t bytes, int* k_pad, int* n_pad) {
  if (!ctx || !k_pad || !n_pad) return set_error(WN_EINVAL, "NULL argument");
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (q < 0 || q >= M->n_shape) return set_error(WN_EINVAL, "shapelet index out of range");
  const ShapeRec& h = M->sh_host[q];
  *k_pad = h.k_pad;
  *n_pad = h.n_pad;
  if (!host_out) return ok();
  const size_t one = (size_t)4 * h.k_pad * h.n_pad;
  if (bytes < one) return set_error(WN_EINVAL, "wn_sky_shapelet_operand_tf32: buffer shorter than 4 k_pad n_pad bytes");
  const size_t need = bytes >= 2 * one ? 2 * one : one;  // hi, and lo when the buffer holds both
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaMemcpy(host_out, M->bop32 + h.b_off, need, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "wn_sky_shapelet_operand_tf32 copy");
  return ok();
}

int wn_predict(wn_ctx* ctx, const wn_obs* obs, int model_id, void* vis_c64, int accumulate, void* stream) {
  TraceRange trace_range(ctx, "wn_predict");
  if (!ctx || !vis_c64) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (accumulate != 0 && accumulate != 1) return set_error(WN_EINVAL, "accumulate must be 0 or 1");
  DeviceGuard g(ctx->device);
  PeelArgs pa;
  int r = run_model(ctx, d, M, static_cast<float2*>(vis_c64), accumulate ? OUT_ACCUM : OUT_STORE, pa,
                    static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

int wn_peel(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t, int gains_f,
            const void* data_c64, void* resid_c64, void* stream) {
  TraceRange trace_range(ctx, "wn_peel");
  if (!ctx || !resid_c64) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  PeelArgs pa;
  if (int r = check_gains(d, gains_c64, gains_t, gains_f, data_c64, pa)) return r;
  DeviceGuard g(ctx->device);
  int r = run_model(ctx, d, M, static_cast<float2*>(resid_c64), OUT_PEEL, pa, static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

int wn_peel_model(wn_ctx* ctx, const wn_obs* obs, const void* gains_c64, int gains_t, int gains_f,
                  const void* data_c64, const void* model_c64, void* resid_c64, void* stream) {
  TraceRange trace_range(ctx, "wn_peel_model");
  if (!ctx || !model_c64 || !resid_c64) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  PeelArgs pa;
  if (int r = check_gains(d, gains_c64, gains_t, gains_f, data_c64, pa)) return r;
  DeviceGuard g(ctx->device);
  int r = launch_peel_model(ctx, d, pa, static_cast<const float2*>(model_c64), static_cast<float2*>(resid_c64),
                            static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

int wn_predict_grad(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t, int gains_f,
                    const void* data_c64, void* resid_c64, const wn_sky_grad* grad_out, double* loss_out,
                    void* stream) {
  TraceRange trace_range(ctx, "wn_predict_grad");
  if (!ctx || !resid_c64 || !grad_out) return set_error(WN_EINVAL, "NULL argument");
  if (resid_c64 == data_c64) return set_error(WN_EINVAL, "wn_predict_grad: resid must not alias data");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  PeelArgs pa;
  if (int r = check_gains(d, gains_c64, gains_t, gains_f, data_c64, pa)) return r;
  if (ctx->precision != WN_PREC_MIXED) return set_error(WN_EINVAL, "wn_predict_grad runs in the mixed precision only");
  DeviceGuard g(ctx->device);
  int r = launch_grad(ctx, d, M, pa, static_cast<float2*>(resid_c64), grad_out, loss_out,
                      static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

int wn_fit_shapelets(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t, int gains_f,
                     const void* data_c64, int n_iter, double tol, double* coeff_inout, double* info, void* stream) {
  TraceRange trace_range(ctx, "wn_fit_shapelets");
  if (!ctx || !coeff_inout) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (M->n_shape < 1 || M->nnz < 1) return set_error(WN_EINVAL, "wn_fit_shapelets: the model has no shapelet coefficients");
  PeelArgs pa;
  if (int r = check_gains(d, gains_c64, gains_t, gains_f, data_c64, pa)) return r;
  if (n_iter < 0 || n_iter > 100000 || !(tol >= 0.0)) return set_error(WN_EINVAL, "wn_fit_shapelets: bad n_iter or tol");
  if (ctx->precision != WN_PREC_MIXED) return set_error(WN_EINVAL, "wn_fit_shapelets runs in the mixed precision only");
  DeviceGuard g(ctx->device);
  int r = launch_fit_shapelets(ctx, d, M, pa, n_iter, tol, coeff_inout, info, static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

int wn_calibrate(wn_ctx* ctx, const wn_obs* obs, const void* model_c64, const void* data_c64, void* gains_c64,
                 int n_iter, void* stream) {
  TraceRange trace_range(ctx, "wn_calibrate");
  if (!ctx || !model_c64 || !data_c64 || !gains_c64) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  if (n_iter < 1 || n_iter > 1000) return set_error(WN_EINVAL, "wn_calibrate: n_iter must be in [1, 1000]");
  if (d.n_ant > 128) return set_error(WN_EINVAL, "wn_calibrate: at most 128 antennas");
  if (((uintptr_t)model_c64 | (uintptr_t)data_c64 | (uintptr_t)gains_c64) & 7)
    return set_error(WN_EINVAL, "wn_calibrate: complex64 arrays must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  int r = launch_calibrate(ctx, d, static_cast<const float2*>(model_c64), static_cast<const float2*>(data_c64),
                           static_cast<float2*>(gains_c64), n_iter, static_cast<cudaStream_t>(stream));
  return r == WN_OK ? ok() : r;
}

// Allocation-free prediction: like wn_predict, but the shapelet launches take their per-row and
// per-channel tables from a fixed device array instead of the context's workspace, so the call
// makes no device allocation.  Points and Gaussians, and the FP64 form, need no scratch at all.
int wn_predict_static(wn_ctx* ctx, const wn_obs* obs, int model_id, void* vis_c64, int accumulate, void* stream) {
  TraceRange trace_range(ctx, "wn_predict_static");
  if (!ctx || !vis_c64) return set_error(WN_EINVAL, "NULL argument");
  ObsDev d;
  if (int r = check_obs(obs, d)) return r;
  Model* M = find_model(ctx, model_id);
  if (!M) return set_error(WN_ENOTFOUND, "unknown model id");
  if (accumulate != 0 && accumulate != 1) return set_error(WN_EINVAL, "accumulate must be 0 or 1");
  if (M->n_shape > 0 && ctx->shape_mode == WN_SHAPE_LUT_BF16X3 && !ctx->lut)
    return set_error(WN_EINVAL, "wn_predict_static: the lookup-table shapelet mode needs its table, built by a first "
                                "wn_predict in that mode");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int mode = accumulate ? OUT_ACCUM : OUT_STORE;
  PeelArgs pa;
  int r = WN_OK;
  if (ctx->precision != WN_PREC_MIXED) {
    r = launch_phasor_fp64(ctx, d, M, static_cast<float2*>(vis_c64), mode, pa, true, st);
  } else {
    const bool have_pg = M->n_point + M->n_gauss > 0;
    if (have_pg || M->n_shape == 0) r = launch_phasor_mixed(ctx, d, M, static_cast<float2*>(vis_c64), mode, pa, st);
    if (r == WN_OK && M->n_shape > 0)
      r = launch_shapelets_static(ctx, d, M, static_cast<float2*>(vis_c64), have_pg ? OUT_ACCUM : mode, pa, st);
  }
  return r == WN_OK ? ok() : r;
}

}  // extern "C"
