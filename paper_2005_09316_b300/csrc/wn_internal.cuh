// Internal definitions shared by the CUDA translation units of libwoden_b300.
// Device helpers: bounded mbarrier waits, TMA bulk copies, double-float phase reduction,
// fast and accurate phasors.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "woden_b300.h"
#include <nvtx3/nvToolsExt.h>

namespace wn {

// Device allocations of the library go through dev_malloc.  g_fail_allocs > 0 (wn_debug_fail_allocs)
// makes that many of the next ones fail as an out-of-memory cudaMalloc would, without calling CUDA:
// host-side fault injection for the allocation-failure paths.
extern std::atomic<int> g_fail_allocs;
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  int n = g_fail_allocs.load();
  while (n > 0)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

constexpr double kC = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
// Gaussian envelope exponent pi^2 / (4 ln 2) (eq:gauss-env), and the shapelet scale pi / sqrt(2 ln 2)
// (eq:scale-shape-x/y).
constexpr double kGaussE = 3.5597074346203355;   // pi^2 / (4 ln 2)
constexpr double kShapeK = 2.6682231827177734;   // pi / sqrt(2 ln 2)
constexpr double kLog2e = 1.4426950408889634;
constexpr int kNmaxLimit = 127;

// Scale k_n of the rescaled Hermite functions g_n = k_n phi_n that the shapelet contraction runs on:
// k_0 = k_1 = 1, k_(n+1) = k_(n-1) sqrt((n+1)/n).  The normalised recurrence
// phi_(n+1) = sqrt(2/(n+1)) x phi_n - sqrt(n/(n+1)) phi_(n-1) then reads g_(n+1) = e_n x g_n - g_(n-1)
// with e_n = sqrt(2/(n+1)) k_(n+1)/k_n: two operations per order instead of three.  The coefficient
// operand carries 1/(k_n1 k_n2), so that sum g C' g = sum phi C phi.  FP64, each step correctly rounded
// (the same value on the host and the device); k_n stays within [1, 4] for n <= 128.
__host__ __device__ inline double herm_k(int n) {
  double km = 1.0, k = 1.0;  // k_(m-1), k_m
  for (int m = 1; m < n; ++m) {
    const double kn = km * sqrt((double)(m + 1) / (double)m);
    km = k;
    k = kn;
  }
  return k;
}

// Packed point / Gaussian component (64 bytes).  Points first, then Gaussians.
struct __align__(16) PGRec {
  // direction cosines l, m and n - 1 = -(l^2+m^2)/(1+sqrt(1-l^2-m^2)), each an unevaluated float pair
  // (x = xh + xl, split from FP64) so the phase argument can be formed in double-float FP32
  float lh, ll, mh, ml, nh, nl;
  double lref;        // log2(nu_ref)
  float lS;           // log2 |S_ref|
  float alpha;        // spectral index
  float sgn;          // sign of S_ref (+1, -1, or 0)
  float ga, gb, gc;   // Gaussian: log2 xi = -(ga u^2 + gb u v + gc v^2) (nu/c)^2 * kGaussE*log2(e)
  float pad0, pad1;
};
static_assert(sizeof(PGRec) == 64, "PGRec layout");

// Packed shapelet header (64 bytes).  The re-phasing frame depends on the phase-centre declination
// of the observation and is formed at launch (shapelet_frame).
struct __align__(16) ShapeRec {
  double l, m, nm1, lref;
  float lS, alpha, sgn;
  float kx_u, kx_v;     // x = (kx_u u' + kx_v v') nu/c : beta1 * K * (sin pa, cos pa)
  float ky_u, ky_v;     // y = (ky_u u' + ky_v v') nu/c : beta2 * K * (cos pa, -sin pa)
  int nmax, k_pad, n_pad;
  int b_off;            // element offset of this shapelet's dense operand in the model's B buffer
};
static_assert(sizeof(ShapeRec) == 80, "ShapeRec layout");

// A resident sky model (device memory owned by the context).
struct Model {
  int n_point = 0, n_gauss = 0, n_shape = 0, nnz = 0;
  PGRec* pg = nullptr;             // [n_point + n_gauss]
  ShapeRec* sh = nullptr;          // [n_shape]
  std::vector<ShapeRec> sh_host;   // host copy of the headers (sizes, offsets)
  __nv_bfloat16* bop = nullptr;    // dense shapelet B operands (hi then lo per shapelet), UMMA layout
  float* bop32 = nullptr;          // the same operands as tf32 hi then lo (K-major, 4-byte elements), shapelet q at b_off
  size_t bop_elems = 0;
  // raw FP64 copies for the FP64 form and the adjoint
  double* raw = nullptr;           // l, m, flux, alpha, nu_ref [n_comp] each; g_maj,g_min,g_pa; s_b1,s_b2,s_pa
  int* s_meta = nullptr;           // s_nmax [n_shape], s_off [n_shape+1], s_n1 [nnz], s_n2 [nnz]
  double* s_coeff = nullptr;       // [nnz]
  int* dmeta = nullptr;            // [3][n_shape]: each shapelet's b_off, k_pad, n_pad (the packers read these)
  std::vector<int> s_off_host, s_nmax_host;
  size_t bytes = 0;
  int n_comp() const { return n_point + n_gauss + n_shape; }
  const double* r_l() const { return raw; }
  const double* r_m() const { return raw + n_comp(); }
  const double* r_flux() const { return raw + 2 * n_comp(); }
  const double* r_alpha() const { return raw + 3 * n_comp(); }
  const double* r_nuref() const { return raw + 4 * n_comp(); }
  const double* r_gmaj() const { return raw + 5 * n_comp(); }
  const double* r_gmin() const { return raw + 5 * n_comp() + n_gauss; }
  const double* r_gpa() const { return raw + 5 * n_comp() + 2 * n_gauss; }
  const double* r_sb1() const { return raw + 5 * n_comp() + 3 * n_gauss; }
  const double* r_sb2() const { return raw + 5 * n_comp() + 3 * n_gauss + n_shape; }
  const double* r_spa() const { return raw + 5 * n_comp() + 3 * n_gauss + 2 * n_shape; }
  const int* m_nmax() const { return s_meta; }
  const int* m_off() const { return s_meta + n_shape; }
  const int* m_n1() const { return s_meta + 2 * n_shape + 1; }
  const int* m_n2() const { return s_meta + 2 * n_shape + 1 + nnz; }
};

}  // namespace wn

struct wn_ctx {
  int device = 0;
  int num_sms = 148;
  int precision = WN_PREC_MIXED;
  int shape_mode = WN_SHAPE_BF16X3;
  int trace = 0;  // NVTX ranges around the entry points (wn_set_trace)
  unsigned* d_err = nullptr;
  std::map<int, wn::Model*> models;
  int next_id = 1;
  // growable workspaces: shapelet prediction tables, and the adjoint's tables and partial sums
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* ws2 = nullptr;
  size_t ws2_bytes = 0;
  float* lut = nullptr;  // basis table of the lookup-table shapelet mode (built on first use)
  float2* k1_part = nullptr;  // partial sums of the split tail tiles of the phasor launch (fixed size)
  float4* static_scratch = nullptr;  // device address of wn_predict_static's file-scope array (set-up)
  float* ws_spec = nullptr;  // spectrum table of the point/Gaussian phasor launch (grow-only)
  size_t ws_spec_bytes = 0;
};
// An NVTX range named after the entry point, for the duration of the call, when the context traces.
// NVTX is header-only: without a tool attached a range costs a few nanoseconds.
struct TraceRange {
  bool on;
  TraceRange(const wn_ctx* ctx, const char* name) : on(ctx && ctx->trace) {
    if (on) nvtxRangePushA(name);
  }
  ~TraceRange() {
    if (on) nvtxRangePop();
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};


namespace wn {

// Output modes of the prediction kernels: store V, add V, write the peel residual D - G V, or subtract
// G V from what the output already holds (a second pass of a peel).
enum OutMode { OUT_STORE = 0, OUT_ACCUM = 1, OUT_PEEL = 2, OUT_SUBG = 3 };

// Gains / peel description passed to kernels.
struct PeelArgs {
  const float2* data = nullptr;   // [rows][F]
  const float2* gains = nullptr;  // [gt][gf][n_ant]
  const int* ant1 = nullptr;
  const int* ant2 = nullptr;
  int gt = 1, gf = 1, n_ant = 0;
};

int set_error(int code, const std::string& msg);

// Raise a kernel's dynamic shared-memory limit to the device maximum, once per (kernel, device).
// Setting it to each launch's own size instead would race between host threads that launch the same
// kernel with different sizes (one thread lowering the limit between another's setting and launch).
cudaError_t allow_max_dynamic_smem(const void* kernel);

// Arguments of the point/Gaussian phasor kernel for one observation (K1).
struct K1Args {
  const double* uvw;
  const double* freq;
  int n_rows, n_chan, n_base;
  int log2L;          // lanes per row pair = 1 << log2L (8..32)
  int chan_block;     // channels per CTA column = L * K
  double nu0;         // log-frequency reference
  float dnu_h, dnu_l; // channel spacing / c as a float pair (uniform channels)
  const PGRec* comps;
  int n_point, n_gauss;
  float2* out;
  int mode;
  PeelArgs peel;
  unsigned* err;
  // single launch only: CTAs 0 .. n_main-1 are whole tiles (grid_x row tiles per channel block); the
  // tiles after them are split into tail_parts component ranges of tail_ct tiles with partial sums in part
  int grid_x = 1, n_main = 0, tail_parts = 1, tail_ct = 0;
  float2* part = nullptr;
};

// One work entry of the batched phasor kernel: request index, row tile, channel block.
struct K1Work {
  int req, bx, by;
};

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------

// Row r = t * n_base + b of the peel: G = g[tg][fg][ant1] * conj(g[tg][fg][ant2]).  Returns false
// (and G = NaN) when an antenna index is out of range; the access is then skipped.
__device__ __forceinline__ bool gain_product(const PeelArgs& p, int row, int n_base, int f, float2& G) {
  int b = row % n_base;
  int t = row / n_base;
  int a1 = __ldg(p.ant1 + b), a2 = __ldg(p.ant2 + b);
  if (a1 < 0 || a1 >= p.n_ant || a2 < 0 || a2 >= p.n_ant) {
    G = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    return false;
  }
  int tg = p.gt == 1 ? 0 : t;
  int fg = p.gf == 1 ? 0 : f;
  const float2* gb = p.gains + ((size_t)tg * p.gf + fg) * p.n_ant;
  float2 g1 = __ldg(gb + a1), g2 = __ldg(gb + a2);
  // g1 * conj(g2)
  G.x = g1.x * g2.x + g1.y * g2.y;
  G.y = g1.y * g2.x - g1.x * g2.y;
  return true;
}

// Phase reduction in double-float arithmetic: frac(t * a) in [-1/2, 1/2] turns, where t = th + tl and
// a = ah + al are unevaluated float sums.  The product error is recovered exactly with an FMA; the
// rounding to the nearest integer uses the 1.5*2^23 shifter (valid for |t*a| < 2^22).
__device__ __forceinline__ float reduce_turns(float th, float tl, float ah, float al) {
  float p = __fmul_rn(th, ah);
  float e = __fmaf_rn(th, ah, -p);
  e = __fmaf_rn(th, al, e);
  e = __fmaf_rn(tl, ah, e);
  const float kShift = 12582912.0f;
  float n = __fsub_rn(__fadd_rn(p, kShift), kShift);
  return __fadd_rn(__fsub_rn(p, n), e);
}

// x rounded to the nearest tf32 (10 explicit mantissa bits, ties away from zero), as an FP32 value with
// the 13 low mantissa bits zero: what a tf32 tensor-core operand reads.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split a double into an unevaluated float pair hi + lo.
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// The phase argument tau = u l + v m + w (n - 1) of one (component, row) in double-float FP32: each
// operand is an unevaluated float pair, products are made exact with an FMA (the two-product of
// Dekker's error-free transformations), the three terms are added with Knuth's two-sum, and the result
// is renormalised into (th, tl).  xuvw = (uh, ul, vh, vl, wh, wl).  The dropped low*low products are
// 2^-48 of each term, so |error| <~ 2^-44 |u| — 3e-10 m on a 5 km baseline, far below what a phase
// accurate to 1e-7 turns needs — and no FP64 instruction is issued.
__device__ __forceinline__ void tau_df(const float* xuvw, const PGRec& c, float& th, float& tl) {
  const float uh = xuvw[0], ul = xuvw[1], vh = xuvw[2], vl = xuvw[3], wh = xuvw[4], wl = xuvw[5];
  const float p1 = __fmul_rn(uh, c.lh);
  float e1 = __fmaf_rn(uh, c.lh, -p1);
  e1 = __fmaf_rn(uh, c.ll, e1);
  e1 = __fmaf_rn(ul, c.lh, e1);
  const float p2 = __fmul_rn(vh, c.mh);
  float e2 = __fmaf_rn(vh, c.mh, -p2);
  e2 = __fmaf_rn(vh, c.ml, e2);
  e2 = __fmaf_rn(vl, c.mh, e2);
  const float p3 = __fmul_rn(wh, c.nh);
  float e3 = __fmaf_rn(wh, c.nh, -p3);
  e3 = __fmaf_rn(wh, c.nl, e3);
  e3 = __fmaf_rn(wl, c.nh, e3);
  const float s = __fadd_rn(p1, p2), bs = __fsub_rn(s, p1);
  const float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bs)), __fsub_rn(p2, bs));
  const float t = __fadd_rn(s, p3), bt = __fsub_rn(t, s);
  const float et = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bt)), __fsub_rn(p3, bt));
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, es)), et);
  th = __fadd_rn(t, lo);
  tl = __fsub_rn(lo, __fsub_rn(th, t));
}

// Fast phasor exp(-2 pi i r) for r in turns, |r| <= 1/2 (MUFU sin/cos; absolute error ~2^-21).
__device__ __forceinline__ float2 phasor_fast(float r) {
  float s, c;
  float a = r * 6.283185307179586f;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(a));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(a));
  return make_float2(c, -s);
}

// Accurate phasor exp(-2 pi i r) via the library's sincospif.
__device__ __forceinline__ float2 phasor_accurate(float r) {
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, -s);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Frame taking (u, v, w) about the phase centre (H0, dec0) to the frame of a component centred at
// (l, m) (Sec. 3.2 after eq:scale-shape-y: the shapelet (u, v) are computed with the phase centre at
// the shapelet's own RA_j, dec_j).  F = R(H_j, dec_j) R(H0, dec0)^T with R the XYZ -> uvw rotation,
// sin dec_j = m cos dec0 + n sin dec0 and H_j - H0 = -atan2(l, n cos dec0 - m sin dec0); F does not
// depend on H0, so H0 = 0.
// Formed without transcendentals: with y = n cos dec0 - m sin dec0, (l, y, sin dec_j) is the unit
// direction of the component, so cos dec_j = sqrt(l^2 + y^2) = r and H_j - H0 = -atan2(l, y) has
// sin = -l / r, cos = y / r (H = 0 at the pole, r = 0).  sd0, cd0 = sin dec0, cos dec0.
__device__ inline void shapelet_frame(double l, double m, double sd0, double cd0, double F[9]) {
  const double n = sqrt(1.0 - l * l - m * m);
  const double sdj = m * cd0 + n * sd0, y = n * cd0 - m * sd0;
  const double cdj = sqrt(l * l + y * y);
  const double shj = cdj > 0.0 ? -l / cdj : 0.0, chj = cdj > 0.0 ? y / cdj : 1.0;
  double rj[9] = {shj, chj, 0.0, -sdj * chj, sdj * shj, cdj, cdj * chj, -cdj * shj, sdj};
  double r0[9] = {0.0, 1.0, 0.0, -sd0, 0.0, cd0, cd0, 0.0, sd0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      F[3 * a + b] = rj[3 * a] * r0[3 * b] + rj[3 * a + 1] * r0[3 * b + 1] + rj[3 * a + 2] * r0[3 * b + 2];
}

// ---- mbarrier / TMA bulk copy (sm_90+ PTX) ---------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit` SM clocks (the kernels use kWaitLimit,
// ~2 s at the B300 clock, far beyond any legitimate wait), raises WN_DEVERR_TIMEOUT and returns false
// so the caller can wind down (drain its own copies and commits, free what it holds, return).
constexpr long long kWaitLimit = 1ll << 32;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err,
                                                  long long limit = kWaitLimit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0 && clock64() - t0 > limit) {
      if (err) atomicOr(err, WN_DEVERR_TIMEOUT);
      return false;
    }
  }
}

// One-dimensional TMA bulk copy global -> shared, completing on an mbarrier (bytes multiple of 16,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace wn

// Launchers (defined in the kernel translation units).
namespace wn {
struct ObsDev {
  int n_ant, n_base, n_time, n_chan, n_rows;
  const double* uvw;
  const double* freq;
  const int* ant1;
  const int* ant2;
  double dec0, dnu, nu0;
  bool uniform;
};
int launch_pack(wn_ctx* ctx, const wn_sky* sky, Model* M, cudaStream_t st);
int launch_repack(wn_ctx* ctx, const wn_sky* sky, Model* M, cudaStream_t st);
int launch_phasor_mixed(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        cudaStream_t st);
int launch_phasor_table(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        cudaStream_t st);
// Workspace of a table-form launch: the spectrum table (spec_bytes of room) and the split tail's partial
// sums (k1_part_bytes).  spec_model / spec_cb name the table spec holds (a launch for the same model and
// channel block, e.g. the next time steps of one observation, reuses it; nullptr / 0: none).
struct KsWork {
  float* spec = nullptr;
  size_t spec_bytes = 0;
  float2* part = nullptr;
  const Model* spec_model = nullptr;
  int spec_cb = 0;
};
size_t phasor_table_spec_bytes(const ObsDev& o, const Model* M);
int launch_phasor_table_ws(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                           KsWork& w, cudaStream_t st);
int launch_phasor_fp64(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                       bool include_shapelets, cudaStream_t st);
int launch_peel_model(wn_ctx* ctx, const ObsDev& o, const PeelArgs& pa, const float2* model, float2* resid,
                      cudaStream_t st);
int launch_shapelets(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                     cudaStream_t st);
int launch_shapelets_static(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                            cudaStream_t st);
size_t static_scratch_entries();
int static_scratch_setup(wn_ctx* ctx);
int grad_constants_setup(wn_ctx* ctx);
int k2_constants_setup();
int pack_constants_setup();
int launch_coeff_mma(wn_ctx* ctx, const ObsDev& o, const Model* M, int q, const PeelArgs& pa, const float2* resid,
                     const float4* rowinfo, const float4* chaninfo, float2* rowg_ws, double* part_c, int* grid_out,
                     cudaStream_t st);
// Per-row gain product g[ant1] conj(g[ant2]) of frequency-independent gains (NaN and the antenna flag for
// an index out of range).
void launch_rowgain(const PeelArgs& pa, int n_rows, int n_base, float2* out, unsigned* err, cudaStream_t st);
int launch_grad(wn_ctx* ctx, const ObsDev& o, const Model* M, const PeelArgs& pa, float2* resid,
                const wn_sky_grad* g, double* loss, cudaStream_t st);
int k1_batched_smem();
size_t k1_part_bytes(int num_sms);
int launch_fit_shapelets(wn_ctx* ctx, const ObsDev& o, Model* M, const PeelArgs& pa, int n_iter, double tol,
                         double* coeff, double* info, cudaStream_t st);
int launch_calibrate(wn_ctx* ctx, const ObsDev& o, const float2* model, const float2* data, float2* gains, int n_iter,
                     cudaStream_t st);
cudaError_t k1_batched_setup();
int k1_batched_args(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                    K1Args* args, int* grid_x, int* grid_y);
cudaError_t k1_batched_launch(const K1Args* reqs, const K1Work* work, const int* n_work, int grid, cudaStream_t st);
// Shapelet launches with caller-supplied tables: chaninfo [n_chan] and rowinfo [rowinfo_cap >= n_rows] float4
// (room for rowinfo_cap / n_rows shapelets' row tables; more shapelets per launch when there is room).
int launch_shapelets_ws(wn_ctx* ctx, const ObsDev& o, const Model* M, float2* out, int mode, const PeelArgs& pa,
                        float4* chaninfo, float4* rowinfo, size_t rowinfo_cap, cudaStream_t st, float2* rowg = nullptr);
}  // namespace wn
