/*
 * woden_b300.h -- C ABI of the B300 (sm_103a) visibility predictor and peeler.
 *
 * The library evaluates the direct measurement equation of Line et al. 2020 (arXiv 2005.09316),
 * Sec. 3 (eq:measure_eq_discrete, eq:env_visi_def):
 *
 *     V(t,b,f) = sum_j S_j(nu_f) xi_j(u,v) exp(-2 pi i (u l_j + v m_j + w (n_j - 1)))
 *
 * with (u,v,w) = uvw(t,b) nu_f / c, S_j(nu) = S_ref,j (nu / nu_ref,j)^alpha_j (Sec. 4.1, Sec. 6),
 * and the envelope xi_j = 1 for points, the elliptical-Gaussian transform (eq:gauss-env,
 * eq:scale-gauss-x/y) for Gaussians, and the coefficient-weighted analytic shapelet transform
 * (eq:shape-env, eq:scale-shape-x/y, eq:basis_FT) for shapelets.  The peel forms
 * R = D - g_ant1 conj(g_ant2) V (Sec. 5.1).  The instrument beam is 1 (Sec. 3.1).
 *
 * Conventions
 *  - Every array pointer in wn_obs, wn_sky and the call arguments is a DEVICE pointer (memory on
 *    the context's GPU) owned by the caller, unless a comment says HOST.  The library never frees
 *    caller memory and keeps no pointer to it after a call returns, except that wn_sky_upload
 *    copies the sky into library-owned device memory (the resident model).
 *  - Complex values are interleaved (re, im) float32 pairs ("complex64"), 8-byte aligned.
 *  - Visibility arrays are [n_time][n_base][n_chan] complex64, channel fastest.
 *  - Baselines are the pairs (ant1[b], ant2[b]) with ant1 < ant2; uvw(t,b) is in metres in the
 *    phase-centre frame and points from ant1 to ant2 (X[ant2] - X[ant1]).
 *  - Calls are asynchronous on the given stream (a cudaStream_t; NULL = the legacy default stream)
 *    unless documented as synchronous.  A call that returns an error launches nothing.
 *  - Return value: WN_OK (0) or a wn_status code; wn_last_error() gives a message for the last
 *    failing call on the calling thread.
 *  - A context's device workspaces (the phasor launch's partial sums of split tail tiles, the
 *    shapelet and adjoint tables) are shared by its calls, so calls on one context that are issued to
 *    different streams must not overlap on the GPU: order them (events), or use one context per
 *    stream.  The serving API (wn_server_*) gives each of its slots its own workspace.
 *  - Device-side faults of the inputs that host checks cannot see (an antenna index outside
 *    [0, n_ant)) are not dereferenced: the kernels skip the access, write NaN for that output and
 *    raise a flag that wn_device_errors() reports.
 *  - Angles are radians; FWHM widths are full widths at half maximum; frequencies are Hz.
 */
#ifndef WODEN_B300_H
#define WODEN_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define WN_API __attribute__((visibility("default")))
#else
#define WN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wn_ctx wn_ctx;

typedef enum {
    WN_OK = 0,
    WN_EINVAL = 1,    /* a size, pointer, index or parameter is out of range */
    WN_ENOMEM = 2,    /* device or host allocation failed */
    WN_ECUDA = 3,     /* a CUDA runtime call failed */
    WN_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    WN_EBUSY = 5,     /* admission refused (serving) */
    WN_ENOTFOUND = 6  /* unknown model id or ticket */
} wn_status;

/* Precision of the point/Gaussian phasor sum. */
typedef enum {
    WN_PREC_MIXED = 0,   /* double-float phase argument, FP32 phasors and sums (default) */
    WN_PREC_FP64 = 1,    /* every step in FP64: the plain reference form, with the per-component constants
                            (log-flux and spectral index, Gaussian quadratic form, shapelet frame and scales)
                            formed once per component per thread block, as the mixed path forms them once */
    WN_PREC_FP64_UNTUNED = 2 /* every step in FP64, the formulas evaluated per visibility as printed (pow for
                                the spectrum, the position angle's cos and sin per evaluation) */
} wn_precision;

/* Precision of the tensor-core shapelet contraction (xi = A C B^T, Sec. 3.2 eq:shape-env). */
typedef enum {
    WN_SHAPE_BF16X3 = 0, /* bf16 hi+lo split of both operands, three products, FP32 accumulate (default) */
    WN_SHAPE_BF16X1 = 1, /* plain bf16 operands, one product, FP32 accumulate */
    WN_SHAPE_LUT_BF16X3 = 2, /* as BF16X3, but the Hermite functions are interpolated linearly from a 1-D table
                                (spacing 1/256, orders 0..127; the look-up tables of Sec. 3.2) instead of the
                                recurrence; the table (6.8 MB) is built once per context */
    WN_SHAPE_TF32 = 3,       /* tf32 operands (both rounded to nearest from FP32, 10 explicit mantissa bits), one
                                product, FP32 accumulate */
    WN_SHAPE_TF32X3 = 4      /* tf32 hi+lo split of both operands (hi = RN_tf32(x), lo = RN_tf32(x - hi)), three
                                products hi*hi + hi*lo + lo*hi, FP32 accumulate: about FP32 accuracy.  The split
                                operands take 8 bytes per element; they fit the kernel's shared memory when the
                                coefficients reach orders n1 + n2 up to 63 (k_pad 64, n_pad 128); a call on a
                                model with a higher order returns WN_EINVAL. */
} wn_shape_mode;

/* Device-side error flags (bit mask) reported by wn_device_errors. */
#define WN_DEVERR_ANTENNA 0x1u  /* an ant1/ant2 entry outside [0, n_ant) met by a peel */
#define WN_DEVERR_TIMEOUT 0x2u  /* a bounded mbarrier / queue wait gave up */
#define WN_DEVERR_SKY     0x4u  /* a sky entry rejected during upload */
#define WN_DEVERR_CALIB   0x8u  /* a calibration solve met a non-positive pivot (its gains were kept) */

/* An observation: baselines, time steps and channels (Sec. 3.2, last paragraph: uvw once per time
 * step, scaled per channel). */
typedef struct {
    int32_t n_ant;          /* antennas, >= 2 */
    int32_t n_base;         /* baselines, >= 1 */
    int32_t n_time;         /* time steps, >= 1 */
    int32_t n_chan;         /* channels, >= 1 */
    const double* uvw;      /* DEVICE [n_time][n_base][3] metres */
    const double* freq_hz;  /* DEVICE [n_chan] Hz, > 0 */
    const int32_t* ant1;    /* DEVICE [n_base] */
    const int32_t* ant2;    /* DEVICE [n_base] */
    double dec0;            /* phase-centre declination (rad); fixes the shapelet re-phasing frame */
    double chan_spacing_hz; /* HOST scalar: 0 for an arbitrary channel list, else the uniform spacing,
                               freq_hz[f] == freq_hz[0] + f * chan_spacing_hz (enables the phasor
                               recurrence across channels) */
    double freq0_hz;        /* HOST scalar: freq_hz[0] (needed on the host to set up the kernels) */
} wn_obs;

/* A sky model: points first, then Gaussians, then shapelets (Sec. 3.1-3.2).  DEVICE pointers. */
typedef struct {
    int32_t n_point, n_gauss, n_shape;
    const double* l;          /* [n_comp] direction cosine, l^2 + m^2 < 1 */
    const double* m;          /* [n_comp] */
    const double* flux;       /* [n_comp] S_ref (Jy); for shapelets the flux multiplying xi (Sec. 3.2) */
    const double* alpha;      /* [n_comp] spectral index */
    const double* nu_ref;     /* [n_comp] reference frequency (Hz), > 0 */
    const double* g_maj;      /* [n_gauss] FWHM major axis (rad) */
    const double* g_min;      /* [n_gauss] FWHM minor axis (rad) */
    const double* g_pa;       /* [n_gauss] position angle, East of North (rad) */
    const double* s_beta1;    /* [n_shape] beta_1 (rad), pairs with the major (PA) axis */
    const double* s_beta2;    /* [n_shape] beta_2 (rad) */
    const double* s_pa;       /* [n_shape] position angle (rad) */
    const int32_t* s_nmax;    /* [n_shape] n_max in [0, 127]; each shapelet is evaluated up to the highest n1 + n2 its triples reach */
    const int32_t* s_off;     /* [n_shape + 1] offsets into the coefficient triples, s_off[0] == 0 */
    const int32_t* s_n1;      /* [nnz] basis order along x (beta_1) */
    const int32_t* s_n2;      /* [nnz] basis order along y (beta_2); n1 + n2 <= n_max */
    const double* s_coeff;    /* [nnz] C[n1,n2] already divided by the integrated flux (Sec. 3.2) */
} wn_sky;

/* Gradient output: DEVICE arrays laid out like wn_sky; entries for absent parts may be NULL. */
typedef struct {
    double* flux;      /* [n_comp] dL/dS_ref */
    double* alpha;     /* [n_comp] dL/dalpha */
    double* l;         /* [n_comp] dL/dl (shapelets: including the re-phasing frame's motion) */
    double* m;         /* [n_comp] dL/dm */
    double* g_maj;     /* [n_gauss] */
    double* g_min;     /* [n_gauss] */
    double* g_pa;      /* [n_gauss] */
    double* s_beta1;   /* [n_shape] */
    double* s_beta2;   /* [n_shape] */
    double* s_pa;      /* [n_shape] */
    double* s_coeff;   /* [nnz] */
} wn_sky_grad;

/* ---- context ------------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` (allocates a small device error word). Synchronous. */
WN_API int wn_create(wn_ctx** out, int device);
/* Destroy a context and every resident model it owns.  Synchronizes the device. */
WN_API void wn_destroy(wn_ctx* ctx);
/* Message for the last non-zero return on the calling thread ("" if none).  Never NULL. */
WN_API const char* wn_last_error(void);
/* Library version string. */
WN_API const char* wn_version(void);
/* Select the point/Gaussian precision (wn_precision) and the shapelet mode (wn_shape_mode). */
WN_API int wn_set_precision(wn_ctx* ctx, int precision, int shape_mode);
/* Tracing (no paper counterpart): with on != 0, every compute entry point of the context (wn_sky_upload,
 * wn_predict, wn_predict_static, wn_peel, wn_peel_model, wn_predict_grad, wn_fit_shapelets, wn_calibrate,
 * wn_server_submit) opens an NVTX range named after itself for the duration of the call, for profilers
 * that record NVTX (ncu --nvtx).  Off by default.  Host-side only: results are unchanged. */
WN_API int wn_set_trace(wn_ctx* ctx, int on);
/* Host-side fault injection for tests (no paper counterpart): the next n device allocations the library
 * makes, in any context or server of the process, fail as an out-of-memory cudaMalloc would, without
 * calling CUDA; the calls that need them return WN_ENOMEM and leave their context usable.  n = 0
 * cancels.  WN_EINVAL for n < 0. */
WN_API int wn_debug_fail_allocs(int n);
/* Read and clear the device error flags (WN_DEVERR_*).  Synchronizes the device. */
WN_API int wn_device_errors(wn_ctx* ctx, uint32_t* flags_out);

/* ---- resident sky models ------------------------------------------------------------------ */

/* Validate and pack a sky into library-owned device memory; *model_id receives its handle.
 * Packing runs in kernels on `stream` (n - 1 computed stably as -(l^2+m^2)/(1+sqrt(1-l^2-m^2)),
 * log-flux, Gaussian quadratic forms, shapelet frames and the dense bf16 coefficient operands).
 * Synchronous: it reads the shapelet sizes back and checks the sky on the device.
 * Errors: WN_EINVAL for negative counts, NULL arrays that are needed, l^2+m^2 >= 1, nu_ref <= 0,
 * n_max outside [0,127], a triple outside the triangle n1+n2 <= n_max, non-monotone s_off. */
WN_API int wn_sky_upload(wn_ctx* ctx, const wn_sky* sky, int* model_id, void* stream);
/* Re-pack a resident model from new parameter values, in place and without allocating (no paper
 * counterpart; for fitting loops that change a model every step).  sky must have the model's component
 * counts; its l, m, flux, alpha, nu_ref, Gaussian axes and position angles, shapelet beta1, beta2,
 * position angles and coefficients (in the model's triple order) are read; its shapelet structure
 * (s_nmax, s_off, s_n1, s_n2) is not: the model keeps the one it was uploaded with.  The packing runs in
 * kernels on `stream`, so later calls on that stream see the new values.  Asynchronous for models of
 * points and Gaussians; with shapelets it ends by reading the packed shapelet headers back to the host
 * (the launches are planned from them), which synchronises `stream`.  Values that wn_sky_upload would
 * reject (l^2 + m^2 >= 1, nu_ref <= 0, a negative width, a non-finite value) are not detected on the
 * host: they raise WN_DEVERR_SKY (wn_device_errors) and the component contributes nothing.
 * WN_ENOTFOUND for an unknown model, WN_EINVAL for different counts or a NULL array that is needed. */
WN_API int wn_sky_update(wn_ctx* ctx, int model_id, const wn_sky* sky, void* stream);
/* Release a resident model.  Synchronous. */
WN_API int wn_sky_free(wn_ctx* ctx, int model_id);
/* Bytes of device memory a resident model holds (admission accounting). */
WN_API int wn_sky_bytes(wn_ctx* ctx, int model_id, size_t* bytes_out);
/* The packed coefficient operand of shapelet q of a resident model, copied to HOST memory (no paper
 * counterpart; for checking the packer).  It holds bf16 hi then lo, k_pad x n_pad each, in the tcgen05
 * canonical K-major layout without swizzle: element (n, k) (n = 2 n2 + {0: Re, 1: Im} of
 * C[n1, n2] (-i)^(n1+n2) / (k_n1 k_n2), k = n1) at ((k/8) (n_pad/8) + n/8) 64 + (n%8) 8 + k%8;
 * hi = RN(float(value)), lo = RN(float(value) - hi), the value formed in FP64.  k_0 = k_1 = 1 and
 * k_(n+1) = k_(n-1) sqrt((n+1)/n) (each step correctly rounded in FP64) are the scales of the Hermite
 * functions g_n = k_n phi_n the contraction runs on (their recurrence takes two operations per order).
 * k_pad and n_pad follow the highest order n1 + n2 the coefficients reach.
 * host_out may be NULL to query k_pad and n_pad; otherwise it must hold bytes >= 4 k_pad n_pad.
 * Synchronous.  WN_ENOTFOUND for an unknown model, WN_EINVAL for q outside [0, n_shape) or a short
 * buffer. */
/* The tf32 copy of the same operand (WN_SHAPE_TF32, WN_SHAPE_TF32X3), copied to HOST memory: k_pad x n_pad
 * FP32 values, each hi = RN_tf32 (ties away from zero) of float(value), in the K-major layout with 8 x 4
 * core matrices: element (n, k) at ((k/4) (n_pad/8) + n/8) 32 + (n%8) 4 + k%4.  When bytes >= 8 k_pad n_pad
 * the remainder operand lo = RN_tf32(float(value) - hi) follows in the same layout.  Same arguments and
 * errors as wn_sky_shapelet_operand (bytes >= 4 k_pad n_pad). */
WN_API int wn_sky_shapelet_operand_tf32(wn_ctx* ctx, int model_id, int q, void* host_out, size_t bytes, int* k_pad,
                                        int* n_pad);
WN_API int wn_sky_shapelet_operand(wn_ctx* ctx, int model_id, int q, void* host_out, size_t bytes, int* k_pad,
                                   int* n_pad);

/* ---- hot path ------------------------------------------------------------------------------ */

/* Predict visibilities (eq:env_visi_def) of a resident model into vis_c64 [T][B][F].
 * accumulate = 0 overwrites vis_c64, 1 adds to it. */
WN_API int wn_predict(wn_ctx* ctx, const wn_obs* obs, int model_id, void* vis_c64, int accumulate, void* stream);

/* Fused peel (Sec. 5.1): resid = data - g[ant1] conj(g[ant2]) V for the resident model.
 * gains_c64 is [gains_t][gains_f][n_ant] complex64 with gains_t in {1, n_time} and gains_f in
 * {1, n_chan} (broadcast when 1).  resid may alias data (each element is read before it is written). */
WN_API int wn_peel(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t, int gains_f,
            const void* data_c64, void* resid_c64, void* stream);

/* Standalone streaming peel of an already predicted model: resid = data - g1 conj(g2) model.
 * HBM-bound (24 bytes per visibility).  resid may alias data or model. */
WN_API int wn_peel_model(wn_ctx* ctx, const wn_obs* obs, const void* gains_c64, int gains_t, int gains_f,
                  const void* data_c64, const void* model_c64, void* resid_c64, void* stream);

/* Gradient of L = sum |data - g1 conj(g2) V|^2 with respect to every sky parameter (analytic adjoint,
 * phasors recomputed, not stored).  grad_out arrays are overwritten; loss_out (DEVICE, 1 double) may be
 * NULL.  resid_c64 (DEVICE [T][B][F] complex64) receives the residual data - G V and serves as the
 * adjoint's input; it must not alias data.  The library allocates its reduction workspace. */
WN_API int wn_predict_grad(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t, int gains_f,
                    const void* data_c64, void* resid_c64, const wn_sky_grad* grad_out, double* loss_out,
                    void* stream);

/* ---- continuous-batching server (requests of uneven size) ------------------------------------ */

/* A scheduler thread admits predict / peel requests by memory, packs the tiles of admitted small
 * requests into one batch run by a persistent phasor kernel replayed from a CUDA graph (shapelets
 * follow per request on the same stream), and keeps up to n_streams batches on the GPU, so requests
 * that arrive while others run are admitted as slots and pool memory free up and their work overlaps.
 * A request above one batch's work budget runs on a stream of its own through the single-request
 * kernels, with that stream's own workspaces (in one launch in arrival order, in chunks of whole time
 * steps small-first; see wn_server_set_order), and keeps the stream until its last launch has
 * completed.  A small request that batching would not help (more than about 1 ms of
 * estimated work, or few tiles with long ones) runs alone through the same kernels, all its steps at
 * once.  Results do not depend on the batch a request ran in (same tiles, same order); a request run
 * alone gives the single-request call's result. */
typedef struct wn_server wn_server;

/* Request states reported by wn_server_poll. */
#define WN_REQ_PENDING 0
#define WN_REQ_ADMITTED 1
#define WN_REQ_RUNNING 2
#define WN_REQ_DONE 3
#define WN_REQ_CANCELLED 4
#define WN_REQ_FAILED 5

/* Create a server on ctx: n_streams batch slots (1..16), a device pool of pool_bytes for the requests'
 * outputs, at most max_inflight admitted requests, observations of at most max_rows (T*B) rows and
 * max_chan channels.  Allocates the pool, per-stream tables (room for four shapelets' row tables) and
 * pinned staging, and captures one graph per stream; a stream that runs a request through the
 * single-request kernels allocates its spectrum table (grown to the largest request it runs) and
 * tail-sum workspace on first use.  Resident
 * models must not be freed while requests that use them are unreleased. */
WN_API int wn_server_create(wn_ctx* ctx, int n_streams, size_t pool_bytes, int max_inflight, int max_rows,
                            int max_chan, wn_server** out);
/* Stop the scheduler and free everything the server owns (waits for batches on the GPU). */
WN_API void wn_server_destroy(wn_server* srv);
/* Queue a request: predict (peel = 0) or peel (peel = 1, with gains [gains_t][gains_f][n_ant] and data
 * as for wn_peel) of resident model model_id on obs (device arrays that stay valid until the request is
 * released; the struct itself is copied).  Channels must be uniformly spaced.  Non-blocking.
 * WN_EBUSY: the output can never fit in the pool; WN_EINVAL: invalid request. */
WN_API int wn_server_submit(wn_server* srv, const wn_obs* obs, int model_id, int peel, const void* gains_c64,
                            int gains_t, int gains_f, const void* data_c64, uint64_t* ticket);
/* State of a request (WN_REQ_*); when done, *vis_out (optional) is the DEVICE address of its
 * [T][B][F] complex64 result in the pool, valid until wn_server_release.  info (optional, 5 doubles):
 * submit, admit, launch and completion times in seconds on the server's clock, and the batch index. */
WN_API int wn_server_poll(wn_server* srv, uint64_t ticket, int* state, void** vis_out, double* info);
/* Block until the request is done, failed or cancelled, or timeout_s passes (WN_ETIMEOUT). */
WN_API int wn_server_wait(wn_server* srv, uint64_t ticket, double timeout_s, void** vis_out, double* info);
/* Copy a finished request's visibilities ([T][B][F] complex64) to dst (DEVICE) on stream. */
WN_API int wn_server_copy(wn_server* srv, uint64_t ticket, void* dst, void* stream);
/* Return a finished request's pool memory and forget it (WN_EBUSY while it is on the GPU). */
WN_API int wn_server_release(wn_server* srv, uint64_t ticket);
/* Cancel a request that has not been admitted yet (WN_EBUSY otherwise). */
WN_API int wn_server_cancel(wn_server* srv, uint64_t ticket);
/* Admission policy for large requests (those whose estimated work exceeds one batch's budget, about
 * 20 ms).  At most max_large_inflight of them (1..16; never more than the slots less one) own a slot at
 * a time.  In the small-first order, among the waiting ones the least estimated work starts first,
 * except that one waiting longer than max_large_wait_s seconds since submission starts before any
 * younger one (0 gives submission order); in arrival order they start in submission order and the wait
 * limit is not used.  Defaults: 1 and 1.0 s.  Takes effect at the next admission; requests already
 * started keep their slot.  WN_EINVAL for a NULL server or values outside those ranges. */
WN_API int wn_server_set_policy(wn_server* srv, int max_large_inflight, double max_large_wait_s);

/* Request orders for wn_server_set_order.
 * WN_SERVE_ARRIVAL (the default): large requests start in submission order, one launch each on the
 *   highest-priority stream.  The large request due next waits for the small requests submitted before
 *   it to finish, and the small requests submitted after it wait until it has started; other small
 *   requests are batched and go out on lower-priority streams as they free up, one batch at a time
 *   while a large request runs.  A large request thus waits only for work submitted before it (and for
 *   blocks of a lower-priority batch that the GPU runs beside it), as in a one-at-a-time queue.
 * WN_SERVE_SMALL_FIRST: small requests go out as soon as a stream is free; large requests run in chunks
 *   of whole time steps on the lowest-priority stream, in the order wn_server_set_policy sets.  The
 *   small requests' latency is far lower; the largest requests' tail is longer. */
#define WN_SERVE_ARRIVAL 0
#define WN_SERVE_SMALL_FIRST 1
/* Set the request order (WN_SERVE_*); takes effect at the next admission.  WN_EINVAL otherwise. */
WN_API int wn_server_set_order(wn_server* srv, int order);
/* stats (6 doubles): batches launched, most batches on the GPU at once, most requests in one batch,
 * requests launched, requests admitted and unreleased, free pool bytes. */
WN_API int wn_server_stats(wn_server* srv, double* stats);

/* ---- allocation-free prediction ------------------------------------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that cannot allocate device memory
 * at prediction time, for example a process whose device memory is fully reserved by another
 * allocator (a framework's caching allocator or a fixed-size pool), or a latency-critical loop that
 * cannot afford cudaMalloc's implicit device synchronisation.  It computes what wn_predict computes,
 * but the shapelet launches take their per-channel and per-row tables from a file-scope device array
 * of 2^18 float4 entries (4 MiB, held by every GPU that loads the library until exit) instead of the
 * context's growable workspace, and nothing in the call allocates.
 * Limits: n_chan rounded up to a multiple of 16, plus n_time * n_base, must not exceed 262144;
 * larger observations are rejected with WN_EINVAL.  The row tables of as many shapelets as the rest of
 * the array holds (up to eight) are summed per launch; a model with more takes further launches that
 * add to the output.
 * The array's device address is looked up once, when the context is created (wn_create, with the
 * context's device current), and kept in the context; the call itself only launches kernels.
 * Each device has its own copy of the array.  Every call on one device shares that copy, which keeps
 * the last call's contents: calls whose work overlaps on the same device (concurrent streams, or
 * several contexts on one device) race on it, so order them; calls on different devices do not.
 * The model must already be resident (wn_sky_upload) and the context created beforehand. */
WN_API int wn_predict_static(wn_ctx* ctx, const wn_obs* obs, int model_id, void* vis_c64, int accumulate, void* stream);

/* ---- visibility-space shapelet fitting ------------------------------------------------------- */

/* Fit the shapelet coefficients of a resident model to data by linear least squares in visibility
 * space.  The model's positions, scales and position angles, and its points and Gaussians, stay
 * fixed.  The visibilities are linear in the coefficients C (eq:shape-env), so the C minimising
 * sum |D - G (V_fixed + V_shapelets(C))|^2 solves the normal equations.  The paper fits in image space
 * (Sec. 2.2); this is the visibility-space counterpart.  Solved by CGLS from the starting
 * coefficients, without forming the normal matrix.  Each iteration is one shapelet contraction and one
 * coefficient adjoint.  It stops after n_iter iterations, or when the normal-equation residual
 * |A^T r| has fallen below tol times its starting value.
 *   gains_c64    device [gains_t][gains_f][n_ant] complex64 (1 or n_time, 1 or n_chan);
 *   data_c64     D, device [n_time][n_base][n_chan] complex64;
 *   coeff_inout  device double [nnz]: every shapelet coefficient of the model, in upload order;
 *                starting values in, fitted values out;
 *   info         host double[4] or NULL: iterations run, final |A^T r| / starting |A^T r|, final and
 *                starting sum |r|^2.
 * On return the model holds the fitted coefficients (later predictions and peels use them).
 * Synchronises `stream` once per iteration and allocates its scratch per call.  WN_EINVAL if the
 * model has no shapelet coefficients or the context is not in the mixed precision. */
WN_API int wn_fit_shapelets(wn_ctx* ctx, const wn_obs* obs, int model_id, const void* gains_c64, int gains_t,
                            int gains_f, const void* data_c64, int n_iter, double tol, double* coeff_inout,
                            double* info, void* stream);

/* ---- gain calibration ------------------------------------------------------------------------- */

/* Fit one complex gain per antenna for every (time, channel): the linearised least squares of Sec. 5.1
 * (eq:peeling-iter), iterated n_iter times (the paper uses 10).  With the model M = g_i conj(g_j) I
 * and residual R = V - M, each iteration solves [A^T A] x = A^T b for the real and imaginary parts of
 * additive gain errors e (the e e* term dropped) and sets g <- g + e.  The overall phase of the gains
 * is not determined by the data, so the gauge is fixed by holding Im(e_0) = 0: antenna 0's imaginary
 * part keeps its starting value.
 *   model_c64  I, device [n_time][n_base][n_chan] complex64: the ideal model (e.g. from wn_predict);
 *   data_c64   V, device [n_time][n_base][n_chan] complex64: the measured visibilities;
 *   gains_c64  device [n_time][n_chan][n_ant] complex64: starting gains in, fitted gains out.
 * Each antenna pair may appear at most once among the baselines (ant1 < ant2).  Requires
 * n_ant <= 128 (the normal matrix of one (time, channel), 2 n_ant - 1 parameters, stays in shared
 * memory) and 1 <= n_iter <= 1000; otherwise WN_EINVAL.  Solves run in FP32.  A problem whose normal
 * matrix is not positive definite (for example an all-zero model) keeps its last gains and sets
 * WN_DEVERR_CALIB.  Asynchronous on `stream`; uses the context's workspace. */
WN_API int wn_calibrate(wn_ctx* ctx, const wn_obs* obs, const void* model_c64, const void* data_c64, void* gains_c64,
                        int n_iter, void* stream);

/* ---- measurement ------------------------------------------------------------------------------ */

/* Measured pipe throughputs of the context's GPU, for the roofline fractions of the phasor kernels (no
 * paper counterpart).  rates (4 doubles, lane operations per second): FP32 FMA, FP32 FMA issued as
 * packed f32x2 (each counting two), MUFU ex2, FP64 FMA.  Each is the best of three timed launches of a
 * kernel running eight independent dependency chains per thread over 8 CTAs of 256 threads per SM;
 * it allocates a small scratch buffer and synchronises its own stream.  Takes a few milliseconds. */
WN_API int wn_pipe_rates(wn_ctx* ctx, double* rates);

/* Component-visibility evaluations per second that the point/Gaussian kernel's channel loop sustains
 * by itself (no paper counterpart): the single-launch kernel's own loop code over component records and
 * spectrum values held in shared memory, four groups of 16 points per group of 16 Gaussians, 12 channels
 * of two rows per lane, one CTA of 512 threads per SM, with no record building, global memory or
 * barriers inside the loop.  The rate the full prediction approaches; its instruction mix, not the FP32
 * peak, sets it.  Best of three timed launches after one warm-up; allocates a small scratch buffer and
 * synchronises its own stream. */
WN_API int wn_phasor_loop_rate(wn_ctx* ctx, double* evals_per_s);

/* Tensor-core and TMEM timings as the shapelet kernel uses them (no paper counterpart).  One CTA per SM
 * issues 2,048 tcgen05 kind::f16 MMAs (M = 128, K = 16, bf16 operands, FP32 accumulator in TMEM) back to
 * back from one thread, with zero operands K-major in shared memory in the shapelet kernel's
 * no-swizzle layout.  out (4 doubles): SM clocks per MMA instruction at N = 128 and at N = 64
 * (issue to completion, averaged over the CTAs), then SM clocks of one 16-column TMEM load and its wait
 * (one warp, alone), and of eight such loads under one wait.  Allocates a small buffer and synchronises
 * its own stream; flags WN_DEVERR_TIMEOUT if a bounded wait gave up. */
WN_API int wn_mma_rate(wn_ctx* ctx, double* out);

/* The same timing for the shapelet kernel's tf32 mode (no paper counterpart): 2,048 tcgen05 kind::tf32 MMAs
 * (M = 128, K = 8, tf32 operands: the same 32 bytes of each operand row as one K = 16 bf16 MMA, FP32
 * accumulator) per CTA, one CTA per SM, zero operands K-major in the kernel's no-swizzle layout.  out
 * (2 doubles): SM clocks per MMA instruction at N = 128 and at N = 64.  Allocates a small buffer and
 * synchronises its own stream. */
WN_API int wn_mma_rate_tf32(wn_ctx* ctx, double* out);

/* The failure path of the kernels' bounded waits, without a fault (no paper counterpart).  A one-thread
 * kernel waits on an mbarrier that nothing ever arrives at, through the same bounded-wait helper as the
 * prediction kernels but with a limit of `seconds` (0 < seconds <= 5) instead of ~2 s; it gives up,
 * raises WN_DEVERR_TIMEOUT in the context's device flags (wn_device_errors) and returns.  The context
 * stays usable.  Synchronous (device-wide); WN_OK once the kernel has returned. */
WN_API int wn_selftest_timeout(wn_ctx* ctx, double seconds);

#ifdef __cplusplus
}
#endif
#endif /* WODEN_B300_H */
