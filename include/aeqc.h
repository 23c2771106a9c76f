/*
 * aeqc.h -- C ABI of libaeqc, the GB300 (sm_103a) hot path of the hybrid
 * compressor of Banerjee et al., "Scalable Hybrid Learning Techniques for
 * Scientific Data Compression" (arXiv:2212.10733):
 *
 *   autoencoder encode/decode (Sec. III Stages 2-3, Eq. (5))
 *   -> error-bounded residual quantization (Sec. III Stage 4)
 *   -> QoI-preserving Lagrange/Newton correction (Sec. III Stage 5, Eq. (6)),
 *      preserving the moments behind n, u_par, T_perp, T_par (Sec. II, Eq. (1)-(4))
 *   -> decompression: decode, add the residual, apply the multipliers
 *      to every value (Sec. III, end of Stage 5).
 *
 * Conventions (every call unless stated otherwise):
 *   - Array arguments are DEVICE pointers owned by the caller, row-major and
 *     contiguous unless a leading dimension (ld) is given.  Host pointers are
 *     named *_host.  Nothing here keeps a pointer after the call returns.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Exceptions: *_create, *_destroy,
 *     *_set_*, *_get_*, aeqc_last_error, *_workspace_size.
 *   - Return value: AEQC_OK (0) or a negative error code; the message of the
 *     last error on the calling thread is aeqc_last_error().  Argument errors
 *     are detected on the host before anything is launched.  Per-histogram
 *     outcomes (non-convergence, verbatim storage, ...) are NOT errors: they
 *     are reported in the uint16 status word of each histogram.
 *   - Histogram layout: x[b][j][i], i (v_par index) fastest, P = n_par*n_perp
 *     values of float64 per histogram (12,168 bytes for the 39 x 39 grid).
 *   - Calls that need temporary device memory take a caller-owned
 *     `workspace` of at least *_workspace_size() bytes (256-byte aligned).
 *     No call allocates device memory except aeqc_model_create,
 *     aeqc_mlp_create, aeqc_model_load and aeqc_mlp_load (which own their
 *     weights until *_destroy).
 *   - Calls on the same stream are ordered; calls on different streams that
 *     share an output, a workspace or a model race.
 */
#ifndef AEQC_H
#define AEQC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes --------------------------------------------------------- */
#define AEQC_OK 0
#define AEQC_EINVAL (-1)        /* bad argument (null pointer, size, alignment) */
#define AEQC_ECUDA (-2)         /* a CUDA runtime call failed */
#define AEQC_ENOMEM (-3)        /* allocation failed (create calls only) */
#define AEQC_ECORRUPT (-4)      /* container header inconsistent */
#define AEQC_EUNSUPPORTED (-5)  /* valid but not supported (grid too large, ...) */

/* ---- per-histogram status bits (uint16) ---------------------------------- */
#define AEQC_ST_CONVERGED 0x0001u        /* Newton round 1 reached tol */
#define AEQC_ST_ROUND2 0x0002u           /* round 2 (damped Newton from 0) ran */
#define AEQC_ST_VERBATIM 0x0004u         /* stored raw: every code escapes, lambda = 0 */
#define AEQC_ST_NONFINITE_INPUT 0x0008u  /* x had a NaN/Inf or a negative value */
#define AEQC_ST_ZERO_IMAGE 0x0010u       /* max(x) == 0: f == 0, codes 0, lambda 0 */
#define AEQC_ST_CODE_ESCAPE 0x0020u      /* at least one escape code (raw value) */
#define AEQC_ST_WARM_REJECTED 0x0040u    /* learned warm start rejected, restarted at 0 */
#define AEQC_ST_ALPHA_RETRY 0x0080u      /* requantized with alpha/4 after a failed check */
#define AEQC_ST_AE_EXACT 0x0100u         /* every code is 0: the decoder alone met the bound */
#define AEQC_ST_OUTLIER_OVERFLOW 0x0200u /* outlier list full: raw values of this
                                            histogram were dropped (data lost) */

/* ---- residual codes (int16) ---------------------------------------------- */
#define AEQC_CODE_ESCAPE (-32768) /* raw value stored in the outlier list */
#define AEQC_CODE_ZERO (-32767)   /* reconstruction level exactly 0 */
#define AEQC_CODE_MAX 32766       /* |q| <= AEQC_CODE_MAX for grid levels */

/* ---- limits --------------------------------------------------------------- */
#define AEQC_MAX_NPAR 64
#define AEQC_MAX_NPERP 64
#define AEQC_MAX_P 1536 /* n_par * n_perp */
#define AEQC_XHAT_LD 1536 /* default leading dimension of decoded rows */

/* ---- velocity grid (Sec. II, Eq. (1)-(4)) -------------------------------- */
typedef struct aeqc_grid {
  int32_t n_par;          /* v_par nodes (index i, fastest), <= AEQC_MAX_NPAR */
  int32_t n_perp;         /* v_perp nodes (index j), <= AEQC_MAX_NPERP */
  const double* vpar_host;  /* HOST [n_par] v_par values */
  const double* vperp_host; /* HOST [n_perp] v_perp values */
  const double* vol;      /* DEVICE [n_perp*n_par] cell volumes, or NULL */
  double vol_uniform;     /* cell volume used when vol == NULL */
  double mass;            /* particle mass m (scales T only; unused by the path) */
} aeqc_grid;

/* ---- method parameters ---------------------------------------------------- */
typedef struct aeqc_params {
  double tau;          /* pointwise bound e = tau * max(x) per histogram */
  double alpha;        /* quantizer share: Delta = 2^floor(log2(2 alpha e)) */
  double step_s;       /* Newton step s of Eq. (6) (1.0) */
  double tol;          /* convergence: max_k |g_k| / S_k <= tol (1e-12) */
  int32_t max_iter;    /* round-1 iteration cap (50) */
  int32_t r2_max_iter; /* round-2 iteration cap (400) */
  int32_t loss;        /* 0: generalised KL, f = x' exp(-lambda.phi) (default);
                          1: L2, f = x' - lambda.phi */
  int32_t warm_iters;  /* warm-start probation iterations (2) */
  double warm_reject;  /* reject the warm start if the residual after
                          warm_iters steps exceeds this (1e-8) */
  double qoi_check;    /* end-to-end moment check (1e-10) */
  int32_t kernel;      /* AEQC_KERNEL_*: correction kernel */
  int32_t reserved;
} aeqc_params;

#define AEQC_KERNEL_FP64 0  /* per-point work in native FP64 (plain form) */
#define AEQC_KERNEL_FAST 1  /* per-point work on the FP32/INT pipes with
                               error-free transforms; FP64 for per-histogram
                               scalars only; same results within tolerance */

/* Fills the defaults listed above (tau = 1e-4, alpha = 0.5). */
void aeqc_params_default(aeqc_params* p);

/* Message of the last error on this thread ("" if none). */
const char* aeqc_last_error(void);

/* Library version string. */
const char* aeqc_version(void);

/* ---- autoencoder model (Sec. III Stage 2, Sec. IV-B) ---------------------- */
#define AEQC_DTYPE_F32 0  /* FP32 weights/activations, FP32 SIMT GEMMs */
#define AEQC_DTYPE_BF16 1 /* BF16 weights/activations, FP32 accumulate, tcgen05;
                             training GEMMs with BF16 operands on tcgen05 too */

#define AEQC_ACT_IDENTITY 0 /* the paper's linear activation */
#define AEQC_ACT_RELU 1

typedef struct aeqc_model_desc {
  int32_t P;        /* input size n_par*n_perp (<= AEQC_MAX_P) */
  int32_t H;        /* hidden width (multiple of 32, <= 1024) */
  int32_t L;        /* latent size (multiple of 8, <= 256) */
  int32_t tied;     /* 1: decoder layers use the encoder weights transposed */
  int32_t act;      /* AEQC_ACT_* for the hidden layers */
  int32_t dtype;    /* AEQC_DTYPE_* of the inference path */
  int32_t n_groups; /* independent models (subdomains, Sec. III Stage 1) */
  int32_t layers;   /* 0 or 2: P -> H -> L -> H -> P; 1: the paper's network,
                       one tied linear layer P -> L -> P (Sec. IV-B, Fig. 2):
                       needs H == L (a multiple of 4, <= 256), tied, FP32;
                       stored as the two-layer net with W2 = I, b2 = b3 = 0,
                       which set_group writes and training keeps (their
                       gradients are zero) */
} aeqc_model_desc;

typedef struct aeqc_model aeqc_model;

/* Creates a model with n_groups zero-initialised parameter sets (weights
 * must be set with aeqc_model_set_group before use).  Allocates the device
 * memory it owns. */
int aeqc_model_create(const aeqc_model_desc* desc, aeqc_model** out);
int aeqc_model_destroy(aeqc_model* m);

/* Launch choices of a model's kernels (no effect on results, only on speed).
 * 0 in a field selects the built-in default.
 *   enc_stages, dec_stages  pipeline depth of the BF16 tensor-core encoder /
 *                           decoder (2..6 / 2..16; reduced to what fits in
 *                           shared memory)
 *   qc_warps_per_sm         warps of the correction kernel per SM (4, 8, 12
 *                           or 16; one CTA per SM) in compress_batch and
 *                           compress_batch_host */
typedef struct aeqc_tuning {
  int32_t enc_stages;
  int32_t dec_stages;
  int32_t qc_warps_per_sm;
  int32_t reserved;
} aeqc_tuning;
int aeqc_model_set_tuning(aeqc_model* m, const aeqc_tuning* t);
int aeqc_model_get_tuning(const aeqc_model* m, aeqc_tuning* t);

/* Device status of the model's tensor-core kernels (encoder, decoder,
 * training GEMMs): every wait inside them is bounded, and one that runs out
 * sets the model's device status word instead of hanging.  Synchronises
 * `stream`, copies the word to *status (0: no wait ran out since the last
 * call; nonzero: the outputs of the calls since then are not valid) and
 * clears it. */
int aeqc_model_device_status(aeqc_model* m, int32_t* status, void* stream);

/* Sets (synchronously) the parameters of one group from HOST float64 arrays:
 * W1 [P][H], b1 [H], W2 [H][L], b2 [L], b3 [H], b4 [P], mu [P], sigma [P]
 * (per-pixel Z-score of x / max(x), Sec. IV-C), and for untied models
 * W3 [L][H], W4 [H][P] (NULL when tied).  Dense layers compute y = W^T x + b.
 * Resets the group's Adam state. */
int aeqc_model_set_group(aeqc_model* m, int32_t group, const double* W1_host,
                         const double* b1_host, const double* W2_host,
                         const double* b2_host, const double* W3_host,
                         const double* b3_host, const double* W4_host,
                         const double* b4_host, const double* mu_host,
                         const double* sigma_host);

/* Reads (synchronously) the FP32 master parameters of one group into HOST
 * float64 arrays with the layouts of aeqc_model_set_group (NULL = skip). */
int aeqc_model_get_group(aeqc_model* m, int32_t group, double* W1_host, double* b1_host,
                         double* W2_host, double* b2_host, double* W3_host,
                         double* b3_host, double* W4_host, double* b4_host,
                         double* mu_host, double* sigma_host);

/* Fits mu/sigma of one group on n training histograms x (device): per pixel
 * mean and max(std, 1e-6) of x / max(x).  Asynchronous. */
int aeqc_fit_normalizer(aeqc_model* m, int32_t group, const double* x, int64_t n,
                        void* workspace, size_t workspace_bytes, void* stream);
size_t aeqc_fit_normalizer_workspace_size(const aeqc_model* m);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) of group `group` on
 * the MSE of Eq. (5) between the normalised batch u = (x/max(x) - mu)/sigma
 * and its reconstruction, computed by the library's own forward and backward
 * kernels: FP32 SIMT GEMMs for an FP32 model; for a BF16 model the GEMMs run
 * on the tensor cores with BF16-rounded operands and FP32 accumulation (the
 * master weights, Adam and the elementwise steps stay FP32).  x_batch
 * [B][P] device float64.  loss_out (device float,
 * may be NULL) receives the batch loss before the step. */
int ae_train_step(aeqc_model* m, const double* x_batch, int64_t B, int32_t group,
                  float lr, float* loss_out, void* workspace, size_t workspace_bytes,
                  void* stream);
size_t ae_train_workspace_size(const aeqc_model* m, int64_t B);

/* Number of trainable parameters of one group: P*H + H + H*L + L
 * (+ L*H untied) + H (+ H*P untied) + P. */
int64_t aeqc_model_param_count(const aeqc_model* m);

/* The loss of ae_train_step and its gradient without updating anything:
 * grad_out (device float32, aeqc_model_param_count entries) in the order
 * W1 [P][H], b1, W2 [H][L], b2, (W3 [L][H]), b3, (W4 [H][P]), b4; tied
 * weights receive the sum of their encoder and decoder uses.  Uses the
 * workspace of ae_train_step. */
int ae_loss_grad(aeqc_model* m, const double* x_batch, int64_t B, int32_t group,
                 float* loss_out, float* grad_out, void* workspace, size_t workspace_bytes,
                 void* stream);

/* Encoder (Sec. III Stage 3): latent [n][L] (float32 for F32 models, bf16
 * for BF16 models) and scale [n] = max(x) per histogram (float64).
 * group_offsets: DEVICE int64 [n_groups+1] row offsets of the subdomains
 * (rows of group g are [off[g], off[g+1])), or NULL for one group. */
int ae_encode(aeqc_model* m, const double* x, int64_t n, const int64_t* group_offsets,
              void* latent, double* scale, void* workspace, size_t workspace_bytes,
              void* stream);
size_t ae_encode_workspace_size(const aeqc_model* m, int64_t n);

/* Decoder from a stored latent: xhat[b][p] = scale[b] (sigma_p y_p + mu_p),
 * float32 rows of leading dimension ld >= P (ld multiple of 4). */
int ae_decode(aeqc_model* m, const void* latent, const double* scale, int64_t n,
              const int64_t* group_offsets, float* xhat, int64_t ld, void* workspace,
              size_t workspace_bytes, void* stream);
size_t ae_decode_workspace_size(const aeqc_model* m, int64_t n);

/* ---- outlier list (escape codes) ------------------------------------------ */
typedef struct aeqc_outliers {
  int64_t capacity; /* entries available in index/value */
  int64_t* count;   /* DEVICE, one int64: entries needed.  Zeroed by the call
                       that fills the list.  If it ends above capacity the
                       excess was dropped and the histograms concerned carry
                       AEQC_ST_OUTLIER_OVERFLOW. */
  int64_t* index;   /* DEVICE [capacity]: flat index b * P + p */
  double* value;    /* DEVICE [capacity]: raw x at that point */
} aeqc_outliers;

/* ---- residual quantizer (Sec. III Stage 4) -------------------------------- */
/* e = tau * s with s = max(x); Delta = 2^floor(log2(2 alpha e));
 * q = round-half-even((x - xhat) / Delta) on the exact real difference;
 * code = q if |q| <= AEQC_CODE_MAX, AEQC_CODE_ZERO when the level 0 is
 * strictly nearer to x than xhat + q Delta, AEQC_CODE_ESCAPE (raw value
 * appended to `out`) for a non-finite xhat or |q| too large.
 * x' = fl64(xhat + q Delta) (0 at the zero code, raw x at escapes), so
 * |x' - x| <= Delta / 2 (+ half an ulp of x') <= alpha e.
 * Inputs: x [n][P], xhat [n][ld] float32.  Outputs: codes [n][P] int16,
 * scale [n], status [n] (ZERO_IMAGE / NONFINITE_INPUT / CODE_ESCAPE /
 * AE_EXACT / VERBATIM), xrec [n][P] (x', may be NULL). */
int residual_quantize(const double* x, const float* xhat, int64_t ld, int64_t n,
                      int32_t P, const aeqc_params* params, int16_t* codes,
                      double* scale, uint16_t* status, aeqc_outliers* out,
                      double* xrec, void* stream);

/* x' from codes: fl64(xhat + q Delta), 0 at AEQC_CODE_ZERO, the outlier
 * list's raw values at escapes; status selects alpha/4 (ALPHA_RETRY) and
 * zero images.  outliers may be NULL when no code escapes. */
int residual_dequantize(const float* xhat, int64_t ld, const int16_t* codes,
                        const aeqc_outliers* outliers, const double* scale,
                        const uint16_t* status, int64_t n, int32_t P,
                        const aeqc_params* params, double* xrec, void* stream);

/* ---- QoI correction (Sec. III Stage 5) ------------------------------------ */
/* Q [n][4] = sum vol phi_k x with phi = (1, v_par, v_perp^2, v_par^2), the
 * linear moments behind n, u_par, T_perp, T_par of Eq. (1)-(4). */
int qoi_moments(const aeqc_grid* grid, const double* x, int64_t n, double* Q,
                void* stream);

/* Solves for lambda [n][4] such that f = x' exp(-lambda.phi) (KL loss) has
 * moments Q, by Newton on the dual, Eq. (6): lambda <- lambda + s M^-1 g,
 * g = sum vol phi f - Q, M = sum vol phi phi^T f; convergence max_k |g_k|/S_k
 * <= tol, S_k = sum vol |phi_k| f, tested before each step; round 2 (damped
 * Newton from 0) for the non-converged.  lambda: in = warm start when
 * use_warm != 0 (probation of warm_iters steps), else ignored; out = result.
 * f_out [n][P] (may be NULL), iters [n] uint8 (steps, saturating),
 * status [n] (CONVERGED / ROUND2 / WARM_REJECTED; none of them = failed). */
int qoi_correct(const aeqc_grid* grid, const double* xrec, const double* Q, int64_t n,
                const aeqc_params* params, int32_t use_warm, double* lambda,
                double* f_out, uint8_t* iters, uint16_t* status, void* stream);

/* ---- fused batch calls ---------------------------------------------------- */
/* Compressed batch, all DEVICE and caller-owned. */
typedef struct aeqc_compressed {
  void* latent;      /* [n][L] model dtype */
  double* scale;     /* [n] max(x) */
  int16_t* codes;    /* [n][P] */
  double* lambda;    /* [n][4] */
  uint8_t* iters;    /* [n] Newton steps */
  uint16_t* status;  /* [n] */
  aeqc_outliers outliers;
  float* features;   /* optional [n][L + 4] float32 (NULL = not written): the
                        warm-start inputs (latent, d_0..d_3), see aeqc_mlp */
} aeqc_compressed;

typedef struct aeqc_mlp aeqc_mlp;

/* Stages 4-5 given decoded histograms xhat [n][ld] float32: targets Q(x),
 * residual quantization against xhat, Newton correction (warm-started by
 * `mlp` when non-NULL: then out->latent is READ as the MLP input, with
 * latent_dtype AEQC_DTYPE_F32/BF16 and latent_dim L), end-to-end check
 * (|f - x| <= tau max(x) at every point and |Q_k(f) - Q_k(x)| / S_k(x) <=
 * qoi_check), one retry with alpha/4 after a failed check, verbatim storage
 * when that fails too or Newton does not converge.  out->latent is not
 * written.  f_out [n][P] (may be NULL) receives the corrected histograms.
 * The workspace (quantize_correct_workspace_size bytes) holds the list of
 * histograms the fast kernel hands to the FP64 kernel. */
int quantize_correct(const aeqc_grid* grid, const double* x, const float* xhat, int64_t ld,
                     int64_t n, const aeqc_params* params, aeqc_mlp* mlp,
                     int32_t latent_dtype, int32_t latent_dim, aeqc_compressed* out,
                     double* f_out, void* workspace, size_t workspace_bytes, void* stream);
size_t quantize_correct_workspace_size(int64_t n);

/* quantize_correct without a caller workspace, for callers that cannot
 * allocate device memory at the point of the call (an allocator-free serving
 * loop, code that runs while another component owns the device memory
 * pool).  The paper has no counterpart: this is a deployment variant of
 * the call above, with the same arguments (minus the workspace), the same
 * kernels and the same results.
 *
 * Its scratch (the list of histograms the fast kernel hands to the FP64
 * kernel, and that list's count) lives in one file-scope device array of
 * the library, sized for AEQC_QC_NOALLOC_MAX_N histograms (about 1 MiB);
 * n above that limit returns AEQC_EINVAL (split the batch).  Nothing is
 * allocated: no cudaMalloc/cudaFree and no allocating library routine.
 * The count is reset on the caller's stream at the start of each call; the
 * list needs no clearing.
 *
 * The first call on each device (with that device current) looks up the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  Every call in the process shares the one
 * array: calls that may overlap on the device (different streams without
 * ordering between them, or concurrent host threads) race on it and give
 * wrong results; serialise them (one stream, or an event between calls). */
#define AEQC_QC_NOALLOC_MAX_N 262144
int quantize_correct_noalloc(const aeqc_grid* grid, const double* x, const float* xhat,
                             int64_t ld, int64_t n, const aeqc_params* params,
                             aeqc_mlp* mlp, int32_t latent_dtype, int32_t latent_dim,
                             aeqc_compressed* out, double* f_out, void* stream);

/* Compression of n histograms (Stages 3-5): encode, decode, targets Q(x),
 * quantize against the decoded xhat, Newton correction (warm-started by
 * `mlp` when non-NULL), end-to-end check (|f - x| <= e at every point and
 * |Q_k(f) - Q_k(x)| / S_k(x) <= qoi_check); a failed check retries once with
 * alpha/4, then stores the histogram verbatim.  Device work only; the host
 * reads nothing back. */
int compress_batch(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid, const double* x,
                   int64_t n, const int64_t* group_offsets, const aeqc_params* params,
                   aeqc_compressed* out, void* workspace, size_t workspace_bytes,
                   void* stream);
size_t compress_batch_workspace_size(const aeqc_model* m, int64_t n);

/* Autotuner of the launch choices (aeqc_tuning) for this model on this batch:
 * times every candidate of each stage (encoder pipeline depths, decoder
 * pipeline depths, correction-kernel CTAs per SM) with CUDA events on
 * `stream`, keeps the fastest in the model and returns it in *best.
 * Arguments as compress_batch (the outputs are written, as by compress_batch
 * with the chosen tuning).  Synchronises the stream; not for use during
 * stream capture.  The paper has no counterpart. */
int aeqc_autotune(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid, const double* x,
                  int64_t n, const int64_t* group_offsets, const aeqc_params* params,
                  aeqc_compressed* out, void* workspace, size_t workspace_bytes, void* stream,
                  aeqc_tuning* best);

/* compress_batch from HOST memory to HOST memory, streamed: the batch is cut
 * into chunks of `chunk` histograms; each chunk's input is copied to the
 * device, compressed and its outputs copied back, on three streams (the
 * caller's for compute, two library-owned ones for the copies) with two
 * device buffers, so the copies of one chunk overlap the compute of the
 * next.  Same results as compress_batch on the whole batch.
 *   x_host   [n][P] float64, host (page-locked for the copies to overlap)
 *   out_host aeqc_compressed whose arrays are HOST arrays of the full batch
 *            (latent [n][L], scale, codes [n][P], lambda [n][4], iters,
 *            status, outliers with global indices; features must be NULL);
 *            outliers.count is written at the end
 *   chunk    histograms per chunk (> 0)
 * Single-group models only (AEQC_EUNSUPPORTED otherwise).  The workspace
 * (compress_batch_host_workspace_size) holds the two device buffers.  On
 * return the work is enqueued; the caller's stream is ordered after the last
 * copy (synchronise it before reading out_host). */
int compress_batch_host(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid,
                        const double* x_host, int64_t n, const aeqc_params* params,
                        aeqc_compressed* out_host, int64_t chunk, void* workspace,
                        size_t workspace_bytes, void* stream);
size_t compress_batch_host_workspace_size(const aeqc_model* m, int64_t chunk,
                                          int64_t outlier_capacity);

/* Decompression (end of Stage 5): decode the latents, x' from the codes,
 * f = x' exp(-lambda.phi) at every point (raw values at escapes, also
 * corrected), f [n][P] float64. */
int decompress_batch(aeqc_model* m, const aeqc_grid* grid, const aeqc_compressed* in,
                     int64_t n, const int64_t* group_offsets, const aeqc_params* params,
                     double* f, void* workspace, size_t workspace_bytes, void* stream);
size_t decompress_batch_workspace_size(const aeqc_model* m, int64_t n);

/* ---- learned warm start (MLP in -> 64 -> 64 -> 4, ReLU) ------------------- */
/* Input per histogram: [latent (L values), d_0..d_3] with the moment defects
 * d_k = (Q_k(x) - Q_k(x')) / S_k(x'); output: the four multipliers.
 * Normalisation of inputs and targets (mean/std) is part of the parameters. */
int aeqc_mlp_create(int32_t n_in, int32_t n_hidden, aeqc_mlp** out);
int aeqc_mlp_destroy(aeqc_mlp* m);
/* HOST float64: W1 [n_in][nh], b1 [nh], W2 [nh][nh], b2 [nh], W3 [nh][4],
 * b3 [4], in_mu/in_sd [n_in], out_mu/out_sd [4].  Resets the Adam state. */
int aeqc_mlp_set(aeqc_mlp* m, const double* W1, const double* b1, const double* W2,
                 const double* b2, const double* W3, const double* b3,
                 const double* in_mu, const double* in_sd, const double* out_mu,
                 const double* out_sd);
int aeqc_mlp_get(aeqc_mlp* m, double* W1, double* b1, double* W2, double* b2, double* W3,
                 double* b3);
/* One Adam step on mean((out - (lambda - out_mu)/out_sd)^2); inputs [B][n_in]
 * float32, target_lambda [B][4] float64 (device). */
int mlp_train_step(aeqc_mlp* m, const float* inputs, const double* target_lambda,
                   int64_t B, float lr, float* loss_out, void* workspace,
                   size_t workspace_bytes, void* stream);
size_t mlp_train_workspace_size(const aeqc_mlp* m, int64_t B);
/* Loss and gradient of mlp_train_step without the update: grad_out (device
 * float32) in the order W1 [n_in][nh], b1, W2 [nh][nh], b2, W3 [nh][4], b3. */
int mlp_loss_grad(aeqc_mlp* m, const float* inputs, const double* target_lambda, int64_t B,
                  float* loss_out, float* grad_out, void* workspace, size_t workspace_bytes,
                  void* stream);
int64_t aeqc_mlp_param_count(const aeqc_mlp* m);
/* lambda0 [n][4] float64 from inputs [n][n_in] float32. */
int mlp_predict(aeqc_mlp* m, const float* inputs, int64_t n, double* lambda0, void* stream);

/* ---- product quantisation of the latents (Sec. III Stage 3, Sec. V-B) ---- */
/* Each subdomain's latent vectors are quantised column by column: K-means
 * with k clusters per latent dimension; a value is stored as its cluster's
 * index (log2 k bits, one uint8 per value here) and decoded as the cluster's
 * centroid, from a float32 PQ table [G][L][k].  The paper gives neither the
 * K-means start nor the iteration count; this library starts from k
 * centroids evenly spaced in the column's range, c_j = lo + (j + 1/2)(hi - lo)/k
 * (float64, rounded to float32), and runs `iters` Lloyd iterations: nearest
 * centroid by float32 |z - c_j| (ties to the lowest index), then each
 * centroid moves to the mean of its members (rounded to float32; a centroid
 * without members stays).  Non-finite latents take no part in training and
 * encode as index 0.  The means are sums of 64-bit fixed-point values
 * (resolution 2^-62 of the column's largest magnitude times the group's row
 * count), so results do not depend on scheduling and lie within
 * 2^-42 max|z| (1M rows per group) of the float64 mean.
 * z: [n][L] latents of latent_dtype (AEQC_DTYPE_F32 / BF16), rows of group g
 * in [group_offsets[g], group_offsets[g+1]) (DEVICE int64 [G+1]; NULL: one
 * group), 2 <= k <= AEQC_PQ_MAX_K, L <= 256, L * (k + 1) <= 10240 for training. */
#define AEQC_PQ_MAX_K 256
size_t pq_train_workspace_size(int32_t G, int32_t L, int32_t k);
int pq_train(const void* z, int32_t latent_dtype, int64_t n, int32_t L,
             const int64_t* group_offsets, int32_t G, int32_t k, int32_t iters, float* table,
             void* workspace, size_t workspace_bytes, void* stream);
/* codes [n][L] uint8: nearest centroid of each value (may be NULL); zq [n][L]
 * in latent_dtype: the decoded latents (may be NULL, may be z itself). */
int pq_encode(const void* z, int32_t latent_dtype, int64_t n, int32_t L,
              const int64_t* group_offsets, int32_t G, int32_t k, const float* table,
              uint8_t* codes, void* zq, void* stream);
/* z [n][L] in latent_dtype from codes and the table (a code >= k decodes to 0). */
int pq_decode(const uint8_t* codes, int64_t n, int32_t L, const int64_t* group_offsets,
              int32_t G, int32_t k, const float* table, int32_t latent_dtype, void* z,
              void* stream);

/* ---- entropy coding of the residual codes ---------------------------------- */
/* The paper hands the quantised residual to MGARD's lossless stage (Sec. III
 * Stage 4; the coded bytes go to the buffer of Stage 5) without fixing a
 * format.  These calls code the int16 codes of each histogram with one
 * Golomb-Rice code:
 *   symbols: AEQC_CODE_ZERO -> 0, a level q -> zigzag(q) + 1 (zigzag(q) = 2q
 *   for q >= 0, -2q - 1 for q < 0), AEQC_CODE_ESCAPE -> 65535;
 *   parameter k in 0..15 per histogram, the one with the fewest bits (ties to
 *   the smaller k);
 *   symbol s: u = s >> k; u < 24: u one-bits, a zero-bit, the k low bits of s
 *   (least significant first); otherwise 24 one-bits and the 16 bits of s;
 *   bit i of a stream is bit (i mod 32) of 32-bit word i / 32, unused high
 *   bits of the last word zero; streams back to back at word offsets.
 * rice_measure: kparam [n] uint8, nbits [n] uint32 and offsets [n + 1] int64
 * (exclusive prefix sum of ceil(nbits / 32); offsets[n] = total words), all
 * DEVICE.  rice_pack: writes every stream at its offset into words
 * (capacity words available; a stream that would not fit is not written, so
 * size words from offsets[n]).  rice_unpack: codes [n][P] from the streams;
 * reads stay inside [offsets[b], offsets[b + 1]) clipped to [0, total_words),
 * so damaged offsets or streams give wrong codes but no stray access. */
size_t rice_workspace_size(int64_t n);
int rice_measure(const int16_t* codes, int64_t n, int32_t P, uint8_t* kparam, uint32_t* nbits,
                 int64_t* offsets, void* workspace, size_t workspace_bytes, void* stream);
int rice_pack(const int16_t* codes, int64_t n, int32_t P, const uint8_t* kparam,
              const int64_t* offsets, uint32_t* words, int64_t capacity, void* stream);
int rice_unpack(const uint32_t* words, int64_t total_words, const int64_t* offsets,
                const uint8_t* kparam, int64_t n, int32_t P, int16_t* codes, void* stream);

/* ---- NRMSE and the error-bound search (Sec. IV-A Eq. (7); Sec. III Stage 4) -- */
/* nrmse_batch: per_hist [n] (DEVICE, may be NULL) = sqrt(mean_p (x - f)^2) /
 * (max x - min x) of each histogram; batch [1] (DEVICE) = the same over all
 * n * P values with the range of the whole batch.  Deterministic (fixed
 * summation order).  x, f: [n][P] float64. */
size_t nrmse_workspace_size(int64_t n);
int nrmse_batch(const double* x, const double* f, int64_t n, int32_t P, double* per_hist,
                double* batch, void* workspace, size_t workspace_bytes, void* stream);
/* The paper finds its residual compressor's error bound automatically for a
 * target accuracy; here the bound is the pointwise tau.  Bisection on
 * log(tau): the first probe is tau_lo, then `probes - 1` midpoints of the
 * bracket; each probe compresses and decompresses the batch (compress_batch,
 * decompress_batch with `base` except tau) and measures the batch NRMSE.
 * Returns the largest probed tau whose NRMSE <= target and that NRMSE
 * (host doubles).  AEQC_EUNSUPPORTED if tau_lo already misses the target
 * or a probe escapes more values than outlier_capacity holds.
 * Synchronizes the stream once per probe.  The workspace holds one
 * compressed batch, the decompressed batch and the calls' workspaces. */
size_t aeqc_bound_search_workspace_size(const aeqc_model* m, int64_t n,
                                        int64_t outlier_capacity);
int aeqc_bound_search(aeqc_model* m, const aeqc_grid* grid, const double* x, int64_t n,
                      const int64_t* group_offsets, const aeqc_params* base, double target,
                      double tau_lo, double tau_hi, int32_t probes, int64_t outlier_capacity,
                      double* tau_out, double* nrmse_out, void* workspace,
                      size_t workspace_bytes, void* stream);

/* ---- checkpoints and the compressed-batch container ----------------------- */
/* The paper stores, per histogram, the codes, the latent and the Lagrange
 * multipliers (Sec. III, Stage 5) next to the trained network (Sec. III,
 * Stage 1); it gives no file format.  These calls define one: little-endian
 * blobs in HOST memory with an 8-byte magic, a version and a header size, so
 * that a reader rejects what it does not know.  All of them are synchronous
 * (they return when every copy has completed).
 *
 * Model checkpoint: header (magic "AEQCMDL1", version 1, 64 bytes: the
 * aeqc_model_desc, floats per group and trainable floats per group), then
 * FP32 params [n_groups][per group] (weights, biases, mu, sigma), Adam first
 * and second moments [n_groups][trainable], int32 Adam step per group.
 * Launch tuning is not saved (it belongs to the machine).  *_save_size gives
 * the exact blob size; *_save needs bytes >= that.  *_load validates the
 * header and the size (AEQC_ECORRUPT on a bad magic, version, descriptor or
 * size: nothing is allocated then) and creates a new model that owns its
 * device memory until aeqc_model_destroy. */
size_t aeqc_model_save_size(const aeqc_model* m);
int aeqc_model_save(const aeqc_model* m, void* blob_host, size_t bytes);
int aeqc_model_load(const void* blob_host, size_t bytes, aeqc_model** out);

/* MLP checkpoint: header (magic "AEQCMLP1", version 1, 40 bytes: n_in,
 * n_hidden, floats of params, trainable floats), FP32 params (weights,
 * biases and the input/output normalisation), Adam moments, int32 step. */
size_t aeqc_mlp_save_size(const aeqc_mlp* m);
int aeqc_mlp_save(const aeqc_mlp* m, void* blob_host, size_t bytes);
int aeqc_mlp_load(const void* blob_host, size_t bytes, aeqc_mlp** out);

/* Batch container: a 192-byte header (magic "AEQCBAT1", version 1, n, P, L,
 * latent dtype, outlier count, total bytes and a table of eight sections as
 * (offset, bytes), offsets 16-byte aligned, increasing, non-overlapping) then
 * the sections latent [n][L] (model dtype), scale [n] f64, codes [n][P]
 * int16, lambda [n][4] f64, iters [n] u8, status [n] u16, outlier index
 * [count] i64 and value [count] f64.  The features array is not stored.
 * pack_size is the blob size for these counts (0 for negative sizes).
 * pack reads the device outlier count (clamped to the list's capacity; a
 * dropped excess is already flagged in the status words), copies every
 * section to blob_host and sets *written; bytes must cover the blob.
 * peek validates the header against `bytes` and returns the counts (any
 * output pointer may be NULL).  unpack validates the same way and copies
 * every section, and the outlier count, into the caller's device arrays
 * (outliers.capacity must hold the count).  A blob that is truncated, or
 * whose magic, version, counts, section table or total size do not agree,
 * returns AEQC_ECORRUPT before anything is copied. */
size_t aeqc_batch_pack_size(int64_t n, int32_t P, int32_t L, int32_t latent_dtype,
                            int64_t outliers);
int aeqc_batch_pack(const aeqc_compressed* in, int64_t n, int32_t P, int32_t L,
                    int32_t latent_dtype, void* blob_host, size_t bytes, size_t* written,
                    void* stream);
int aeqc_batch_peek(const void* blob_host, size_t bytes, int64_t* n, int32_t* P, int32_t* L,
                    int32_t* latent_dtype, int64_t* outliers);
int aeqc_batch_unpack(const void* blob_host, size_t bytes, aeqc_compressed* out, void* stream);

/* ---- multi-GPU partitioning (host) ---------------------------------------- */
/* Each processor trains and compresses its own subdomains with no exchange
 * of data (Sec. III Stage 1; Sec. IV-B, distributed training), and the
 * per-processor buffers are written one after another (Sec. III, the
 * output stage).  On one node with several GPUs (one process per GPU) whole
 * subdomains are the unit: aeqc_partition_lpt assigns them to ranks by the
 * longest-processing-time rule on their histogram counts, and
 * aeqc_exclusive_scan turns per-rank compressed byte counts into output
 * offsets.  Host pointers, synchronous, deterministic: every rank that calls
 * them with the same arguments gets the same answer, so no collective is
 * needed to agree on the assignment.
 *
 * aeqc_partition_lpt: counts_host[n_groups] (>= 0) histograms per subdomain;
 * owner_host[n_groups] receives the rank of each subdomain and
 * load_host[n_ranks] (may be NULL) the histograms per rank.  Subdomains are
 * taken in decreasing count (equal counts: lower index first) and each goes
 * to the rank with the least load so far (equal loads: lower rank), so the
 * largest load is at most (4/3 - 1/(3 n_ranks)) of the best possible.
 * AEQC_EINVAL for n_groups < 0, n_ranks < 1, a negative count or null arrays.
 *
 * aeqc_exclusive_scan: offsets_host[n + 1] with offsets[0] = 0 and
 * offsets[r + 1] = offsets[r] + sizes_host[r]; AEQC_EINVAL for n < 0, a
 * negative size, null arrays or a total beyond INT64_MAX. */
int aeqc_partition_lpt(const int64_t* counts_host, int32_t n_groups, int32_t n_ranks,
                       int32_t* owner_host, int64_t* load_host);
int aeqc_exclusive_scan(const int64_t* sizes_host, int32_t n, int64_t* offsets_host);

#ifdef __cplusplus
}
#endif
#endif /* AEQC_H */
