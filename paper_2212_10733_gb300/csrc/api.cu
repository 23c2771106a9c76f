// C-ABI entry points of libaeqc: argument validation on the host, then the
// device work of each call enqueued on the caller's stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>

#include "model.cuh"
#include "workspace.cuh"

namespace aeqc {

static thread_local char g_err[512] = {0};

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = 0; }

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(AEQC_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
  return AEQC_OK;
}

int raise_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> raised;
  int dev = 0;
  AEQC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& cur = raised[std::make_pair(func, dev)];
  if (cur >= bytes) return AEQC_OK;
  AEQC_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
  return AEQC_OK;
}

int make_grid(const aeqc_grid* g, GridK* k) {
  AEQC_CHECK_ARG(g, "null grid");
  AEQC_CHECK_ARG(g->n_par >= 1 && g->n_par <= AEQC_MAX_NPAR, "grid: n_par=%d out of range",
                 g->n_par);
  AEQC_CHECK_ARG(g->n_perp >= 1 && g->n_perp <= AEQC_MAX_NPERP,
                 "grid: n_perp=%d out of range", g->n_perp);
  AEQC_CHECK_ARG(g->n_par * g->n_perp <= AEQC_MAX_P, "grid: n_par*n_perp > %d", AEQC_MAX_P);
  AEQC_CHECK_ARG(g->vpar_host && g->vperp_host, "grid: null vpar/vperp");
  AEQC_CHECK_ARG(g->vol || (std::isfinite(g->vol_uniform) && g->vol_uniform > 0.0),
                 "grid: vol_uniform must be positive when vol is NULL");
  memset(k, 0, sizeof(*k));
  k->n_par = g->n_par;
  k->n_perp = g->n_perp;
  k->P = g->n_par * g->n_perp;
  k->has_vol = g->vol != nullptr;
  k->vol = g->vol;
  k->vol_uniform = g->vol_uniform;
  for (int i = 0; i < g->n_par; ++i) {
    AEQC_CHECK_ARG(std::isfinite(g->vpar_host[i]), "grid: non-finite v_par");
    k->vpar[i] = g->vpar_host[i];
  }
  for (int j = 0; j < g->n_perp; ++j) {
    AEQC_CHECK_ARG(std::isfinite(g->vperp_host[j]), "grid: non-finite v_perp");
    k->vperp2[j] = g->vperp_host[j] * g->vperp_host[j];
  }
  return AEQC_OK;
}

int make_params(const aeqc_params* p, ParamsK* k) {
  AEQC_CHECK_ARG(p, "null params");
  AEQC_CHECK_ARG(std::isfinite(p->tau) && p->tau > 0.0, "params: tau must be positive");
  AEQC_CHECK_ARG(std::isfinite(p->alpha) && p->alpha > 0.0 && p->alpha <= 0.5,
                 "params: alpha must be in (0, 0.5]");
  AEQC_CHECK_ARG(std::isfinite(p->step_s) && p->step_s > 0.0, "params: step_s must be positive");
  AEQC_CHECK_ARG(std::isfinite(p->tol) && p->tol >= 0.0, "params: tol must be >= 0");
  AEQC_CHECK_ARG(p->max_iter >= 0 && p->max_iter <= 10000, "params: max_iter out of range");
  AEQC_CHECK_ARG(p->r2_max_iter >= 0 && p->r2_max_iter <= 10000,
                 "params: r2_max_iter out of range");
  AEQC_CHECK_ARG(p->loss == 0 || p->loss == 1, "params: loss must be 0 (KL) or 1 (L2)");
  AEQC_CHECK_ARG(p->warm_iters >= 0 && p->warm_iters <= p->max_iter,
                 "params: warm_iters must be in [0, max_iter]");
  AEQC_CHECK_ARG(p->kernel == AEQC_KERNEL_FP64 || p->kernel == AEQC_KERNEL_FAST,
                 "params: unknown kernel %d", p->kernel);
  k->tau = p->tau;
  k->alpha = p->alpha;
  k->step_s = p->step_s;
  k->tol = p->tol;
  k->warm_reject = p->warm_reject;
  k->qoi_check = p->qoi_check;
  k->max_iter = p->max_iter;
  k->r2_max_iter = p->r2_max_iter;
  k->loss = p->loss;
  k->warm_iters = p->warm_iters;
  k->alpha4 = p->alpha * 0.25;
  {
    // exact powers of two 2 alpha = 2^e (frexp gives mantissa 0.5 exactly)
    int e2 = 0, e24 = 0, et = 0;
    const double m2 = std::frexp(2.0 * p->alpha, &e2), m24 = std::frexp(2.0 * k->alpha4, &e24);
    const double mt = std::frexp(p->tau, &et);
    k->bw_int = m2 == 0.5 && m24 == 0.5 && p->tau >= DBL_MIN && 2.0 * k->alpha4 >= DBL_MIN;
    k->a2_e[0] = e2 - 1;
    k->a2_e[1] = e24 - 1;
    k->tau_e = et - 1;  // tau in [2^tau_e, 2^(tau_e + 1))
    k->tau_m = (unsigned long long)std::ldexp(mt, 53);  // exact: 53-bit significand
  }
  k->tau_f = (float)p->tau;
  k->step_f = (float)p->step_s;
  k->tol_f = (float)p->tol;
  k->warm_reject_f = (float)p->warm_reject;
  k->qoi_check_f = (float)p->qoi_check;
  return AEQC_OK;
}

static bool aligned(const void* p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// Stages 4-5 on decoded histograms (shared by quantize_correct and
// compress_batch).
static size_t qc_ws(long long n) { return ws_round(sizeof(int) * (size_t)(n > 0 ? n : 1)) + kWsAlign; }

static int run_quantize_correct(const GridK& gk, const ParamsK& pk, int kernel,
                                const double* x, const float* xhat, long long ld, long long n,
                                aeqc_mlp* mlp, int latent_dtype, int latent_dim,
                                aeqc_compressed* out, double* f_out, char* ws, size_t ws_bytes,
                                cudaStream_t s, long long row0 = 0, bool reset_count = true,
                                int warps_per_sm = 0) {
  WsCarver c(ws, ws_bytes);
  int* fb_list = c.take<int>((size_t)n);
  int* fb_count = c.take<int>(1);
  if (!c.ok()) return set_error(AEQC_EINVAL, "quantize_correct: workspace too small");
  if (reset_count) AEQC_CUDA_TRY(cudaMemsetAsync(out->outliers.count, 0, sizeof(int64_t), s));
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x;
  a.xhat = xhat;
  a.ldx = ld;
  a.n = n;
  a.row0 = row0;
  a.grid = gk;
  a.prm = pk;
  a.codes = out->codes;
  a.scale = out->scale;
  a.lambda = out->lambda;
  a.iters = out->iters;
  a.status = out->status;
  a.out = make_outliers(&out->outliers);
  a.features = out->features;
  a.latent.ptr = out->latent;
  a.latent.L = latent_dim;
  a.latent.bf16 = latent_dtype == AEQC_DTYPE_BF16;
  a.use_mlp = mlp != nullptr;
  if (mlp) a.mlp = mlp_kernel_view(mlp);
  a.f_out = f_out;
  int rc = make_fast_grid(gk, &a.fg);
  if (rc) return rc;
  a.fb_list = fb_list;
  a.fb_count = fb_count;
  return kernel == AEQC_KERNEL_FAST ? launch_fused_fast(a, s, warps_per_sm)
                                    : launch_fused_fp64(a, s);
}

}  // namespace aeqc

using namespace aeqc;

extern "C" const char* aeqc_last_error(void) { return g_err; }

extern "C" const char* aeqc_version(void) { return "aeqc 0.1 (sm_103a)"; }

extern "C" void aeqc_params_default(aeqc_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tau = 1e-4;
  p->alpha = 0.5;
  p->step_s = 1.0;
  p->tol = 1e-12;
  p->max_iter = 50;
  p->r2_max_iter = 400;
  p->loss = 0;
  p->warm_iters = 2;
  p->warm_reject = 1e-8;
  p->qoi_check = 1e-10;
  p->kernel = AEQC_KERNEL_FP64;
}

// ---- residual quantizer ----------------------------------------------------

extern "C" int residual_quantize(const double* x, const float* xhat, int64_t ld, int64_t n,
                                 int32_t P, const aeqc_params* params, int16_t* codes,
                                 double* scale, uint16_t* status, aeqc_outliers* out,
                                 double* xrec, void* stream) {
  clear_error();
  ParamsK pk;
  int rc = make_params(params, &pk);
  if (rc) return rc;
  AEQC_CHECK_ARG(n >= 0, "residual_quantize: negative n");
  AEQC_CHECK_ARG(P > 0 && P <= AEQC_MAX_P, "residual_quantize: P out of range");
  AEQC_CHECK_ARG(ld >= P, "residual_quantize: ld < P");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(x && xhat && codes && scale && status, "residual_quantize: null array");
  OutliersK ok = make_outliers(out);
  if (out) AEQC_CHECK_ARG(out->count && (out->capacity == 0 || (out->index && out->value)),
                          "residual_quantize: incomplete outlier list");
  return launch_quantize(x, xhat, ld, n, P, pk, codes, scale, status, ok, xrec,
                         static_cast<cudaStream_t>(stream));
}

extern "C" int residual_dequantize(const float* xhat, int64_t ld, const int16_t* codes,
                                   const aeqc_outliers* outliers, const double* scale,
                                   const uint16_t* status, int64_t n, int32_t P,
                                   const aeqc_params* params, double* xrec, void* stream) {
  clear_error();
  ParamsK pk;
  int rc = make_params(params, &pk);
  if (rc) return rc;
  AEQC_CHECK_ARG(n >= 0, "residual_dequantize: negative n");
  AEQC_CHECK_ARG(P > 0 && P <= AEQC_MAX_P && ld >= P, "residual_dequantize: bad P/ld");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(xhat && codes && scale && status && xrec, "residual_dequantize: null array");
  OutliersK ok = make_outliers(outliers);
  return launch_dequantize(xhat, ld, codes, outliers ? &ok : nullptr, scale, status, n, P, pk,
                           xrec, static_cast<cudaStream_t>(stream));
}

// ---- QoI correction --------------------------------------------------------

extern "C" int qoi_moments(const aeqc_grid* grid, const double* x, int64_t n, double* Q,
                           void* stream) {
  clear_error();
  GridK gk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  AEQC_CHECK_ARG(n >= 0, "qoi_moments: negative n");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(x && Q, "qoi_moments: null array");
  return launch_moments(gk, x, n, Q, static_cast<cudaStream_t>(stream));
}

extern "C" int qoi_correct(const aeqc_grid* grid, const double* xrec, const double* Q,
                           int64_t n, const aeqc_params* params, int32_t use_warm,
                           double* lambda, double* f_out, uint8_t* iters, uint16_t* status,
                           void* stream) {
  clear_error();
  GridK gk;
  ParamsK pk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  if ((rc = make_params(params, &pk))) return rc;
  AEQC_CHECK_ARG(n >= 0, "qoi_correct: negative n");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(xrec && Q && lambda && iters && status, "qoi_correct: null array");
  return launch_newton(gk, xrec, Q, n, pk, use_warm ? 1 : 0, lambda, f_out, iters, status,
                       static_cast<cudaStream_t>(stream));
}

// ---- autoencoder -----------------------------------------------------------

extern "C" size_t ae_encode_workspace_size(const aeqc_model* m, int64_t n) {
  return m ? encode_ws(m, n) : 0;
}
extern "C" size_t ae_decode_workspace_size(const aeqc_model* m, int64_t n) {
  return m ? decode_ws(m, n) : 0;
}

extern "C" int ae_encode(aeqc_model* m, const double* x, int64_t n,
                         const int64_t* group_offsets, void* latent, double* scale,
                         void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m, "ae_encode: null model");
  AEQC_CHECK_ARG(n >= 0, "ae_encode: negative n");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(x && latent && scale, "ae_encode: null array");
  AEQC_CHECK_ARG(group_offsets || m->d.n_groups == 1,
                 "ae_encode: group_offsets required for a model with %d groups",
                 m->d.n_groups);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= encode_ws(m, n),
                 "ae_encode: workspace of %zu bytes needed", encode_ws(m, n));
  AEQC_CHECK_ARG(aligned(workspace, kWsAlign), "ae_encode: workspace not 256-byte aligned");
  AEQC_CHECK_ARG(m->d.dtype == AEQC_DTYPE_F32 || m->d.dtype == AEQC_DTYPE_BF16,
                 "ae_encode: bad dtype");
  return run_encode(m, x, n, reinterpret_cast<const long long*>(group_offsets), latent, scale,
                    static_cast<char*>(workspace), workspace_bytes,
                    static_cast<cudaStream_t>(stream));
}

extern "C" int ae_decode(aeqc_model* m, const void* latent, const double* scale, int64_t n,
                         const int64_t* group_offsets, float* xhat, int64_t ld,
                         void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m, "ae_decode: null model");
  AEQC_CHECK_ARG(n >= 0, "ae_decode: negative n");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(latent && scale && xhat, "ae_decode: null array");
  AEQC_CHECK_ARG(ld >= m->d.P && ld % 4 == 0, "ae_decode: ld must be >= P and a multiple of 4");
  AEQC_CHECK_ARG(group_offsets || m->d.n_groups == 1,
                 "ae_decode: group_offsets required for a model with %d groups",
                 m->d.n_groups);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= decode_ws(m, n),
                 "ae_decode: workspace of %zu bytes needed", decode_ws(m, n));
  AEQC_CHECK_ARG(aligned(workspace, kWsAlign), "ae_decode: workspace not 256-byte aligned");
  return run_decode(m, latent, scale, n, reinterpret_cast<const long long*>(group_offsets), xhat,
                    ld, static_cast<char*>(workspace), workspace_bytes,
                    static_cast<cudaStream_t>(stream));
}

// ---- fused batch calls -----------------------------------------------------

static size_t xhat_bytes(const aeqc_model* m, long long n) {
  (void)m;
  return ws_round(sizeof(float) * (size_t)n * AEQC_XHAT_LD);
}

extern "C" size_t compress_batch_workspace_size(const aeqc_model* m, int64_t n) {
  if (!m || n <= 0) return 0;
  size_t a = encode_ws(m, n), b = decode_ws(m, n);
  size_t c = qc_ws(n);  // the fallback list reuses the hidden-layer buffer
  size_t r = a > b ? a : b;
  return xhat_bytes(m, n) + (r > c ? r : c);
}

extern "C" size_t quantize_correct_workspace_size(int64_t n) { return qc_ws(n); }

extern "C" size_t decompress_batch_workspace_size(const aeqc_model* m, int64_t n) {
  if (!m || n <= 0) return 0;
  return xhat_bytes(m, n) + decode_ws(m, n);
}

extern "C" int compress_batch(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid,
                              const double* x, int64_t n, const int64_t* group_offsets,
                              const aeqc_params* params, aeqc_compressed* out,
                              void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  GridK gk;
  ParamsK pk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  if ((rc = make_params(params, &pk))) return rc;
  AEQC_CHECK_ARG(m && out, "compress_batch: null argument");
  AEQC_CHECK_ARG(m->d.P == gk.P, "compress_batch: model P=%d but grid has %d cells", m->d.P,
                 gk.P);
  AEQC_CHECK_ARG(n >= 0, "compress_batch: negative n");
  AEQC_CHECK_ARG(group_offsets || m->d.n_groups == 1,
                 "compress_batch: group_offsets required for a model with %d groups",
                 m->d.n_groups);
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(x && out->latent && out->scale && out->codes && out->lambda && out->iters &&
                     out->status,
                 "compress_batch: null array");
  AEQC_CHECK_ARG(out->outliers.count &&
                     (out->outliers.capacity == 0 || (out->outliers.index && out->outliers.value)),
                 "compress_batch: outlier list needs a count (and arrays when capacity > 0)");
  size_t need = compress_batch_workspace_size(m, n);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need,
                 "compress_batch: workspace of %zu bytes needed", need);
  AEQC_CHECK_ARG(aligned(workspace, kWsAlign), "compress_batch: workspace not aligned");
  if (mlp) AEQC_CHECK_ARG(mlp->nin == m->d.L + 4, "compress_batch: MLP expects %d inputs, "
                          "latent + 4 = %d", mlp->nin, m->d.L + 4);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* xhat = reinterpret_cast<float*>(ws);
  char* rest = ws + xhat_bytes(m, n);
  size_t rest_bytes = workspace_bytes - xhat_bytes(m, n);
  const long long* goff = reinterpret_cast<const long long*>(group_offsets);
  if ((rc = run_encode(m, x, n, goff, out->latent, out->scale, rest, rest_bytes, s))) return rc;
  if ((rc = run_decode(m, out->latent, out->scale, n, goff, xhat, AEQC_XHAT_LD, rest,
                       rest_bytes, s)))
    return rc;
  return run_quantize_correct(gk, pk, params->kernel, x, xhat, AEQC_XHAT_LD, n, mlp,
                              m->d.dtype, m->d.L, out, nullptr, rest, rest_bytes, s, 0, true,
                              m->tuning.qc_warps_per_sm);
}

// ---- launch tuning --------------------------------------------------------------

extern "C" int aeqc_model_set_tuning(aeqc_model* m, const aeqc_tuning* t) {
  clear_error();
  AEQC_CHECK_ARG(m && t, "aeqc_model_set_tuning: null argument");
  AEQC_CHECK_ARG(t->enc_stages == 0 || (t->enc_stages >= 2 && t->enc_stages <= 6),
                 "aeqc_model_set_tuning: enc_stages must be 0 or in [2, 6]");
  AEQC_CHECK_ARG(t->dec_stages == 0 || (t->dec_stages >= 2 && t->dec_stages <= 16),
                 "aeqc_model_set_tuning: dec_stages must be 0 or in [2, 16]");
  AEQC_CHECK_ARG(t->qc_warps_per_sm >= 0 && t->qc_warps_per_sm <= 16 && t->qc_warps_per_sm % 4 == 0,
                 "aeqc_model_set_tuning: qc_warps_per_sm must be 0, 4, 8, 12 or 16");
  m->tuning = *t;
  m->tuning.reserved = 0;
  return AEQC_OK;
}

extern "C" int aeqc_model_get_tuning(const aeqc_model* m, aeqc_tuning* t) {
  clear_error();
  AEQC_CHECK_ARG(m && t, "aeqc_model_get_tuning: null argument");
  *t = m->tuning;
  return AEQC_OK;
}

extern "C" int aeqc_model_device_status(aeqc_model* m, int32_t* status, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m && status, "aeqc_model_device_status: null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  AEQC_CUDA_TRY(cudaMemcpyAsync(&v, m->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AEQC_CUDA_TRY(cudaMemsetAsync(m->dev_err, 0, sizeof(int), s));
  AEQC_CUDA_TRY(cudaStreamSynchronize(s));
  *status = v;
  return AEQC_OK;
}

namespace aeqc {

// mean time of `reps` calls of f after one untimed call, CUDA events on s
template <typename F>
static int time_calls(cudaStream_t s, int reps, F f, float* ms) {
  int rc = f();
  if (rc) return rc;
  cudaEvent_t e0, e1;
  AEQC_CUDA_TRY(cudaEventCreate(&e0));
  AEQC_CUDA_TRY(cudaEventCreate(&e1));
  AEQC_CUDA_TRY(cudaEventRecord(e0, s));
  for (int r = 0; r < reps && !rc; ++r) rc = f();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return set_error(AEQC_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
  *ms = t / reps;
  return AEQC_OK;
}

}  // namespace aeqc

extern "C" int aeqc_autotune(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid,
                             const double* x, int64_t n, const int64_t* group_offsets,
                             const aeqc_params* params, aeqc_compressed* out, void* workspace,
                             size_t workspace_bytes, void* stream, aeqc_tuning* best) {
  // one ordinary call validates the arguments and leaves the decoded rows in
  // the workspace
  int rc = compress_batch(m, mlp, grid, x, n, group_offsets, params, out, workspace,
                          workspace_bytes, stream);
  if (rc) return rc;
  AEQC_CHECK_ARG(best, "aeqc_autotune: null best");
  if (n == 0) {
    *best = m->tuning;
    return AEQC_OK;
  }
  GridK gk;
  ParamsK pk;
  make_grid(grid, &gk);
  make_params(params, &pk);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* xhat = reinterpret_cast<float*>(ws);
  char* rest = ws + xhat_bytes(m, n);
  const size_t rest_bytes = workspace_bytes - xhat_bytes(m, n);
  const long long* goff = reinterpret_cast<const long long*>(group_offsets);
  aeqc_tuning t = m->tuning;
  const int reps = 2;
  if (m->d.dtype == AEQC_DTYPE_BF16) {
    float bt = 1e30f;
    int bv = t.enc_stages;
    for (int v = 2; v <= 6; ++v) {
      m->tuning.enc_stages = v;
      float ms = 0.f;
      if ((rc = time_calls(s, reps, [&]() {
             return run_encode(m, x, n, goff, out->latent, out->scale, rest, rest_bytes, s);
           }, &ms)))
        break;
      if (ms < bt) bt = ms, bv = v;
    }
    m->tuning.enc_stages = bv;
    t.enc_stages = bv;
    bt = 1e30f;
    bv = t.dec_stages;
    for (int v = 4; v <= 16 && !rc; v += 4) {
      m->tuning.dec_stages = v;
      float ms = 0.f;
      if ((rc = time_calls(s, reps, [&]() {
             return run_decode(m, out->latent, out->scale, n, goff, xhat, AEQC_XHAT_LD, rest,
                               rest_bytes, s);
           }, &ms)))
        break;
      if (ms < bt) bt = ms, bv = v;
    }
    m->tuning.dec_stages = bv;
    t.dec_stages = bv;
  }
  if (!rc && params->kernel == AEQC_KERNEL_FAST) {
    float bt = 1e30f;
    int bv = t.qc_warps_per_sm;
    for (int v = 4; v <= 16; v += 4) {
      float ms = 0.f;
      if ((rc = time_calls(s, reps, [&]() {
             return run_quantize_correct(gk, pk, params->kernel, x, xhat, AEQC_XHAT_LD, n, mlp,
                                         m->d.dtype, m->d.L, out, nullptr, rest, rest_bytes, s,
                                         0, true, v);
           }, &ms)))
        break;
      if (ms < bt) bt = ms, bv = v;
    }
    t.qc_warps_per_sm = bv;
  }
  m->tuning = t;
  if (rc) return rc;
  *best = t;
  // the outputs as compress_batch writes them with the chosen tuning
  return compress_batch(m, mlp, grid, x, n, group_offsets, params, out, workspace,
                        workspace_bytes, stream);
}

extern "C" int quantize_correct(const aeqc_grid* grid, const double* x, const float* xhat,
                                int64_t ld, int64_t n, const aeqc_params* params,
                                aeqc_mlp* mlp, int32_t latent_dtype, int32_t latent_dim,
                                aeqc_compressed* out, double* f_out, void* workspace,
                                size_t workspace_bytes, void* stream) {
  clear_error();
  GridK gk;
  ParamsK pk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  if ((rc = make_params(params, &pk))) return rc;
  AEQC_CHECK_ARG(out, "quantize_correct: null out");
  AEQC_CHECK_ARG(workspace && workspace_bytes >= qc_ws(n) && aligned(workspace, kWsAlign),
                 "quantize_correct: 256-byte aligned workspace of %zu bytes needed", qc_ws(n));
  AEQC_CHECK_ARG(n >= 0, "quantize_correct: negative n");
  AEQC_CHECK_ARG(ld >= gk.P, "quantize_correct: ld < P");
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(x && xhat && out->scale && out->codes && out->lambda && out->iters &&
                     out->status,
                 "quantize_correct: null array");
  AEQC_CHECK_ARG(out->outliers.count &&
                     (out->outliers.capacity == 0 || (out->outliers.index && out->outliers.value)),
                 "quantize_correct: outlier list needs a count (and arrays when capacity > 0)");
  AEQC_CHECK_ARG(latent_dtype == AEQC_DTYPE_F32 || latent_dtype == AEQC_DTYPE_BF16,
                 "quantize_correct: bad latent dtype");
  if (mlp || out->features) {
    AEQC_CHECK_ARG(out->latent && latent_dim > 0, "quantize_correct: latent input required");
  }
  if (mlp)
    AEQC_CHECK_ARG(mlp->nin == latent_dim + 4, "quantize_correct: MLP expects %d inputs",
                   mlp->nin);
  return run_quantize_correct(gk, pk, params->kernel, x, xhat, ld, n, mlp, latent_dtype,
                              latent_dim, out, f_out, static_cast<char*>(workspace),
                              workspace_bytes, static_cast<cudaStream_t>(stream));
}

// ---- compress_batch from host memory, streamed ---------------------------------

namespace aeqc {

// copy streams, created once per device and kept for the process lifetime
struct CopyStreams {
  cudaStream_t h2d = nullptr, d2h = nullptr;
};
static std::mutex g_cs_mu;
static CopyStreams g_cs[64];

static int copy_streams(CopyStreams* out) {
  int dev = 0;
  AEQC_CUDA_TRY(cudaGetDevice(&dev));
  AEQC_CHECK_ARG(dev >= 0 && dev < 64, "compress_batch_host: device ordinal %d >= 64", dev);
  std::lock_guard<std::mutex> lock(g_cs_mu);
  if (!g_cs[dev].h2d) {
    AEQC_CUDA_TRY(cudaStreamCreateWithFlags(&g_cs[dev].h2d, cudaStreamNonBlocking));
    AEQC_CUDA_TRY(cudaStreamCreateWithFlags(&g_cs[dev].d2h, cudaStreamNonBlocking));
  }
  *out = g_cs[dev];
  return AEQC_OK;
}

// one device buffer of the pipeline
struct HostChunkBuf {
  double* x;
  void* latent;
  double* scale;
  int16_t* codes;
  double* lambda;
  uint8_t* iters;
  uint16_t* status;
  char* ws;
  size_t ws_bytes;
};

static size_t host_buf_bytes(const aeqc_model* m, long long chunk) {
  const size_t esz = m->d.dtype == AEQC_DTYPE_BF16 ? 2 : 4;
  WsSize w;
  w.add<double>((size_t)chunk * m->d.P);
  w.add<char>((size_t)chunk * m->d.L * esz);
  w.add<double>((size_t)chunk);
  w.add<int16_t>((size_t)chunk * m->d.P);
  w.add<double>((size_t)chunk * 4);
  w.add<uint8_t>((size_t)chunk);
  w.add<uint16_t>((size_t)chunk);
  w.add<char>(compress_batch_workspace_size(m, chunk));
  return w.bytes;
}

static bool carve_buf(WsCarver& c, const aeqc_model* m, long long chunk, HostChunkBuf& b) {
  const size_t esz = m->d.dtype == AEQC_DTYPE_BF16 ? 2 : 4;
  b.x = c.take<double>((size_t)chunk * m->d.P);
  b.latent = c.take<char>((size_t)chunk * m->d.L * esz);
  b.scale = c.take<double>((size_t)chunk);
  b.codes = c.take<int16_t>((size_t)chunk * m->d.P);
  b.lambda = c.take<double>((size_t)chunk * 4);
  b.iters = c.take<uint8_t>((size_t)chunk);
  b.status = c.take<uint16_t>((size_t)chunk);
  b.ws_bytes = compress_batch_workspace_size(m, chunk);
  b.ws = c.take<char>(b.ws_bytes);
  return c.ok();
}

}  // namespace aeqc

extern "C" size_t compress_batch_host_workspace_size(const aeqc_model* m, int64_t chunk,
                                                     int64_t outlier_capacity) {
  if (!m || chunk <= 0) return 0;
  WsSize w;
  w.add<long long>(1);                                       // outlier count
  w.add<long long>((size_t)(outlier_capacity > 0 ? outlier_capacity : 1));  // indices
  w.add<double>((size_t)(outlier_capacity > 0 ? outlier_capacity : 1));     // values
  return w.bytes + 2 * host_buf_bytes(m, chunk) + kWsAlign;
}

// The chunked pipeline of compress_batch_host on the caller's stream s and the
// library's copy streams, with the caller-owned events ev (h2d done, compute
// done, d2h done, per buffer).  Returns at the first error; the caller joins
// the copy streams then.
static int host_pipeline(aeqc_model* m, aeqc_mlp* mlp, const GridK& gk, const ParamsK& pk,
                         const aeqc_params* params, const double* x_host, long long n,
                         const aeqc_compressed& o, long long chunk, void* workspace,
                         size_t workspace_bytes, cudaStream_t s, const CopyStreams& cs,
                         cudaEvent_t (&ev)[2][3]) {
  int rc = AEQC_OK;
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  long long* d_count = c.take<long long>(1);
  const long long cap = o.outliers.capacity;
  long long* d_index = c.take<long long>((size_t)(cap > 0 ? cap : 1));
  double* d_value = c.take<double>((size_t)(cap > 0 ? cap : 1));
  HostChunkBuf buf[2];
  if (!carve_buf(c, m, chunk, buf[0]) || !carve_buf(c, m, chunk, buf[1]))
    return set_error(AEQC_EINVAL, "compress_batch_host: workspace too small");
  const size_t esz = m->d.dtype == AEQC_DTYPE_BF16 ? 2 : 4;
  const int P = m->d.P, L = m->d.L;
  // the copy streams start after the work already on the caller's stream
  cudaEvent_t start;
  AEQC_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  AEQC_CUDA_TRY(cudaEventRecord(start, s));
  AEQC_CUDA_TRY(cudaStreamWaitEvent(cs.h2d, start, 0));
  AEQC_CUDA_TRY(cudaStreamWaitEvent(cs.d2h, start, 0));
  cudaEventDestroy(start);
  AEQC_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(long long), s));
  const long long nchunks = (n + chunk - 1) / chunk;
  rc = AEQC_OK;
  for (long long ci = 0; ci < nchunks && rc == AEQC_OK; ++ci) {
    const int b = (int)(ci & 1);
    HostChunkBuf& B = buf[b];
    const long long c0 = ci * chunk, rows = (c0 + chunk <= n) ? chunk : n - c0;
    // input: after the compute of chunk ci - 2 has read this buffer
    if (ci >= 2) AEQC_CUDA_TRY(cudaStreamWaitEvent(cs.h2d, ev[b][1], 0));
    AEQC_CUDA_TRY(cudaMemcpyAsync(B.x, x_host + c0 * P, sizeof(double) * rows * P,
                                  cudaMemcpyHostToDevice, cs.h2d));
    AEQC_CUDA_TRY(cudaEventRecord(ev[b][0], cs.h2d));
    // compute: after the input and after the copy-out of chunk ci - 2
    AEQC_CUDA_TRY(cudaStreamWaitEvent(s, ev[b][0], 0));
    if (ci >= 2) AEQC_CUDA_TRY(cudaStreamWaitEvent(s, ev[b][2], 0));
    aeqc_compressed dc;
    memset(&dc, 0, sizeof(dc));
    dc.latent = B.latent;
    dc.scale = B.scale;
    dc.codes = B.codes;
    dc.lambda = B.lambda;
    dc.iters = B.iters;
    dc.status = B.status;
    dc.outliers.capacity = cap;
    dc.outliers.count = reinterpret_cast<int64_t*>(d_count);
    dc.outliers.index = reinterpret_cast<int64_t*>(d_index);
    dc.outliers.value = d_value;
    float* xhat = reinterpret_cast<float*>(B.ws);
    char* rest = B.ws + ws_round(sizeof(float) * (size_t)rows * AEQC_XHAT_LD);
    const size_t rest_bytes = B.ws_bytes - ws_round(sizeof(float) * (size_t)rows * AEQC_XHAT_LD);
    if ((rc = run_encode(m, B.x, rows, nullptr, dc.latent, dc.scale, rest, rest_bytes, s))) break;
    if ((rc = run_decode(m, dc.latent, dc.scale, rows, nullptr, xhat, AEQC_XHAT_LD, rest,
                         rest_bytes, s)))
      break;
    if ((rc = run_quantize_correct(gk, pk, params->kernel, B.x, xhat, AEQC_XHAT_LD, rows, mlp,
                                   m->d.dtype, L, &dc, nullptr, rest, rest_bytes, s, c0,
                                   false, m->tuning.qc_warps_per_sm)))
      break;
    AEQC_CUDA_TRY(cudaEventRecord(ev[b][1], s));
    // outputs
    AEQC_CUDA_TRY(cudaStreamWaitEvent(cs.d2h, ev[b][1], 0));
    char* lat_h = static_cast<char*>(o.latent) + (size_t)c0 * L * esz;
    AEQC_CUDA_TRY(cudaMemcpyAsync(lat_h, B.latent, (size_t)rows * L * esz,
                                  cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaMemcpyAsync(o.scale + c0, B.scale, sizeof(double) * rows,
                                  cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaMemcpyAsync(o.codes + c0 * P, B.codes, sizeof(int16_t) * rows * P,
                                  cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaMemcpyAsync(o.lambda + c0 * 4, B.lambda, sizeof(double) * rows * 4,
                                  cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaMemcpyAsync(o.iters + c0, B.iters, rows, cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaMemcpyAsync(o.status + c0, B.status, sizeof(uint16_t) * rows,
                                  cudaMemcpyDeviceToHost, cs.d2h));
    AEQC_CUDA_TRY(cudaEventRecord(ev[b][2], cs.d2h));
  }
  if (rc == AEQC_OK) {
    // the outlier list after the last compute, then the caller's stream waits
    // for every copy
    cudaError_t e = cudaStreamWaitEvent(cs.d2h, ev[(nchunks - 1) & 1][1], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(o.outliers.count, d_count, sizeof(long long), cudaMemcpyDeviceToHost,
                          cs.d2h);
    if (e == cudaSuccess && cap > 0)
      e = cudaMemcpyAsync(o.outliers.index, d_index, sizeof(long long) * cap,
                          cudaMemcpyDeviceToHost, cs.d2h);
    if (e == cudaSuccess && cap > 0)
      e = cudaMemcpyAsync(o.outliers.value, d_value, sizeof(double) * cap,
                          cudaMemcpyDeviceToHost, cs.d2h);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0][2], cs.d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[0][2], 0);
    if (e != cudaSuccess)
      rc = set_error(AEQC_ECUDA, "compress_batch_host: %s", cudaGetErrorString(e));
  }
  return rc;
}

extern "C" int compress_batch_host(aeqc_model* m, aeqc_mlp* mlp, const aeqc_grid* grid,
                                   const double* x_host, int64_t n, const aeqc_params* params,
                                   aeqc_compressed* out_host, int64_t chunk, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  clear_error();
  GridK gk;
  ParamsK pk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  if ((rc = make_params(params, &pk))) return rc;
  AEQC_CHECK_ARG(m && out_host, "compress_batch_host: null argument");
  if (m->d.n_groups != 1)
    return set_error(AEQC_EUNSUPPORTED, "compress_batch_host: single-group models only");
  AEQC_CHECK_ARG(m->d.P == gk.P, "compress_batch_host: model P=%d but grid has %d cells",
                 m->d.P, gk.P);
  AEQC_CHECK_ARG(n >= 0 && chunk > 0, "compress_batch_host: need n >= 0 and chunk > 0");
  if (n == 0) return AEQC_OK;
  const aeqc_compressed& o = *out_host;
  AEQC_CHECK_ARG(x_host && o.latent && o.scale && o.codes && o.lambda && o.iters && o.status &&
                     o.outliers.count && !o.features,
                 "compress_batch_host: null output array (or features set)");
  AEQC_CHECK_ARG(o.outliers.capacity == 0 || (o.outliers.index && o.outliers.value),
                 "compress_batch_host: outlier arrays missing");
  if (mlp) AEQC_CHECK_ARG(mlp->nin == m->d.L + 4, "compress_batch_host: MLP expects %d inputs",
                          mlp->nin);
  if (chunk > n) chunk = n;
  const size_t need = compress_batch_host_workspace_size(m, chunk, o.outliers.capacity);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need && aligned(workspace, kWsAlign),
                 "compress_batch_host: 256-byte aligned workspace of %zu bytes needed", need);
  CopyStreams cs;
  if ((rc = copy_streams(&cs))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[2][3] = {};
  for (int b = 0; b < 2 && rc == AEQC_OK; ++b)
    for (int k = 0; k < 3 && rc == AEQC_OK; ++k) {
      const cudaError_t e = cudaEventCreateWithFlags(&ev[b][k], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        ev[b][k] = nullptr;
        rc = set_error(AEQC_ECUDA, "compress_batch_host: event: %s", cudaGetErrorString(e));
      }
    }
  if (rc == AEQC_OK)
    rc = host_pipeline(m, mlp, gk, pk, params, x_host, n, o, chunk, workspace, workspace_bytes,
                       s, cs, ev);
  if (rc != AEQC_OK) {
    // no copy into or out of the caller's host buffers may still be in
    // flight when the error returns
    cudaStreamSynchronize(cs.h2d);
    cudaStreamSynchronize(cs.d2h);
  }
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 3; ++k)
      if (ev[b][k]) cudaEventDestroy(ev[b][k]);
  return rc;
}

extern "C" int decompress_batch(aeqc_model* m, const aeqc_grid* grid,
                                const aeqc_compressed* in, int64_t n,
                                const int64_t* group_offsets, const aeqc_params* params,
                                double* f, void* workspace, size_t workspace_bytes,
                                void* stream) {
  clear_error();
  GridK gk;
  ParamsK pk;
  int rc = make_grid(grid, &gk);
  if (rc) return rc;
  if ((rc = make_params(params, &pk))) return rc;
  AEQC_CHECK_ARG(m && in, "decompress_batch: null argument");
  AEQC_CHECK_ARG(m->d.P == gk.P, "decompress_batch: model P=%d but grid has %d cells", m->d.P,
                 gk.P);
  AEQC_CHECK_ARG(n >= 0, "decompress_batch: negative n");
  AEQC_CHECK_ARG(group_offsets || m->d.n_groups == 1,
                 "decompress_batch: group_offsets required for a model with %d groups",
                 m->d.n_groups);
  if (n == 0) return AEQC_OK;
  AEQC_CHECK_ARG(in->latent && in->scale && in->codes && in->lambda && in->status && f,
                 "decompress_batch: null array");
  size_t need = decompress_batch_workspace_size(m, n);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need,
                 "decompress_batch: workspace of %zu bytes needed", need);
  AEQC_CHECK_ARG(aligned(workspace, kWsAlign), "decompress_batch: workspace not aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* xhat = reinterpret_cast<float*>(ws);
  char* rest = ws + xhat_bytes(m, n);
  size_t rest_bytes = workspace_bytes - xhat_bytes(m, n);
  const long long* goff = reinterpret_cast<const long long*>(group_offsets);
  if ((rc = run_decode(m, in->latent, in->scale, n, goff, xhat, AEQC_XHAT_LD, rest, rest_bytes,
                       s)))
    return rc;
  OutliersK ok = make_outliers(&in->outliers);
  return launch_apply(gk, xhat, AEQC_XHAT_LD, in->codes, in->outliers.count ? &ok : nullptr,
                      in->scale, in->lambda, in->status, n, 0, pk, f, s);
}

// ---- quantize_correct without a caller workspace -----------------------------
// The scratch of quantize_correct (deferred-histogram list + its count, laid
// out exactly as qc_ws(AEQC_QC_NOALLOC_MAX_N) carves it) in one file-scope
// device array; every call shares it.

namespace aeqc {

constexpr size_t kNoAllocScratchBytes =
    (sizeof(int) * (size_t)AEQC_QC_NOALLOC_MAX_N + kWsAlign - 1) / kWsAlign * kWsAlign +
    kWsAlign;

static __device__ __align__(256) char g_qc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_qc_scratch_mu;
static char* g_qc_scratch_ptr[kNoAllocMaxDevices] = {};

// Address of the array on the current device, looked up once per device.
static int qc_scratch_current_device(char** out) {
  int dev = 0;
  AEQC_CUDA_TRY(cudaGetDevice(&dev));
  AEQC_CHECK_ARG(dev >= 0 && dev < kNoAllocMaxDevices,
                 "quantize_correct_noalloc: device ordinal %d >= %d", dev, kNoAllocMaxDevices);
  std::lock_guard<std::mutex> lock(g_qc_scratch_mu);
  if (!g_qc_scratch_ptr[dev]) {
    void* p = nullptr;
    AEQC_CUDA_TRY(cudaGetSymbolAddress(&p, g_qc_scratch));
    g_qc_scratch_ptr[dev] = static_cast<char*>(p);
  }
  *out = g_qc_scratch_ptr[dev];
  return AEQC_OK;
}

}  // namespace aeqc

extern "C" int quantize_correct_noalloc(const aeqc_grid* grid, const double* x,
                                        const float* xhat, int64_t ld, int64_t n,
                                        const aeqc_params* params, aeqc_mlp* mlp,
                                        int32_t latent_dtype, int32_t latent_dim,
                                        aeqc_compressed* out, double* f_out, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(n <= AEQC_QC_NOALLOC_MAX_N,
                 "quantize_correct_noalloc: n=%lld exceeds the static scratch limit of %d "
                 "histograms; split the batch or use quantize_correct",
                 (long long)n, AEQC_QC_NOALLOC_MAX_N);
  char* scratch = nullptr;
  int rc = qc_scratch_current_device(&scratch);
  if (rc) return rc;
  return quantize_correct(grid, x, xhat, ld, n, params, mlp, latent_dtype, latent_dim, out,
                          f_out, scratch, kNoAllocScratchBytes, stream);
}
