// Learned warm start for the Newton correction: a 3-layer MLP
// (latent + 4 moment defects -> nh -> nh -> 4 multipliers, ReLU) trained on
// (input, Newton solution) pairs by the library's own forward/backward
// kernels and Adam.  The paper has no learned warm start; plain Newton from
// zero stays the fallback and the judge of its error (Stage 5, Eq. (6)).
#include <string.h>

#include <vector>

#include "model.cuh"
#include "qc_common.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

__global__ void mlp_normalize_kernel(const float* in, long long B, int nin, const float* mu,
                                     const float* sd, float* u) {
  long long cnt = B * nin;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    int k = (int)(t % nin);
    u[t] = (in[t] - mu[k]) / sd[k];
  }
}

// dout = 2 (o - t) / (B 4) with t = (lambda - out_mu) / out_sd; rowloss[b]
__global__ void mlp_loss_kernel(const float* o, const double* lam, long long B,
                                const float* omu, const float* osd, float* dout,
                                float* rowloss) {
  long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = 0.f;
  const float sc = 2.f / ((float)B * 4.f);
  for (int k = 0; k < 4; ++k) {
    float t = (float)((lam[b * 4 + k] - (double)omu[k]) / (double)osd[k]);
    float d = o[b * 4 + k] - t;
    s = fmaf(d, d, s);
    dout[b * 4 + k] = sc * d;
  }
  rowloss[b] = s;
}

__global__ void mlp_loss_finish_kernel(const float* rowloss, long long B, float* out) {
  if (threadIdx.x || blockIdx.x) return;
  double t = 0.0;
  for (long long b = 0; b < B; ++b) t += rowloss[b];
  *out = (float)(t / ((double)B * 4.0));
}

__global__ void mlp_predict_kernel(const MlpK m, const float* in, long long n, double* lam) {
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n) return;
  double l0[4];
  const float* row = in + b * m.nin;
  dev::mlp_eval_warp(m, [&](int k) { return __ldg(row + k); }, l0, lane);
  if (lane < 4) lam[b * 4 + lane] = l0[lane];
}

}  // namespace
}  // namespace aeqc

using namespace aeqc;

extern "C" int aeqc_mlp_create(int32_t n_in, int32_t n_hidden, aeqc_mlp** out) {
  clear_error();
  AEQC_CHECK_ARG(out, "aeqc_mlp_create: null out");
  AEQC_CHECK_ARG(n_in >= 5 && n_in <= 1024, "aeqc_mlp_create: n_in=%d out of range", n_in);
  AEQC_CHECK_ARG(n_hidden >= 1 && n_hidden <= 64, "aeqc_mlp_create: n_hidden must be <= 64");
  aeqc_mlp* m = new aeqc_mlp();
  memset(m, 0, sizeof(*m));
  m->nin = n_in;
  m->nh = n_hidden;
  const long long ni = n_in, nh = n_hidden;
  long long o = 0;
  m->oW1 = o; o += ni * nh;
  m->ob1 = o; o += nh;
  m->oW2 = o; o += nh * nh;
  m->ob2 = o; o += nh;
  m->oW3 = o; o += nh * 4;
  m->ob3 = o; o += 4;
  m->n_train = o;
  m->oimu = o; o += ni;
  m->oisd = o; o += ni;
  m->oomu = o; o += 4;
  m->oosd = o; o += 4;
  m->n_all = o;
  size_t bytes = sizeof(float) * (size_t)(m->n_all + 2 * m->n_train);
  char* base = nullptr;
  if (cudaMalloc(&base, bytes) != cudaSuccess) {
    delete m;
    return set_error(AEQC_ENOMEM, "aeqc_mlp_create: cudaMalloc failed");
  }
  cudaMemset(base, 0, bytes);
  m->params = reinterpret_cast<float*>(base);
  m->adam_m = m->params + m->n_all;
  m->adam_v = m->adam_m + m->n_train;
  std::vector<float> ones(ni, 1.f);
  cudaMemcpy(m->params + m->oisd, ones.data(), ni * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(m->params + m->oosd, ones.data(), 4 * sizeof(float), cudaMemcpyHostToDevice);
  *out = m;
  return AEQC_OK;
}

extern "C" int aeqc_mlp_destroy(aeqc_mlp* m) {
  clear_error();
  if (!m) return AEQC_OK;
  cudaFree(m->params);
  delete m;
  return AEQC_OK;
}

static int mlp_copy_in(float* dst, const double* src, long long cnt) {
  if (!src) return AEQC_OK;
  std::vector<float> t(cnt);
  for (long long i = 0; i < cnt; ++i) t[i] = (float)src[i];
  AEQC_CUDA_TRY(cudaMemcpy(dst, t.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
  return AEQC_OK;
}

extern "C" int aeqc_mlp_set(aeqc_mlp* m, const double* W1, const double* b1, const double* W2,
                            const double* b2, const double* W3, const double* b3,
                            const double* in_mu, const double* in_sd, const double* out_mu,
                            const double* out_sd) {
  clear_error();
  AEQC_CHECK_ARG(m && W1 && b1 && W2 && b2 && W3 && b3 && in_mu && in_sd && out_mu && out_sd,
                 "aeqc_mlp_set: null argument");
  const long long ni = m->nin, nh = m->nh;
  for (long long k = 0; k < ni; ++k)
    AEQC_CHECK_ARG(in_sd[k] > 0.0, "aeqc_mlp_set: in_sd must be positive");
  for (int k = 0; k < 4; ++k)
    AEQC_CHECK_ARG(out_sd[k] > 0.0, "aeqc_mlp_set: out_sd must be positive");
  int rc;
  if ((rc = mlp_copy_in(m->params + m->oW1, W1, ni * nh))) return rc;
  if ((rc = mlp_copy_in(m->params + m->ob1, b1, nh))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oW2, W2, nh * nh))) return rc;
  if ((rc = mlp_copy_in(m->params + m->ob2, b2, nh))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oW3, W3, nh * 4))) return rc;
  if ((rc = mlp_copy_in(m->params + m->ob3, b3, 4))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oimu, in_mu, ni))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oisd, in_sd, ni))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oomu, out_mu, 4))) return rc;
  if ((rc = mlp_copy_in(m->params + m->oosd, out_sd, 4))) return rc;
  AEQC_CUDA_TRY(cudaMemset(m->adam_m, 0, 2 * m->n_train * sizeof(float)));
  m->step = 0;
  return AEQC_OK;
}

extern "C" int aeqc_mlp_get(aeqc_mlp* m, double* W1, double* b1, double* W2, double* b2,
                            double* W3, double* b3) {
  clear_error();
  AEQC_CHECK_ARG(m, "aeqc_mlp_get: null mlp");
  AEQC_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<float> t(m->n_train);
  AEQC_CUDA_TRY(cudaMemcpy(t.data(), m->params, m->n_train * sizeof(float),
                           cudaMemcpyDeviceToHost));
  const long long ni = m->nin, nh = m->nh;
  auto out = [&](double* d, long long off, long long cnt) {
    if (d)
      for (long long i = 0; i < cnt; ++i) d[i] = t[off + i];
  };
  out(W1, m->oW1, ni * nh);
  out(b1, m->ob1, nh);
  out(W2, m->oW2, nh * nh);
  out(b2, m->ob2, nh);
  out(W3, m->oW3, nh * 4);
  out(b3, m->ob3, 4);
  return AEQC_OK;
}

extern "C" size_t mlp_train_workspace_size(const aeqc_mlp* m, int64_t B) {
  if (!m || B <= 0) return 0;
  WsSize w;
  w.add<float>((size_t)B * m->nin);  // u
  w.add<float>((size_t)B * m->nh);   // h1
  w.add<float>((size_t)B * m->nh);   // h2
  w.add<float>((size_t)B * 4);       // o
  w.add<float>((size_t)B * 4);       // dout
  w.add<float>((size_t)B * m->nh);   // dh2
  w.add<float>((size_t)B * m->nh);   // dh1
  w.add<float>((size_t)B);           // row losses
  w.add<float>(m->n_train);          // gradient
  w.add<float>(1);
  return w.bytes;
}

static int mlp_loss_grad_impl(aeqc_mlp* m, const float* in, const double* lam, int64_t B,
                              float* loss_out, float* grad_ext, void* workspace,
                              size_t workspace_bytes, void* stream, float** grad_used) {
  AEQC_CHECK_ARG(m && in && lam, "mlp_train_step: null argument");
  AEQC_CHECK_ARG(B > 0, "mlp_train_step: B must be positive");
  size_t need = mlp_train_workspace_size(m, B);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need,
                 "mlp_train_step: workspace of %zu bytes needed", need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ni = m->nin, nh = m->nh;
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  float* u = c.take<float>((size_t)B * ni);
  float* h1 = c.take<float>((size_t)B * nh);
  float* h2 = c.take<float>((size_t)B * nh);
  float* o = c.take<float>((size_t)B * 4);
  float* dout = c.take<float>((size_t)B * 4);
  float* dh2 = c.take<float>((size_t)B * nh);
  float* dh1 = c.take<float>((size_t)B * nh);
  float* rowloss = c.take<float>(B);
  float* grad = c.take<float>(m->n_train);
  float* lscratch = c.take<float>(1);
  if (grad_ext) grad = grad_ext;
  *grad_used = grad;
  float* P = m->params;
  int rc;
#define TRY(e) \
  do {                    \
    if ((rc = (e))) return rc; \
  } while (0)
  mlp_normalize_kernel<<<256, 256, 0, s>>>(in, B, ni, P + m->oimu, P + m->oisd, u);
  TRY(check_launch("mlp_normalize_kernel"));
  TRY(gemm_bias(B, nh, ni, u, ni, P + m->oW1, nh, 1, P + m->ob1, AEQC_ACT_RELU, h1, s));
  TRY(gemm_bias(B, nh, nh, h1, nh, P + m->oW2, nh, 1, P + m->ob2, AEQC_ACT_RELU, h2, s));
  TRY(gemm_bias(B, 4, nh, h2, nh, P + m->oW3, 4, 1, P + m->ob3, AEQC_ACT_IDENTITY, o, s));
  mlp_loss_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(o, lam, B, P + m->oomu,
                                                              P + m->oosd, dout, rowloss);
  TRY(check_launch("mlp_loss_kernel"));
  mlp_loss_finish_kernel<<<1, 1, 0, s>>>(rowloss, B, loss_out ? loss_out : lscratch);
  TRY(check_launch("mlp_loss_finish_kernel"));
  float *gW1 = grad + m->oW1, *gb1 = grad + m->ob1, *gW2 = grad + m->oW2, *gb2 = grad + m->ob2;
  float *gW3 = grad + m->oW3, *gb3 = grad + m->ob3;
  TRY(launch_colsum(dout, B, 4, gb3, s));
  TRY(gemm_plain(nh, 4, (int)B, h2, 1, nh, dout, 4, 1, gW3, 4, 0.f, s));
  TRY(gemm_plain(B, nh, 4, dout, 4, 1, P + m->oW3, 1, 4, dh2, nh, 0.f, s));
  TRY(launch_relu_mask(dh2, h2, (long long)B * nh, s));
  TRY(launch_colsum(dh2, B, nh, gb2, s));
  TRY(gemm_plain(nh, nh, (int)B, h1, 1, nh, dh2, nh, 1, gW2, nh, 0.f, s));
  TRY(gemm_plain(B, nh, nh, dh2, nh, 1, P + m->oW2, 1, nh, dh1, nh, 0.f, s));
  TRY(launch_relu_mask(dh1, h1, (long long)B * nh, s));
  TRY(launch_colsum(dh1, B, nh, gb1, s));
  TRY(gemm_plain(ni, nh, (int)B, u, 1, ni, dh1, nh, 1, gW1, nh, 0.f, s));
#undef TRY
  return AEQC_OK;
}

extern "C" int64_t aeqc_mlp_param_count(const aeqc_mlp* m) { return m ? m->n_train : 0; }

extern "C" int mlp_loss_grad(aeqc_mlp* m, const float* in, const double* lam, int64_t B,
                             float* loss_out, float* grad_out, void* workspace,
                             size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(grad_out, "mlp_loss_grad: null grad_out");
  float* g = nullptr;
  return mlp_loss_grad_impl(m, in, lam, B, loss_out, grad_out, workspace, workspace_bytes,
                            stream, &g);
}

extern "C" int mlp_train_step(aeqc_mlp* m, const float* in, const double* lam, int64_t B,
                              float lr, float* loss_out, void* workspace,
                              size_t workspace_bytes, void* stream) {
  clear_error();
  float* grad = nullptr;
  int rc = mlp_loss_grad_impl(m, in, lam, B, loss_out, nullptr, workspace, workspace_bytes,
                              stream, &grad);
  if (rc) return rc;
  return launch_adam(m->params, grad, m->adam_m, m->adam_v, m->n_train, lr, ++m->step,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int mlp_predict(aeqc_mlp* m, const float* in, int64_t n, double* lam0,
                           void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m && in && lam0, "mlp_predict: null argument");
  AEQC_CHECK_ARG(n >= 0, "mlp_predict: negative n");
  if (n == 0) return AEQC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_predict_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(mlp_kernel_view(m), in, n, lam0);
  return check_launch("mlp_predict_kernel");
}
