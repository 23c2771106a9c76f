// Autoencoder model object: parameters, Adam state, folded inference weights,
// the encoder/decoder GEMM chains and the training step (Sec. III Stages 2-3,
// Eq. (5); Sec. IV-B: dense layers with tied weights and linear activation,
// Adam, Z-score normalisation).
#include <cuda_bf16.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "gemm_tc.cuh"
#include "model.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

// ---- inference copies -------------------------------------------------------

struct PrepArgs {
  const float* par;  // group params
  float* inf;        // group inference block
  __nv_bfloat16* bf;  // group bf16 block or null
  int P, H, L, tied, Kp1;
  long long oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, omu, osig;
  long long iE1B, iE1b, iE2B, iD1B, iD2B, iD2b;
  long long bE1B, bE2B, bD1B, bD2B;
};

// grid.y = group; grid.x strides over the elements of the largest array
__global__ void prepare_kernel(PrepArgs a, long long group_params, long long group_inf,
                               long long group_bf16) {
  const int g = blockIdx.y;
  const float* par = a.par + g * group_params;
  float* inf = a.inf + g * group_inf;
  __nv_bfloat16* bf = a.bf ? a.bf + g * group_bf16 : nullptr;
  const float* W1 = par + a.oW1;
  const float* W2 = par + a.oW2;
  const float* W3 = par + a.oW3;
  const float* W4 = par + a.oW4;
  const float* mu = par + a.omu;
  const float* sig = par + a.osig;
  const int P = a.P, H = a.H, L = a.L;
  long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  // enc1B [H][P] = W1[p][h] / sigma_p ; bf16 copy padded to Kp1 columns
  for (long long t = t0; t < (long long)H * a.Kp1; t += st) {
    int h = (int)(t / a.Kp1), p = (int)(t - (long long)h * a.Kp1);
    float v = p < P ? W1[(long long)p * H + h] / sig[p] : 0.f;
    if (p < P) inf[a.iE1B + (long long)h * P + p] = v;
    if (bf) bf[a.bE1B + t] = __float2bfloat16_rn(v);
  }
  // enc2B [L][H] = W2[h][l]
  for (long long t = t0; t < (long long)L * H; t += st) {
    int l = (int)(t / H), h = (int)(t - (long long)l * H);
    float v = W2[(long long)h * L + l];
    inf[a.iE2B + t] = v;
    if (bf) bf[a.bE2B + t] = __float2bfloat16_rn(v);
  }
  // dec1B [H][L] = W3[l][h] (tied: W2[h][l])
  for (long long t = t0; t < (long long)H * L; t += st) {
    int h = (int)(t / L), l = (int)(t - (long long)h * L);
    float v = a.tied ? W2[(long long)h * L + l] : W3[(long long)l * H + h];
    inf[a.iD1B + t] = v;
    if (bf) bf[a.bD1B + t] = __float2bfloat16_rn(v);
  }
  // dec2B [P][H] = sigma_p W4[h][p] (tied: sigma_p W1[p][h]); dec2b = sigma b4 + mu
  for (long long t = t0; t < (long long)P * H; t += st) {
    int p = (int)(t / H), h = (int)(t - (long long)p * H);
    float w = a.tied ? W1[(long long)p * H + h] : W4[(long long)h * P + p];
    float v = sig[p] * w;
    inf[a.iD2B + t] = v;
    if (bf) bf[a.bD2B + t] = __float2bfloat16_rn(v);
  }
  for (long long t = t0; t < P; t += st) {
    inf[a.iD2b + t] = sig[t] * par[a.ob4 + t] + mu[t];
  }
}

// enc1b[h] = b1[h] - sum_p (W1[p][h] / sigma_p) mu_p   (one warp per h)
__global__ void prepare_bias_kernel(const float* params, float* inf, int P, int H,
                                    long long oW1, long long ob1, long long omu,
                                    long long osig, long long iE1b, long long group_params,
                                    long long group_inf) {
  const int g = blockIdx.y;
  const float* par = params + g * group_params;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= H) return;
  double s = 0.0;
  for (int p = lane; p < P; p += 32)
    s += (double)par[oW1 + (long long)p * H + warp] / par[osig + p] * par[omu + p];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) inf[g * group_inf + iE1b + warp] = (float)(par[ob1 + warp] - s);
}

// ---- training helpers -------------------------------------------------------

// u[b][p] = (x[b][p] / max(x_b) - mu_p) / sigma_p   (one block per row)
__global__ void normalize_kernel(const double* x, int P, const float* mu, const float* sig,
                                 float* u) {
  __shared__ double red[32];
  const long long b = blockIdx.x;
  const double* xb = x + b * P;
  double s = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double v = xb[p];
    if (v > s) s = v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, s, o);
    s = v > s ? v : s;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_xor_sync(0xffffffffu, s, o);
      s = v > s ? v : s;
    }
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  double inv = (s > 0.0 && isfinite(s)) ? 1.0 / s : 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x)
    u[b * P + p] = (float)((xb[p] * inv - (double)mu[p]) / (double)sig[p]);
}

// dy = 2 (y - u) / (B P); rowloss[b] = sum_p (y - u)^2   (one block per row)
__global__ void mse_grad_kernel(const float* y, const float* u, int P, float scale2,
                                float* dy, float* rowloss) {
  __shared__ float red[32];
  const long long b = blockIdx.x;
  float s = 0.f;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float d = y[b * P + p] - u[b * P + p];
    s = fmaf(d, d, s);
    dy[b * P + p] = scale2 * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rowloss[b] = t;
  }
}

__global__ void loss_finish_kernel(const float* rowloss, long long B, float inv_count,
                                   float* loss_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (long long b = 0; b < B; ++b) t += rowloss[b];
  *loss_out = (float)(t * inv_count);
}

// d[b][c] *= (h[b][c] > 0) for ReLU (h = act(pre), so pre > 0 <=> h > 0)
__global__ void relu_mask_kernel(float* d, const float* h, long long count) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    if (!(h[t] > 0.f)) d[t] = 0.f;
}

// out[c] = sum_b d[b][c] (fixed order over b)
__global__ void colsum_kernel(const float* d, long long B, int C, float* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (long long b = 0; b < B; ++b) s += d[b * C + c];
  out[c] = s;
}

// Adam (Kingma & Ba): the decay factors b1, b2 and their complements
// omb1 = 1 - beta1, omb2 = 1 - beta2 are each rounded from their exact values
// (1.f - 0.999f would be 1.3e-5 off 0.001, against the bias correction c2
// computed from the exact beta2).
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, long long cnt,
                            float lr, float b1, float b2, float omb1, float omb2, float eps,
                            float c1, float c2) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    float gr = g[t];
    float mt = b1 * m[t] + omb1 * gr;
    float vt = b2 * v[t] + omb2 * gr * gr;
    m[t] = mt;
    v[t] = vt;
    w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

// normaliser: scale per row, then per-pixel mean / std of x / s
__global__ void rowmax_kernel(const double* x, long long n, int P, double* s) {
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n) return;
  double m = 0.0;
  for (int p = lane; p < P; p += 32) {
    double v = x[b * P + p];
    if (v > m) m = v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if (lane == 0) s[b] = m;
}

__global__ void pixel_stats_kernel(const double* x, const double* s, long long n, int P,
                                   float* mu, float* sig) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double acc = 0.0;
  for (long long b = 0; b < n; ++b) {
    double inv = s[b] > 0.0 ? 1.0 / s[b] : 0.0;
    acc += x[b * P + p] * inv;
  }
  double mean = acc / (double)n, var = 0.0;
  for (long long b = 0; b < n; ++b) {
    double inv = s[b] > 0.0 ? 1.0 / s[b] : 0.0;
    double d = x[b * P + p] * inv - mean;
    var += d * d;
  }
  double sd = sqrt(var / (double)n);
  mu[p] = (float)mean;
  sig[p] = (float)(sd > 1e-6 ? sd : 1e-6);
}

GemmArgs gemm0() {
  GemmArgs a;
  memset(&a, 0, sizeof(a));
  a.alpha = 1.f;
  a.n_groups = 1;
  return a;
}

// C[M][N] (ldc) = op(A) op(B): A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
int gemm_plain_impl(long long M, int N, int K, const float* A, long long sam, long long sak,
               const float* B, long long sbk, long long sbn, float* C, long long ldc,
               float beta, cudaStream_t s) {
  GemmArgs a = gemm0();
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.sam = sam; a.sak = sak;
  a.B = B; a.sbk = sbk; a.sbn = sbn;
  a.C = C; a.ldc = ldc;
  a.epi = EPI_PLAIN;
  a.beta = beta;
  return launch_gemm(a, s);
}

int gemm_bias_impl(long long M, int N, int K, const float* A, long long sam, const float* B,
                   long long sbk, long long sbn, const float* bias, int act, float* C,
                   cudaStream_t s) {
  GemmArgs a = gemm0();
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.sam = sam; a.sak = 1;
  a.B = B; a.sbk = sbk; a.sbn = sbn;
  a.C = C; a.ldc = N;
  a.epi = EPI_BIAS_ACT;
  a.act = act;
  a.bias = bias;
  return launch_gemm(a, s);
}

}  // namespace

int gemm_plain(long long M, int N, int K, const float* A, long long sam, long long sak,
               const float* B, long long sbk, long long sbn, float* C, long long ldc,
               float beta, cudaStream_t s) {
  return gemm_plain_impl(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, beta, s);
}
int gemm_bias(long long M, int N, int K, const float* A, long long sam, const float* B,
              long long sbk, long long sbn, const float* bias, int act, float* C,
              cudaStream_t s) {
  return gemm_bias_impl(M, N, K, A, sam, B, sbk, sbn, bias, act, C, s);
}
int launch_colsum(const float* d, long long B, int C, float* out, cudaStream_t s) {
  colsum_kernel<<<(C + 255) / 256, 256, 0, s>>>(d, B, C, out);
  return check_launch("colsum_kernel");
}
int launch_relu_mask(float* d, const float* h, long long count, cudaStream_t s) {
  relu_mask_kernel<<<256, 256, 0, s>>>(d, h, count);
  return check_launch("relu_mask_kernel");
}
int launch_adam(float* w, const float* g, float* m, float* v, long long cnt, float lr,
                int t, cudaStream_t s) {
  float c1 = (float)(1.0 - pow(0.9, t)), c2 = (float)(1.0 - pow(0.999, t));
  adam_kernel<<<512, 256, 0, s>>>(w, g, m, v, cnt, lr, 0.9f, 0.999f, (float)(1.0 - 0.9),
                                  (float)(1.0 - 0.999), 1e-8f, c1, c2);
  return check_launch("adam_kernel");
}

// ---------------------------------------------------------------------------

int model_prepare(aeqc_model* m, cudaStream_t s) {
  if (!m->dirty) return AEQC_OK;
  const aeqc_model_desc& d = m->d;
  PrepArgs a;
  a.par = m->params;
  a.inf = m->inf;
  a.bf = static_cast<__nv_bfloat16*>(m->inf_bf16);
  a.P = d.P; a.H = d.H; a.L = d.L; a.tied = d.tied; a.Kp1 = m->Kp1;
  a.oW1 = m->oW1; a.ob1 = m->ob1; a.oW2 = m->oW2; a.ob2 = m->ob2; a.oW3 = m->oW3;
  a.ob3 = m->ob3; a.oW4 = m->oW4; a.ob4 = m->ob4; a.omu = m->omu; a.osig = m->osig;
  a.iE1B = m->iE1B; a.iE1b = m->iE1b; a.iE2B = m->iE2B; a.iD1B = m->iD1B;
  a.iD2B = m->iD2B; a.iD2b = m->iD2b;
  a.bE1B = m->bE1B; a.bE2B = m->bE2B; a.bD1B = m->bD1B; a.bD2B = m->bD2B;
  dim3 grid(256, d.n_groups);
  prepare_kernel<<<grid, 256, 0, s>>>(a, m->n_group, m->n_inf, m->n_bf16);
  int rc = check_launch("prepare_kernel");
  if (rc) return rc;
  dim3 g2((d.H * 32 + 255) / 256, d.n_groups);
  prepare_bias_kernel<<<g2, 256, 0, s>>>(m->params, m->inf, d.P, d.H, m->oW1, m->ob1,
                                         m->omu, m->osig, m->iE1b, m->n_group, m->n_inf);
  rc = check_launch("prepare_bias_kernel");
  if (rc) return rc;
  m->dirty = false;
  return AEQC_OK;
}

size_t encode_ws(const aeqc_model* m, long long n) {
  WsSize w;
  w.add<float>((size_t)n * m->d.H);
  w.add<int>(m->d.n_groups + 1);
  return w.bytes;
}
size_t decode_ws(const aeqc_model* m, long long n) { return encode_ws(m, n); }

int run_encode(aeqc_model* m, const double* x, long long n, const long long* group_off,
               void* latent, double* scale, char* ws, size_t ws_bytes, cudaStream_t s) {
  const aeqc_model_desc& d = m->d;
  int rc = model_prepare(m, s);
  if (rc) return rc;
  WsCarver c(ws, ws_bytes);
  float* h1 = c.take<float>((size_t)n * d.H);
  int* tile_off = c.take<int>(d.n_groups + 1);
  if (!c.ok()) return set_error(AEQC_EINVAL, "ae_encode: workspace too small");
  int G = group_off ? d.n_groups : 1;
  if (G > 1) {
    rc = launch_tile_offsets(group_off, G, 128, tile_off, s);
    if (rc) return rc;
  }
  if (d.dtype == AEQC_DTYPE_BF16)
    return run_encode_tc(m, x, n, group_off, tile_off, G, latent, scale, m->dev_err, s);
  GemmArgs a = gemm0();
  a.M = n; a.N = d.H; a.K = d.P;
  a.A = x; a.sam = d.P; a.sak = 1; a.a_f64 = 1;
  a.B = m->inf + m->iE1B; a.sbk = 1; a.sbn = d.P;
  a.C = h1; a.ldc = d.H;
  a.epi = EPI_ROWSCALE_BIAS_ACT; a.act = d.act;
  a.bias = m->inf + m->iE1b;
  a.group_stride_B = m->n_inf; a.group_stride_bias = m->n_inf;
  a.scale_out = scale;
  a.n_groups = G; a.group_off = group_off; a.tile_off = tile_off;
  a.max_tiles = (n + 127) / 128 + G;
  rc = launch_gemm(a, s);
  if (rc) return rc;
  GemmArgs b = a;
  b.N = d.L; b.K = d.H;
  b.A = h1; b.sam = d.H; b.a_f64 = 0;
  b.B = m->inf + m->iE2B; b.sbn = d.H;
  b.C = static_cast<float*>(latent); b.ldc = d.L;
  b.epi = EPI_BIAS_ACT; b.act = AEQC_ACT_IDENTITY;
  b.bias = m->params + m->ob2;
  b.group_stride_bias = m->n_group;
  b.scale_out = nullptr;
  return launch_gemm(b, s);
}

int run_decode(aeqc_model* m, const void* latent, const double* scale, long long n,
               const long long* group_off, float* xhat, long long ld, char* ws,
               size_t ws_bytes, cudaStream_t s) {
  const aeqc_model_desc& d = m->d;
  int rc = model_prepare(m, s);
  if (rc) return rc;
  WsCarver c(ws, ws_bytes);
  float* h3 = c.take<float>((size_t)n * d.H);
  int* tile_off = c.take<int>(d.n_groups + 1);
  if (!c.ok()) return set_error(AEQC_EINVAL, "ae_decode: workspace too small");
  int G = group_off ? d.n_groups : 1;
  if (G > 1) {
    rc = launch_tile_offsets(group_off, G, 128, tile_off, s);
    if (rc) return rc;
  }
  if (d.dtype == AEQC_DTYPE_BF16)
    return run_decode_tc(m, latent, scale, n, group_off, tile_off, G, xhat, ld, m->dev_err, s);
  GemmArgs a = gemm0();
  a.M = n; a.N = d.H; a.K = d.L;
  a.A = latent; a.sam = d.L; a.sak = 1;
  a.B = m->inf + m->iD1B; a.sbk = 1; a.sbn = d.L;
  a.C = h3; a.ldc = d.H;
  a.epi = EPI_BIAS_ACT; a.act = d.act;
  a.bias = m->params + m->ob3;
  a.group_stride_B = m->n_inf; a.group_stride_bias = m->n_group;
  a.n_groups = G; a.group_off = group_off; a.tile_off = tile_off;
  a.max_tiles = (n + 127) / 128 + G;
  rc = launch_gemm(a, s);
  if (rc) return rc;
  GemmArgs b = a;
  b.N = d.P; b.K = d.H;
  b.A = h3; b.sam = d.H;
  b.B = m->inf + m->iD2B; b.sbn = d.H;
  b.C = xhat; b.ldc = ld;
  b.epi = EPI_DENORM;
  b.bias = m->inf + m->iD2b;
  b.group_stride_bias = m->n_inf;
  b.scale_in = scale;
  return launch_gemm(b, s);
}

MlpK mlp_kernel_view(const aeqc_mlp* m) {
  MlpK k;
  k.W1 = m->params + m->oW1;
  k.b1 = m->params + m->ob1;
  k.W2 = m->params + m->oW2;
  k.b2 = m->params + m->ob2;
  k.W3 = m->params + m->oW3;
  k.b3 = m->params + m->ob3;
  k.in_mu = m->params + m->oimu;
  k.in_sd = m->params + m->oisd;
  k.out_mu = m->params + m->oomu;
  k.out_sd = m->params + m->oosd;
  k.nin = m->nin;
  k.nh = m->nh;
  return k;
}

}  // namespace aeqc

using namespace aeqc;

// ---------------------------------------------------------------------------
// C ABI: model
// ---------------------------------------------------------------------------

extern "C" int aeqc_model_create(const aeqc_model_desc* desc, aeqc_model** out) {
  clear_error();
  AEQC_CHECK_ARG(desc && out, "aeqc_model_create: null argument");
  const aeqc_model_desc d = *desc;
  AEQC_CHECK_ARG(d.P > 0 && d.P <= AEQC_MAX_P, "aeqc_model_create: P=%d out of range", d.P);
  AEQC_CHECK_ARG(d.layers == 0 || d.layers == 1 || d.layers == 2,
                 "aeqc_model_create: layers=%d", d.layers);
  if (d.layers == 1) {
    AEQC_CHECK_ARG(d.H == d.L && d.L > 0 && d.L <= 256 && d.L % 4 == 0 && d.tied,
                   "aeqc_model_create: one layer needs H == L, a multiple of 4 in [4, 256], "
                   "tied (H=%d, L=%d)", d.H, d.L);
    if (d.dtype != AEQC_DTYPE_F32)
      return set_error(AEQC_EUNSUPPORTED, "aeqc_model_create: one-layer models are FP32");
  } else {
    AEQC_CHECK_ARG(d.H > 0 && d.H <= 1024 && d.H % 32 == 0,
                   "aeqc_model_create: H=%d must be a multiple of 32 in [32, 1024]", d.H);
    AEQC_CHECK_ARG(d.L > 0 && d.L <= 256 && d.L % 8 == 0,
                   "aeqc_model_create: L=%d must be a multiple of 8 in [8, 256]", d.L);
  }
  AEQC_CHECK_ARG(d.act == AEQC_ACT_IDENTITY || d.act == AEQC_ACT_RELU,
                 "aeqc_model_create: bad act");
  AEQC_CHECK_ARG(d.dtype == AEQC_DTYPE_F32 || d.dtype == AEQC_DTYPE_BF16,
                 "aeqc_model_create: bad dtype");
  AEQC_CHECK_ARG(d.n_groups >= 1 && d.n_groups <= 65536, "aeqc_model_create: bad n_groups");
  if (d.dtype == AEQC_DTYPE_BF16 && !tc_shape_ok(d.H, d.L))
    return set_error(AEQC_EUNSUPPORTED,
                     "aeqc_model_create: BF16 models need H a multiple of 64 in [64, 512] and "
                     "L in {16, 32} (H=%d, L=%d)", d.H, d.L);
  aeqc_model* m = new aeqc_model();
  m->step.assign(d.n_groups, 0);  // new aeqc_model() zero-initialises the rest
  m->d = d;
  const long long P = d.P, H = d.H, L = d.L;
  long long o = 0;
  m->oW1 = o; o += P * H;
  m->ob1 = o; o += H;
  m->oW2 = o; o += H * L;
  m->ob2 = o; o += L;
  m->oW3 = o; if (!d.tied) o += L * H;
  m->ob3 = o; o += H;
  m->oW4 = o; if (!d.tied) o += H * P;
  m->ob4 = o; o += P;
  m->n_train = o;
  m->omu = o; o += P;
  m->osig = o; o += P;
  m->n_group = (o + 63) / 64 * 64;
  long long q = 0;
  m->iE1B = q; q += H * P;
  m->iE1b = q; q += H;
  m->iE2B = q; q += L * H;
  m->iD1B = q; q += H * L;
  m->iD2B = q; q += P * H;
  m->iD2b = q; q += P;
  m->n_inf = (q + 63) / 64 * 64;
  m->Kp1 = (d.P + 63) / 64 * 64;
  long long r = 0;
  m->bE1B = r; r += H * m->Kp1;
  m->bE2B = r; r += L * H;
  m->bD1B = r; r += H * L;
  m->bD2B = r; r += P * H;
  m->n_bf16 = (r + 63) / 64 * 64;
  const long long G = d.n_groups;
  // params, adam_m, adam_v contiguous (saved as one block); the inference
  // copy starts on a 256-byte boundary (vector loads of its bias rows)
  const long long inf_off = (G * m->n_group + 2 * G * m->n_train + 63) / 64 * 64;
  size_t bytes = sizeof(float) * (size_t)(inf_off + G * m->n_inf) + 256;  // + the device error word
  size_t bbytes = d.dtype == AEQC_DTYPE_BF16 ? sizeof(__nv_bfloat16) * (size_t)(G * m->n_bf16) : 0;
  char* base = nullptr;
  if (cudaMalloc(&base, bytes) != cudaSuccess) {
    delete m;
    return set_error(AEQC_ENOMEM, "aeqc_model_create: cudaMalloc(%zu) failed", bytes);
  }
  if (cudaMemset(base, 0, bytes) != cudaSuccess) {
    cudaFree(base);
    delete m;
    return set_error(AEQC_ECUDA, "aeqc_model_create: cudaMemset failed");
  }
  m->params = reinterpret_cast<float*>(base);
  m->adam_m = m->params + G * m->n_group;
  m->adam_v = m->adam_m + G * m->n_train;
  m->inf = m->params + inf_off;
  m->dev_err = reinterpret_cast<int*>(m->inf + G * m->n_inf);
  if (bbytes) {
    if (cudaMalloc(&m->inf_bf16, bbytes) != cudaSuccess) {
      cudaFree(base);
      delete m;
      return set_error(AEQC_ENOMEM, "aeqc_model_create: cudaMalloc(%zu) failed", bbytes);
    }
    cudaMemset(m->inf_bf16, 0, bbytes);
  }
  // sigma = 1 so an unset model is well defined
  std::vector<float> ones(P, 1.f);
  for (long long g = 0; g < G; ++g)
    cudaMemcpy(m->params + g * m->n_group + m->osig, ones.data(), P * sizeof(float),
               cudaMemcpyHostToDevice);
  m->dirty = true;
  *out = m;
  return AEQC_OK;
}

extern "C" int aeqc_model_destroy(aeqc_model* m) {
  clear_error();
  if (!m) return AEQC_OK;
  cudaFree(m->params);
  if (m->inf_bf16) cudaFree(m->inf_bf16);
  delete m;
  return AEQC_OK;
}

static int copy_in(float* dst, const double* src, long long cnt) {
  if (!src) return AEQC_OK;
  std::vector<float> tmp(cnt);
  for (long long t = 0; t < cnt; ++t) tmp[t] = (float)src[t];
  AEQC_CUDA_TRY(cudaMemcpy(dst, tmp.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
  return AEQC_OK;
}
static int copy_out(double* dst, const float* src, long long cnt) {
  if (!dst) return AEQC_OK;
  std::vector<float> tmp(cnt);
  AEQC_CUDA_TRY(cudaMemcpy(tmp.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost));
  for (long long t = 0; t < cnt; ++t) dst[t] = tmp[t];
  return AEQC_OK;
}

extern "C" int aeqc_model_set_group(aeqc_model* m, int32_t group, const double* W1,
                                    const double* b1, const double* W2, const double* b2,
                                    const double* W3, const double* b3, const double* W4,
                                    const double* b4, const double* mu, const double* sigma) {
  clear_error();
  AEQC_CHECK_ARG(m, "aeqc_model_set_group: null model");
  AEQC_CHECK_ARG(group >= 0 && group < m->d.n_groups, "aeqc_model_set_group: bad group %d",
                 group);
  const bool one = m->d.layers == 1;
  AEQC_CHECK_ARG(W1 && b1 && (one || (W2 && b2 && b3)) && b4 && mu && sigma,
                 "aeqc_model_set_group: null parameter array");
  AEQC_CHECK_ARG(m->d.tied || (W3 && W4), "aeqc_model_set_group: untied model needs W3, W4");
  const long long P = m->d.P, H = m->d.H, L = m->d.L;
  for (long long p = 0; p < P; ++p)
    AEQC_CHECK_ARG(sigma[p] > 0.0, "aeqc_model_set_group: sigma must be positive");
  float* g = m->params + group * m->n_group;
  int rc;
  if ((rc = copy_in(g + m->oW1, W1, P * H))) return rc;
  if ((rc = copy_in(g + m->ob1, b1, H))) return rc;
  if (one) {  // the second layer is the identity and its biases zero
    std::vector<double> eye((size_t)H * L, 0.0), zero((size_t)H, 0.0);
    for (long long i = 0; i < H; ++i) eye[(size_t)i * L + i] = 1.0;
    if ((rc = copy_in(g + m->oW2, eye.data(), H * L))) return rc;
    if ((rc = copy_in(g + m->ob2, zero.data(), L))) return rc;
    if ((rc = copy_in(g + m->ob3, zero.data(), H))) return rc;
  } else {
    if ((rc = copy_in(g + m->oW2, W2, H * L))) return rc;
    if ((rc = copy_in(g + m->ob2, b2, L))) return rc;
    if ((rc = copy_in(g + m->ob3, b3, H))) return rc;
  }
  if (!m->d.tied) {
    if ((rc = copy_in(g + m->oW3, W3, L * H))) return rc;
    if ((rc = copy_in(g + m->oW4, W4, H * P))) return rc;
  }
  if ((rc = copy_in(g + m->ob4, b4, P))) return rc;
  if ((rc = copy_in(g + m->omu, mu, P))) return rc;
  if ((rc = copy_in(g + m->osig, sigma, P))) return rc;
  AEQC_CUDA_TRY(cudaMemset(m->adam_m + group * m->n_train, 0, m->n_train * sizeof(float)));
  AEQC_CUDA_TRY(cudaMemset(m->adam_v + group * m->n_train, 0, m->n_train * sizeof(float)));
  m->step[group] = 0;
  m->dirty = true;
  return AEQC_OK;
}

extern "C" int aeqc_model_get_group(aeqc_model* m, int32_t group, double* W1, double* b1,
                                    double* W2, double* b2, double* W3, double* b3,
                                    double* W4, double* b4, double* mu, double* sigma) {
  clear_error();
  AEQC_CHECK_ARG(m, "aeqc_model_get_group: null model");
  AEQC_CHECK_ARG(group >= 0 && group < m->d.n_groups, "aeqc_model_get_group: bad group");
  AEQC_CUDA_TRY(cudaDeviceSynchronize());
  const long long P = m->d.P, H = m->d.H, L = m->d.L;
  const float* g = m->params + group * m->n_group;
  int rc;
  if ((rc = copy_out(W1, g + m->oW1, P * H))) return rc;
  if ((rc = copy_out(b1, g + m->ob1, H))) return rc;
  if ((rc = copy_out(W2, g + m->oW2, H * L))) return rc;
  if ((rc = copy_out(b2, g + m->ob2, L))) return rc;
  if (!m->d.tied) {
    if ((rc = copy_out(W3, g + m->oW3, L * H))) return rc;
    if ((rc = copy_out(W4, g + m->oW4, H * P))) return rc;
  }
  if ((rc = copy_out(b3, g + m->ob3, H))) return rc;
  if ((rc = copy_out(b4, g + m->ob4, P))) return rc;
  if ((rc = copy_out(mu, g + m->omu, P))) return rc;
  if ((rc = copy_out(sigma, g + m->osig, P))) return rc;
  return AEQC_OK;
}

extern "C" size_t aeqc_fit_normalizer_workspace_size(const aeqc_model* m) {
  (void)m;
  return 0;
}

extern "C" int aeqc_fit_normalizer(aeqc_model* m, int32_t group, const double* x, int64_t n,
                                   void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m && x, "aeqc_fit_normalizer: null argument");
  AEQC_CHECK_ARG(group >= 0 && group < m->d.n_groups, "aeqc_fit_normalizer: bad group");
  AEQC_CHECK_ARG(n > 0, "aeqc_fit_normalizer: n must be positive");
  size_t need = sizeof(double) * (size_t)n;
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need,
                 "aeqc_fit_normalizer: workspace of %zu bytes needed", need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* sc = static_cast<double*>(workspace);
  rowmax_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(x, n, m->d.P, sc);
  int rc = check_launch("rowmax_kernel");
  if (rc) return rc;
  float* g = m->params + group * m->n_group;
  pixel_stats_kernel<<<(m->d.P + 127) / 128, 128, 0, s>>>(x, sc, n, m->d.P, g + m->omu,
                                                          g + m->osig);
  rc = check_launch("pixel_stats_kernel");
  m->dirty = true;
  return rc;
}

// ---------------------------------------------------------------------------
// C ABI: training step (Eq. (5) loss, Adam)
// ---------------------------------------------------------------------------

extern "C" size_t ae_train_workspace_size(const aeqc_model* m, int64_t B) {
  if (!m || B <= 0) return 0;
  const size_t P = m->d.P, H = m->d.H, L = m->d.L;
  WsSize w;
  w.add<float>(B * P);  // u
  w.add<float>(B * H);  // h1
  w.add<float>(B * L);  // z
  w.add<float>(B * H);  // h3
  w.add<float>(B * P);  // y
  w.add<float>(B * P);  // dy
  w.add<float>(B * H);  // dh3 / dpre3
  w.add<float>(B * L);  // dz
  w.add<float>(B * H);  // dh1 / dpre1
  w.add<float>(B);      // row losses
  w.add<float>(m->n_train);  // gradients
  w.add<float>(1);      // scratch loss
  if (m->d.dtype == AEQC_DTYPE_BF16)  // split-K partial tiles of the tensor-core GEMMs
    w.add<float>((size_t)gemm_tc_scratch_elems(B, (int)P, (int)H));
  return w.bytes;
}

// Forward + backward of one batch: loss and gradient (into grad_ext when
// given, else into the workspace); returns the gradient pointer in *grad_used.
static int loss_grad_impl(aeqc_model* m, const double* x, int64_t B, int32_t group,
                          float* loss_out, float* grad_ext, void* workspace,
                          size_t workspace_bytes, void* stream, float** grad_used) {
  AEQC_CHECK_ARG(m && x, "ae_train_step: null argument");
  AEQC_CHECK_ARG(B > 0, "ae_train_step: B must be positive");
  AEQC_CHECK_ARG(group >= 0 && group < m->d.n_groups, "ae_train_step: bad group");
  size_t need = ae_train_workspace_size(m, B);
  AEQC_CHECK_ARG(workspace && workspace_bytes >= need,
                 "ae_train_step: workspace of %zu bytes needed", need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = m->d.P, H = m->d.H, L = m->d.L, act = m->d.act;
  const bool tied = m->d.tied;
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  float* u = c.take<float>((size_t)B * P);
  float* h1 = c.take<float>((size_t)B * H);
  float* z = c.take<float>((size_t)B * L);
  float* h3 = c.take<float>((size_t)B * H);
  float* y = c.take<float>((size_t)B * P);
  float* dy = c.take<float>((size_t)B * P);
  float* dh3 = c.take<float>((size_t)B * H);
  float* dz = c.take<float>((size_t)B * L);
  float* dh1 = c.take<float>((size_t)B * H);
  float* rowloss = c.take<float>(B);
  float* grad = c.take<float>(m->n_train);
  float* lscratch = c.take<float>(1);
  const long long kscr_n =
      m->d.dtype == AEQC_DTYPE_BF16 ? gemm_tc_scratch_elems(B, m->d.P, m->d.H) : 0;
  float* kscr = kscr_n ? c.take<float>((size_t)kscr_n) : nullptr;
  if (grad_ext) grad = grad_ext;
  *grad_used = grad;
  float* par = m->params + group * m->n_group;
  const float *W1 = par + m->oW1, *b1 = par + m->ob1, *W2 = par + m->oW2, *b2 = par + m->ob2;
  const float *W3 = par + m->oW3, *b3 = par + m->ob3, *W4 = par + m->oW4, *b4 = par + m->ob4;
  // the BF16 model trains on the tensor cores (BF16 operands, FP32
  // accumulation; FP32 master weights and Adam), the FP32 model on FP32 SIMT
  const bool tc = m->d.dtype == AEQC_DTYPE_BF16;
  int* err = m->dev_err;
  auto fwd = [&](long long M, int N, int K, const float* A, long long sam, const float* Bm,
                 long long sbk, long long sbn, const float* bias, int ac, float* C,
                 cudaStream_t st) {
    return tc ? gemm_tc_bias(M, N, K, A, sam, Bm, sbk, sbn, bias, ac, C, kscr, kscr_n, err, st)
              : gemm_bias(M, N, K, A, sam, Bm, sbk, sbn, bias, ac, C, st);
  };
  auto prod = [&](long long M, int N, int K, const float* A, long long sam, long long sak,
                  const float* Bm, long long sbk, long long sbn, float* C, long long ldc,
                  float beta, cudaStream_t st) {
    return tc ? gemm_tc_plain(M, N, K, A, sam, sak, Bm, sbk, sbn, C, ldc, beta, kscr, kscr_n,
                              err, st)
              : gemm_plain(M, N, K, A, sam, sak, Bm, sbk, sbn, C, ldc, beta, st);
  };
  int rc;
#define TRY(e) \
  do {                    \
    if ((rc = (e))) return rc; \
  } while (0)
  normalize_kernel<<<(unsigned)B, 256, 0, s>>>(x, P, par + m->omu, par + m->osig, u);
  TRY(check_launch("normalize_kernel"));
  // forward: h1 = act(u W1 + b1); z = h1 W2 + b2; h3 = act(z W3' + b3); y = h3 W4' + b4
  TRY(fwd(B, H, P, u, P, W1, H, 1, b1, act, h1, s));
  TRY(fwd(B, L, H, h1, H, W2, L, 1, b2, AEQC_ACT_IDENTITY, z, s));
  if (tied) TRY(fwd(B, H, L, z, L, W2, 1, L, b3, act, h3, s));
  else TRY(fwd(B, H, L, z, L, W3, H, 1, b3, act, h3, s));
  if (tied) TRY(fwd(B, P, H, h3, H, W1, 1, H, b4, AEQC_ACT_IDENTITY, y, s));
  else TRY(fwd(B, P, H, h3, H, W4, P, 1, b4, AEQC_ACT_IDENTITY, y, s));
  // loss and dy
  mse_grad_kernel<<<(unsigned)B, 256, 0, s>>>(y, u, P, 2.f / ((float)B * (float)P), dy,
                                              rowloss);
  TRY(check_launch("mse_grad_kernel"));
  loss_finish_kernel<<<1, 1, 0, s>>>(rowloss, B, 1.f / ((float)B * (float)P),
                                     loss_out ? loss_out : lscratch);
  TRY(check_launch("loss_finish_kernel"));
  float *gW1 = grad + m->oW1, *gb1 = grad + m->ob1, *gW2 = grad + m->oW2, *gb2 = grad + m->ob2;
  float *gW3 = grad + m->oW3, *gb3 = grad + m->ob3, *gW4 = grad + m->oW4, *gb4 = grad + m->ob4;
  // layer 4
  colsum_kernel<<<(P + 255) / 256, 256, 0, s>>>(dy, B, P, gb4);
  TRY(check_launch("colsum_kernel"));
  if (tied) TRY(prod(P, H, (int)B, dy, 1, P, h3, H, 1, gW1, H, 0.f, s));
  else TRY(prod(H, P, (int)B, h3, 1, H, dy, P, 1, gW4, P, 0.f, s));
  if (tied) TRY(prod(B, H, P, dy, P, 1, W1, H, 1, dh3, H, 0.f, s));
  else TRY(prod(B, H, P, dy, P, 1, W4, 1, P, dh3, H, 0.f, s));
  if (act == AEQC_ACT_RELU) {
    relu_mask_kernel<<<256, 256, 0, s>>>(dh3, h3, (long long)B * H);
    TRY(check_launch("relu_mask_kernel"));
  }
  // layer 3
  colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(dh3, B, H, gb3);
  TRY(check_launch("colsum_kernel"));
  if (tied) TRY(prod(H, L, (int)B, dh3, 1, H, z, L, 1, gW2, L, 0.f, s));
  else TRY(prod(L, H, (int)B, z, 1, L, dh3, H, 1, gW3, H, 0.f, s));
  if (tied) TRY(prod(B, L, H, dh3, H, 1, W2, L, 1, dz, L, 0.f, s));
  else TRY(prod(B, L, H, dh3, H, 1, W3, 1, H, dz, L, 0.f, s));
  // layer 2
  colsum_kernel<<<(L + 255) / 256, 256, 0, s>>>(dz, B, L, gb2);
  TRY(check_launch("colsum_kernel"));
  TRY(prod(H, L, (int)B, h1, 1, H, dz, L, 1, gW2, L, tied ? 1.f : 0.f, s));
  TRY(prod(B, H, L, dz, L, 1, W2, 1, L, dh1, H, 0.f, s));
  if (act == AEQC_ACT_RELU) {
    relu_mask_kernel<<<256, 256, 0, s>>>(dh1, h1, (long long)B * H);
    TRY(check_launch("relu_mask_kernel"));
  }
  // layer 1
  colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(dh1, B, H, gb1);
  TRY(check_launch("colsum_kernel"));
  TRY(prod(P, H, (int)B, u, 1, P, dh1, H, 1, gW1, H, tied ? 1.f : 0.f, s));
  if (m->d.layers == 1) {  // the identity layer and its zero biases do not train
    AEQC_CUDA_TRY(cudaMemsetAsync(gW2, 0, sizeof(float) * (size_t)H * L, s));
    AEQC_CUDA_TRY(cudaMemsetAsync(gb2, 0, sizeof(float) * (size_t)L, s));
    AEQC_CUDA_TRY(cudaMemsetAsync(gb3, 0, sizeof(float) * (size_t)H, s));
  }
#undef TRY
  return AEQC_OK;
}

extern "C" int64_t aeqc_model_param_count(const aeqc_model* m) { return m ? m->n_train : 0; }

extern "C" int ae_loss_grad(aeqc_model* m, const double* x, int64_t B, int32_t group,
                            float* loss_out, float* grad_out, void* workspace,
                            size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(grad_out, "ae_loss_grad: null grad_out");
  float* g = nullptr;
  return loss_grad_impl(m, x, B, group, loss_out, grad_out, workspace, workspace_bytes, stream,
                        &g);
}

extern "C" int ae_train_step(aeqc_model* m, const double* x, int64_t B, int32_t group,
                             float lr, float* loss_out, void* workspace,
                             size_t workspace_bytes, void* stream) {
  clear_error();
  float* grad = nullptr;
  int rc = loss_grad_impl(m, x, B, group, loss_out, nullptr, workspace, workspace_bytes,
                          stream, &grad);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int t = ++m->step[group];
  rc = launch_adam(m->params + group * m->n_group, grad, m->adam_m + group * m->n_train,
                   m->adam_v + group * m->n_train, m->n_train, lr, t, s);
  m->dirty = true;
  return rc;
}
