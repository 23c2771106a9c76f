// Model and MLP objects behind the opaque C-ABI handles.
#pragma once

#include <vector>

#include "aeqc_internal.cuh"
#include "gemm_simt.cuh"

struct aeqc_model {
  aeqc_model_desc d;
  // --- per-group parameter block, FP32, device --------------------------------
  // layout (floats) of one group's trainable parameters, then mu, sigma
  long long oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, n_train, omu, osig, n_group;
  float* params;  // [n_groups][n_group]
  float* adam_m;  // [n_groups][n_train]
  float* adam_v;
  std::vector<int> step;  // Adam step per group (host)
  // --- inference copies (FP32, folded normalisation), per group ---------------
  //   enc1B [H][P]   = (W1[p][h] / sigma_p)^T         enc1b [H] = b1 - W1f^T mu
  //   enc2B [L][H]   = W2^T                            (bias b2)
  //   dec1B [H][L]   = W3^T (tied: W2)                 (bias b3)
  //   dec2B [P][H]   = (sigma_p W4[h][p])^T            dec2b [P] = sigma (.) b4 + mu
  long long iE1B, iE1b, iE2B, iD1B, iD2B, iD2b, n_inf;
  float* inf;  // [n_groups][n_inf]
  // BF16 copies of the inference weights (tcgen05 path), K padded to 64
  void* inf_bf16;
  long long bE1B, bE2B, bD1B, bD2B, n_bf16;
  int Kp1;  // P padded to a multiple of 64
  int* dev_err;  // device word: nonzero after a tensor-core kernel gave up a wait
  aeqc_tuning tuning;  // launch choices (zero: defaults)
  bool dirty;
};

struct aeqc_mlp {
  int nin, nh;
  long long oW1, ob1, oW2, ob2, oW3, ob3, n_train, oimu, oisd, oomu, oosd, n_all;
  float* params;
  float* adam_m;
  float* adam_v;
  int step;
};

namespace aeqc {

int model_prepare(aeqc_model* m, cudaStream_t s);
aeqc::MlpK mlp_kernel_view(const aeqc_mlp* m);

// encoder/decoder GEMM chains (FP32 SIMT or BF16 tcgen05 by model dtype)
int run_encode(aeqc_model* m, const double* x, long long n, const long long* group_off,
               void* latent, double* scale, char* ws, size_t ws_bytes, cudaStream_t s);
int run_decode(aeqc_model* m, const void* latent, const double* scale, long long n,
               const long long* group_off, float* xhat, long long ld, char* ws,
               size_t ws_bytes, cudaStream_t s);
size_t encode_ws(const aeqc_model* m, long long n);
size_t decode_ws(const aeqc_model* m, long long n);

// BF16 tcgen05 encoder/decoder (ae_tc.cu)
bool tc_shape_ok(int H, int L);
int run_encode_tc(aeqc_model* m, const double* x, long long n, const long long* group_off,
                  const int* tile_off, int G, void* latent, double* scale, int* err,
                  cudaStream_t s);
int run_decode_tc(aeqc_model* m, const void* latent, const double* scale, long long n,
                  const long long* group_off, const int* tile_off, int G, float* xhat,
                  long long ld, int* err, cudaStream_t s);

}  // namespace aeqc

namespace aeqc {
// small training kernels shared by the autoencoder and MLP steps (model.cu)
int launch_colsum(const float* d, long long B, int C, float* out, cudaStream_t s);
int launch_relu_mask(float* d, const float* h, long long count, cudaStream_t s);
int launch_adam(float* w, const float* g, float* m, float* v, long long cnt, float lr,
                int t, cudaStream_t s);
int gemm_plain(long long M, int N, int K, const float* A, long long sam, long long sak,
               const float* B, long long sbk, long long sbn, float* C, long long ldc,
               float beta, cudaStream_t s);
int gemm_bias(long long M, int N, int K, const float* A, long long sam, const float* B,
              long long sbk, long long sbn, const float* bias, int act, float* C,
              cudaStream_t s);
}  // namespace aeqc
