// FP32 SIMT GEMM launcher (gemm_simt.cu).
#pragma once

#include "aeqc_internal.cuh"

namespace aeqc {

enum GemmEpi {
  EPI_PLAIN = 0,              // C = alpha * acc + beta * C
  EPI_BIAS_ACT = 1,           // C = act(acc + bias[n])
  EPI_ROWSCALE_BIAS_ACT = 2,  // C = act(acc / s_m + bias[n]), s_m = max_k A(m,k) (FP64 A)
  EPI_DENORM = 3,             // C = s_m * (acc + bias[n]), s_m = scale_in[m]
};

struct GemmArgs {
  long long M;  // rows (all groups)
  int N, K;
  const void* A;           // float, or double when a_f64
  long long sam, sak;      // A(m,k) = A[m*sam + k*sak]
  int a_f64;
  const float* B;          // B(k,n) = B[k*sbk + n*sbn] (+ g * group_stride_B)
  long long sbk, sbn;
  float* C;
  long long ldc;
  int epi, act;
  const float* bias;       // [N] (+ g * group_stride_bias) or null
  long long group_stride_B, group_stride_bias;
  float alpha, beta;
  double* scale_out;       // EPI_ROWSCALE_BIAS_ACT: writes s_m (may be null)
  const double* scale_in;  // EPI_DENORM
  // groups: rows [group_off[g], group_off[g+1]) use B_g; tile_off = prefix of
  // ceil(rows_g / 128) (both device arrays); n_groups <= 1 means one group
  int n_groups;
  const long long* group_off;
  const int* tile_off;
  long long max_tiles;     // grid.y for the grouped launch (>= tile_off[G])
};

int launch_gemm(const GemmArgs& a, cudaStream_t s);

// tile_off[G+1] from group_off[G+1] (device), for grouped launches.
int launch_tile_offsets(const long long* group_off, int n_groups, int tile_rows,
                        int* tile_off, cudaStream_t s);

}  // namespace aeqc
