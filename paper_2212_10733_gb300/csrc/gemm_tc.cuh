// Tensor-core GEMMs of the BF16 model's training step (gemm_tc.cu).
#pragma once

#include <string.h>

#include "aeqc_internal.cuh"

namespace aeqc {

// C[M][N] (ldc) = A B + beta C with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]; operands rounded to BF16, FP32 accumulation.
// A timed-out internal wait sets *err (device word) to a nonzero value.
int gemm_tc_plain(long long M, int N, int K, const float* A, long long sam, long long sak,
                  const float* B, long long sbk, long long sbn, float* C, long long ldc,
                  float beta, int* err, cudaStream_t s);

// C[M][N] (ldc = N) = act(A B + bias[n]) with A(m,k) = A[m*sam + k].
int gemm_tc_bias(long long M, int N, int K, const float* A, long long sam, const float* B,
                 long long sbk, long long sbn, const float* bias, int act, float* C, int* err,
                 cudaStream_t s);

}  // namespace aeqc
