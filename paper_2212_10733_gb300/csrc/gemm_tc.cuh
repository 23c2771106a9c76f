// Tensor-core GEMMs of the BF16 model's training step (gemm_tc.cu).
#pragma once

#include <string.h>

#include "aeqc_internal.cuh"

namespace aeqc {

// C[M][N] (ldc) = A B + beta C with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]; operands rounded to BF16, FP32 accumulation.
// scratch (device, scratch_elems floats, may be null) holds the partial tiles
// when a long K is split over more CTAs; the sum over the splits is taken in
// a fixed order.  A timed-out internal wait sets *err (device word) nonzero.
int gemm_tc_plain(long long M, int N, int K, const float* A, long long sam, long long sak,
                  const float* B, long long sbk, long long sbn, float* C, long long ldc,
                  float beta, float* scratch, long long scratch_elems, int* err,
                  cudaStream_t s);

// C[M][N] (ldc = N) = act(A B + bias[n]) with A(m,k) = A[m*sam + k].
int gemm_tc_bias(long long M, int N, int K, const float* A, long long sam, const float* B,
                 long long sbk, long long sbn, const float* bias, int act, float* C,
                 float* scratch, long long scratch_elems, int* err, cudaStream_t s);

// floats of split-K scratch the training step of a B-row batch provides
long long gemm_tc_scratch_elems(long long B, int P, int H);

}  // namespace aeqc
