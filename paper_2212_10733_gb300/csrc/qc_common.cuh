// Device helpers shared by the correction kernels: exact quantizer decision,
// 4x4 Cholesky, warp reductions, point iteration, warm-start MLP evaluation.
#pragma once

#include <cuda_bf16.h>

#include "aeqc_internal.cuh"

namespace aeqc {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
// max with the "keep s unless v > s" semantics of max(x) (NaN never wins)
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double u = __shfl_xor_sync(FULL, v, o);
    v = (u > v) ? u : v;
  }
  return v;
}

// (j, i) walker over p = lane, lane + 32, ... for row-major [j][i] grids.
struct PointIter {
  int p, i, j, n_par;
  __device__ __forceinline__ PointIter(int lane, int npar) : p(lane), n_par(npar) {
    j = lane / npar;
    i = lane - j * npar;
  }
  __device__ __forceinline__ void next() {
    p += 32;
    i += 32;
    while (i >= n_par) {
      i -= n_par;
      ++j;
    }
  }
};

// Bin width Delta = 2^floor(log2(2 alpha e)) for e = tau * s (Stage 4).
// 2^floor(log2 v) is read off the bit pattern of v = (2 alpha) (tau s): the
// exponent field of a normal number, the leading mantissa bit of a subnormal.
// Returns 0 for v == 0 and NaN for a non-finite v.
__device__ __forceinline__ double bin_width(double tau, double s, double alpha) {
  const double e = __dmul_rn(tau, s);
  const double v = __dmul_rn(__dmul_rn(2.0, alpha), e);
  const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long E = u >> 52;
  if (E == 0x7ff) return __longlong_as_double(0x7ff8000000000000LL);
  if (E > 0) return __longlong_as_double((long long)(E << 52));
  if (u == 0) return 0.0;
  return __longlong_as_double((long long)(1ull << (63 - __clzll((long long)u))));
}

// Exact quantizer decision for one point (Stage 4), FP64 form.
// q = round-half-even((x - xh)/Delta) on the exact difference: the rounded
// difference d and its TwoSum error err; the rounding is monotone, so d sits
// on the exact side of each tie point (k + 1/2) Delta or on it, where err
// decides.  Then the zero level wins when strictly nearer: for x >= 0 that
// is g < 0 or g > 2x with g = xh + q Delta (TwoSum again for g == 2x).
// Writes x' and returns the int16 code.
__device__ __forceinline__ int quant_point_fp64(double x, double xh, double dl, double* xp) {
  if (!isfinite(xh)) {
    *xp = x;
    return AEQC_CODE_ESCAPE;
  }
  double d = __dsub_rn(x, xh);
  double bb = __dsub_rn(d, x);
  double err = __dadd_rn(__dsub_rn(x, __dsub_rn(d, bb)), __dsub_rn(-xh, bb));
  double t = __ddiv_rn(d, dl);
  double fl = floor(t);
  double mid = __dadd_rn(fl, 0.5);
  double q;
  if (t > mid) q = fl + 1.0;
  else if (t < mid) q = fl;
  else if (err > 0.0) q = fl + 1.0;
  else if (err < 0.0) q = fl;
  else q = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
  if (!(q <= (double)AEQC_CODE_MAX && q >= -(double)AEQC_CODE_MAX)) {
    *xp = x;
    return AEQC_CODE_ESCAPE;
  }
  double qd = __dmul_rn(q, dl);
  double gs = __dadd_rn(xh, qd);
  double b2 = __dsub_rn(gs, xh);
  double ge = __dadd_rn(__dsub_rn(xh, __dsub_rn(gs, b2)), __dsub_rn(qd, b2));
  double two_x = __dmul_rn(2.0, x);
  if (gs < 0.0 || gs > two_x || (gs == two_x && ge > 0.0)) {
    *xp = 0.0;
    return AEQC_CODE_ZERO;
  }
  *xp = gs;
  return (int)q;
}

// Solve M d = r, M symmetric positive definite (upper triangle given as the
// 10 entries m00 m01 m02 m03 m11 m12 m13 m22 m23 m33), by Cholesky.
// Returns 0 on success, -1 when a pivot is not positive or d is not finite.
__device__ __forceinline__ int chol_solve4(const double m[10], const double r[4], double d[4]) {
  double a[4][4];
  a[0][0] = m[0]; a[0][1] = m[1]; a[0][2] = m[2]; a[0][3] = m[3];
  a[1][1] = m[4]; a[1][2] = m[5]; a[1][3] = m[6];
  a[2][2] = m[7]; a[2][3] = m[8];
  a[3][3] = m[9];
  a[1][0] = a[0][1]; a[2][0] = a[0][2]; a[3][0] = a[0][3];
  a[2][1] = a[1][2]; a[3][1] = a[1][3]; a[3][2] = a[2][3];
  double L[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int l = 0; l < 4; ++l) L[k][l] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int l = 0; l <= k; ++l) {
      double s = a[k][l];
#pragma unroll
      for (int q = 0; q < l; ++q) s -= L[k][q] * L[l][q];
      if (k == l) {
        if (!(s > 0.0)) return -1;
        L[k][k] = sqrt(s);
      } else {
        L[k][l] = s / L[l][l];
      }
    }
  }
  double y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double s = r[k];
#pragma unroll
    for (int q = 0; q < k; ++q) s -= L[k][q] * y[q];
    y[k] = s / L[k][k];
  }
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    double s = y[k];
#pragma unroll
    for (int q = k + 1; q < 4; ++q) s -= L[q][k] * d[q];
    d[k] = s / L[k][k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!isfinite(d[k])) return -1;
  return 0;
}

// Separated exponent of the KL correction f = x' exp(-lambda.phi):
// exp(-lambda.phi) = a_i * b_j with a_i = exp(-(lambda0 + v (lambda1 + v lambda3)))
// and b_j = exp(-lambda2 v_perp^2).  Written with explicit roundings so every
// kernel (compress, check, decompress) produces the same bits.
__device__ __forceinline__ double corr_a(const double lam[4], double v) {
  return exp(-__fma_rn(__fma_rn(lam[3], v, lam[1]), v, lam[0]));
}
__device__ __forceinline__ double corr_b(const double lam[4], double v2) {
  return exp(-__dmul_rn(lam[2], v2));
}
__device__ __forceinline__ double corr_kl(double xp, double a, double b) {
  return __dmul_rn(__dmul_rn(xp, a), b);
}
// L2 variant f = x' - lambda.phi
__device__ __forceinline__ double corr_l2(double xp, const double lam[4], double v, double v2) {
  return __dsub_rn(xp, __fma_rn(lam[2], v2, __fma_rn(__fma_rn(lam[3], v, lam[1]), v, lam[0])));
}

// max_k |g_k| / S_k (S_k floored at 1e-300); NaN if anything is non-finite.
__device__ __forceinline__ double scaled_residual(const double g[4], const double S[4]) {
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!isfinite(g[k]) || !isfinite(S[k])) return __longlong_as_double(0x7ff8000000000000LL);
    double den = S[k] > 0.0 ? S[k] : 1e-300;
    double v = fabs(g[k]) / den;
    r = v > r ? v : r;
  }
  return r;
}

__device__ __forceinline__ float load_latent(const LatentK& z, long long b, int l) {
  if (z.bf16) {
    const __nv_bfloat16* p = static_cast<const __nv_bfloat16*>(z.ptr);
    return __bfloat162float(p[b * z.L + l]);
  }
  return static_cast<const float*>(z.ptr)[b * z.L + l];
}

// Warm-start MLP (in -> nh -> nh -> 4, ReLU) for one histogram, evaluated by
// one warp in FP32; in_k(k) returns raw input k (latent values, then the four
// moment defects).  nh <= 64.  Every lane returns the same lambda0.
template <typename In>
__device__ __forceinline__ void mlp_eval_warp(const MlpK& m, In in_k, double lam0[4],
                                              int lane) {
  const int nin = m.nin, nh = m.nh;
  // this lane's two hidden units (o = lane, lane + 32)
  float h1a = 0.f, h1b = 0.f;
  for (int k = 0; k < nin; ++k) {
    float u = (in_k(k) - __ldg(m.in_mu + k)) / __ldg(m.in_sd + k);
    if (lane < nh) h1a = fmaf(__ldg(m.W1 + k * nh + lane), u, h1a);
    if (lane + 32 < nh) h1b = fmaf(__ldg(m.W1 + k * nh + lane + 32), u, h1b);
  }
  h1a = lane < nh ? fmaxf(h1a + __ldg(m.b1 + lane), 0.f) : 0.f;
  h1b = lane + 32 < nh ? fmaxf(h1b + __ldg(m.b1 + lane + 32), 0.f) : 0.f;
  float h2a = 0.f, h2b = 0.f;
  for (int k = 0; k < nh; ++k) {
    float hk = __shfl_sync(FULL, k < 32 ? h1a : h1b, k & 31);
    if (lane < nh) h2a = fmaf(__ldg(m.W2 + k * nh + lane), hk, h2a);
    if (lane + 32 < nh) h2b = fmaf(__ldg(m.W2 + k * nh + lane + 32), hk, h2b);
  }
  h2a = lane < nh ? fmaxf(h2a + __ldg(m.b2 + lane), 0.f) : 0.f;
  h2b = lane + 32 < nh ? fmaxf(h2b + __ldg(m.b2 + lane + 32), 0.f) : 0.f;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    float s = 0.f;
    if (lane < nh) s = fmaf(__ldg(m.W3 + lane * 4 + o), h2a, s);
    if (lane + 32 < nh) s = fmaf(__ldg(m.W3 + (lane + 32) * 4 + o), h2b, s);
    s = wsumf(s);
    lam0[o] = ((double)s + (double)__ldg(m.b3 + o)) * (double)__ldg(m.out_sd + o) +
              (double)__ldg(m.out_mu + o);
  }
}

// Append the escape points of one histogram (codes in shared memory) to the
// outlier list; returns 1 if the list overflowed for this histogram.
__device__ __forceinline__ int append_outliers(const OutliersK& o, const int16_t* codes,
                                               const double* raw, int P, long long row,
                                               int lane) {
  int cnt = 0;
  for (int p = lane; p < P; p += 32) cnt += codes[p] == AEQC_CODE_ESCAPE;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) cnt += __shfl_xor_sync(FULL, cnt, s);
  if (cnt == 0) return 0;
  long long base = 0;
  if (lane == 0) base = (long long)atomicAdd((unsigned long long*)o.count, (unsigned long long)cnt);
  base = __shfl_sync(FULL, base, 0);
  long long run = base;
  for (int p0 = 0; p0 < P; p0 += 32) {
    int p = p0 + lane;
    int pred = p < P && codes[p] == AEQC_CODE_ESCAPE;
    unsigned bal = __ballot_sync(FULL, pred);
    long long pos = run + __popc(bal & ((1u << lane) - 1u));
    if (pred && pos < o.capacity) {
      o.index[pos] = row * (long long)P + p;
      o.value[pos] = raw[p];
    }
    run += __popc(bal);
  }
  return (base + cnt > o.capacity) ? 1 : 0;
}

}  // namespace dev
}  // namespace aeqc
