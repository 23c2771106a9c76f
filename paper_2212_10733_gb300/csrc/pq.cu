// Product quantisation of the latent space (Sec. III Stage 3, Sec. V-B):
// per subdomain and latent dimension, K-means with k clusters; a latent value
// is stored as the index of its nearest centroid and decoded as the centroid.
//
// Training runs Lloyd iterations from k centroids evenly spaced in the
// column's range.  Each iteration is one pass over the latents: the nearest
// centroid is chosen in float32 (ties to the lowest index), and the members'
// sum is accumulated as a 64-bit fixed-point integer (value * 2^s with s set
// from the column's largest magnitude and the group's row count, so that no
// sum can overflow).  Integer sums are order-independent, so the result does
// not depend on scheduling; each value is rounded to 2^-s, at most 2^-(s+1)
// away, which moves a mean by far less than half a float32 ulp of the column's
// range.  The new centroid is the sum over the count, rounded to float32; a
// centroid without members stays.
#include <cuda_bf16.h>
#include <math.h>

#include "aeqc_internal.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

constexpr int PQ_THREADS = 256;

__device__ __forceinline__ float load_z(const void* z, int bf16, long long i) {
  if (bf16) return __bfloat162float(static_cast<const __nv_bfloat16*>(z)[i]);
  return static_cast<const float*>(z)[i];
}

__device__ __forceinline__ void store_z(void* z, int bf16, long long i, float v) {
  if (bf16) static_cast<__nv_bfloat16*>(z)[i] = __float2bfloat16_rn(v);
  else static_cast<float*>(z)[i] = v;
}

// float <-> int32 key with the same order (finite values)
__device__ __forceinline__ int order_key(float v) {
  const int b = __float_as_int(v);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float key_value(int k) {
  return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF);
}

__device__ __forceinline__ long long group_lo(const long long* off, int g, long long n) {
  return off ? off[g] : 0;
}
__device__ __forceinline__ long long group_hi(const long long* off, int g, long long n) {
  return off ? off[g + 1] : n;
}

// nearest of k centroids (float32 distances, lowest index on ties)
__device__ __forceinline__ int nearest(float v, const float* c, int k) {
  float best = fabsf(v - c[0]);
  int arg = 0;
  for (int j = 1; j < k; ++j) {
    const float d = fabsf(v - c[j]);
    if (d < best) {
      best = d;
      arg = j;
    }
  }
  return arg;
}

// Elements of group g handled by this block: rows off[g] + blockIdx.x * R +
// tr + i * gridDim.x * R, dimension d (R = rows per block step).
#define PQ_FOR_ELEMENTS(body)                                                    \
  do {                                                                           \
    const int g = blockIdx.y;                                                    \
    const long long r0 = group_lo(off, g, n), r1 = group_hi(off, g, n);          \
    const int R = PQ_THREADS / L;                                                \
    const int d = threadIdx.x % L, tr = threadIdx.x / L;                         \
    if (tr < R) {                                                                \
      for (long long r = r0 + (long long)blockIdx.x * R + tr; r < r1;            \
           r += (long long)gridDim.x * R) {                                      \
        const long long e = r * L + d;                                           \
        body                                                                     \
      }                                                                          \
    }                                                                            \
  } while (0)

__global__ void pq_clear_kernel(int* keys, long long* acc, unsigned long long* cnt, int GL,
                                int k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < GL * k; t += gridDim.x * blockDim.x) {
    acc[t] = 0;
    cnt[t] = 0;
    if (t < GL) {
      keys[2 * t] = 0x7FFFFFFF;    // running minimum
      keys[2 * t + 1] = (int)0x80000000;  // running maximum
    }
  }
}

__global__ void pq_minmax_kernel(const void* z, int bf16, long long n, int L,
                                 const long long* off, int* keys) {
  __shared__ int smin[PQ_THREADS], smax[PQ_THREADS];
  int mn = 0x7FFFFFFF, mx = (int)0x80000000;
  PQ_FOR_ELEMENTS({
    const float v = load_z(z, bf16, e);
    if (isfinite(v)) {  // a non-finite latent takes no part in training
      mn = min(mn, order_key(v));
      mx = max(mx, order_key(v));
    }
  });
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  if ((int)threadIdx.x < L) {  // fold the block's rows of dimension threadIdx.x
    const int R = PQ_THREADS / L;
    for (int t = 1; t < R; ++t) {
      mn = min(mn, smin[threadIdx.x + t * L]);
      mx = max(mx, smax[threadIdx.x + t * L]);
    }
    const int gd = blockIdx.y * L + threadIdx.x;
    atomicMin(&keys[2 * gd], mn);
    atomicMax(&keys[2 * gd + 1], mx);
  }
}

// start centroids and the fixed-point scale of each (group, dimension)
__global__ void pq_init_kernel(const int* keys, const long long* off, long long n, int G, int L,
                               int k, float* table, int* shift) {
  const int gd = blockIdx.x * blockDim.x + threadIdx.x;
  if (gd >= G * L) return;
  const int g = gd / L;
  const long long ng = group_hi(off, g, n) - group_lo(off, g, n);
  float* c = table + (long long)gd * k;
  if (ng <= 0) {
    for (int j = 0; j < k; ++j) c[j] = 0.f;
    shift[gd] = 0;
    return;
  }
  if (keys[2 * gd] > keys[2 * gd + 1]) {  // no finite value in the column
    for (int j = 0; j < k; ++j) c[j] = 0.f;
    shift[gd] = 0;
    return;
  }
  const double lo = (double)key_value(keys[2 * gd]), hi = (double)key_value(keys[2 * gd + 1]);
  for (int j = 0; j < k; ++j) c[j] = __double2float_rn(lo + (j + 0.5) * (hi - lo) / k);
  // |value| < 2^e; the sum of ng values stays below 2^62
  const double amax = fmax(fabs(lo), fabs(hi));
  int e = 0;
  if (amax > 0.0) frexp(amax, &e);
  int lg = 0;
  while (lg < 40 && (1ll << lg) < ng) ++lg;
  int s = 62 - lg - e;
  if (s > 1000) s = 1000;
  shift[gd] = amax > 0.0 ? s : 0;
}

// assign every value to its nearest centroid and add it to the cluster's
// fixed-point sum (shared-memory totals of the block, then one global add
// per cluster)
__global__ void pq_accum_kernel(const void* z, int bf16, long long n, int L, const long long* off,
                                int k, const float* table, const int* shift, long long* acc,
                                unsigned long long* cnt) {
  // rows of k + 1 entries: the lanes of a warp (consecutive dimensions) read
  // the same centroid index j in different banks
  extern __shared__ __align__(16) unsigned char sm[];
  const int ks = k + 1;
  float* c = reinterpret_cast<float*>(sm);                                  // [L][k + 1]
  long long* sacc = reinterpret_cast<long long*>(c + ((L * ks + 1) & ~1));  // [L][k + 1]
  unsigned long long* scnt = reinterpret_cast<unsigned long long*>(sacc + L * ks);
  const int g = blockIdx.y;
  for (int t = threadIdx.x; t < L * k; t += blockDim.x) {
    const int dd = t / k, j = t - dd * k;
    c[dd * ks + j] = table[(long long)g * L * k + t];
    sacc[dd * ks + j] = 0;
    scnt[dd * ks + j] = 0;
  }
  __syncthreads();
  const int dd = threadIdx.x % L;
  const double sc = ldexp(1.0, shift[g * L + dd]);
  PQ_FOR_ELEMENTS({
    const float v = load_z(z, bf16, e);
    if (isfinite(v)) {
      const int j = nearest(v, c + d * ks, k);
      atomicAdd(reinterpret_cast<unsigned long long*>(&sacc[d * ks + j]),
                (unsigned long long)__double2ll_rn((double)v * sc));
      atomicAdd(&scnt[d * ks + j], 1ull);
    }
  });
  __syncthreads();
  for (int t = threadIdx.x; t < L * k; t += blockDim.x) {
    const int dd = t / k, j = t - dd * k;
    if (scnt[dd * ks + j]) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&acc[(long long)g * L * k + t]),
                (unsigned long long)sacc[dd * ks + j]);
      atomicAdd(&cnt[(long long)g * L * k + t], scnt[dd * ks + j]);
    }
  }
}

__global__ void pq_update_kernel(int GL, int k, const int* shift, long long* acc,
                                 unsigned long long* cnt, float* table) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= GL * k) return;
  if (cnt[t]) {
    const double mean = ldexp((double)acc[t] / (double)cnt[t], -shift[t / k]);
    table[t] = __double2float_rn(mean);
  }
  acc[t] = 0;
  cnt[t] = 0;
}

__global__ void pq_encode_kernel(const void* z, int bf16, long long n, int L, const long long* off,
                                 int k, const float* table, uint8_t* codes, void* zq) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* c = reinterpret_cast<float*>(sm);  // [L][k + 1], as in pq_accum_kernel
  const int ks = k + 1;
  const int g = blockIdx.y;
  for (int t = threadIdx.x; t < L * k; t += blockDim.x) {
    const int dd = t / k;
    c[dd * ks + (t - dd * k)] = table[(long long)g * L * k + t];
  }
  __syncthreads();
  PQ_FOR_ELEMENTS({
    const float v = load_z(z, bf16, e);
    const int j = nearest(v, c + d * ks, k);
    if (codes) codes[e] = (uint8_t)j;
    if (zq) store_z(zq, bf16, e, c[d * ks + j]);
  });
}

__global__ void pq_decode_kernel(const uint8_t* codes, long long n, int L, const long long* off,
                                 int k, const float* table, int bf16, void* z) {
  PQ_FOR_ELEMENTS({
    const int j = codes[e];
    store_z(z, bf16, e, j < k ? table[((long long)g * L + d) * k + j] : 0.f);
  });
}

int pq_check(int32_t latent_dtype, int64_t n, int32_t L, int32_t G, int32_t k) {
  AEQC_CHECK_ARG(latent_dtype == AEQC_DTYPE_F32 || latent_dtype == AEQC_DTYPE_BF16,
                 "pq: latent dtype %d", latent_dtype);
  AEQC_CHECK_ARG(n >= 0, "pq: n < 0");
  AEQC_CHECK_ARG(L >= 1 && L <= PQ_THREADS, "pq: L=%d out of range", L);
  AEQC_CHECK_ARG(G >= 1 && G <= 65535, "pq: G=%d out of range", G);
  AEQC_CHECK_ARG(k >= 2 && k <= AEQC_PQ_MAX_K, "pq: k=%d out of range", k);
  return AEQC_OK;
}

dim3 pq_grid(int G) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int c = (8 * sms + G - 1) / G;
  if (c < 1) c = 1;
  if (c > 4096) c = 4096;
  return dim3((unsigned)c, (unsigned)G);
}

size_t accum_smem(int L, int k) {
  const size_t e = (size_t)L * (k + 1);
  return sizeof(float) * ((e + 1) & ~(size_t)1) + 16 * e;
}

}  // namespace
}  // namespace aeqc

using namespace aeqc;

extern "C" size_t pq_train_workspace_size(int32_t G, int32_t L, int32_t k) {
  if (G < 1 || L < 1 || k < 2) return 0;
  WsSize w;
  const size_t GL = (size_t)G * L;
  w.add<int>(2 * GL);
  w.add<int>(GL);
  w.add<long long>(GL * k);
  w.add<unsigned long long>(GL * k);
  return w.bytes;
}

extern "C" int pq_train(const void* z, int32_t latent_dtype, int64_t n, int32_t L,
                        const int64_t* group_offsets, int32_t G, int32_t k, int32_t iters,
                        float* table, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  int rc = pq_check(latent_dtype, n, L, G, k);
  if (rc) return rc;
  AEQC_CHECK_ARG(table && workspace && (z || n == 0), "pq_train: null pointer");
  AEQC_CHECK_ARG(G == 1 || group_offsets, "pq_train: G > 1 needs group_offsets");
  AEQC_CHECK_ARG(iters >= 0 && iters <= 10000, "pq_train: iters=%d", iters);
  AEQC_CHECK_ARG(workspace_bytes >= pq_train_workspace_size(G, L, k),
                 "pq_train: workspace too small");
  const size_t sm = accum_smem(L, k);
  AEQC_CHECK_ARG(sm <= 200 * 1024, "pq_train: L * k = %d too large", L * k);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long* off = reinterpret_cast<const long long*>(group_offsets);
  const int GL = G * L, bf16 = latent_dtype == AEQC_DTYPE_BF16;
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  int* keys = c.take<int>(2 * (size_t)GL);
  int* shift = c.take<int>(GL);
  long long* acc = c.take<long long>((size_t)GL * k);
  unsigned long long* cnt = c.take<unsigned long long>((size_t)GL * k);
  AEQC_CHECK_ARG(c.ok(), "pq_train: workspace not 256-byte aligned");
  const int nb = (GL * k + 255) / 256;
  pq_clear_kernel<<<nb, 256, 0, s>>>(keys, acc, cnt, GL, k);
  const dim3 grid = pq_grid(G);
  pq_minmax_kernel<<<grid, PQ_THREADS, 0, s>>>(z, bf16, n, L, off, keys);
  pq_init_kernel<<<(GL + 127) / 128, 128, 0, s>>>(keys, off, n, G, L, k, table, shift);
  rc = check_launch("pq_init_kernel");
  if (rc) return rc;
  if (sm > 48 * 1024) {
    rc = raise_smem_limit((const void*)pq_accum_kernel, (int)sm);
    if (rc) return rc;
  }
  for (int it = 0; it < iters; ++it) {
    pq_accum_kernel<<<grid, PQ_THREADS, sm, s>>>(z, bf16, n, L, off, k, table, shift, acc, cnt);
    pq_update_kernel<<<nb, 256, 0, s>>>(GL, k, shift, acc, cnt, table);
  }
  return check_launch("pq_accum_kernel");
}

extern "C" int pq_encode(const void* z, int32_t latent_dtype, int64_t n, int32_t L,
                         const int64_t* group_offsets, int32_t G, int32_t k, const float* table,
                         uint8_t* codes, void* zq, void* stream) {
  clear_error();
  int rc = pq_check(latent_dtype, n, L, G, k);
  if (rc) return rc;
  AEQC_CHECK_ARG(table && (z || n == 0) && (codes || zq), "pq_encode: null pointer");
  AEQC_CHECK_ARG(G == 1 || group_offsets, "pq_encode: G > 1 needs group_offsets");
  if (n == 0) return AEQC_OK;
  const size_t sm = sizeof(float) * (size_t)L * (k + 1);
  AEQC_CHECK_ARG(sm <= 200 * 1024, "pq_encode: L * k = %d too large", L * k);
  if (sm > 48 * 1024) {
    rc = raise_smem_limit((const void*)pq_encode_kernel, (int)sm);
    if (rc) return rc;
  }
  pq_encode_kernel<<<pq_grid(G), PQ_THREADS, sm, static_cast<cudaStream_t>(stream)>>>(
      z, latent_dtype == AEQC_DTYPE_BF16, n, L, reinterpret_cast<const long long*>(group_offsets),
      k, table, codes, zq);
  return check_launch("pq_encode_kernel");
}

extern "C" int pq_decode(const uint8_t* codes, int64_t n, int32_t L, const int64_t* group_offsets,
                         int32_t G, int32_t k, const float* table, int32_t latent_dtype, void* z,
                         void* stream) {
  clear_error();
  int rc = pq_check(latent_dtype, n, L, G, k);
  if (rc) return rc;
  AEQC_CHECK_ARG(table && ((codes && z) || n == 0), "pq_decode: null pointer");
  AEQC_CHECK_ARG(G == 1 || group_offsets, "pq_decode: G > 1 needs group_offsets");
  if (n == 0) return AEQC_OK;
  pq_decode_kernel<<<pq_grid(G), PQ_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
      codes, n, L, reinterpret_cast<const long long*>(group_offsets), k, table,
      latent_dtype == AEQC_DTYPE_BF16, z);
  return check_launch("pq_decode_kernel");
}
