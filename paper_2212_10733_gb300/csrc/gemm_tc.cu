// Training products of the BF16 model on the 5th-generation tensor cores:
// the forward layers and the gradient products of Eq. (5) (Sec. III Stage 2,
// Adam with FP32 master weights, Sec. IV-B).  C = epi(op(A) op(B)) with FP32
// operands in any strides: eight loading warps round them to BF16 and write
// 128 x 64 tiles in the 128-byte-swizzled K-major layout of the shared-memory
// descriptors (coalesced along whichever operand index has unit stride), one
// thread issues tcgen05.mma (M = 128, N = 128, K = 16) into an FP32
// accumulator in tensor memory, and the loading warps apply the epilogue.
// Rows or columns past M, N and the K tail are zero in the tiles.
#include <cuda_bf16.h>

#include "gemm_tc.cuh"
#include "tc_ptx.cuh"

namespace aeqc {
namespace {

using namespace tc;

constexpr int TBM = 128;                  // rows of C per CTA
constexpr int TBN = 128;                  // columns of C per CTA (one MMA N)
constexpr int TKB = 64;                   // K per stage
constexpr int TNS = 3;                    // stages
constexpr int TLOAD = 8;                  // loading / epilogue warps
constexpr int TTHREADS = (TLOAD + 1) * 32;
constexpr uint32_t T_TILE = 128 * 128;    // one 128 x 64 BF16 tile

struct TcGemm {
  int M, N, K;
  const float* A;
  long long sam, sak;  // A(m, k) = A[m sam + k sak]
  const float* B;
  long long sbk, sbn;  // B(k, n) = B[k sbk + n sbn]
  float* C;
  long long ldc;
  int bias_act, act;   // 1: C = act(acc + bias[n]); 0: C = alpha acc + beta C
  const float* bias;
  float alpha, beta;
  int kbs;             // K blocks per split (blockIdx.z)
  float* part;         // split K: raw FP32 tiles [split][M][N], else null
  int* err;
};

// tile rows r0 + r (r < 128), columns k0 + k (k < 64): element
// src[(r0 + r) sr + (k0 + k) sk] rounded to BF16, zero outside R x K
__device__ __forceinline__ void fill_tile(uint8_t* dst, const float* src, long long sr,
                                          long long sk, int r0, int R, int k0, int K, int t) {
  const bool kfast = sk == 1;  // consecutive threads on consecutive k, else on consecutive r
  constexpr int PER = 128 * TKB / (TLOAD * 32);
  // every load of the tile in flight before the first store
  float v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = t + i * (TLOAD * 32);
    const int r = kfast ? idx >> 6 : idx & 127;
    const int k = kfast ? idx & 63 : idx >> 7;
    const int gr = r0 + r, gk = k0 + k;
    v[i] = gr < R && gk < K ? __ldg(src + (long long)gr * sr + (long long)gk * sk) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = t + i * (TLOAD * 32);
    const int r = kfast ? idx >> 6 : idx & 127;
    const int k = kfast ? idx & 63 : idx >> 7;
    *reinterpret_cast<__nv_bfloat16*>(dst + swz128(r, k >> 3) + (k & 7) * 2) =
        __float2bfloat16_rn(v[i]);
  }
}

__global__ void __launch_bounds__(TTHREADS, 1) gemm_tc_kernel(const TcGemm a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                           ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TNS * 2 * T_TILE);
  uint64_t* empty = full + TNS;
  uint64_t* acc_full = empty + TNS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
  // this CTA's K blocks (split K: a range of them, never empty)
  const int kb_lo = blockIdx.z * a.kbs;
  const int kb_hi = min((a.K + TKB - 1) / TKB, kb_lo + a.kbs);
  const int nk = kb_hi - kb_lo;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TNS; ++s) {
      mbar_init(&full[s], TLOAD * 32);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    fence_barrier_init();
  }
  if (warp == TLOAD) tmem_alloc(tmem_slot, TBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == TLOAD) {
    if (lane == 0) {
      const uint32_t id = idesc_bf16(TBM, TBN);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % TNS;
        if (!mbar_wait(&full[s], (kb / TNS) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ab = smem_u32(sm + s * 2 * T_TILE), bb = ab + T_TILE;
#pragma unroll
        for (int kk = 0; kk < TKB / 16; ++kk)
          mma_bf16(tmem, desc_k128(ab + kk * 32), desc_k128(bb + kk * 32), id, (kb | kk) != 0);
        mma_commit(&empty[s]);
      }
      // arrives once every MMA issued above has completed
      mma_commit(acc_full);
      if (!ok) atomicExch(a.err, 1);
    }
    __syncwarp();
  } else {
    const int t = threadIdx.x;
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TNS;
      if (kb >= TNS && !mbar_wait(&empty[s], ((kb / TNS) & 1) ^ 1)) {
        ok = false;
        break;
      }
      uint8_t* at = sm + s * 2 * T_TILE;
      fill_tile(at, a.A, a.sam, a.sak, m0, a.M, (kb_lo + kb) * TKB, a.K, t);
      fill_tile(at + T_TILE, a.B, a.sbn, a.sbk, n0, a.N, (kb_lo + kb) * TKB, a.K, t);
      fence_proxy_async_smem();
      tc_fence_before();
      mbar_arrive(&full[s]);
    }
    if (ok && !mbar_wait(acc_full, 0)) ok = false;
    if (ok) {
      tc_fence_after();
      // every MMA has completed: the stages serve as transposition blocks
      // (32 x 33 floats per warp), so that each store instruction writes 32
      // consecutive columns of one row
      const int q = warp & 3, half = warp >> 2;
      float* stg = reinterpret_cast<float*>(sm) + warp * 32 * 33;
      for (int c = half * (TBN / 2); c < (half + 1) * (TBN / 2); c += 32) {
        if (n0 + c >= a.N) break;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[i];
        __syncwarp();
        const int n = n0 + c + lane;
        const float bn = a.bias_act && a.bias && n < a.N ? __ldg(a.bias + n) : 0.f;
        for (int rr = 0; rr < 32; ++rr) {
          const int m = m0 + q * 32 + rr;
          if (m < a.M && n < a.N) {
            float val = stg[rr * 33 + lane];
            if (a.part) {  // split K: the raw sum of this K range
              a.part[((long long)blockIdx.z * a.M + m) * a.N + n] = val;
              continue;
            }
            float* cp = a.C + (long long)m * a.ldc + n;
            if (a.bias_act) {
              val += bn;
              if (a.act == AEQC_ACT_RELU) val = fmaxf(val, 0.f);
            } else {
              val = a.beta != 0.f ? fmaf(a.alpha, val, a.beta * *cp) : a.alpha * val;
            }
            *cp = val;
          }
        }
        __syncwarp();
      }
    }
    if (!ok) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TLOAD) {
    tc_fence_after();
    tmem_dealloc(tmem, TBN);
  }
}

// split K: C = epi(sum over the splits of the partial tiles), summed in split
// order (deterministic)
__global__ void splitk_reduce_kernel(const TcGemm a, int splits) {
  const long long mn = (long long)a.M * a.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < mn;
       i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += a.part[z * mn + i];
    const int m = (int)(i / a.N), n = (int)(i - (long long)m * a.N);
    float* cp = a.C + (long long)m * a.ldc + n;
    if (a.bias_act) {
      acc += a.bias ? __ldg(a.bias + n) : 0.f;
      if (a.act == AEQC_ACT_RELU) acc = fmaxf(acc, 0.f);
    } else {
      acc = a.beta != 0.f ? fmaf(a.alpha, acc, a.beta * *cp) : a.alpha * acc;
    }
    *cp = acc;
  }
}

int launch_tc(TcGemm a, float* scratch, long long scratch_elems, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return AEQC_OK;
  const int smem = TNS * 2 * T_TILE + 8 * (2 * TNS + 1) + 16 + 1024;
  {
    const int rc = raise_smem_limit((const void*)gemm_tc_kernel, smem);
    if (rc) return rc;
  }
  const int gx = (a.M + TBM - 1) / TBM, gy = (a.N + TBN - 1) / TBN;
  const int nk = (a.K + TKB - 1) / TKB;
  // few output tiles and a long K (the products with 128 batch rows and
  // K = P or H): split K over more CTAs, at least two K blocks each, as far as
  // the scratch holds the partial tiles
  int splits = 1;
  if (nk >= 4 && gx * gy < 64) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    splits = min(nk / 2, (sms + gx * gy - 1) / (gx * gy));
    const long long mn = (long long)a.M * a.N;
    if (scratch == nullptr || mn <= 0) splits = 1;
    else if ((long long)splits * mn > scratch_elems) splits = (int)(scratch_elems / mn);
    if (splits < 2) splits = 1;
  }
  a.kbs = (nk + splits - 1) / splits;
  splits = nk > 0 ? (nk + a.kbs - 1) / a.kbs : 1;  // no empty split
  a.part = splits > 1 ? scratch : nullptr;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)splits);
  gemm_tc_kernel<<<grid, TTHREADS, smem, s>>>(a);
  int rc = check_launch("gemm_tc_kernel");
  if (rc || splits == 1) return rc;
  const long long mn = (long long)a.M * a.N;
  const long long nb = (mn + 255) / 256 < 4096 ? (mn + 255) / 256 : 4096;
  splitk_reduce_kernel<<<(unsigned)nb, 256, 0, s>>>(a, splits);
  return check_launch("splitk_reduce_kernel");
}

}  // namespace

int gemm_tc_plain(long long M, int N, int K, const float* A, long long sam, long long sak,
                  const float* B, long long sbk, long long sbn, float* C, long long ldc,
                  float beta, float* scratch, long long scratch_elems, int* err,
                  cudaStream_t s) {
  TcGemm a;
  memset(&a, 0, sizeof(a));
  a.M = (int)M; a.N = N; a.K = K;
  a.A = A; a.sam = sam; a.sak = sak;
  a.B = B; a.sbk = sbk; a.sbn = sbn;
  a.C = C; a.ldc = ldc;
  a.alpha = 1.f;
  a.beta = beta;
  a.err = err;
  return launch_tc(a, scratch, scratch_elems, s);
}

int gemm_tc_bias(long long M, int N, int K, const float* A, long long sam, const float* B,
                 long long sbk, long long sbn, const float* bias, int act, float* C,
                 float* scratch, long long scratch_elems, int* err, cudaStream_t s) {
  TcGemm a;
  memset(&a, 0, sizeof(a));
  a.M = (int)M; a.N = N; a.K = K;
  a.A = A; a.sam = sam; a.sak = 1;
  a.B = B; a.sbk = sbk; a.sbn = sbn;
  a.C = C; a.ldc = N;
  a.bias_act = 1;
  a.act = act;
  a.bias = bias;
  a.alpha = 1.f;
  a.err = err;
  return launch_tc(a, scratch, scratch_elems, s);
}

long long gemm_tc_scratch_elems(long long B, int P, int H) {
  const long long w = 16 * B * (long long)(P > H ? P : H);
  return w < (1ll << 24) ? w : (1ll << 24);
}

}  // namespace aeqc
