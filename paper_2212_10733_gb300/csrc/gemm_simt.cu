// FP32 SIMT GEMM for the autoencoder's dense layers (y = W^T x + b, Sec. IV-B)
// in the plain FP32 form, and for the training products behind the gradient
// of Eq. (5).  C[m][n] = epilogue(sum_k A(m,k) B(k,n)) with strided operands,
// 128x128x8 CTA tiles, 8x8 outputs per thread, register-prefetched double
// buffering.  Grouped: rows are split into groups (subdomains) that each use
// their own B and bias; no tile straddles two groups.
#include "gemm_simt.cuh"

namespace aeqc {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

// the narrow-layer kernel below takes the row-scale layer with N <= 8
#define A_NARROW_OK(a)                                                                    \
  ((a).a_f64 && (a).epi == EPI_ROWSCALE_BIAS_ACT && (a).N <= 8 && (a).sak == 1 &&         \
   (a).M < (1ll << 36))

__device__ __forceinline__ float act_apply(int act, float v) {
  return act == AEQC_ACT_RELU ? fmaxf(v, 0.f) : v;
}

// Tile t of the launch -> (group, first row, end row of the group).
__device__ __forceinline__ bool tile_of(const GemmArgs& a, long long t, int* g, long long* r0,
                                        long long* rend) {
  if (a.n_groups <= 1) {
    *g = 0;
    *r0 = t * BM;
    *rend = a.M;
    return *r0 < a.M;
  }
  int lo = 0, hi = a.n_groups;
  if (t >= a.tile_off[hi]) return false;
  while (hi - lo > 1) {  // last group whose first tile <= t
    int mid = (lo + hi) >> 1;
    if (a.tile_off[mid] <= t) lo = mid;
    else hi = mid;
  }
  *g = lo;
  *r0 = a.group_off[lo] + (t - a.tile_off[lo]) * BM;
  *rend = a.group_off[lo + 1];
  return true;
}

template <bool A_F64>
__global__ void __launch_bounds__(NT, 2) gemm_kernel(const GemmArgs a) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  __shared__ double rowmax_s[BM];

  int g;
  long long r0, rend;
  if (!tile_of(a, blockIdx.y, &g, &r0, &rend)) return;
  const int n0 = blockIdx.x * BN;
  const float* B = a.B + (long long)g * a.group_stride_B;
  const float* bias = a.bias ? a.bias + (long long)g * a.group_stride_bias : nullptr;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // loader mapping, 128 rows x 8 k, 4 elements per thread:
  //   k-contiguous operand:   row = tid/2, k = (tid&1)*4 + e
  //   row-contiguous operand: k = tid/32, row = (tid&31)*4 + e
  const bool a_kc = A_F64 || a.sak == 1;
  const bool b_kc = a.sbk == 1;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float ra[4], rb[4];
  double rmax = 0.0;

  auto load_a = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int r, k;
      if (a_kc) {
        r = tid >> 1;
        k = (tid & 1) * 4 + e;
      } else {
        k = tid >> 5;
        r = (tid & 31) * 4 + e;
      }
      long long gr = r0 + r;
      int gk = k0 + k;
      float v = 0.f;
      if (gr < rend && gk < a.K) {
        if (A_F64) {
          double d = static_cast<const double*>(a.A)[gr * a.sam + (long long)gk * a.sak];
          if (d > rmax) rmax = d;  // max(x) semantics: NaN and negatives never win
          v = (float)d;
        } else {
          v = static_cast<const float*>(a.A)[gr * a.sam + (long long)gk * a.sak];
        }
      }
      ra[e] = v;
    }
  };
  auto load_b = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int c, k;
      if (b_kc) {
        c = tid >> 1;
        k = (tid & 1) * 4 + e;
      } else {
        k = tid >> 5;
        c = (tid & 31) * 4 + e;
      }
      int gc = n0 + c, gk = k0 + k;
      rb[e] = (gc < a.N && gk < a.K) ? B[(long long)gk * a.sbk + (long long)gc * a.sbn] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (a_kc) As[buf][(tid & 1) * 4 + e][tid >> 1] = ra[e];
      else As[buf][tid >> 5][(tid & 31) * 4 + e] = ra[e];
      if (b_kc) Bs[buf][(tid & 1) * 4 + e][tid >> 1] = rb[e];
      else Bs[buf][tid >> 5][(tid & 31) * 4 + e] = rb[e];
    }
  };

  const int nk = (a.K + BK - 1) / BK;
  load_a(0);
  load_b(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load_a((kt + 1) * BK);
      load_b((kt + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }

  if (A_F64) {
    // the two loader threads of a row combine their partial maxima
    double o = __shfl_xor_sync(0xffffffffu, rmax, 1);
    rmax = o > rmax ? o : rmax;
    if ((tid & 1) == 0) {
      rowmax_s[tid >> 1] = rmax;
      long long gr = r0 + (tid >> 1);
      if (a.scale_out && blockIdx.x == 0 && gr < rend) a.scale_out[gr] = rmax;
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    const long long gr = r0 + r;
    if (gr >= rend) continue;
    float rs = 1.f;
    if (a.epi == EPI_DENORM) rs = (float)a.scale_in[gr];
    if (A_F64) {
      double s = rowmax_s[r];
      rs = (s > 0.0 && isfinite(s)) ? (float)(1.0 / s) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
      const int gc = n0 + c;
      if (gc >= a.N) continue;
      float v = acc[i][j];
      float* dst = a.C + gr * a.ldc + gc;
      const float bb = bias ? bias[gc] : 0.f;
      switch (a.epi) {
        case EPI_PLAIN:
          v = a.beta != 0.f ? fmaf(a.alpha, v, a.beta * *dst) : a.alpha * v;
          break;
        case EPI_BIAS_ACT:
          v = act_apply(a.act, v + bb);
          break;
        case EPI_ROWSCALE_BIAS_ACT:
          v = act_apply(a.act, fmaf(v, rs, bb));
          break;
        default:  // EPI_DENORM
          v = rs * (v + bb);
          break;
      }
      *dst = v;
    }
  }
}

__global__ void tile_offsets_kernel(const long long* group_off, int G, int tile_rows,
                                     int* tile_off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  tile_off[0] = 0;
  for (int g = 0; g < G; ++g) {
    long long rows = group_off[g + 1] - group_off[g];
    acc += (int)((rows + tile_rows - 1) / tile_rows);
    tile_off[g + 1] = acc;
  }
}

}  // namespace

// The first encoder layer of a narrow network (N <= 8 outputs, FP64 input
// rows with unit stride, the row-scale epilogue): the 128 x 128 tiles above
// would leave most of their FMAs idle, so one warp takes one row instead:
// lanes stride over k, accumulate N products each and the row maximum (on the
// bit patterns: non-negative doubles up to +inf order like their bits, so the
// maximum over them and +0 is the FP64 "d > max" maximum, NaN and negatives
// never winning), then reduce across the warp.  Same epilogue as above.
template <int NN>
__global__ void __launch_bounds__(256) rowscale_narrow_kernel(const GemmArgs a) {
  const int lane = threadIdx.x & 31;
  const long long m = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (m >= a.M) return;
  int g = 0;
  if (a.n_groups > 1) {  // last group whose first row <= m
    int lo = 0, hi = a.n_groups;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.group_off[mid] <= m) lo = mid;
      else hi = mid;
    }
    g = lo;
  }
  const double* Ar = static_cast<const double*>(a.A) + m * a.sam;
  const float* B = a.B + (long long)g * a.group_stride_B;
  const float* bias = a.bias ? a.bias + (long long)g * a.group_stride_bias : nullptr;
  float acc[NN];
#pragma unroll
  for (int n = 0; n < NN; ++n) acc[n] = 0.f;
  unsigned long long kmax = 0ull;  // +0
  for (int k = lane; k < a.K; k += 32) {
    const double d = __ldg(Ar + k);
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    if (u <= 0x7FF0000000000000ull && u > kmax) kmax = u;
    const float v = (float)d;
#pragma unroll
    for (int n = 0; n < NN; ++n)
      if (n < a.N) acc[n] = fmaf(v, __ldg(B + (long long)k * a.sbk + (long long)n * a.sbn), acc[n]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ko = __shfl_xor_sync(0xffffffffu, kmax, o);
    kmax = ko > kmax ? ko : kmax;
#pragma unroll
    for (int n = 0; n < NN; ++n) acc[n] += __shfl_xor_sync(0xffffffffu, acc[n], o);
  }
  const double sm = __longlong_as_double((long long)kmax);
  const float rs = (sm > 0.0 && isfinite(sm)) ? (float)(1.0 / sm) : 0.f;
  if (lane == 0 && a.scale_out) a.scale_out[m] = sm;
#pragma unroll
  for (int n = 0; n < NN; ++n)
    if (lane == n && n < a.N)
      a.C[m * a.ldc + n] = act_apply(a.act, fmaf(acc[n], rs, bias ? __ldg(bias + n) : 0.f));
}

// The last decoder layer of a narrow network (K <= 8 inputs, the denormalising
// epilogue): one warp per row, the row's K inputs held by every lane, lanes
// over the output columns (coalesced stores); each output sums its K
// products in k order from zero, as the tiled kernel does.
template <int KK>
__global__ void __launch_bounds__(256) denorm_narrow_kernel(const GemmArgs a) {
  const int lane = threadIdx.x & 31;
  const long long m = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (m >= a.M) return;
  int g = 0;
  if (a.n_groups > 1) {
    int lo = 0, hi = a.n_groups;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.group_off[mid] <= m) lo = mid;
      else hi = mid;
    }
    g = lo;
  }
  const float* Ar = static_cast<const float*>(a.A) + m * a.sam;
  const float* B = a.B + (long long)g * a.group_stride_B;
  const float* bias = a.bias ? a.bias + (long long)g * a.group_stride_bias : nullptr;
  float av[KK];
#pragma unroll
  for (int k = 0; k < KK; ++k) av[k] = k < a.K ? __ldg(Ar + k) : 0.f;
  const float rs = (float)a.scale_in[m];
  float* Cr = a.C + m * a.ldc;
  for (int n = lane; n < a.N; n += 32) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < KK; ++k)
      if (k < a.K) acc = fmaf(av[k], __ldg(B + (long long)k * a.sbk + (long long)n * a.sbn), acc);
    Cr[n] = rs * (acc + (bias ? __ldg(bias + n) : 0.f));
  }
}

// A layer of at most 8 inputs and 8 outputs (the narrow network's middle
// layers): one thread per row, each output summing its K products in k order
// from zero, as the tiled kernel does.
__global__ void __launch_bounds__(256) bias_act_tiny_kernel(const GemmArgs a) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.M) return;
  int g = 0;
  if (a.n_groups > 1) {
    int lo = 0, hi = a.n_groups;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.group_off[mid] <= m) lo = mid;
      else hi = mid;
    }
    g = lo;
  }
  const float* Ar = static_cast<const float*>(a.A) + m * a.sam;
  const float* B = a.B + (long long)g * a.group_stride_B;
  const float* bias = a.bias ? a.bias + (long long)g * a.group_stride_bias : nullptr;
  float av[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) av[k] = k < a.K ? Ar[k] : 0.f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    if (n >= a.N) break;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < a.K) acc = fmaf(av[k], __ldg(B + (long long)k * a.sbk + (long long)n * a.sbn), acc);
    a.C[m * a.ldc + n] = act_apply(a.act, acc + (bias ? __ldg(bias + n) : 0.f));
  }
}

int launch_gemm(const GemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return AEQC_OK;
  if (!a.a_f64 && a.epi == EPI_BIAS_ACT && a.N <= 8 && a.K <= 8 && a.sak == 1 &&
      a.M < (1ll << 40)) {
    bias_act_tiny_kernel<<<(unsigned)((a.M + 255) / 256), 256, 0, s>>>(a);
    return check_launch("bias_act_tiny_kernel");
  }
  if (!a.a_f64 && a.epi == EPI_DENORM && a.K <= 8 && a.sak == 1 && a.M < (1ll << 36)) {
    const unsigned blocks = (unsigned)((a.M + 7) / 8);
    if (a.K <= 4) denorm_narrow_kernel<4><<<blocks, 256, 0, s>>>(a);
    else denorm_narrow_kernel<8><<<blocks, 256, 0, s>>>(a);
    return check_launch("denorm_narrow_kernel");
  }
  if (A_NARROW_OK(a)) {
    const unsigned blocks = (unsigned)((a.M + 7) / 8);
    if (a.N <= 4) rowscale_narrow_kernel<4><<<blocks, 256, 0, s>>>(a);
    else rowscale_narrow_kernel<8><<<blocks, 256, 0, s>>>(a);
    return check_launch("rowscale_narrow_kernel");
  }
  long long tiles = a.n_groups <= 1 ? (a.M + BM - 1) / BM : a.max_tiles;
  if (tiles > 2147483647LL || tiles > 65535LL * 65535LL)
    return set_error(AEQC_EUNSUPPORTED, "gemm: too many row tiles");
  dim3 grid((a.N + BN - 1) / BN, (unsigned)tiles);
  if (tiles > 65535) {
    // grid.y is limited to 65535: split into several launches over row ranges
    GemmArgs b = a;
    if (a.n_groups > 1)
      return set_error(AEQC_EUNSUPPORTED, "gemm: grouped launch with > 65535 tiles");
    for (long long t0 = 0; t0 < tiles; t0 += 65535) {
      long long nt = tiles - t0 < 65535 ? tiles - t0 : 65535;
      long long row0 = t0 * BM;
      b.M = a.M - row0;
      b.A = a.a_f64 ? (const void*)(static_cast<const double*>(a.A) + row0 * a.sam)
                    : (const void*)(static_cast<const float*>(a.A) + row0 * a.sam);
      b.C = a.C + row0 * a.ldc;
      b.scale_out = a.scale_out ? a.scale_out + row0 : nullptr;
      b.scale_in = a.scale_in ? a.scale_in + row0 : nullptr;
      dim3 g2(grid.x, (unsigned)nt);
      if (a.a_f64) gemm_kernel<true><<<g2, NT, 0, s>>>(b);
      else gemm_kernel<false><<<g2, NT, 0, s>>>(b);
      int rc = check_launch("gemm_kernel");
      if (rc != AEQC_OK) return rc;
    }
    return AEQC_OK;
  }
  if (a.a_f64) gemm_kernel<true><<<grid, NT, 0, s>>>(a);
  else gemm_kernel<false><<<grid, NT, 0, s>>>(a);
  return check_launch("gemm_kernel");
}

int launch_tile_offsets(const long long* group_off, int n_groups, int tile_rows,
                        int* tile_off, cudaStream_t s) {
  tile_offsets_kernel<<<1, 32, 0, s>>>(group_off, n_groups, tile_rows, tile_off);
  return check_launch("tile_offsets_kernel");
}

}  // namespace aeqc
