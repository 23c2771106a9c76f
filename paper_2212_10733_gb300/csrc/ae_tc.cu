// BF16 autoencoder forward on the 5th-generation tensor cores (Stage 3 of
// Sec. III; the tied linear network of Sec. IV-B): tcgen05.mma with FP32
// accumulators in tensor memory, weights streamed by TMA; persistent kernels
// (one CTA per SM) walking tiles of 128 histograms.
//
// Encoder (one kernel): h = act((x W1') / s + b1') then z = h W2 + b2, with
// W1' = W1 / sigma and b1' = b1 - W1'^T mu folded on the host side, s the
// per-histogram maximum.  The FP64 input rows are read once: eight converter
// warps load them, take the row maximum and write BF16 operand tiles into
// shared memory in the 128-byte-swizzled K-major layout the MMA reads; h goes
// from tensor memory through shared memory (BF16) into the second MMA, so
// neither h nor the BF16 copy of x touches HBM.
//
// Decoder (one kernel): h = act(z W3 + b3) then xhat = s (h W4' + b4'), with
// W4' = sigma W4 and b4' = sigma b4 + mu; h goes from the first layer's
// accumulator back into tensor memory as packed BF16 and is the A operand of
// the second layer, W4 streams through a shared-memory ring, and the output
// tiles of 128 columns are double-buffered in tensor memory; their FP32 rows
// leave through TMA stores, so that the stores of one tile overlap the MMAs of
// the next.
#include <cuda_bf16.h>
#include <string.h>

#include "model.cuh"
#include "tc_ptx.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

using namespace tc;

constexpr int BM = 128;       // rows (histograms) per tile
constexpr int KB = 64;        // K per stage: 64 bf16 = one 128-byte swizzle row
constexpr int NCONV = 8;      // converter / epilogue warps
constexpr int WARP_TMA = 8;   // TMA producer, TMEM owner
constexpr int WARP_MMA = 9;   // MMA issuer
constexpr int NTHREADS = 320;
constexpr uint32_t A_STAGE = BM * 128;  // bytes of one A stage (128 rows x 128 B)
// the encoder: sixteen converter warps (eight rows of each A stage apiece),
// then its TMA and MMA warps
constexpr int ENC_NCONV = 16;
constexpr int ENC_RPW = BM / ENC_NCONV;
constexpr int ENC_WARP_TMA = ENC_NCONV;
constexpr int ENC_WARP_MMA = ENC_NCONV + 1;
constexpr int ENC_NTHREADS = (ENC_NCONV + 2) * 32;

// error word values (device)
constexpr int ERR_TIMEOUT = 1;

__device__ __forceinline__ unsigned long long f64_key(unsigned long long u) {
  // order-preserving map of a double's bits to a signed 64-bit key
  return u ^ (((unsigned long long)((long long)u >> 63)) & 0x7FFFFFFFFFFFFFFFull);
}

// BF16 bits of a double (given as its two 32-bit words), round to nearest
// even (values below the BF16 normal range become zero, above it infinity).
// The high word carries sign, exponent
// and 20 mantissa bits; any set bit of the low word only matters as a sticky
// bit below the rounding position, so it is OR-ed into bit 0 of the high word.
// Round half to even at bit 13 then gives the BF16 significand; the exponent
// is rebiased when it is in the BF16 normal range.
__device__ __forceinline__ uint32_t bf16_of_f64_words(uint32_t hi, uint32_t lo) {
  const uint32_t sign = (hi >> 16) & 0x8000u;
  const uint32_t a = (hi & 0x7FFFFFFFu) | (lo != 0u ? 1u : 0u);
  const uint32_t r = a + 0xFFFu + ((a >> 13) & 1u);
  // the rounded magnitude with the exponent rebased to BF16's: below 128 the
  // value is under the BF16 normal range (flushed to zero), from 0x7F80 up it
  // overflows to infinity; a NaN input (a above infinity's pattern) gives
  // the quiet NaN.  Clamps and selects, not branches, since the zero row of
  // every histogram makes lanes diverge.
  const int t = (int)(r >> 13) - (896 << 7);
  const uint32_t m = t < 128 ? 0u : (uint32_t)min(t, 0x7F80);
  return sign | (a > 0x7FF00000u ? 0x7FC0u : m);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float act_f(int act, float v) {
  return act == AEQC_ACT_RELU ? fmaxf(v, 0.f) : v;
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// tile t -> group, first row, end row (grouped batches: tiles never straddle
// two groups); false for the spare CTAs of a grouped launch
struct TileInfo {
  int g;
  long long m0, mend;
};

__device__ __forceinline__ bool tile_info(int t, long long n, int G, const long long* goff,
                                          const int* toff, TileInfo& ti) {
  if (G <= 1) {
    ti.g = 0;
    ti.m0 = (long long)t * BM;
    ti.mend = n;
    return ti.m0 < n;
  }
  if (t >= toff[G]) return false;
  int lo = 0, hi = G - 1;  // largest g with toff[g] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  ti.g = lo;
  ti.m0 = goff[lo] + (long long)(t - toff[lo]) * BM;
  ti.mend = goff[lo + 1];
  return ti.m0 < ti.mend;
}

struct EncArgs {
  const double* x;
  long long n;
  long long ntiles;  // tiles to walk (grouped: an upper bound, spare tiles skipped)
  int P, Kp, H, L, act, G, ns;
  const long long* goff;
  const int* toff;
  const float* b1;  // enc1b, group stride b1_gs
  long long b1_gs;
  const float* b2;  // b2, group stride b2_gs
  long long b2_gs;
  __nv_bfloat16* latent;
  double* scale;
  int* err;
};

// shared memory of the encoder, offsets from a 1024-byte aligned base
struct EncSmem {
  uint32_t stage_bytes, off_b, w2, rowmax, bars, total;
  __host__ __device__ EncSmem(int H, int L, int ns) {
    const uint32_t b_bytes = (uint32_t)H * 128;
    stage_bytes = A_STAGE + b_bytes;
    off_b = A_STAGE;
    uint32_t o = stage_bytes * ns;
    const uint32_t h1 = (uint32_t)BM * H * 2;  // E2 operand reuses the stages
    if (o < h1) o = h1;
    w2 = o;
    o += (uint32_t)(H / KB) * L * 128;
    rowmax = o;
    o += BM * 8;
    bars = o;
    o += 8 * (3 * ns + 4) + 16;
    total = o;
  }
};

// Persistent: one CTA per SM walks the tiles t = blockIdx.x, + gridDim.x, ...
// (tiles are numbered group by group, so the CTAs working at one time share a
// few groups' weights in L2).  Tensor memory is allocated and the barriers
// initialised once; the stage ring continues across tiles, and the per-tile
// barriers (acc_full, h1_full, w2_full, lat_full) complete once per tile, so
// tile iteration i waits on parity i & 1.  The BF16 h tile of the second MMA
// aliases the stage ring, so the next tile's operand writes (A by the
// converters, W1 and W2 by the TMA warp) start after lat_full of this tile.
__global__ void __launch_bounds__(ENC_NTHREADS, 1)
    enc_tc_kernel(const __grid_constant__ CUtensorMap mapW1,
                  const __grid_constant__ CUtensorMap mapW2, const EncArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                           ~uintptr_t(1023));
  const EncSmem L(a.H, a.L, a.ns);
  const int ns = a.ns;
  uint64_t* full_a = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* full_b = full_a + ns;
  uint64_t* empty = full_b + ns;
  uint64_t* w2_full = empty + ns;
  uint64_t* acc_full = w2_full + 1;
  uint64_t* h1_full = acc_full + 1;
  uint64_t* lat_full = h1_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(lat_full + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* rowmax = reinterpret_cast<double*>(sm + L.rowmax);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = a.H, nkb = a.Kp / KB, nh = (H + 255) / 256, hn = H < 256 ? H : 256;
  const uint32_t tcols = H <= 32 ? 32 : (H <= 64 ? 64 : (H <= 128 ? 128 : (H <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full_a[s], ENC_NCONV * 32);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(w2_full, 1);
    mbar_init(acc_full, 1);
    mbar_init(h1_full, ENC_NCONV * 32);
    mbar_init(lat_full, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == ENC_WARP_TMA) tmem_alloc(tmem_slot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(a.err, ERR_TIMEOUT);
  };

  if (warp == ENC_WARP_TMA) {
    if (lane == 0) {
      prefetch_tmap(&mapW1);
      prefetch_tmap(&mapW2);
      int it = 0;  // stage ring position
      int iter = 0;
      for (long long t = blockIdx.x; t < a.ntiles && !*abort_flag; t += gridDim.x) {
        TileInfo ti;
        if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
        // the previous tile's second MMA has read h (aliasing the stages) and W2
        if (iter > 0 && !mbar_wait(lat_full, (iter - 1) & 1)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(w2_full, (uint32_t)(H / KB) * a.L * 128);
        for (int k2 = 0; k2 < H / KB; ++k2)
          tma_load_3d(sm + L.w2 + k2 * a.L * 128, &mapW2, w2_full, k2 * KB, 0, ti.g);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % ns;
          const uint32_t ph = (it / ns) & 1;
          if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
            ok = false;
            break;
          }
          uint8_t* bst = sm + s * L.stage_bytes + L.off_b;
          mbar_arrive_expect_tx(&full_b[s], (uint32_t)H * 128);
          for (int j = 0; j < nh; ++j)
            tma_load_3d(bst + j * 256 * 128, &mapW1, &full_b[s], kb * KB, j * 256, ti.g);
        }
        if (!ok) {
          fail();
          break;
        }
        ++iter;
      }
    }
    __syncwarp();
  } else if (warp == ENC_WARP_MMA) {
    if (lane == 0) {
      const uint32_t id1 = idesc_bf16(BM, hn);
      const uint32_t id2 = idesc_bf16(BM, a.L);
      int it = 0, iter = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        TileInfo ti;
        if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
        const uint32_t tp = iter & 1;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % ns;
          const uint32_t ph = (it / ns) & 1;
          if (*abort_flag || !mbar_wait(&full_a[s], ph) || !mbar_wait(&full_b[s], ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = smem_u32(sm + s * L.stage_bytes);
          const uint32_t bbase = abase + L.off_b;
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk)
            for (int j = 0; j < nh; ++j)
              mma_bf16(tmem + j * 256, desc_k128(abase + kk * 32),
                       desc_k128(bbase + j * 256 * 128 + kk * 32), id1, (kb | kk) != 0);
          mma_commit(&empty[s]);
        }
        mma_commit(acc_full);
        if (ok && (!mbar_wait(h1_full, tp) || !mbar_wait(w2_full, tp))) ok = false;
        if (ok) {
          tc_fence_after();
          const uint32_t hbase = smem_u32(sm), wbase = smem_u32(sm + L.w2);
          for (int k2 = 0; k2 < H / KB; ++k2)
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk)
              mma_bf16(tmem, desc_k128(hbase + k2 * A_STAGE + kk * 32),
                       desc_k128(wbase + k2 * a.L * 128 + kk * 32), id2, (k2 | kk) != 0);
        }
        mma_commit(lat_full);
        ++iter;
      }
      if (!ok) fail();
    }
    __syncwarp();
  } else {
    // ---- converters / epilogue: sixteen warps, ENC_RPW rows each ----
    const int q = warp & 3, part = warp >> 2;
    const int r = q * 32 + lane;
    // stage and phase of the ring position, advanced by one per K block
    // (no division by the runtime stage count on the converters' path)
    int s_ring = 0, iter = 0;
    uint32_t ph_ring = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      TileInfo ti;
      if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
      const int rows = (int)min((long long)BM, ti.mend - ti.m0);
      const uint32_t tp = iter & 1;
      // FP64 rows -> BF16 swizzled A tiles, row maxima on the raw bits as
      // signed 64-bit integers: exact among non-negative values (which order
      // like their bits) and below any of them for negatives; a row without a
      // non-negative value is redone exactly after the main loop
      long long mraw[ENC_RPW];
#pragma unroll
      for (int i = 0; i < ENC_RPW; ++i) mraw[i] = (long long)0x8000000000000000ull;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = s_ring;
        const uint32_t ph = ph_ring;
        if (++s_ring == ns) {
          s_ring = 0;
          ph_ring ^= 1u;
        }
        if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
          ok = false;
          break;
        }
        uint8_t* ast = sm + s * L.stage_bytes;
        const int k0 = kb * KB + 2 * lane;
        unsigned long long v0[ENC_RPW], v1[ENC_RPW];
#pragma unroll
        for (int i = 0; i < ENC_RPW; ++i) {
          const int rw = warp * ENC_RPW + i;
          v0[i] = 0;
          v1[i] = 0;
          if (rw < rows) {
            const double* xr = a.x + (ti.m0 + rw) * (long long)a.P;
            if (k0 < a.P) v0[i] = (unsigned long long)__double_as_longlong(__ldg(xr + k0));
            if (k0 + 1 < a.P)
              v1[i] = (unsigned long long)__double_as_longlong(__ldg(xr + k0 + 1));
          }
        }
#pragma unroll
        for (int i = 0; i < ENC_RPW; ++i) {
          const int rw = warp * ENC_RPW + i;
          if (k0 < a.P) mraw[i] = max(mraw[i], (long long)v0[i]);
          if (k0 + 1 < a.P) mraw[i] = max(mraw[i], (long long)v1[i]);
          const uint32_t packed =
              bf16_of_f64_words((uint32_t)(v0[i] >> 32), (uint32_t)v0[i]) |
              (bf16_of_f64_words((uint32_t)(v1[i] >> 32), (uint32_t)v1[i]) << 16);
          *reinterpret_cast<uint32_t*>(ast + swz128(rw, lane >> 2) + (lane & 3) * 4) = packed;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        mbar_arrive(&full_a[s]);
      }
      if (!ok) break;
      // row maxima: lanes hold partial maxima of rows warp * ENC_RPW + i
#pragma unroll
      for (int i = 0; i < ENC_RPW; ++i) {
        long long k = mraw[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k = max(k, (long long)__shfl_xor_sync(0xffffffffu, k, o));
        const int rw = warp * ENC_RPW + i;
        if (k < 0 && rw < rows) {
          // no non-negative value: the exact maximum on order-preserving keys
          const double* xr = a.x + (ti.m0 + rw) * (long long)a.P;
          long long kk = (long long)f64_key(0xFFF0000000000000ull);
          for (int p = lane; p < a.P; p += 32)
            kk = max(kk,
                     (long long)f64_key((unsigned long long)__double_as_longlong(__ldg(xr + p))));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            kk = max(kk, (long long)__shfl_xor_sync(0xffffffffu, kk, o));
          k = (long long)f64_key((unsigned long long)kk);
        }
        if (lane == 0) rowmax[rw] = __longlong_as_double(k);
      }
      named_sync(1, ENC_NCONV * 32);
      // ---- E1 epilogue: TMEM -> act(acc / s + b1) -> BF16 swizzled h tile ----
      if (!mbar_wait(acc_full, tp)) {
        ok = false;
        break;
      }
      tc_fence_after();
      {
        const double srow = rowmax[r];
        const float rs = (srow > 0.0 && isfinite(srow)) ? (float)(1.0 / srow) : 0.f;
        const float* b1 = a.b1 + ti.g * a.b1_gs;
        // 32-column slices of h, dealt round robin to the four warps of a
        // lane quarter
        for (int c = part * 32; c < H; c += 4 * 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
          uint8_t* hb = sm + (c / KB) * A_STAGE;
          const int ch0 = (c % KB) / 8;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            uint4 w;
            w.x = pack_bf16(act_f(a.act, fmaf(v[8 * u + 0], rs, __ldg(b1 + c + 8 * u + 0))),
                            act_f(a.act, fmaf(v[8 * u + 1], rs, __ldg(b1 + c + 8 * u + 1))));
            w.y = pack_bf16(act_f(a.act, fmaf(v[8 * u + 2], rs, __ldg(b1 + c + 8 * u + 2))),
                            act_f(a.act, fmaf(v[8 * u + 3], rs, __ldg(b1 + c + 8 * u + 3))));
            w.z = pack_bf16(act_f(a.act, fmaf(v[8 * u + 4], rs, __ldg(b1 + c + 8 * u + 4))),
                            act_f(a.act, fmaf(v[8 * u + 5], rs, __ldg(b1 + c + 8 * u + 5))));
            w.w = pack_bf16(act_f(a.act, fmaf(v[8 * u + 6], rs, __ldg(b1 + c + 8 * u + 6))),
                            act_f(a.act, fmaf(v[8 * u + 7], rs, __ldg(b1 + c + 8 * u + 7))));
            *reinterpret_cast<uint4*>(hb + swz128(r, ch0 + u)) = w;
          }
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      mbar_arrive(h1_full);
      // ---- E2 epilogue: latent = acc + b2 (BF16), scale = s; every converter
      // warp waits for the second MMA, whose operand h aliases the next
      // tile's stages ----
      if (!mbar_wait(lat_full, tp)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (warp < 4) {
        if (!*abort_flag) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16), v);
          if (r < rows) {
            const float* b2 = a.b2 + ti.g * a.b2_gs;
            uint32_t* dst = reinterpret_cast<uint32_t*>(a.latent + (ti.m0 + r) * a.L);
            for (int l = 0; l < a.L; l += 2)
              dst[l >> 1] = pack_bf16(v[l] + __ldg(b2 + l), v[l + 1] + __ldg(b2 + l + 1));
          }
        }
      } else if (warp < 8) {
        const int rr = (warp - 4) * 32 + lane;
        if (rr < rows) a.scale[ti.m0 + rr] = rowmax[rr];
      }
      tc_fence_before();
      ++iter;
    }
    if (!ok) fail();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == ENC_WARP_TMA) {
    tc_fence_after();
    tmem_dealloc(tmem, tcols);
  }
}

// ---------------------------------------------------------------------------
// decoder

struct DecArgs {
  const __nv_bfloat16* latent;
  const double* scale;
  long long n;
  long long ntiles;  // tiles to walk (grouped: an upper bound, spare tiles skipped)
  int P, H, L, act, G, ns;
  const long long* goff;
  const int* toff;
  const __nv_bfloat16* W3;  // dec1B [H][L] per group, group stride w3_gs (elements)
  long long w3_gs;
  const float* b3;  // group stride b3_gs
  long long b3_gs;
  const float* b4;  // dec2b [P], group stride b4_gs
  long long b4_gs;
  float* xhat;
  long long ld;
  int tma;  // 1: full tiles of xhat are written by TMA stores through mapX
  int* err;
};

// Decoder layout: D1 operands (latent tile and one chunk of W3) and the W4
// stage ring in shared memory; h lives in tensor memory (the A operand of
// the second layer).  offsets from a 1024-byte aligned base
constexpr int DNT = 128;                    // output columns per accumulator use
constexpr uint32_t D_STAGE = DNT * 128;     // one W4 stage: 128 rows x 64 bf16 of K
constexpr uint32_t TM_ACC = 256;            // TMEM column of the first accumulator

constexpr uint32_t D_OUT = 32 * 128;        // one output box: 32 rows x 32 FP32

struct DecSmem {
  uint32_t d1a, d1b, stages, stg, bars, total;
  __host__ __device__ explicit DecSmem(int ns) {
    d1a = 0;                 // latent tile: 128 rows x 128 B (K padded to 64)
    d1b = A_STAGE;           // W3 chunk: up to 128 rows x 128 B
    stages = 2 * A_STAGE;    // W4 ring
    uint32_t o = stages + (uint32_t)ns * D_STAGE;
    // per epilogue warp two output boxes in the 128-byte-swizzled layout the
    // TMA store reads (the rows of a partial tile reuse them as a 32 x 33
    // transposition block)
    stg = o;
    o += NCONV * 2 * D_OUT;
    bars = o;
    o += 8 * (2 * ns + 8) + 16;
    total = o;
  }
};

// h (packed BF16) from a tensor-memory accumulator: 32 columns of one row
// per thread, b3 added, activation, two values per 32-bit TMEM column
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T: A in tensor memory, one row per lane, two
// bf16 of K per 32-bit column (even k in the low half), 8 columns per K = 16
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Persistent like the encoder: one CTA per SM walks the tiles.  Per tile the
// accumulator is used H / 128 times for the first layer (chunks of 128 hidden
// units, their epilogue writing packed BF16 h into tensor memory) and then
// once per 128 output columns for the second (A = h from tensor memory, B =
// W4 from the ring); the uses alternate between two TMEM accumulators, with
// acc_full / acc_empty counted over all uses of the CTA.  The TMA warp streams
// W4 independently of the first layer (separate shared memory), so it runs
// ahead into the next tile as far as the ring allows.
__global__ void __launch_bounds__(NTHREADS, 1)
    dec_tc_kernel(const __grid_constant__ CUtensorMap mapW4, const __grid_constant__ CUtensorMap mapX,
                  const DecArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                           ~uintptr_t(1023));
  const DecSmem L(a.ns);
  const int ns = a.ns;
  uint64_t* full_b = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* empty = full_b + ns;
  uint64_t* d1_ops = empty + ns;       // latent + W3 chunk written (converter warps)
  uint64_t* h_full = d1_ops + 1;       // every chunk of h stored in TMEM
  uint64_t* acc_full = h_full + 1;     // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = a.H, nk2 = H / KB, nchunk = (H + DNT - 1) / DNT;
  const int ntiles = (a.P + DNT - 1) / DNT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(d1_ops, NCONV * 32);
    mbar_init(h_full, NCONV * 32);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], NCONV * 32);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == WARP_TMA) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(a.err, ERR_TIMEOUT);
  };

  if (warp == WARP_TMA) {
    if (lane == 0) {
      prefetch_tmap(&mapW4);
      if (a.tma) prefetch_tmap(&mapX);
      int it = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < a.ntiles && ok && !*abort_flag; t += gridDim.x) {
        TileInfo ti;
        if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
        for (int j = 0; j < ntiles && ok; ++j)
          for (int k2 = 0; k2 < nk2; ++k2, ++it) {
            const int s = it % ns;
            const uint32_t ph = (it / ns) & 1;
            if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&full_b[s], D_STAGE);
            tma_load_3d(sm + L.stages + s * D_STAGE, &mapW4, &full_b[s], k2 * KB, j * DNT, ti.g);
          }
      }
      if (!ok) fail();
    }
    __syncwarp();
  } else if (warp == WARP_MMA) {
    if (lane == 0) {
      const uint32_t id2 = idesc_bf16(BM, DNT);
      int it = 0, iter = 0, J = 0, nd1 = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        TileInfo ti;
        if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
        // first layer, chunk by chunk: acc = latent W3[chunk]^T
        for (int c = 0; c < nchunk && ok; ++c, ++J, ++nd1) {
          const int buf = J & 1, cw = min(DNT, H - c * DNT);
          if (!mbar_wait(d1_ops, nd1 & 1) ||
              (J >= 2 && !mbar_wait(&acc_empty[buf], ((J >> 1) - 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = smem_u32(sm + L.d1a), bbase = smem_u32(sm + L.d1b);
          const uint32_t id1 = idesc_bf16(BM, cw);
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk)
            mma_bf16(tmem + TM_ACC + buf * DNT, desc_k128(abase + kk * 32),
                     desc_k128(bbase + kk * 32), id1, kk != 0);
          mma_commit(&acc_full[buf]);
        }
        if (!ok) break;
        // second layer: 128 output columns per accumulator use, A = h (TMEM)
        if (!mbar_wait(h_full, iter & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int j = 0; j < ntiles && ok; ++j, ++J) {
          const int buf = J & 1;
          if (J >= 2 && !mbar_wait(&acc_empty[buf], ((J >> 1) - 1) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int k2 = 0; k2 < nk2; ++k2, ++it) {
            const int s = it % ns;
            const uint32_t ph = (it / ns) & 1;
            if (*abort_flag || !mbar_wait(&full_b[s], ph)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t bbase = smem_u32(sm + L.stages + s * D_STAGE);
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk)
              mma_bf16_ta(tmem + TM_ACC + buf * DNT, tmem + (uint32_t)(k2 * 32 + kk * 8),
                          desc_k128(bbase + kk * 32), id2, (k2 | kk) != 0);
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[buf]);
        }
        ++iter;
      }
      if (!ok) fail();
    }
    __syncwarp();
  } else {
    const int t_ = threadIdx.x;
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint8_t* obox = sm + L.stg + warp * 2 * D_OUT;  // this warp's two output boxes
    int ob = 0;                                     // box the next TMA store reads
    int J = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      TileInfo ti;
      if (!tile_info((int)t, a.n, a.G, a.goff, a.toff, ti)) continue;
      const int rows = (int)min((long long)BM, ti.mend - ti.m0);
      // ---- first layer, chunk by chunk: operands, then h = act(acc + b3)
      // as packed BF16 into tensor memory ----
      // latent: 128 rows x 8 chunks of 16 B; chunk c holds k = 8c..8c+7
      for (int idx = t_; idx < BM * 8; idx += NCONV * 32) {
        const int rw = idx >> 3, c = idx & 7;
        uint4 w = make_uint4(0, 0, 0, 0);
        if (rw < rows && c * 8 < a.L)
          w = *reinterpret_cast<const uint4*>(a.latent + (ti.m0 + rw) * a.L + c * 8);
        *reinterpret_cast<uint4*>(sm + L.d1a + swz128(rw, c)) = w;
      }
      const __nv_bfloat16* W3 = a.W3 + ti.g * a.w3_gs;
      const float* b3 = a.b3 + ti.g * a.b3_gs;
      for (int ch = 0; ch < nchunk; ++ch, ++J) {
        const int cw = min(DNT, H - ch * DNT), buf = J & 1;
        // W3 rows [ch * 128, ch * 128 + cw), K zero-padded to 64 (the previous
        // chunk's MMA has completed: its accumulator was drained below)
        for (int idx = t_; idx < cw * 8; idx += NCONV * 32) {
          const int rw = idx >> 3, c = idx & 7;
          uint4 w = make_uint4(0, 0, 0, 0);
          if (c * 8 < a.L)
            w = *reinterpret_cast<const uint4*>(W3 + (long long)(ch * DNT + rw) * a.L + c * 8);
          *reinterpret_cast<uint4*>(sm + L.d1b + swz128(rw, c)) = w;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        mbar_arrive(d1_ops);
        if (!mbar_wait(&acc_full[buf], (J >> 1) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int cpw = cw / 2;  // columns of the chunk per warp half
        for (int col = half * cpw; col < (half + 1) * cpw; col += 32) {
          float v[32];
          tmem_ld32(tmem + lane_base + TM_ACC + (uint32_t)(buf * DNT + col), v);
          const int hc = ch * DNT + col;
          uint32_t u[16];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            u[i] = pack_bf16(act_f(a.act, v[2 * i] + __ldg(b3 + hc + 2 * i)),
                             act_f(a.act, v[2 * i + 1] + __ldg(b3 + hc + 2 * i + 1)));
          tmem_st16(tmem + lane_base + (uint32_t)(hc / 2), u);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      tc_fence_before();
      mbar_arrive(h_full);
      // ---- second layer per 128-column tile: xhat = s (acc + b4) ----
      // each thread holds one row; a warp's 32 rows x 32 columns go to shared
      // memory in the layout of the TMA store and leave as one box.  A tile
      // that ends inside the batch (its group ends mid-tile) takes plain
      // stores through a transposition block instead: a box would also cover
      // the first rows of the next group
      const float* b4 = a.b4 + ti.g * a.b4_gs;
      const float rs = r < rows ? (float)a.scale[ti.m0 + r] : 0.f;
      const bool by_tma = a.tma && (rows == BM || ti.mend == a.n);
      const bool warp_rows = q * 32 < rows;
      for (int j = 0; j < ntiles; ++j, ++J) {
        const int buf = J & 1;
        if (ok && (*abort_flag || !mbar_wait(&acc_full[buf], (J >> 1) & 1))) ok = false;
        if (ok) {
          tc_fence_after();
#pragma unroll 1
          for (int cc = 0; cc < DNT / 2; cc += 32) {
            const int col = half * (DNT / 2) + cc, p0 = j * DNT + col;
            if (p0 >= a.P) break;
            float v[32];
            tmem_ld32(tmem + lane_base + TM_ACC + (uint32_t)(buf * DNT + col), v);
            // b4 of the 32 columns: the same address in every lane
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const float4 b = __ldg(reinterpret_cast<const float4*>(b4 + p0 + i));
              v[i] = rs * (v[i] + (p0 + i < a.P ? b.x : 0.f));
              v[i + 1] = rs * (v[i + 1] + (p0 + i + 1 < a.P ? b.y : 0.f));
              v[i + 2] = rs * (v[i + 2] + (p0 + i + 2 < a.P ? b.z : 0.f));
              v[i + 3] = rs * (v[i + 3] + (p0 + i + 3 < a.P ? b.w : 0.f));
            }
            if (by_tma) {
              uint8_t* box = obox + ob * D_OUT;
              if (lane == 0) bulk_wait_read<1>();  // the store that last read this box
              __syncwarp();
#pragma unroll
              for (int c = 0; c < 8; ++c)
                *reinterpret_cast<float4*>(box + swz128(lane, c)) =
                    make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
              fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0 && warp_rows) {
                tma_store_2d(&mapX, box, p0, (int)(ti.m0 + q * 32));
                bulk_commit();
              }
              ob ^= 1;
            } else {
              float* tb = reinterpret_cast<float*>(obox);
              if (lane == 0) bulk_wait_read<0>();
              __syncwarp();
#pragma unroll
              for (int i = 0; i < 32; ++i) tb[lane * 33 + i] = v[i];
              __syncwarp();
              const int pc = p0 + lane;
              for (int rr = 0; rr < 32; ++rr) {
                const int row = q * 32 + rr;
                if (row < rows && pc < a.P) a.xhat[(ti.m0 + row) * a.ld + pc] = tb[rr * 33 + lane];
              }
              __syncwarp();
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
      }
    }
    // the boxes stay in shared memory until their stores have completed
    if (lane == 0) bulk_wait_all();
    __syncwarp();
    if (!ok) fail();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WARP_TMA) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- host side ---------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D BF16 tensor [G][rows][cols] (cols contiguous, group stride gstride
// elements) read in boxes of 64 columns x box_rows rows, 128-byte swizzle
int make_map(CUtensorMap* map, const void* base, int cols, int rows, int G, long long gstride,
             int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(AEQC_ECUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)G};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)gstride * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                  strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(AEQC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return AEQC_OK;
}

// 2-D FP32 tensor [rows][cols] with row pitch ld elements, written in boxes of
// 32 columns x 32 rows from a 128-byte-swizzled shared-memory layout; false
// where the tensor map cannot describe the output (unaligned base or pitch)
bool make_out_map(CUtensorMap* map, float* base, int cols, long long rows, long long ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld & 3) != 0 || ld < cols ||
      rows <= 0 || rows > 0x7FFFFFFFll - BM)
    return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Shapes the tensor-core path takes: H a multiple of 64 up to 512, L = 16 or 32.
bool tc_shape_ok(int H, int L) {
  return H % 64 == 0 && H >= 64 && H <= 512 && (L == 16 || L == 32);
}

// one CTA per SM (each takes the whole shared memory), at most one per tile
unsigned persistent_grid(long long ntiles) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (unsigned)(ntiles < sms ? (ntiles > 0 ? ntiles : 1) : sms);
}

int run_encode_tc(aeqc_model* m, const double* x, long long n, const long long* group_off,
                  const int* tile_off, int G, void* latent, double* scale, int* err,
                  cudaStream_t s) {
  const aeqc_model_desc& d = m->d;
  const __nv_bfloat16* bf = static_cast<const __nv_bfloat16*>(m->inf_bf16);
  CUtensorMap mW1, mW2;
  int rc = make_map(&mW1, bf + m->bE1B, m->Kp1, d.H, d.n_groups, m->n_bf16, d.H < 256 ? d.H : 256);
  if (rc) return rc;
  if ((rc = make_map(&mW2, bf + m->bE2B, d.H, d.L, d.n_groups, m->n_bf16, d.L))) return rc;
  EncArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x;
  a.n = n;
  a.P = d.P;
  a.Kp = m->Kp1;
  a.H = d.H;
  a.L = d.L;
  a.act = d.act;
  a.G = G;
  a.goff = group_off;
  a.toff = tile_off;
  a.b1 = m->inf + m->iE1b;
  a.b1_gs = m->n_inf;
  a.b2 = m->params + m->ob2;
  a.b2_gs = m->n_group;
  a.latent = static_cast<__nv_bfloat16*>(latent);
  a.scale = scale;
  a.err = err;
  // stages: as many as fit next to the W2 tile
  // stages: the tuned depth (else 6), reduced to what fits next to the W2 tile
  int ns = m->tuning.enc_stages >= 2 && m->tuning.enc_stages <= 6 ? m->tuning.enc_stages : 6;
  while (ns > 2 && EncSmem(d.H, d.L, ns).total + 1024 > 227 * 1024) --ns;
  a.ns = ns;
  const size_t smem = EncSmem(d.H, d.L, ns).total + 1024;
  if (smem > 227 * 1024) return set_error(AEQC_EUNSUPPORTED, "encoder tile does not fit (H=%d)", d.H);
  {
    const int rc = raise_smem_limit((const void*)enc_tc_kernel, 227 * 1024);
    if (rc) return rc;
  }
  a.ntiles = G > 1 ? (n + BM - 1) / BM + G : (n + BM - 1) / BM;
  enc_tc_kernel<<<persistent_grid(a.ntiles), ENC_NTHREADS, smem, s>>>(mW1, mW2, a);
  return check_launch("enc_tc_kernel");
}

int run_decode_tc(aeqc_model* m, const void* latent, const double* scale, long long n,
                  const long long* group_off, const int* tile_off, int G, float* xhat,
                  long long ld, int* err, cudaStream_t s) {
  const aeqc_model_desc& d = m->d;
  const __nv_bfloat16* bf = static_cast<const __nv_bfloat16*>(m->inf_bf16);
  CUtensorMap mW4;
  int rc = make_map(&mW4, bf + m->bD2B, d.H, d.P, d.n_groups, m->n_bf16, DNT);
  if (rc) return rc;
  DecArgs a;
  memset(&a, 0, sizeof(a));
  a.latent = static_cast<const __nv_bfloat16*>(latent);
  a.scale = scale;
  a.n = n;
  a.P = d.P;
  a.H = d.H;
  a.L = d.L;
  a.act = d.act;
  a.G = G;
  a.goff = group_off;
  a.toff = tile_off;
  a.W3 = bf + m->bD1B;
  a.w3_gs = m->n_bf16;
  a.b3 = m->params + m->ob3;
  a.b3_gs = m->n_group;
  a.b4 = m->inf + m->iD2b;
  a.b4_gs = m->n_inf;
  a.xhat = xhat;
  a.ld = ld;
  a.err = err;
  // full tiles of xhat leave through TMA stores where a tensor map can
  // describe the output
  CUtensorMap mX;
  memset(&mX, 0, sizeof(mX));
  a.tma = make_out_map(&mX, xhat, d.P, n, ld) ? 1 : 0;
  // the W4 ring: the tuned depth, else four stages (measured at 1M histograms,
  // H = 512: 2 / 4 / 6 / 8 stages 12.4 / 11.9 / 12.1 / 13.2 ms per 4M; deeper
  // rings leave the SM less L1 cache for the bias, latent and W3 loads),
  // reduced to what fits next to the output boxes
  const int cap = m->tuning.dec_stages >= 2 && m->tuning.dec_stages <= 16 ? m->tuning.dec_stages
                                                                          : 4;
  int ns = 2;
  while (ns < cap && DecSmem(ns + 1).total + 1024 <= 227 * 1024) ++ns;
  a.ns = ns;
  const size_t smem = DecSmem(ns).total + 1024;
  if (smem > 227 * 1024) return set_error(AEQC_EUNSUPPORTED, "decoder tile does not fit (H=%d)", d.H);
  {
    const int rc = raise_smem_limit((const void*)dec_tc_kernel, 227 * 1024);
    if (rc) return rc;
  }
  a.ntiles = G > 1 ? (n + BM - 1) / BM + G : (n + BM - 1) / BM;
  dec_tc_kernel<<<persistent_grid(a.ntiles), NTHREADS, smem, s>>>(mW4, mX, a);
  return check_launch("dec_tc_kernel");
}

}  // namespace aeqc
