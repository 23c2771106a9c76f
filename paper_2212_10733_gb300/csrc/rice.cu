// Entropy coding of the residual codes (the lossless stage the paper leaves to
// MGARD's Huffman/Zstd, Sec. III Stage 4; its output is part of the buffer of
// Stage 5): one Golomb-Rice code per histogram.
//
// Symbols: the zero-level code -> 0, a level q -> zigzag(q) + 1, the escape
// code -> 65535.  Per histogram the parameter k in 0..15 with the fewest bits
// (ties to the smaller k).  Per symbol s: u = s >> k; if u < 24: u one-bits, a
// zero-bit, the k low bits of s (least significant first); else 24 one-bits
// and the 16 bits of s.  Bit i of a histogram's stream is bit (i mod 32) of
// 32-bit word i / 32, unused high bits zero; streams are stored back to back
// at word offsets given by an exclusive prefix sum.
//
// rice_measure: warp per histogram, the sixteen candidate lengths summed
// per lane and reduced.  rice_pack: warp per histogram, each 32-symbol step
// places its bit patterns with a warp prefix sum of their lengths and ORs
// them into the histogram's stream in shared memory, which is then copied
// out.  rice_unpack: one thread per histogram reads its stream through a
// 64-bit bit buffer (reads never leave the histogram's words) and the warp
// writes the decoded codes through shared memory in contiguous rows.
#include "aeqc_internal.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

constexpr int RW = 4;           // warps per CTA (measure, pack)
constexpr int RCAP = 24;        // unary prefix cap
constexpr int RMAXBITS = 40;    // longest code
constexpr int RSLOT = (AEQC_MAX_P * RMAXBITS + 31) / 32;  // words of the longest stream
constexpr int SCAN_B = 1024;    // elements per scan block

__device__ __forceinline__ unsigned rice_symbol(int code) {
  if (code == AEQC_CODE_ZERO) return 0u;
  if (code == AEQC_CODE_ESCAPE) return 65535u;
  return (code >= 0 ? 2u * (unsigned)code : 2u * (unsigned)(-code) - 1u) + 1u;
}

__device__ __forceinline__ int rice_code(unsigned s) {
  if (s == 0u) return AEQC_CODE_ZERO;
  if (s == 65535u) return AEQC_CODE_ESCAPE;
  const unsigned z = s - 1u;
  return (z & 1u) ? -(int)((z + 1u) >> 1) : (int)(z >> 1);
}

__device__ __forceinline__ int rice_bits(unsigned s, int k) {
  const unsigned u = s >> k;
  return u < (unsigned)RCAP ? (int)u + 1 + k : RCAP + 16;
}

__global__ void __launch_bounds__(RW * 32) rice_measure_kernel(const int16_t* codes, long long n,
                                                               int P, uint8_t* kparam,
                                                               uint32_t* nbits,
                                                               long long* wcount) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * RW;
  for (long long b = (long long)blockIdx.x * RW + (threadIdx.x >> 5); b < n; b += nw) {
    const int16_t* cb = codes + b * P;
    int tot[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) tot[k] = 0;
    for (int p = lane; p < P; p += 32) {
      const unsigned s = rice_symbol(cb[p]);
#pragma unroll
      for (int k = 0; k < 16; ++k) tot[k] += rice_bits(s, k);
    }
    int best = 0x7FFFFFFF, arg = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      int t = tot[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (t < best) {
        best = t;
        arg = k;
      }
    }
    if (lane == 0) {
      kparam[b] = (uint8_t)arg;
      nbits[b] = (uint32_t)best;
      wcount[b] = (best + 31) / 32;
    }
  }
}

// exclusive prefix sum of wcount [n] into off [n + 1], three passes
__global__ void scan_block_sums(const long long* v, long long n, long long* bsum) {
  __shared__ long long s[32];
  const long long i0 = (long long)blockIdx.x * SCAN_B;
  long long acc = 0;
  for (int t = threadIdx.x; t < SCAN_B; t += blockDim.x)
    if (i0 + t < n) acc += v[i0 + t];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void scan_sums_serial(long long* bsum, long long nb, long long* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long run = 0;
  for (long long i = 0; i < nb; ++i) {
    const long long v = bsum[i];
    bsum[i] = run;
    run += v;
  }
  *total = run;
}

// SCAN_B threads: one element each
__global__ void scan_apply(const long long* v, long long n, const long long* bsum, long long* off) {
  __shared__ long long wsum[SCAN_B / 32];
  const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long x = i < n ? v[i] : 0;
  long long inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long t = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const long long before = (w ? wsum[w - 1] : 0) + inc - x;
  if (i < n) off[i] = bsum[blockIdx.x] + before;
}

__global__ void scan_total(const long long* total, long long n, long long* off) { off[n] = *total; }

__global__ void __launch_bounds__(RW * 32) rice_pack_kernel(const int16_t* codes, long long n,
                                                            int P, const uint8_t* kparam,
                                                            const long long* off, uint32_t* words,
                                                            long long capacity) {
  __shared__ uint32_t slot[RW][RSLOT];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint32_t* st = slot[wi];
  const long long nw = (long long)gridDim.x * RW;
  for (long long b = (long long)blockIdx.x * RW + wi; b < n; b += nw) {
    const int16_t* cb = codes + b * P;
    const int k = kparam[b] & 15;
    const int nwords = (P * RMAXBITS + 31) / 32;
    for (int t = lane; t < nwords; t += 32) st[t] = 0u;
    __syncwarp();
    long long base = 0;
    for (int p0 = 0; p0 < P; p0 += 32) {
      const int p = p0 + lane;
      int len = 0;
      unsigned long long v = 0ull;
      if (p < P) {
        const unsigned s = rice_symbol(cb[p]);
        const unsigned u = s >> k;
        if (u < (unsigned)RCAP) {
          len = (int)u + 1 + k;
          v = ((1ull << u) - 1ull) | ((unsigned long long)(s & ((1u << k) - 1u)) << (u + 1));
        } else {
          len = RCAP + 16;
          v = ((1ull << RCAP) - 1ull) | ((unsigned long long)s << RCAP);
        }
      }
      int inc = len;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const long long at = base + inc - len;
      if (len) {
        const int w0 = (int)(at >> 5), sh = (int)(at & 31);
        atomicOr(&st[w0], (uint32_t)(v << sh));
        const unsigned long long rest = sh ? (v >> (32 - sh)) : (v >> 32);
        if (rest) {
          atomicOr(&st[w0 + 1], (uint32_t)rest);
          if (rest >> 32) atomicOr(&st[w0 + 2], (uint32_t)(rest >> 32));
        }
      }
      base += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    const long long w0 = off[b], wc = (base + 31) >> 5;
    if (w0 >= 0 && w0 + wc <= capacity)
      for (int t = lane; t < (int)wc; t += 32) words[w0 + t] = st[t];
    __syncwarp();
  }
}

// Pack with every lane coding its own run of ceil(P / 32) >= 32 consecutive
// symbols (so every run has at least 32 bits and a 32-bit word is shared by
// at most two neighbouring lanes): one prefix sum of the run lengths per
// histogram, then each lane appends its patterns to a 64-bit buffer and
// stores whole words; the word it shares with the previous lane goes through
// shared memory and is merged after the run.
__global__ void __launch_bounds__(RW * 32) rice_pack_seg_kernel(const int16_t* codes,
                                                                long long n, int P,
                                                                const uint8_t* kparam,
                                                                const long long* off,
                                                                uint32_t* words,
                                                                long long capacity) {
  __shared__ int16_t sc[RW][AEQC_MAX_P];
  __shared__ uint32_t head[RW][32], tail[RW][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int ppl = (P + 31) / 32;
  const int p0 = min(P, lane * ppl), p1 = min(P, p0 + ppl);
  const int16_t* run = &sc[wi][p0];  // run[p - p0] for p in [p0, p1)
  const long long nw = (long long)gridDim.x * RW;
  for (long long b = (long long)blockIdx.x * RW + wi; b < n; b += nw) {
    const int16_t* cb = codes + b * P;
    for (int p = lane; p < P; p += 32) sc[wi][p] = cb[p];
    __syncwarp();
    const int k = kparam[b] & 15;
    long long len = 0;
    for (int p = p0; p < p1; ++p) len += rice_bits(rice_symbol(run[p - p0]), k);
    long long inc = len;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const long long S = inc - len, total = __shfl_sync(0xffffffffu, inc, 31);
    const long long w0 = off[b], wc = (total + 31) >> 5;
    if (w0 >= 0 && w0 + wc <= capacity) {  // the same for the whole warp
      const bool shared_head = (S & 31) != 0;
      unsigned long long buf = 0ull;
      int cnt = (int)(S & 31);
      long long wpos = S >> 5;
      bool first = true;
      auto emit = [&](uint32_t wv) {
        if (first && shared_head) head[wi][lane] = wv;
        else words[w0 + wpos] = wv;
        first = false;
        ++wpos;
      };
      for (int p = p0; p < p1; ++p) {
        const unsigned s = rice_symbol(run[p - p0]);
        const unsigned u = s >> k;
        unsigned long long v;
        int l;
        if (u < (unsigned)RCAP) {
          l = (int)u + 1 + k;
          v = ((1ull << u) - 1ull) | ((unsigned long long)(s & ((1u << k) - 1u)) << (u + 1));
        } else {
          l = RCAP + 16;
          v = ((1ull << RCAP) - 1ull) | ((unsigned long long)s << RCAP);
        }
        const unsigned long long carry = cnt ? (v >> (64 - cnt)) : 0ull;  // cnt < 32 here
        buf |= v << cnt;
        cnt += l;
        if (cnt >= 32) {
          emit((uint32_t)buf);
          buf = (buf >> 32) | (carry << 32);
          cnt -= 32;
          if (cnt >= 32) {
            emit((uint32_t)buf);
            buf >>= 32;
            cnt -= 32;
          }
        }
      }
      if (cnt > 0) {  // the run's last, partial word
        const uint32_t wv = (uint32_t)buf;
        if (first && shared_head) head[wi][lane] = wv;  // the whole run in one shared word
        else if (lane < 31) tail[wi][lane] = wv;        // shared with the next run
        else words[w0 + wpos] = wv;                     // the stream's last word
      }
      __syncwarp();
      if (shared_head) words[w0 + (S >> 5)] = head[wi][lane] | tail[wi][lane - 1];
    }
    __syncwarp();
  }
}

// One thread per histogram decodes 32 symbols at a time into shared memory;
// the warp then writes each of its 32 histograms' 32 codes as one contiguous
// 64-byte store (instead of 32 scattered 2-byte stores per instruction).
// Launched with 128 threads (4 warps) per block.
__global__ void __launch_bounds__(128, 6) rice_unpack_kernel(const uint32_t* words,
                                                          long long total_words,
                                                          const long long* off,
                                                          const uint8_t* kparam, long long n,
                                                          int P, int16_t* codes) {
  __shared__ int stage[4][32][33];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long b0 = ((long long)blockIdx.x * 4 + wi) * 32;  // the warp's first histogram
  const long long b = b0 + lane;
  const bool live = b < n;
  long long w = 0, wend = 0;
  int k = 0;
  if (live) {
    w = off[b];
    wend = off[b + 1];
    if (w < 0) w = 0;
    if (wend > total_words) wend = total_words;
    k = kparam[b] & 15;
  }
  unsigned long long buf = 0ull;
  int have = 0;  // valid bits in buf
  auto refill = [&]() {
    while (have <= 32) {
      const unsigned long long x = w < wend ? (unsigned long long)words[w] : 0ull;
      ++w;
      buf |= x << have;
      have += 32;
    }
  };
  for (int c0 = 0; c0 < P; c0 += 32) {
    const int m = min(32, P - c0);
    if (live) {
      for (int i = 0; i < m; ++i) {
        refill();
        // unary prefix: count of trailing ones, at most RCAP
        int u = __ffsll((long long)~buf) - 1;  // buf has at least 33 bits
        if (u < 0 || u > RCAP) u = RCAP;
        unsigned sy;
        if (u < RCAP) {
          buf >>= (u + 1);
          have -= u + 1;
          refill();
          sy = ((unsigned)u << k) | (unsigned)(buf & ((1ull << k) - 1ull));
          buf >>= k;
          have -= k;
        } else {
          buf >>= RCAP;
          have -= RCAP;
          refill();
          sy = (unsigned)(buf & 0xFFFFull);
          buf >>= 16;
          have -= 16;
        }
        stage[wi][lane][i] = rice_code(sy);
      }
    }
    __syncwarp();
    for (int h = 0; h < 32; ++h) {
      const long long bh = b0 + h;
      if (bh < n && lane < m) codes[bh * P + c0 + lane] = (int16_t)stage[wi][h][lane];
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace aeqc

using namespace aeqc;

extern "C" size_t rice_workspace_size(int64_t n) {
  if (n < 0) return 0;
  WsSize w;
  w.add<long long>((size_t)n + 1);
  w.add<long long>((size_t)(n + SCAN_B - 1) / SCAN_B + 1);
  w.add<long long>(1);
  return w.bytes;
}

extern "C" int rice_measure(const int16_t* codes, int64_t n, int32_t P, uint8_t* kparam,
                            uint32_t* nbits, int64_t* offsets, void* workspace,
                            size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(n >= 0 && P >= 1 && P <= AEQC_MAX_P, "rice_measure: bad sizes");
  AEQC_CHECK_ARG((n == 0 || (codes && kparam && nbits)) && offsets && workspace,
                 "rice_measure: null pointer");
  AEQC_CHECK_ARG(workspace_bytes >= rice_workspace_size(n), "rice_measure: workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  long long* wc = c.take<long long>((size_t)n + 1);
  const long long nb = (n + SCAN_B - 1) / SCAN_B;
  long long* bsum = c.take<long long>((size_t)nb + 1);
  long long* total = c.take<long long>(1);
  AEQC_CHECK_ARG(c.ok(), "rice_measure: workspace not 256-byte aligned");
  long long* off = reinterpret_cast<long long*>(offsets);
  if (n == 0) {
    AEQC_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), s));
    return AEQC_OK;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + RW - 1) / RW;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  rice_measure_kernel<<<(unsigned)blocks, RW * 32, 0, s>>>(codes, n, P, kparam, nbits, wc);
  scan_block_sums<<<(unsigned)nb, 256, 0, s>>>(wc, n, bsum);
  scan_sums_serial<<<1, 32, 0, s>>>(bsum, nb, total);
  scan_apply<<<(unsigned)nb, SCAN_B, 0, s>>>(wc, n, bsum, off);
  scan_total<<<1, 1, 0, s>>>(total, n, off);
  return check_launch("rice_measure");
}

extern "C" int rice_pack(const int16_t* codes, int64_t n, int32_t P, const uint8_t* kparam,
                         const int64_t* offsets, uint32_t* words, int64_t capacity, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(n >= 0 && P >= 1 && P <= AEQC_MAX_P && capacity >= 0, "rice_pack: bad sizes");
  AEQC_CHECK_ARG(n == 0 || (codes && kparam && offsets && words), "rice_pack: null pointer");
  if (n == 0) return AEQC_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + RW - 1) / RW;
  const long long* off = reinterpret_cast<const long long*>(offsets);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (P >= 32 * 31 + 1) {  // runs of at least 32 symbols per lane
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    rice_pack_seg_kernel<<<(unsigned)blocks, RW * 32, 0, s>>>(codes, n, P, kparam, off, words,
                                                               capacity);
    return check_launch("rice_pack_seg_kernel");
  }
  if (blocks > (long long)sms * 7) blocks = (long long)sms * 7;
  rice_pack_kernel<<<(unsigned)blocks, RW * 32, 0, s>>>(codes, n, P, kparam, off, words,
                                                          capacity);
  return check_launch("rice_pack_kernel");
}

extern "C" int rice_unpack(const uint32_t* words, int64_t total_words, const int64_t* offsets,
                           const uint8_t* kparam, int64_t n, int32_t P, int16_t* codes,
                           void* stream) {
  clear_error();
  AEQC_CHECK_ARG(n >= 0 && P >= 1 && P <= AEQC_MAX_P && total_words >= 0,
                 "rice_unpack: bad sizes");
  AEQC_CHECK_ARG(n == 0 || (offsets && kparam && codes && (words || total_words == 0)),
                 "rice_unpack: null pointer");
  if (n == 0) return AEQC_OK;
  rice_unpack_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      words, total_words, reinterpret_cast<const long long*>(offsets), kparam, n, P, codes);
  // 128 threads = 4 warps x 32 histograms per block
  return check_launch("rice_unpack_kernel");
}
