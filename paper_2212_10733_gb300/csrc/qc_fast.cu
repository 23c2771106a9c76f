// Residual quantization and QoI correction with the per-point work on the
// integer and FP32 pipes.  On GB300 the FP64 pipe runs at ~1/58 of the FP32
// rate and a warp-wide FP64 instruction costs the same with one active lane as
// with 32, so the per-histogram algebra runs in double-float arithmetic (pairs
// of floats, ~48-bit significands) on the FP32 pipe as well; FP64 is used only
// where a result must equal the oracle's bit for bit (the bin width Delta) and
// to hand the multipliers out as float64.  One warp per histogram; x', the
// residual and the codes stay in shared memory for the Newton passes.
//
// Quantizer (Stage 4), exactly: with Delta = 2^k, x and xhat become integers
// X = floor(x 2^(F-k)), Xh = floor(xhat 2^(F-k)) by bit manipulation, with an
// "inexact" flag when bits are dropped.  D = X - Xh lies within one unit of the
// exact scaled difference, so its fractional part decides round-half-even
// except when it is exactly one half and bits were dropped; the zero-level
// test (g < 0 or g > 2x) is decided the same way.  Those rare ambiguous points
// use the exact FP64 routine.
//
// Correction (Stage 5, Eq. (6)): with r = x - x' and t = lambda.phi,
//   g(lambda) = sum vol phi (x' e^{-t} - x) = -R - M lambda + H(lambda),
//   R = sum vol phi r,  M = sum vol phi phi^T x',  H = sum vol phi x' h(t),
//   h(t) = e^{-t} - 1 + t = t^2/2 - t^3/6 + ...
// R and M do not depend on lambda: one pass accumulates them exactly as
// integer sums (on the affine grid v_par = b (i - i_c) + c0, v_perp^2 = d2 j^2
// every weight is a small integer polynomial).  H is second order; each pass
// sums it in FP32 together with a bound on the rounding error of those sums,
// and repeats the pass with error-free (TwoSum) accumulation if the bound
// exceeds 1e-13 S_k.  Newton steps use M as the Jacobian (a chord step: M is
// the exact Jacobian at lambda = 0, and the iteration contracts at a rate
// ~|t|); the 4x4 solve runs in FP32 on the unit-diagonal scaled M with one
// double-float refinement step.  Each step after the first costs one FP32 pass,
// which also performs the end-to-end check.  Histograms the fast path cannot
// certify (non-finite or negative input, large lambda, no convergence, an
// ambiguous check, verbatim storage) go to a list the FP64 kernel completes.
#include <math.h>
#include <string.h>

#include "qc_common.cuh"

namespace aeqc {
namespace {

using namespace dev;

// One CTA per SM with up to sixteen warps, one histogram per warp at a time.
// Measured on the precision workload: sixteen warps in one CTA run 14 % faster
// than the same sixteen warps as four CTAs of four (same registers, same
// shared memory per warp, same histogram-to-SM mapping).
constexpr int FW_MAX = 16;

struct FastWS {
  float xp[AEQC_MAX_P];  // x' (float) for the Newton passes
  union {
    int16_t rho[AEQC_MAX_P];  // round((x - x') / Delta 2^15) for the end-to-end check
    struct {
      double ta[AEQC_MAX_NPAR], tb[AEQC_MAX_NPERP];  // exponential tables for f_out
    } t;
  };
};

// float(v) for |v| < 2^22 without a conversion instruction (those issue to the
// slow FP64 pipe on this GPU): 1.5 2^23 + v is exact and read off its bits
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.f;
}

// ---- double-float arithmetic (Dekker / Knuth error-free transformations) ---
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return quick_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  return quick_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df x, float f) {
  const float p = __fmul_rn(x.hi, f);
  const float e = __fmaf_rn(x.lo, f, __fmaf_rn(x.hi, f, -p));
  return quick_sum(p, e);
}
__device__ __forceinline__ df df_add_f(df x, float f) {
  const df s = two_sum(x.hi, f);
  return quick_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ float exp2i(int n) {  // 2^n for n in [-126, 127]
  return __int_as_float((n + 127) << 23);
}
__device__ __forceinline__ df df_ldexp(df x, int n) {  // n in [-126, 127]; exact for normal results
  const float f = exp2i(n);
  return {x.hi * f, x.lo * f};
}
// the top 48 bits of an int64 as a float pair (relative error <= 2^-48)
__device__ __forceinline__ df df_from_ll(long long v) {
  if (v == 0) return {0.f, 0.f};
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << lz;
  const int e = 63 - lz;
  // top 24 bits (leading bit set) straight into a float's fields; the next
  // 24 as two exact 12-bit halves (int->float conversion instructions issue
  // to the FP64 pipe on this GPU)
  float hi = __int_as_float(((e + 127) << 23) | (int)((m >> 40) & 0x7FFFFFull));
  const unsigned l24 = (unsigned)((m >> 16) & 0xFFFFFFull);
  const float l24f = fmaf(__int_as_float(0x4B000000 | (int)(l24 >> 12)) - 8388608.f, 4096.f,
                          __int_as_float(0x4B000000 | (int)(l24 & 0xFFFu)) - 8388608.f);
  float lo = __fmul_rn(l24f, exp2i(e - 47));
  if (v < 0) {
    hi = -hi;
    lo = -lo;
  }
  return quick_sum(hi, lo);
}

// hi + lo as a double on the integer pipe, for a pair with |lo| <= ulp(hi)
// (as quick_sum leaves it): hi's 24-bit significand widened to 53 bits plus
// lo aligned to it, lo's bits below the 53 truncated (the result is within one
// unit in the last place of hi + lo).  A zero, subnormal or non-finite hi takes
// the FP64 conversion.
__device__ __forceinline__ double df_to_double(df x) {
  const unsigned uh = __float_as_uint(x.hi), ul = __float_as_uint(x.lo);
  const int eh = (int)((uh >> 23) & 0xffu), el = (int)((ul >> 23) & 0xffu);
  if (eh == 0 || eh == 255) return (double)x.hi + (double)x.lo;
  // hi = S 2^(eh - 179) with S in [2^52, 2^53)
  long long S = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;
  int e = eh;
  if (el != 0) {
    // lo = L 2^(el - 150) = L 2^(el - eh + 29) units of hi's last place
    const long long L = (long long)((ul & 0x7fffffu) | 0x800000u);
    const int sh = eh - el - 29;  // >= -5 for |lo| <= ulp(hi)
    const long long Ls = sh <= 0 ? (L << (-sh)) : (sh < 63 ? (L >> sh) : 0ll);
    S += ((uh ^ ul) >> 31) ? -Ls : Ls;
    if (S >= (1ll << 53)) {
      S >>= 1;
      ++e;
    } else if (S < (1ll << 52)) {
      S <<= 1;
      --e;
    }
  }
  const unsigned long long bits = ((unsigned long long)(uh >> 31) << 63) |
                                  ((unsigned long long)(e + 896) << 52) |
                                  ((unsigned long long)S & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// ---- integer decomposition of the inputs ----------------------------------

// binary exponent E of a positive finite double: d in [2^(E-1), 2^E)
__device__ __forceinline__ int exponent_of(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int E = (int)(u >> 52) & 0x7ff;
  if (E) return E - 1022;
  return (63 - __clzll((long long)u)) - 1073;  // subnormal
}

// Fixed point of the quantizer: units of Delta 2^-QF.
constexpr int QF = 38;

// Per-histogram constants of the integer quantizer.
struct QConst {
  double dl;  // Delta = 2^k
  float dl_f;
  int k;
  int cx;    // floor(x 2^(QF-k)) = (mantissa << 10) >> (cx - E), E the exponent field
  int ch;    // trunc(xhat 2^(QF-k)) = (mantissa << 40) >> (ch - E)
  int thr;   // exponent field of xhat at or above which |q| > 32766 for sure
};

// floor(log2(2 alpha fl(tau s))) for 2 alpha = 2^a2e and tau, s > 0 normal, on
// the integer pipe (the FP64 pipe issues one warp instruction in ~60 cycles
// on this GPU): fl(tau s) = 2^(et + es + top + carry) (1 + f) with top set
// when the significand product P = mt ms (in [2^104, 2^106)) reaches 2^105,
// and carry when rounding P to 53 bits, to nearest even, overflows into the
// next binade; scaling by 2^a2e is exact.  Results outside the normal range
// are rejected by the caller, as the FP64 form of bin_width would be.
__device__ __forceinline__ int bin_exp_int(unsigned long long mt, int et, unsigned long long us,
                                           int a2e) {
  const unsigned long long ms = (us & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int es = (int)(us >> 52) - 1023;
  const unsigned long long lo = mt * ms, hi = __umul64hi(mt, ms);
  const int top = (int)(hi >> 41);
  const unsigned long long sig = top ? ((hi << 11) | (lo >> 53)) : ((hi << 12) | (lo >> 52));
  const unsigned long long rb = top ? (lo >> 52) & 1ull : (lo >> 51) & 1ull;
  // sig = 2^53 - 1 is odd: a set round bit rounds it up (to even) whatever
  // the sticky bits
  const int carry = (rb && sig == (1ull << 53) - 1ull) ? 1 : 0;
  return et + es + top + carry + a2e;
}

__device__ __forceinline__ bool make_qconst(const ParamsK& pr, double s, int level, QConst& c) {
  const unsigned long long us = (unsigned long long)__double_as_longlong(s);
  if (pr.bw_int && (us >> 52) != 0) {  // s > 0 and normal
    c.k = bin_exp_int(pr.tau_m, pr.tau_e, us, pr.a2_e[level]);
    if (c.k < -1022 || c.k > 1023) return false;
    c.dl = __longlong_as_double((long long)(c.k + 1023) << 52);
  } else {
    c.dl = bin_width(pr.tau, s, level ? pr.alpha4 : pr.alpha);
    if (!(c.dl > 0.0) || !isfinite(c.dl)) return false;
    c.k = exponent_of(c.dl) - 1;
  }
  const int IBx = exponent_of(s) - c.k;  // s / Delta < 2^IBx
  c.cx = 1085 + c.k - QF;
  c.ch = 190 + c.k - QF;
  // |xhat| >= 2^(61 - QF + k) = 2^23 Delta > s + 32766 Delta: certain escape
  c.thr = 127 + 61 - QF + c.k;
  // x < 2^(IBx + QF) <= 2^60 units; Delta and the scale factors of the moment
  // sums (vol Delta 2^-30, vol Delta 2^-38) stay normal floats
  const bool ok = IBx >= 1 && IBx <= 22 && c.k - 64 >= -100 && c.k + 20 <= 100;
  c.dl_f = ok ? exp2i(c.k) : 0.f;
  return ok;
}

// |x| as a float (mantissa truncated; 0 below the float range) from the bit
// pattern u of a double, on the integer pipe
__device__ __forceinline__ float float_of_bits(unsigned long long u) {
  const int E = (int)(u >> 52) & 0x7ff;
  if (E <= 896) return 0.f;
  if (E >= 1151) return __int_as_float(0x7f800000);
  return __int_as_float(((E - 896) << 23) | (int)((u >> 29) & 0x7FFFFFull));
}

struct PointQ {
  int code;
  long long rho;  // (x - x') / Delta * 2^38 (within two units)
  long long xpw;  // x' / Delta * 2^38 (within one unit)
  float xpf;      // x' (float)
};

// The exact FP64 routine for the rare points whose integer decision falls in
// an ambiguity band.
__device__ __noinline__ PointQ quant_point_hard(double x, float xh, double dl) {
  PointQ o;
  double xpd;
  o.code = quant_point_fp64(x, (double)xh, dl, &xpd);
  o.xpw = __double2ll_rn(ldexp(__ddiv_rn(xpd, dl), QF));
  // x in the same units (exact: x < 2^23 Delta), so that rho = X - X'
  o.rho = __double2ll_rn(ldexp(__ddiv_rn(x, dl), QF)) - o.xpw;
  o.xpf = (float)xpd;
  return o;
}

// Quantizer decision for one point (x finite, x >= 0), exact where it is
// not flagged.  With u = Delta 2^-38, X = floor(x / u) and Xh = trunc(xhat / u)
// come from the bit patterns; the exact scaled difference (x - xhat) / u is
// D + e with D = X - Xh and e in (-1, 2).  With t = D + 2^37, q = floor(t / 2^38)
// is the round-half-even index unless t's fraction is within two units of a
// multiple of 2^38 (a tie or an uncertain rounding): that point is flagged.
// rho = D - q 2^38 is the residual (x - xhat - q Delta) / u within the same
// (-1, 2) units; the zero level wins iff |x - xhat - q Delta| > x, decided on
// |rho| - X unless within three units (flagged).  Escapes (|q| > 32766 or a
// non-finite or huge xhat) are flagged too.  A flagged point's outputs here
// are zero; the caller completes it with the exact FP64 routine.
struct PointF {
  int code;       // q, or AEQC_CODE_ZERO (0 when flagged)
  long long xpw;  // x' / u within one unit (0 when flagged or at the zero level)
  long long rho;  // (x - x') / u within two units (0 when flagged)
  float xpf;      // x' as a float (0 when flagged or at the zero level)
  bool hard;
};

__device__ __forceinline__ PointF quant_point_fast(double x, float xh, const QConst& c) {
  const unsigned long long ux = (unsigned long long)__double_as_longlong(x);
  const int E = (int)(ux >> 52);  // x >= 0: no sign bit
  // mantissa with its implicit bit at bits 10..62; a subnormal x gives X = 0
  const unsigned long long M10 =
      ((ux & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(E != 0) << 52)) << 10;
  const long long X = (long long)(M10 >> min(c.cx - E, 63));
  const unsigned v = __float_as_uint(xh);
  const int Eh = (v >> 23) & 0xff;
  const bool esc_h = Eh >= c.thr;  // |q| > 32766 for sure, or a non-finite xhat
  const unsigned long long m40 = (unsigned long long)((v & 0x7fffffu) | (Eh ? 0x800000u : 0u))
                                 << 40;
  const long long mag = (long long)(m40 >> min(max(c.ch - (Eh ? Eh : 1), 0), 63));
  const long long D = X - ((v >> 31) ? -mag : mag);
  const long long t = D + (1ll << (QF - 1));
  const int q = (int)(t >> QF);
  const bool band = ((t + 2) & ((1ll << QF) - 1)) < 4;
  const long long rho = D - ((long long)q << QF);
  const long long uz = (rho < 0 ? -rho : rho) - X;  // |r| - x in units
  const bool zero = uz > 3;
  const bool band2 = (unsigned long long)(uz + 3) <= 6ull;
  PointF o;
  o.hard = band || band2 || esc_h || q > AEQC_CODE_MAX || q < -AEQC_CODE_MAX;
  const bool keep = !o.hard && !zero;
  o.code = o.hard ? 0 : (zero ? AEQC_CODE_ZERO : q);
  o.xpw = keep ? X - rho : 0ll;
  o.rho = o.hard ? 0ll : (zero ? X : rho);
  // |q| < 2^22 wherever the value is kept
  o.xpf = keep ? fmaf(small_int_to_float(q), c.dl_f, xh) : 0.f;
  return o;
}

// The lambda-independent moments of one quantization level, double-float.
struct Moments {
  df R[4];       // sum vol phi_k (x - x')
  df M[10];      // upper triangle of sum vol phi phi^T x' (m00 m01 m02 m03 m11 ...)
  float S[4];    // sum vol |phi_k| x'
  unsigned flags;  // CODE_ESCAPE / AE_EXACT
};

// Sums over the warp of 32 64-bit values held by every lane, scattered:
// lane k returns the total of value k.  Recursive halving: at each step a
// lane keeps the half of its values selected by its lane bit and adds its
// partner's copy of that half (the totals are bounded on the host so that
// they fit).
// Warp sums of four double-float values held by every lane: the total of
// value k ends in lanes 8k..8k+7 (halving over lane bits 4 and 3, then a
// butterfly over the remaining three bits), added error-free.
__device__ __forceinline__ df df_reduce_scatter4(const df (&a)[4], int lane) {
  const bool u4 = (lane & 16) != 0, u3 = (lane & 8) != 0;
  df v[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const df send = u4 ? a[i] : a[2 + i];
    const df keep = u4 ? a[2 + i] : a[i];
    v[i] = df_add(keep, df{__shfl_xor_sync(FULL, send.hi, 16), __shfl_xor_sync(FULL, send.lo, 16)});
  }
  const df send = u3 ? v[0] : v[1];
  df x = df_add(u3 ? v[1] : v[0],
                df{__shfl_xor_sync(FULL, send.hi, 8), __shfl_xor_sync(FULL, send.lo, 8)});
#pragma unroll
  for (int o = 4; o > 0; o >>= 1)
    x = df_add(x, df{__shfl_xor_sync(FULL, x.hi, o), __shfl_xor_sync(FULL, x.lo, o)});
  return x;
}

__device__ __forceinline__ long long reduce_scatter32(long long (&v)[32], int lane) {
#pragma unroll
  for (int o = 16, n = 16; o >= 1; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const long long send = up ? v[i] : v[n + i];
      const long long keep = up ? v[n + i] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, o);
    }
  }
  return v[0];
}

// Each lane walks down (part of) grid columns, so that the weights in i are
// constants of the lane and the weights in j are the same for the whole warp:
// one column sum per power of j replaces the per-point products.  Part 1:
// lane i owns column i (i < 32, when the grid has at least 32 columns).
// Part 2: the remaining columns, each cut into row chunks so that most lanes
// take one chunk.
struct Seg {
  int c, j0, j1;  // column, rows [j0, j1)
};

__device__ __forceinline__ void lane_segments(const FastGridK& fg, int n_par, int n_perp,
                                              int lane, Seg& s1, Seg& s2) {
  const int cw = n_par >= 32 ? 32 : 0, rw = n_par - cw;
  s1.c = lane;
  s1.j0 = 0;
  s1.j1 = cw ? n_perp : 0;
  s2.c = cw;
  s2.j0 = s2.j1 = 0;
  if (rw) {
    const int nchunk = fg.seg_nchunk;  // 32 / rw >= 1
    const int rpc = fg.seg_rpc;        // ceil(n_perp / nchunk)
    if (lane < rw * nchunk) {
      const int chunk = (lane * fg.seg_mul) >> 16;  // lane / rw
      s2.c = cw + lane - chunk * rw;
      s2.j0 = chunk * rpc;
      s2.j1 = min(n_perp, s2.j0 + rpc);
    }
  }
}

// Column sums of one segment: X' j^(2q) (split at bit 31), rho j^(2q)
// (q = 0, 1) and x' (float).
struct ColSums {
  long long b[3], a[3], u[2];
  float xs;
};

// a + b c for unsigned 32-bit b, c (one wide multiply-add)
__device__ __forceinline__ long long mad_wide(long long a, unsigned b, unsigned c) {
  return (long long)((unsigned long long)a + (unsigned long long)b * (unsigned long long)c);
}

__device__ __forceinline__ void colsum_add(ColSums& cs, long long xpw, long long rho, float xpf,
                                           unsigned j2, unsigned j4) {
  // x' >= 0 here, below 2^60 units: two unsigned 32-bit parts (31 + 29 bits)
  const unsigned xl = (unsigned)xpw & 0x7FFFFFFFu, xu = (unsigned)(xpw >> 31);
  cs.b[0] += xl;
  cs.b[1] = mad_wide(cs.b[1], xl, j2);
  cs.b[2] = mad_wide(cs.b[2], xl, j4);
  cs.a[0] += xu;
  cs.a[1] = mad_wide(cs.a[1], xu, j2);
  cs.a[2] = mad_wide(cs.a[2], xu, j4);
  // |rho| <= 2^37 and the grid's sum of j^2 is below 2^25 (host check):
  // every total stays below 2^62.  rho j2 from rho's two words, modulo 2^64
  // (two's complement: the exact product).
  cs.u[0] += rho;
  cs.u[1] = mad_wide(cs.u[1] + (long long)((unsigned long long)((unsigned)(rho >> 32) * j2) << 32),
                     (unsigned)rho, j2);
  cs.xs += xpf;
}

// Quantize one segment (column sg.c, rows [j0, j1)): codes to cb (global), x'
// and the residual (in Delta 2^-15) to shared memory, column sums to cs.  One
// straight-line body per point; the flagged points (a bit per row of the
// segment, at most 64 rows) are completed after the walk.
__device__ __forceinline__ void quant_segment(const Seg& sg, int n_par, const double* xb,
                                              const float* xhb, const QConst& c, FastWS& w,
                                              int16_t* cb, ColSums& cs, int& esc,
                                              int& nonzero) {
  cs = ColSums{{0, 0, 0}, {0, 0, 0}, {0, 0}, 0.f};
  unsigned long long flagged = 0;
  int nz = 0;
  int p = sg.j0 * n_par + sg.c;
  // loads issued two points ahead of the work
  double xn = sg.j0 < sg.j1 ? __ldg(xb + p) : 0.0;
  float hn = sg.j0 < sg.j1 ? __ldg(xhb + p) : 0.f;
  double xn2 = sg.j0 + 1 < sg.j1 ? __ldg(xb + p + n_par) : 0.0;
  float hn2 = sg.j0 + 1 < sg.j1 ? __ldg(xhb + p + n_par) : 0.f;
  unsigned j2 = (unsigned)(sg.j0 * sg.j0);
#pragma unroll 1
  for (int j = sg.j0; j < sg.j1; ++j, p += n_par) {
    const double x = xn;
    const float xh = hn;
    xn = xn2;
    hn = hn2;
    if (j + 2 < sg.j1) {
      xn2 = __ldg(xb + p + 2 * n_par);
      hn2 = __ldg(xhb + p + 2 * n_par);
    }
    const PointF o = quant_point_fast(x, xh, c);
    cb[p] = (int16_t)o.code;
    w.xp[p] = o.xpf;
    w.rho[p] = (int16_t)((o.rho + (1ll << 22)) >> 23);
    nz |= o.code;
    if (o.hard) flagged |= 1ull << (j - sg.j0);
    colsum_add(cs, o.xpw, o.rho, o.xpf, j2, j2 * j2);
    j2 += 2 * j + 1;  // (j + 1)^2
  }
  nonzero |= nz;
  // the flagged points: the exact FP64 routine (out of line), outputs stored
  // and moments added
  while (flagged) {
    const int j = sg.j0 + __ffsll((long long)flagged) - 1;
    flagged &= flagged - 1;
    const int pf = j * n_par + sg.c;
    const PointQ o = quant_point_hard(__ldg(xb + pf), __ldg(xhb + pf), c.dl);
    cb[pf] = (int16_t)o.code;
    w.xp[pf] = o.xpf;
    w.rho[pf] = (int16_t)((o.rho + (1ll << 22)) >> 23);
    esc |= o.code == AEQC_CODE_ESCAPE;
    nonzero |= o.code != 0;
    colsum_add(cs, o.xpw, o.rho, o.xpf, (unsigned)(j * j), (unsigned)(j * j * j * j));
  }
}

// Quantize the histogram (row xb, decoded row xhb): codes to cb (global),
// x' and the residual to shared memory, and the moments.
__device__ void phase_a(const GridK& g, const FastGridK& fg, const double* xb,
                        const float* xhb, const QConst& c, FastWS& w, int16_t* cb, Moments& mo,
                        int lane) {
  Seg sg1, sg2;
  lane_segments(fg, g.n_par, g.n_perp, lane, sg1, sg2);
  int esc = 0, nonzero = 0;
  ColSums c1, c2;
  quant_segment(sg1, g.n_par, xb, xhb, c, w, cb, c1, esc, nonzero);
  quant_segment(sg2, g.n_par, xb, xhb, c, w, cb, c2, esc, nonzero);
  // fold with the powers of i - i_c: U_q over weights 1, ic, ic^2, j^2 and T
  // over (ic^r j^(2q)) in the order T00 T10 T20 T30 T40 T01 T11 T21 T02, the
  // latter as Tb + 2^31 Ta
  long long U[4], Tb[9], Ta[9];
  {
    const long long i1 = sg1.c - fg.i_c, i2 = sg2.c - fg.i_c;
    const long long p1[5] = {1, i1, i1 * i1, i1 * i1 * i1, i1 * i1 * i1 * i1};
    const long long p2[5] = {1, i2, i2 * i2, i2 * i2 * i2, i2 * i2 * i2 * i2};
    const int rq[9][2] = {{0, 0}, {1, 0}, {2, 0}, {3, 0}, {4, 0}, {0, 1}, {1, 1}, {2, 1}, {0, 2}};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int r = rq[k][0], q = rq[k][1];
      Tb[k] = c1.b[q] * p1[r] + c2.b[q] * p2[r];
      Ta[k] = c1.a[q] * p1[r] + c2.a[q] * p2[r];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) U[r] = c1.u[0] * p1[r] + c2.u[0] * p2[r];
    U[3] = c1.u[1] + c2.u[1];
  }
  const float b_f = fg.b_f, c0_f = fg.c0_f;
  float s1 = c1.xs * fabsf(fmaf(b_f, small_int_to_float(sg1.c - fg.i_c), c0_f)) +
             c2.xs * fabsf(fmaf(b_f, small_int_to_float(sg2.c - fg.i_c), c0_f));
  __syncwarp();
  // exact warp totals (the host bounds them below 2^62), scattered over the
  // lanes: lane k holds total k of (U0..U3, Tb0..Tb8, Ta0..Ta8); each lane
  // converts one total to double-float
  long long v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i)
    v[i] = i < 4 ? U[i] : (i < 13 ? Tb[i - 4] : (i < 22 ? Ta[i - 13] : 0ll));
  df mine = df_from_ll(reduce_scatter32(v, lane));
  {
    const df ta = {__shfl_down_sync(FULL, mine.hi, 9), __shfl_down_sync(FULL, mine.lo, 9)};
    if (lane >= 4 && lane < 13) mine = df_add(df_ldexp(ta, 31), mine);  // T = Tb + 2^31 Ta
  }
  float S1 = s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S1 += __shfl_xor_sync(FULL, S1, o);
  const df vol = {fg.vol_h, fg.vol_l};
  const df sr = df_ldexp(vol, c.k - QF), sm = sr;
  // moment j = m(p, q) in lane j < 9, (p, q) in the order of the T totals:
  // m(p, q) = vol Delta 2^-38 d2^q sum_r C(p,r) b^r c0^(p-r) T[r][q]
  df mj;
  {
    const int jj = lane < 9 ? lane : 0;
    const int pj = jj < 5 ? jj : (jj < 8 ? jj - 5 : 0), qj = jj < 5 ? 0 : (jj < 8 ? 1 : 2);
    df acc = {0.f, 0.f};
#pragma unroll
    for (int r = 0; r <= 4; ++r) {
      const int src = 4 + (qj == 0 ? r : (qj == 1 ? 5 + min(r, 2) : 8));
      const df tr = {__shfl_sync(FULL, mine.hi, src), __shfl_sync(FULL, mine.lo, src)};
      if (r <= pj) acc = df_add(acc, df_mul(df{fg.coef_h[pj][r], fg.coef_l[pj][r]}, tr));
    }
    mj = df_mul(sm, df_mul(df{fg.d2q_h[qj], fg.d2q_l[qj]}, acc));
  }
  df mm[9], u[4];
#pragma unroll
  for (int j = 0; j < 9; ++j) mm[j] = df{__shfl_sync(FULL, mj.hi, j), __shfl_sync(FULL, mj.lo, j)};
#pragma unroll
  for (int q = 0; q < 4; ++q) u[q] = df{__shfl_sync(FULL, mine.hi, q), __shfl_sync(FULL, mine.lo, q)};
  const df b = {fg.coef_h[1][1], fg.coef_l[1][1]};   // C(1,1) b = b
  const df c0 = {fg.coef_h[1][0], fg.coef_l[1][0]};  // C(1,0) c0 = c0
  const df d2 = {fg.d2q_h[1], fg.d2q_l[1]};
  // R_k = vol Delta 2^-38 sum phi_k rho, phi = (1, v, w, v^2), v = b ic + c0
  mo.R[0] = df_mul(sr, u[0]);
  mo.R[1] = df_mul(sr, df_add(df_mul(b, u[1]), df_mul(c0, u[0])));
  mo.R[2] = df_mul(sr, df_mul(d2, u[3]));
  {
    const df cc[3] = {{fg.coef_h[2][0], fg.coef_l[2][0]},
                      {fg.coef_h[2][1], fg.coef_l[2][1]},
                      {fg.coef_h[2][2], fg.coef_l[2][2]}};
    df acc = df_mul(cc[0], u[0]);
    acc = df_add(acc, df_mul(cc[1], u[1]));
    acc = df_add(acc, df_mul(cc[2], u[2]));
    mo.R[3] = df_mul(sr, acc);
  }
  // mm: m00 m10 m20 m30 m40 m01 m11 m21 m02
  mo.M[0] = mm[0]; mo.M[1] = mm[1]; mo.M[2] = mm[5]; mo.M[3] = mm[2];
  mo.M[4] = mm[2]; mo.M[5] = mm[6]; mo.M[6] = mm[3];
  mo.M[7] = mm[8]; mo.M[8] = mm[7];
  mo.M[9] = mm[4];
  mo.S[0] = mm[0].hi;
  mo.S[1] = fg.vol_h * S1;
  mo.S[2] = mm[5].hi;
  mo.S[3] = mm[2].hi;
  mo.flags = 0;
  if (__any_sync(FULL, esc)) mo.flags |= AEQC_ST_CODE_ESCAPE;
  if (!__any_sync(FULL, nonzero)) mo.flags |= AEQC_ST_AE_EXACT;
}

struct PassOut {
  df H[4];
  float Habs[4];  // bounds on the sums of |terms| (for the FP32 rounding bound)
  float tmax;     // bound on |t| over the grid points (segment end points)
  float errmax;   // largest FP32 check value |x' e^{-t} - x| of the points
  // row (lane & 3) of J = dH/dlambda = sum vol phi phi^T x' h'(t), in FP32
  // (its rounding is bounded in the certificate of round1_fast)
  float J[4];
  int viol, uncertain;
};

// t = lambda.phi in exact integer weights: t = a0 + a1 ic + a3 ic^2 + a2 j^2
// (ic = i - i_c), the coefficients as float pairs so that no weight carries a
// systematic rounding error.
struct TCoef {
  float h[4], l[4];  // a0, a1, a2 (j^2), a3 (ic^2)
};

__device__ __forceinline__ TCoef make_tcoef(const FastGridK& fg, const df lam[4]) {
  const df c0 = {fg.coef_h[1][0], fg.coef_l[1][0]}, b = {fg.coef_h[1][1], fg.coef_l[1][1]};
  const df c00 = {fg.coef_h[2][0], fg.coef_l[2][0]}, c21 = {fg.coef_h[2][1], fg.coef_l[2][1]};
  const df bb = {fg.coef_h[2][2], fg.coef_l[2][2]}, d2 = {fg.d2q_h[1], fg.d2q_l[1]};
  const df a0 = df_add(lam[0], df_add(df_mul(lam[1], c0), df_mul(lam[3], c00)));
  const df a1 = df_add(df_mul(lam[1], b), df_mul(lam[3], c21));
  const df a2 = df_mul(lam[2], d2);
  const df a3 = df_mul(lam[3], bb);
  TCoef t;
  t.h[0] = a0.hi; t.l[0] = a0.lo;
  t.h[1] = a1.hi; t.l[1] = a1.lo;
  t.h[2] = a2.hi; t.l[2] = a2.lo;
  t.h[3] = a3.hi; t.l[3] = a3.lo;
  return t;
}

// One pass at lambda: H(lambda) and the end-to-end check.  EXACT selects
// TwoSum accumulation of H (used when the FP32 sums' error bound is too wide).
// The points are walked in the segments of phase_a: on a segment t = A +
// a2 j^2 with A a constant, and one column sum of y and of y j^2 per segment
// gives all four sums.
__device__ void pass_warp(const GridK& g, const FastGridK& fg, const FastWS& w,
                          const QConst& c, const TCoef& tc, float e_lo, float e_hi, PassOut& o,
                          int lane, const bool EXACT) {
  df a[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // sums of y, y ic, y ic^2, y j^2
  float ab1 = 0.f, tmax = 0.f, errmax = 0.f;
  // sums of z = x' h'(t) over the monomials v^p w^q of phi phi^T, in the
  // order m00 m10 m20 m30 m40 m01 m11 m21 m02 (w^q as j^(2q), d2^q later)
  float jz[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float cq = c.dl_f * 3.0517578125e-05f, dq = -12582912.f * cq;  // Delta 2^-15
  // x' h(t), x' h'(t) and the check value of one point (the largest check
  // value decides the check after the walk); h'(t) = 1 - e^-t = t - h(t)
  auto point = [&](int p, float t, float& z) -> float {
    const float xp = w.xp[p];
    const float h =
        t * t * fmaf(-t, fmaf(-t, fmaf(-t, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f);
    // Delta rho from its 2^-15 fixed point: exact, see small_int_to_float
    const float drho = fmaf(__int_as_float(0x4B400000 + (int)w.rho[p]), cq, dq);
    const float hmt = h - t;
    errmax = fmaxf(errmax, fabsf(fmaf(xp, hmt, -drho)));
    z = -xp * hmt;
    return xp * h;
  };
  Seg sg[2];
  lane_segments(fg, g.n_par, g.n_perp, lane, sg[0], sg[1]);
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {
    const Seg& sgm = sg[part];
    const float icf = small_int_to_float(sgm.c - fg.i_c), ic2f = icf * icf;
    // t = A + a2 j^2 with A = a0 + a1 ic + a3 ic^2 fixed on the segment, A in
    // double-float (error below 2^-44 tb), so that a point's t carries one
    // FP32 rounding relative to t itself
    df A = df_add(df{tc.h[0], tc.l[0]}, df_mul_f(df{tc.h[1], tc.l[1]}, icf));
    A = df_add(A, df_mul_f(df{tc.h[3], tc.l[3]}, ic2f));
    const float ah = A.hi, al = A.lo;
    df s0 = {0.f, 0.f}, s3 = {0.f, 0.f};
    float z0 = 0.f, z1 = 0.f, z2 = 0.f;  // sums of z, z j^2, z j^4
    float jf = small_int_to_float(sgm.j0), j2f = jf * jf;
    // |t| is largest at an end of the segment (t is monotone in j^2): a bound
    // over every point of the segment, x' = 0 included
    if (sgm.j1 > sgm.j0) {
      const float jl = small_int_to_float(sgm.j1 - 1);
      tmax = fmaxf(tmax, fmaxf(fabsf(fmaf(tc.h[2], j2f, ah)), fabsf(fmaf(tc.h[2], jl * jl, ah))));
    }
    int p = sgm.j0 * g.n_par + sgm.c;
    for (int j = sgm.j0; j < sgm.j1; ++j, p += g.n_par) {
      const float t = fmaf(tc.h[2], j2f, ah) + fmaf(tc.l[2], j2f, al);
      float z;
      const float y = point(p, t, z);
      z0 += z;
      z1 = fmaf(z, j2f, z1);
      z2 = fmaf(z, j2f * j2f, z2);
      if (EXACT) {
        s0 = df_add_f(s0, y);
        s3 = df_add_f(s3, y * j2f);
      } else {
        s0.hi += y;
        s3.hi = fmaf(y, j2f, s3.hi);
      }
      j2f = fmaf(2.f, jf, j2f + 1.f);  // (j + 1)^2
      jf += 1.f;
    }
    if (EXACT) {
      a[0] = df_add(a[0], s0);
      a[1] = df_add(a[1], df_mul_f(s0, icf));
      a[2] = df_add(a[2], df_mul_f(s0, ic2f));
      a[3] = df_add(a[3], s3);
    } else {
      a[0].hi += s0.hi;
      a[1].hi = fmaf(s0.hi, icf, a[1].hi);
      a[2].hi = fmaf(s0.hi, ic2f, a[2].hi);
      a[3].hi += s3.hi;
    }
    ab1 = fmaf(s0.hi, fabsf(icf), ab1);  // y >= 0
    {
      // the segment's column at v = b ic + c0 (FP32: J only enters the
      // certificate with its rounding bounded)
      const float v = fmaf(fg.b_f, icf, fg.c0_f), v2 = v * v;
      jz[0] += z0;
      jz[1] = fmaf(z0, v, jz[1]);
      jz[2] = fmaf(z0, v2, jz[2]);
      jz[3] = fmaf(z0, v2 * v, jz[3]);
      jz[4] = fmaf(z0, v2 * v2, jz[4]);
      jz[5] += z1;
      jz[6] = fmaf(z1, v, jz[6]);
      jz[7] = fmaf(z1, v2, jz[7]);
      jz[8] += z2;
    }
  }
  // warp totals of the J sums; lane k (mod 4) keeps row k of J:
  // J[k][l] = vol d2^q m(p, q) for phi_k phi_l = v^p w^q
#pragma unroll
  for (int i = 0; i < 9; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jz[i] += __shfl_xor_sync(FULL, jz[i], o);
  }
  {
    const float vh = fg.vol_h, vd = vh * fg.d2q_h[1], vdd = vh * fg.d2q_h[2];
    const float m00 = vh * jz[0], m10 = vh * jz[1], m20 = vh * jz[2], m30 = vh * jz[3],
                m40 = vh * jz[4], m01 = vd * jz[5], m11 = vd * jz[6], m21 = vd * jz[7],
                m02 = vdd * jz[8];
    const int k = lane & 3;
    // rows: (1, v, w, v^2) times (1, v, w, v^2)
    o.J[0] = k == 0 ? m00 : (k == 1 ? m10 : (k == 2 ? m01 : m20));
    o.J[1] = k == 0 ? m10 : (k == 1 ? m20 : (k == 2 ? m11 : m30));
    o.J[2] = k == 0 ? m01 : (k == 1 ? m11 : (k == 2 ? m02 : m21));
    o.J[3] = k == 0 ? m20 : (k == 1 ? m30 : (k == 2 ? m21 : m40));
  }
  // warp totals of the four sums, scattered (total k in lanes 8k..8k+7), in
  // double-float; then H_k in lane k and every total and H broadcast
  const df Ak = df_reduce_scatter4(a, lane);
  float B1 = ab1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) B1 += __shfl_xor_sync(FULL, B1, o);
  df A[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) A[k] = df{__shfl_sync(FULL, Ak.hi, 8 * k), __shfl_sync(FULL, Ak.lo, 8 * k)};
  const df vol = {fg.vol_h, fg.vol_l};
  // H_k = vol sum phi_k y with phi = (1, v, w, v^2), v = b ic + c0, w = d2 j^2:
  // H0 = vol A0, H1 = vol (b A1 + c0 A0), H2 = vol d2 A3,
  // H3 = vol (b^2 A2 + 2 b c0 A1 + c0^2 A0); lane k forms H_k
  df hk;
  {
    // H_k = vol (a0 A0 + a1 A1 + a2 A2 + a3 A3) with per-lane coefficients
    // (1,0,0,0), (c0,b,0,0), (0,0,0,d2), (c0^2,2bc0,b^2,0): no divergence
    const int k = lane & 3;
    const df zero = {0.f, 0.f};
    const df a0 = k == 0 ? df{1.f, 0.f}
                         : (k == 1 ? df{fg.coef_h[1][0], fg.coef_l[1][0]}
                                   : (k == 3 ? df{fg.coef_h[2][0], fg.coef_l[2][0]} : zero));
    const df a1 = k == 1 ? df{fg.coef_h[1][1], fg.coef_l[1][1]}
                         : (k == 3 ? df{fg.coef_h[2][1], fg.coef_l[2][1]} : zero);
    const df a2 = k == 3 ? df{fg.coef_h[2][2], fg.coef_l[2][2]} : zero;
    const df a3 = k == 2 ? df{fg.d2q_h[1], fg.d2q_l[1]} : zero;
    df acc = df_add(df_mul(a0, A[0]), df_mul(a1, A[1]));
    acc = df_add(acc, df_add(df_mul(a2, A[2]), df_mul(a3, A[3])));
    hk = df_mul(vol, acc);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) o.H[k] = df{__shfl_sync(FULL, hk.hi, k), __shfl_sync(FULL, hk.lo, k)};
  const df c0 = {fg.coef_h[1][0], fg.coef_l[1][0]}, b = {fg.coef_h[1][1], fg.coef_l[1][1]};
  const df c00 = {fg.coef_h[2][0], fg.coef_l[2][0]}, c21 = {fg.coef_h[2][1], fg.coef_l[2][1]};
  const df bb = {fg.coef_h[2][2], fg.coef_l[2][2]}, d2 = {fg.d2q_h[1], fg.d2q_l[1]};
  // y >= 0 (h >= 0, x' >= 0), so A0, A2, A3 are sums of non-negative terms
  const float vh = fg.vol_h;
  o.Habs[0] = vh * fabsf(A[0].hi);
  o.Habs[1] = vh * (fabsf(b.hi) * B1 + fabsf(c0.hi) * fabsf(A[0].hi));
  o.Habs[2] = vh * d2.hi * fabsf(A[3].hi);
  o.Habs[3] = vh * (bb.hi * fabsf(A[2].hi) + fabsf(c21.hi) * B1 + c00.hi * fabsf(A[0].hi));
  float tm = tmax, em = errmax;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    tm = fmaxf(tm, __shfl_xor_sync(FULL, tm, s));
    em = fmaxf(em, __shfl_xor_sync(FULL, em, s));
  }
  o.tmax = tm * 1.000001f;  // the end points' FP32 rounding
  o.errmax = em;
  o.viol = em > e_hi;
  o.uncertain = em > e_lo;
}

// FP32 Cholesky of the unit-diagonal scaling of M (the chord Jacobian).
struct Chol {
  float L[4][4];
  float inv[4];  // 1 / L_kk (the solves multiply: no division sequences)
  float d[4];    // 1 / sqrt(M_kk)
  bool ok;
};

__device__ __forceinline__ void chol_factor(const df M[10], Chol& ch) {
  float a[4][4];
  const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  ch.ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float mk = M[idx[k][k]].hi;
    ch.ok = ch.ok && mk > 0.f;
    ch.d[k] = mk > 0.f ? rsqrtf(mk) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) a[k][l] = M[idx[k][l]].hi * ch.d[k] * ch.d[l];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int l = 0; l < 4; ++l) ch.L[k][l] = 0.f;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int l = 0; l <= k; ++l) {
      float s = a[k][l];
#pragma unroll
      for (int q = 0; q < l; ++q) s = fmaf(-ch.L[k][q], ch.L[l][q], s);
      if (k == l) {
        ch.ok = ch.ok && s > 1e-6f;  // cond(M) beyond ~1e6: leave it to FP64
        // approximate square root: the factor only shapes the chord steps,
        // whose residuals are always formed with the exact M
        const float r = s > 0.f ? rsqrtf(s) : 1.f;
        ch.L[k][k] = s > 0.f ? s * r : 1.f;
        ch.inv[k] = r;
      } else {
        ch.L[k][l] = s * ch.inv[l];
      }
    }
  }
}

// delta = M^-1 r in FP32 through the scaled factorisation
__device__ __forceinline__ void chol_solve(const Chol& ch, const float r[4], float dlt[4]) {
  float y[4], z[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float s = r[k] * ch.d[k];
#pragma unroll
    for (int q = 0; q < k; ++q) s = fmaf(-ch.L[k][q], y[q], s);
    y[k] = s * ch.inv[k];
  }
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    float s = y[k];
#pragma unroll
    for (int q = k + 1; q < 4; ++q) s = fmaf(-ch.L[q][k], z[q], s);
    z[k] = s * ch.inv[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) dlt[k] = z[k] * ch.d[k];
}

struct NewtonState {
  int check_viol;  // end-to-end violation at the final lambda (valid when converged)
  float gres[4];   // |g_k| / S_k at the final lambda
};

// Round 1 of Eq. (6) with the chord Jacobian M from lam (in/out).
// Returns 1 converged, 0 not converged, -1 defer (precision guards).
__device__ int round1_fast(const GridK& g, const FastGridK& fg, const FastWS& w,
                           const QConst& c, const Moments& mo, const Chol& ch, df lam[4],
                           int max_iter, float step, float tol, float e, float s, int* iters,
                           float* r0, float* rlast, NewtonState& ns, int lane) {
  // lane k (mod 4) owns row k of M and component k of R: the matrix-vector
  // products run one row per lane and are gathered by shuffles
  const int kr = lane & 3;
  df rowM[4];
  {
    const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
#pragma unroll
    for (int l = 0; l < 4; ++l)
      rowM[l] = kr == 0 ? mo.M[idx[0][l]]
                        : (kr == 1 ? mo.M[idx[1][l]] : (kr == 2 ? mo.M[idx[2][l]] : mo.M[idx[3][l]]));
  }
  const df Rk = kr == 0 ? mo.R[0] : (kr == 1 ? mo.R[1] : (kr == 2 ? mo.R[2] : mo.R[3]));
  // 1 / S_k once per histogram: the residual tests multiply
  float invS[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) invS[k] = mo.S[k] > 1e-30f ? 1.f / mo.S[k] : 1e30f;
  // Error budget of g (absolute, per moment k), so that "converged" proves
  // |g_k| <= tol S_k with S_k = sum vol |phi_k| f at the final lambda:
  //  * moments: the residual is summed in units of Delta 2^-38 within two
  //    units per point, x' within one unit (its error enters as M lambda):
  //    Delta wk (2^-37 + 2^-38 tb), wk = vol sum |phi_k| over the grid;
  //  * the double-float assembly of g: below 2e-15 S_k;
  //  * H (after a pass, a bound on sum vol |phi_k| |x' h| in Habs):
  //    summation <= 3.5e-6 Habs in FP32 (none with TwoSum accumulation);
  //    terms: x' to float (2^-23), t to float (|dt| <= 2.1 u |t| + 2^-43 tb,
  //    |h'(t)| <= 1.06 |t|: 4.7 u relative to h), h's polynomial in FP32:
  //    <= 8e-7 Habs + 1.2e-13 tb tmax S_k; the series for h cut after t^5:
  //    |t|^6 e^|t| / 720 <= 0.003 t^4 h(t) for |t| <= 0.05;
  //  * S_k at f is at least S_k(x') (1 - tmax).
  // The budget is kept as one number, max_k err_k / S_k.
  bool force_pass = false;  // converged at lambda = 0: repeat the iteration with the check
  float erel = 0.f;
  for (int it = 0;; ++it) {
    df H[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float Jr[4] = {0.f, 0.f, 0.f, 0.f};  // row kr of dH/dlambda at lambda (after a pass)
    const bool zero_lam =
        lam[0].hi == 0.f && lam[1].hi == 0.f && lam[2].hi == 0.f && lam[3].hi == 0.f;
    int viol = 0, unc = 0;
    bool did_pass = false;
    float tmax = 0.f, errmax = 0.f, pmargin = 0.f;
    const float tb = fabsf(lam[0].hi) + fabsf(lam[1].hi) * fg.vmax + fabsf(lam[2].hi) * fg.wmax +
                     fabsf(lam[3].hi) * fg.vmax * fg.vmax;
    erel = 2e-15f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      erel = fmaxf(erel, fg.wk[k] * c.dl_f * fmaf(3.7e-12f, tb, 7.3e-12f) * invS[k] + 2e-15f);
    auto do_pass = [&]() {
      // FP32 rounding of the check (x' e^{-t} - x evaluated as x'(h - t) - Delta rho)
      // plus the 2^-15 Delta fixed point of rho
      const float margin = 4e-7f * (s * tb + c.dl_f) + 3.0517578125e-05f * c.dl_f + 1e-30f;
      PassOut po;
      const TCoef tc = make_tcoef(fg, lam);
      // FP32 sums first; again with TwoSum accumulation when their error bound
      // (<= 50 FP32 roundings per lane: 50 u sum|terms|) is too wide.  One
      // call site for both (the kernel is bound by instruction fetch).
      bool redo = false;
#pragma unroll 1
      for (int rep = 0; rep < 2; ++rep) {
        pass_warp(g, fg, w, c, tc, e - margin, e + margin, po, lane, rep != 0);
        if (rep) break;
#pragma unroll
        for (int k = 0; k < 4; ++k) redo = redo || 3.5e-6f * po.Habs[k] > 1e-13f * mo.S[k];
        if (!redo) break;
      }
      const float t2 = po.tmax * po.tmax;
      const float hrel = (redo ? 8e-7f : 4.3e-6f) + 0.003f * t2 * t2;
      float eh = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        H[k] = po.H[k];
        Jr[k] = po.J[k];
        eh = fmaxf(eh, hrel * po.Habs[k] * invS[k]);
      }
      erel += eh + 1.2e-13f * tb * po.tmax;
      viol = po.viol;
      unc = po.uncertain;
      did_pass = true;
      tmax = po.tmax;
      errmax = po.errmax;
      pmargin = margin;
    };
    if (!zero_lam || force_pass) do_pass();
    // g_k = -R_k - (M lambda)_k + H_k, row k in lane k, gathered; at
    // lambda = 0, g = -R (t = 0 on every point, so H = 0 even after a pass)
    df gk[4];
    {
      df gl = df_neg(Rk);
      if (!zero_lam) {
        df ml = df_mul(rowM[0], lam[0]);
#pragma unroll
        for (int l = 1; l < 4; ++l) ml = df_add(ml, df_mul(rowM[l], lam[l]));
        const df Hk = kr == 0 ? H[0] : (kr == 1 ? H[1] : (kr == 2 ? H[2] : H[3]));
        gl = df_add(df_neg(df_add(Rk, ml)), Hk);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        gk[k] = df{__shfl_sync(FULL, gl.hi, k), __shfl_sync(FULL, gl.lo, k)};
    }
    // residual bound (|g_k| + err_k) / (S_k (1 - tmax)); the floor err_k alone
    // must leave room below tol, else the histogram goes to the FP64 kernel
    // 1 / (1 - t) <= 1 + 1.06 t for t <= 0.05 (tmax > 0.05 defers below)
    const float sf = fmaf(1.06f, tmax, 1.f);
    const float floor_r = erel * sf;
    float res = 0.f;
    bool finite_ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float rk = fabsf(gk[k].hi) * invS[k] * sf + floor_r;
      finite_ok = finite_ok && isfinite(rk);
      ns.gres[k] = rk;
      res = fmaxf(res, rk);
    }
    if (it == 0) *r0 = res;
    *rlast = res;
    *iters = it;
    if (!finite_ok) return 0;
    if (tmax > 0.05f || floor_r > 0.5f * tol) return -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (fabsf(H[k].hi) > 1e-5f * mo.S[k]) return -1;
    if (res <= tol) {
      if (!did_pass) {  // lambda = 0 converged: still check every point
        force_pass = true;
        --it;
        continue;
      }
      if (unc && !viol) return -1;
      ns.check_viol = viol;
      return 1;
    }
    if (it == max_iter) return 0;
    // chord step with one refinement: delta = M^-1 g, then M^-1 (g - M delta).
    // The first step from lambda = 0 goes without the refinement: its FP32
    // error (~1e-6 of the step) is part of g at the next lambda, where the
    // pass measures it and the next step removes it.
    float r[4], d1[4], d2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = gk[k].hi;
    chol_solve(ch, r, d1);
    if (zero_lam) {
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] = df{step * d1[k], 0.f};
      continue;
    }
    df rd1;  // g - M d1 in row kr (double-float), reused by the certificate
    {
      df md = df_mul_f(rowM[0], d1[0]);
#pragma unroll
      for (int l = 1; l < 4; ++l) md = df_add(md, df_mul_f(rowM[l], d1[l]));
      const df gl = kr == 0 ? gk[0] : (kr == 1 ? gk[1] : (kr == 2 ? gk[2] : gk[3]));
      rd1 = df_add(gl, df_neg(md));
      const float rl = rd1.hi;
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = __shfl_sync(FULL, rl, k);
    }
    chol_solve(ch, r, d2);
    // Newton correction from the Jacobian of H that the pass measured:
    // g(l + d) = g(l) - M d + J d + R2 with J = sum vol phi phi^T x' h'(t), so
    // d3 = M^-1 (J (d1 + d2)) makes d1 + d2 + d3 solve (M - J) d = g up to
    // terms of second order (|J| is of order |t| |M|).  Without a pass,
    // lambda = 0 and J = 0.
    float dd[4], d3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) dd[k] = d1[k] + d2[k];
    float vk = 0.f;  // (J dd)_k in lane k
    if (did_pass) {
      vk = fmaf(Jr[3], dd[3], fmaf(Jr[2], dd[2], fmaf(Jr[1], dd[1], Jr[0] * dd[0])));
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = __shfl_sync(FULL, vk, k);
      chol_solve(ch, r, d3);
    }
    // Certificate after a pass (unit step d = d1 + d2 + d3): in row k,
    //   g_k(l + d) = (g - M dd)_k + (J dd - M d3 + J d3)_k + e_J + R2_k,
    // the first term in double-float, the second in FP32 (roundings within
    // 1e-6 of the sum of the magnitudes of its products, which also covers
    // dd's rounding of d1 + d2); e_J, the FP32 error of J, is below
    // 1e-5 tmax e^tmax tb_d S_k (|h'(t)| <= |t| e^|t|, about 70 roundings
    // per sum; tb_d bounds |d.phi| on the grid); the remainder of the
    // expansion is |R2_k| <= e^tt tb_d^2 S_k / 2 (h'' = e^-t, tt = tmax + tb_d).
    // g itself carries at most err_k (the budget above, its x' term widened
    // to the new lambda), and S_k at the new f is at least S_k (1 - tt).  The
    // pointwise check moves by at most x'max e^tmax (e^tb_d - 1).  When both
    // bounds hold, the step is taken and the histogram converged without the
    // pass at the new lambda.
    if (did_pass && step == 1.f && !viol && !unc) {
      float dn[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) dn[k] = dd[k] + d3[k];
      const float tbd = (fabsf(dn[0]) + fabsf(dn[1]) * fg.vmax + fabsf(dn[2]) * fg.wmax +
                         fabsf(dn[3]) * fg.vmax * fg.vmax) *
                        1.000001f;
      const float tt = tmax + tbd;
      if (tt < 0.05f) {
        const float grow = (1.f + 1.1f * tt) * 1.01f;  // e^tt for tt < 0.05, padded
        // residual of the solve, row k in lane k: g - M dd = (g - M d1) - M d2,
        // the second product in FP32 (|d2| ~ 1e-6 |d1|; its rounding in cabs)
        const float Sk = kr == 0 ? mo.S[0] : (kr == 1 ? mo.S[1] : (kr == 2 ? mo.S[2] : mo.S[3]));
        float rs = rd1.hi, corr = vk + rd1.lo, cabs = 0.f;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          rs = fmaf(-rowM[l].hi, d2[l], rs);
          corr = fmaf(Jr[l] - rowM[l].hi, d3[l], corr);
          cabs = fmaf(fabsf(Jr[l]) + fabsf(rowM[l].hi),
                      fabsf(dd[l]) + fabsf(d2[l]) + fabsf(d3[l]), cabs);
        }
        cabs += fabsf(rs);
        const float ek = erel * Sk +
                         3.7e-12f * c.dl_f * tbd *
                             (kr == 0 ? fg.wk[0] : (kr == 1 ? fg.wk[1] : (kr == 2 ? fg.wk[2] : fg.wk[3]))) +
                         1e-6f * cabs + Sk * grow * tbd * fmaf(1e-5f, tmax, 0.5f * tbd);
        const float bk = fabsf(rs + corr) + ek;
        const float rel = bk *
                          (kr == 0 ? invS[0] : (kr == 1 ? invS[1] : (kr == 2 ? invS[2] : invS[3]))) *
                          fmaf(1.06f, tt, 1.f);
        float worst = rel;
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) worst = fmaxf(worst, __shfl_xor_sync(FULL, worst, o));
        const float xpmax = s + 2.f * c.dl_f;
        if (worst <= tol && errmax + pmargin + xpmax * grow * tbd * 1.01f <= e) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            lam[k] = df_add_f(lam[k], d1[k]);
            lam[k] = df_add_f(lam[k], d2[k]);
            lam[k] = df_add_f(lam[k], d3[k]);
            ns.gres[k] = __shfl_sync(FULL, rel, k);
          }
          *iters = it + 1;
          *rlast = worst;
          ns.check_viol = 0;
          return 1;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      lam[k] = df_add_f(lam[k], step * d1[k]);
      lam[k] = df_add_f(lam[k], step * d2[k]);
      lam[k] = df_add_f(lam[k], step * d3[k]);
    }
  }
}

// Cold paths of fast_histogram, kept out of line: the kernel is bound by
// instruction fetch, so the common path should span as few cache lines as
// possible.  The kernel parameters are __grid_constant__, so these take them
// by reference without a copy.
struct WarmGuess {
  float l[4];
};

__device__ __noinline__ WarmGuess warm_guess(const FusedArgs& a, long long b, float d0, float d1,
                                             float d2, float d3, int lane) {
  const float dfeat[4] = {d0, d1, d2, d3};
  const int L = a.latent.L;
  double l0[4];
  mlp_eval_warp(
      a.mlp, [&](int k) { return k < L ? load_latent(a.latent, b, k) : dfeat[k - L]; }, l0,
      lane);
  WarmGuess o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.l[k] = (float)l0[k];
  return o;
}

// f = x' exp(-lambda.phi) with the rounding of the decompression kernel
__device__ __noinline__ void write_corrected(const FusedArgs& a, long long b, double dl,
                                             double lamd, FastWS& w, int lane) {
  const GridK& g = a.grid;
  double* fb = a.f_out + b * (long long)g.P;
  const int16_t* cb = a.codes + b * (long long)g.P;
  const double* xb = a.x + b * (long long)g.P;
  const float* xhb = a.xhat + b * a.ldx;
  double ld[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ld[k] = __shfl_sync(FULL, lamd, k);
  for (int i = lane; i < g.n_par; i += 32) w.t.ta[i] = corr_a(ld, g.vpar[i]);
  for (int j = lane; j < g.n_perp; j += 32) w.t.tb[j] = corr_b(ld, g.vperp2[j]);
  __syncwarp();
  PointIter pi(lane, g.n_par);
  for (; pi.p < g.P; pi.next()) {
    const int code = cb[pi.p];
    double xpd;
    if (code == AEQC_CODE_ESCAPE) xpd = __ldg(xb + pi.p);
    else if (code == AEQC_CODE_ZERO) xpd = 0.0;
    else xpd = __dadd_rn((double)__ldg(xhb + pi.p), __dmul_rn((double)code, dl));
    fb[pi.p] = corr_kl(xpd, w.t.ta[pi.i], w.t.tb[pi.j]);
  }
}

__device__ __noinline__ int write_outliers(const FusedArgs& a, long long b, int lane) {
  const int P = a.grid.P;
  return append_outliers(a.out, a.codes + b * (long long)P, a.x + b * (long long)P, P,
                         a.row0 + b, lane);
}

__device__ __noinline__ void write_features(const FusedArgs& a, long long b, float d0, float d1,
                                            float d2, float d3, int lane) {
  const LatentK& z = a.latent;
  float* fr = a.features + b * (long long)(z.L + 4);
  for (int l = lane; l < z.L; l += 32) fr[l] = load_latent(z, b, l);
  const float d = lane == 0 ? d0 : (lane == 1 ? d1 : (lane == 2 ? d2 : d3));
  if (lane < 4) fr[z.L + lane] = d;
}

// Verbatim storage after a certain end-to-end violation at both levels (the
// oracle's result for it: every code escapes, the raw values go to the
// outlier list, lambda = 0, f = x); out of line, since it is rare.
__device__ __noinline__ void write_verbatim(const FusedArgs& a, long long b, double s, unsigned st,
                                            int total_it, float d0, float d1, float d2,
                                            float d3, int lane) {
  const int P = a.grid.P;
  int16_t* cb = a.codes + b * (long long)P;
  const double* xb = a.x + b * (long long)P;
  for (int p = lane; p < P; p += 32) cb[p] = (int16_t)AEQC_CODE_ESCAPE;
  if (a.f_out) {
    double* fb = a.f_out + b * (long long)P;
    for (int p = lane; p < P; p += 32) fb[p] = __ldg(xb + p);
  }
  __syncwarp();
  if (a.out.count && append_outliers(a.out, cb, xb, P, a.row0 + b, lane))
    st |= AEQC_ST_OUTLIER_OVERFLOW;
  if (a.features) {
    const LatentK& z = a.latent;
    float* fr = a.features + b * (long long)(z.L + 4);
    for (int l = lane; l < z.L; l += 32) fr[l] = load_latent(z, b, l);
    const float d = lane == 0 ? d0 : (lane == 1 ? d1 : (lane == 2 ? d2 : d3));
    if (lane < 4) fr[z.L + lane] = d;
  }
  if (lane < 4) a.lambda[b * 4 + lane] = 0.0;
  if (lane == 0) {
    a.scale[b] = s;
    a.iters[b] = (uint8_t)(total_it > 255 ? 255 : total_it);
    a.status[b] = (uint16_t)st;
  }
  __syncwarp();
}

__device__ void fast_histogram(const FusedArgs& a, FastWS& w, long long b, int lane) {
  const GridK& g = a.grid;
  const ParamsK& pr = a.prm;
  const FastGridK& fg = a.fg;
  const int P = g.P;
  const double* xb = a.x + b * (long long)P;
  const float* xhb = a.xhat + b * a.ldx;
  int16_t* cb = a.codes + b * (long long)P;
  // max(x) and input validity, on the bit patterns (no FP64 compares); the
  // decoded row is fetched into L2 meanwhile, for the quantizer's loads
  for (int o = lane * 32; o < P; o += 32 * 32) asm volatile("prefetch.L2 [%0];" ::"l"(xhb + o));
  if (lane == 0) asm volatile("prefetch.L2 [%0];" ::"l"(xhb + P - 1));
  unsigned long long umax = 0;
  int bad = 0;
  // eight loads in flight per lane;
  // a point past the end reads as +0
#pragma unroll 1
  for (int p0 = lane; p0 < P; p0 += 32 * 8) {
    unsigned long long u[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int p = p0 + 32 * q;
      u[q] = p < P ? (unsigned long long)__double_as_longlong(__ldg(xb + p)) : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (u[q] <= 0x7FEFFFFFFFFFFFFFull) umax = u[q] > umax ? u[q] : umax;  // finite, >= +0
      else bad |= u[q] != 0x8000000000000000ull;                            // -0 counts as 0
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, umax, s);
    umax = o > umax ? o : umax;
  }
  bad = __any_sync(FULL, bad);
  const double s = __longlong_as_double((long long)umax);
  bool defer = bad || umax == 0;
  unsigned st = 0;
  df lam[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  int total_it = 0;
  float dfeat[4] = {0.f, 0.f, 0.f, 0.f};
  bool done = false, verbatim = false;
  const float s_f = float_of_bits(umax);  // s to 24 bits (margins only)
  // not unrolled: one copy of the quantizer and of the Newton loop serves both
  // levels (alpha, then alpha / 4)
#pragma unroll 1
  for (int level = 0; level < 2 && !defer && !done; ++level) {
    QConst c;
    if (!make_qconst(pr, s, level, c)) {
      defer = true;
      break;
    }
    Moments mo;
    phase_a(g, fg, xb, xhb, c, w, cb, mo, lane);
    st = mo.flags | (level ? AEQC_ST_ALPHA_RETRY : 0u) | (st & AEQC_ST_WARM_REJECTED);
    Chol ch;
    chol_factor(mo.M, ch);
    if (!ch.ok) {
      defer = true;
      break;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] = df{0.f, 0.f};
    int warm = 0;
    if (level == 0) {
      if (a.use_mlp || a.features) {  // the warm-start inputs d_k
#pragma unroll
        for (int k = 0; k < 4; ++k) dfeat[k] = mo.S[k] > 0.f ? mo.R[k].hi / mo.S[k] : 0.f;
      }
      if (a.use_mlp) {
        const WarmGuess l0 = warm_guess(a, b, dfeat[0], dfeat[1], dfeat[2], dfeat[3], lane);
        warm = 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float v = l0.l[k];
          warm = warm && isfinite(v);
          lam[k] = df{isfinite(v) ? v : 0.f, 0.f};
        }
        if (!warm) st |= AEQC_ST_WARM_REJECTED;
      }
    }
    // e = tau max(x) in FP32 (relative error ~2^-22, inside the check's margin)
    const float e = pr.tau_f * s_f;
    NewtonState ns;
    ns.check_viol = 0;
    int conv, it1 = 0, itw = 0;
    float r0 = 0.f, rw = 0.f;
    const float tol = pr.tol_f, step = pr.step_f;
    // one call site of the Newton loop: phase 0 the warm-start probation,
    // phase 1 its continuation, phase 2 the start from zero
    for (int phase = warm ? 0 : 2;;) {
      const int cap = phase == 0 ? pr.warm_iters
                                 : (phase == 1 ? pr.max_iter - pr.warm_iters : pr.max_iter);
      int itx = 0;
      float ra = 0.f, rb = 0.f;
      conv = round1_fast(g, fg, w, c, mo, ch, lam, cap, step, tol, e, s_f, &itx, &ra, &rb, ns,
                         lane);
      if (phase != 0) {
        it1 = itx;
        break;
      }
      itw = itx;
      r0 = ra;
      rw = rb;
      if (conv != 0) break;
      if (!isfinite(rw) || !isfinite(r0) || rw > pr.warm_reject_f || rw > r0) {
        st |= AEQC_ST_WARM_REJECTED;
#pragma unroll
        for (int k = 0; k < 4; ++k) lam[k] = df{0.f, 0.f};
        phase = 2;
      } else {
        phase = 1;
      }
    }
    total_it += itw + it1;
    if (conv != 1) {  // round 2 and verbatim storage belong to the FP64 kernel
      defer = true;
      break;
    }
    st |= AEQC_ST_CONVERGED;
    bool qoi_ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) qoi_ok = qoi_ok && ns.gres[k] <= pr.qoi_check_f;
    if (!ns.check_viol && qoi_ok) done = true;
    else if (level == 1) {
      // a certain pointwise violation at alpha / 4 too: verbatim, as the
      // oracle stores it; a moment check that fails only by its error bound
      // goes to the FP64 kernel
      if (ns.check_viol) verbatim = true;
      else defer = true;
    }
  }
  if (verbatim && !defer) {
    write_verbatim(a, b, s, (st & AEQC_ST_WARM_REJECTED) | AEQC_ST_VERBATIM | AEQC_ST_ALPHA_RETRY,
                   total_it, dfeat[0], dfeat[1], dfeat[2], dfeat[3], lane);
    return;
  }
  if (defer || !done) {
    if (lane == 0) {
      const int slot = atomicAdd(a.fb_count, 1);
      a.fb_list[slot] = (int)b;
    }
    __syncwarp();
    return;
  }
  // the multipliers as float64: lane k converts lambda_k (one warp instruction
  // sequence serves all four)
  double lamd = 0.0;
  {
    const int k = lane & 3;
    const df lk = k == 0 ? lam[0] : (k == 1 ? lam[1] : (k == 2 ? lam[2] : lam[3]));
    lamd = df_to_double(lk);
  }
  // outputs (the codes are in place)
  if (a.f_out) {
    const double dl =
        bin_width(pr.tau, s, (st & AEQC_ST_ALPHA_RETRY) ? pr.alpha * 0.25 : pr.alpha);
    write_corrected(a, b, dl, lamd, w, lane);
  }
  if (a.out.count && (st & AEQC_ST_CODE_ESCAPE)) {
    if (write_outliers(a, b, lane)) st |= AEQC_ST_OUTLIER_OVERFLOW;
  }
  if (a.features)
    write_features(a, b, dfeat[0], dfeat[1], dfeat[2], dfeat[3], lane);
  if (lane < 4) a.lambda[b * 4 + lane] = lamd;
  if (lane == 0) {
    a.scale[b] = s;
    a.iters[b] = (uint8_t)(total_it > 255 ? 255 : total_it);
    a.status[b] = (uint16_t)st;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(FW_MAX * 32, 1)
    fused_fast_kernel(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FastWS& w = reinterpret_cast<FastWS*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int fw = blockDim.x >> 5;
  const long long nw = (long long)gridDim.x * fw;
  for (long long b = (long long)blockIdx.x * fw + (threadIdx.x >> 5); b < a.n; b += nw)
    fast_histogram(a, w, b, lane);
}

void split_df(double v, float* h, float* l) {
  *h = (float)v;
  *l = (float)(v - (double)*h);
}

}  // namespace

int make_fast_grid(const GridK& g, FastGridK* out) {
  FastGridK f;
  memset(&f, 0, sizeof(f));
  *out = f;
  if (g.has_vol || g.n_par < 2 || g.n_perp < 2) return AEQC_OK;
  // integer weights must stay below 2^24 (|i - i_c|^4, j^4) and the x' sums
  // of one lane below 2^62
  if (g.n_par > 64 || g.n_perp > 64) return AEQC_OK;
  const double b = (g.vpar[g.n_par - 1] - g.vpar[0]) / (double)(g.n_par - 1);
  if (!(b > 0.0)) return AEQC_OK;
  double vmax = 0.0;
  for (int i = 0; i < g.n_par; ++i) vmax = fmax(vmax, fabs(g.vpar[i]));
  int ic = (int)llround(-g.vpar[0] / b);  // index nearest to v_par = 0
  if (ic < 0) ic = 0;
  if (ic > g.n_par - 1) ic = g.n_par - 1;
  const double c0 = g.vpar[ic];
  for (int i = 0; i < g.n_par; ++i)
    if (fabs(g.vpar[i] - (b * (i - ic) + c0)) > 1e-13 * vmax) return AEQC_OK;
  if (g.vperp2[0] != 0.0) return AEQC_OK;
  const double d2 = g.vperp2[1];
  if (!(d2 > 0.0)) return AEQC_OK;
  for (int j = 0; j < g.n_perp; ++j)
    if (fabs(g.vperp2[j] - d2 * (double)j * (double)j) > 1e-13 * g.vperp2[g.n_perp - 1])
      return AEQC_OK;
  // exact 64-bit moment sums: for every weight (i - i_c)^r j^(2q) of the
  // moments, the sum of |weight| over the grid stays below 2^31, so that the
  // totals of X' (split at bit 31: parts below 2^31 and 2^29) stay below 2^62;
  // the residual rho (|rho| <= 2^37) enters only with the weights 1, i - i_c,
  // (i - i_c)^2 and j^2, whose sums must stay below 2^25
  {
    double wsum[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < g.n_perp; ++j)
      for (int i = 0; i < g.n_par; ++i) {
        const double a = fabs((double)(i - ic)), j2 = (double)j * j;
        const double wt[9] = {1, a, a * a, a * a * a, a * a * a * a, j2, a * j2, a * a * j2,
                              j2 * j2};
        for (int q = 0; q < 9; ++q) wsum[q] += wt[q];
      }
    for (int q = 0; q < 9; ++q)
      if (!(wsum[q] < 2147483648.0)) return AEQC_OK;
    if (!(wsum[0] < 33554432.0 && wsum[1] < 33554432.0 && wsum[2] < 33554432.0 &&
          wsum[5] < 33554432.0))
      return AEQC_OK;
  }
  // vol sum |phi_k| over the grid, rounded up: per-point rounding of the
  // residual and of x' enters the moments with at most these weights
  {
    double w[4] = {0, 0, 0, 0};
    for (int j = 0; j < g.n_perp; ++j)
      for (int i = 0; i < g.n_par; ++i) {
        w[0] += 1.0;
        w[1] += fabs(g.vpar[i]);
        w[2] += g.vperp2[j];
        w[3] += g.vpar[i] * g.vpar[i];
      }
    for (int k = 0; k < 4; ++k) f.wk[k] = (float)(w[k] * g.vol_uniform * 1.001);
  }
  f.ok = 1;
  f.i_c = ic;
  f.b = b;
  f.c0 = c0;
  f.d2 = d2;
  split_df(g.vol_uniform, &f.vol_h, &f.vol_l);
  split_df(1.0, &f.d2q_h[0], &f.d2q_l[0]);
  split_df(d2, &f.d2q_h[1], &f.d2q_l[1]);
  split_df(d2 * d2, &f.d2q_h[2], &f.d2q_l[2]);
  const double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0},
                              {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  for (int p = 0; p < 5; ++p)
    for (int r = 0; r < 5; ++r) {
      const double cf = r <= p ? binom[p][r] * pow(b, r) * pow(c0, p - r) : 0.0;
      split_df(cf, &f.coef_h[p][r], &f.coef_l[p][r]);
    }
  f.b_f = (float)b;
  f.c0_f = (float)c0;
  f.vmax = (float)vmax;
  f.wmax = (float)g.vperp2[g.n_perp - 1];
  {
    const int rw = g.n_par - (g.n_par >= 32 ? 32 : 0);  // >= 1 (n_par in [2, 64])
    f.seg_nchunk = 32 / rw;
    f.seg_rpc = (g.n_perp + f.seg_nchunk - 1) / f.seg_nchunk;
    f.seg_mul = (65536 + rw - 1) / rw;
    for (int l = 0; l < 32; ++l)
      if ((l * f.seg_mul) >> 16 != l / rw) return AEQC_OK;  // never: 2^16 > 32 rw
  }
  *out = f;
  return AEQC_OK;
}

int launch_fused_fast(const FusedArgs& a_in, cudaStream_t s, int warps_per_sm) {
  if (a_in.n <= 0) return AEQC_OK;
  FusedArgs a = a_in;
  if (!a.fg.ok || a.prm.loss != 0 || a.grid.has_vol) return launch_fused_fp64(a, s);
  AEQC_CUDA_TRY(cudaMemsetAsync(a.fb_count, 0, sizeof(int), s));
  // warps per CTA (= per SM): the tuned count, else sixteen
  const int fw = warps_per_sm >= 4 && warps_per_sm <= FW_MAX && warps_per_sm % 4 == 0
                     ? warps_per_sm
                     : FW_MAX;
  const size_t smem = sizeof(FastWS) * fw;
  {
    const int rc = raise_smem_limit((const void*)fused_fast_kernel, (int)smem);
    if (rc) return rc;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (a.n + fw - 1) / fw;
  if (blocks > sms) blocks = sms;
  fused_fast_kernel<<<(unsigned)blocks, fw * 32, smem, s>>>(a);
  int rc = check_launch("fused_fast_kernel");
  if (rc) return rc;
  return launch_fused_fp64_list(a, a.fb_list, a.fb_count, s);
}

}  // namespace aeqc
