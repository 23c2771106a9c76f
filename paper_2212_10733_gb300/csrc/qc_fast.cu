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

constexpr int FW = 4;  // warps per CTA

struct FastWS {
  float xp[AEQC_MAX_P];   // x' (float) for the Newton passes
  float rho[AEQC_MAX_P];  // (x - x') / Delta (float) for the end-to-end check
  int16_t codes[AEQC_MAX_P];
  double ta[AEQC_MAX_NPAR], tb[AEQC_MAX_NPERP];  // exponential tables for f_out
};

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
__device__ __forceinline__ df df_ldexp(df x, int n) {  // exact for normal results
  return {ldexpf(x.hi, n), ldexpf(x.lo, n)};
}
__device__ __forceinline__ df df_wsum(df x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df y = {__shfl_xor_sync(FULL, x.hi, o), __shfl_xor_sync(FULL, x.lo, o)};
    x = df_add(x, y);
  }
  return x;
}
// the top 48 bits of an int64 as a float pair (relative error <= 2^-48)
__device__ __forceinline__ df df_from_ll(long long v) {
  if (v == 0) return {0.f, 0.f};
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << lz;
  const int e = 63 - lz;
  float hi = __fmul_rn(__uint2float_rn((unsigned)(m >> 40)), exp2i(e - 23));
  float lo = __fmul_rn(__uint2float_rn((unsigned)((m >> 16) & 0xFFFFFFull)), exp2i(e - 47));
  if (v < 0) {
    hi = -hi;
    lo = -lo;
  }
  return quick_sum(hi, lo);
}

// ---- integer decomposition of the inputs ----------------------------------

// floor(x 2^sh) of a finite double x >= 0 given its bits; inexact |= bits dropped.
__device__ __forceinline__ long long fix_f64(unsigned long long u, int sh, bool& inexact) {
  const int E = (int)(u >> 52) & 0x7ff;
  unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  int e2;
  if (E == 0) {
    e2 = -1074 + sh;
  } else {
    M |= 1ull << 52;
    e2 = E - 1075 + sh;
  }
  if (e2 >= 0) return (long long)(M << e2);  // small: the value is below 2^60
  const int r = -e2;
  if (r >= 64) {
    inexact |= M != 0;
    return 0;
  }
  inexact |= (M & ((1ull << r) - 1ull)) != 0;
  return (long long)(M >> r);
}

// floor(xh 2^sh) of a finite float given its bits (two's complement result).
__device__ __forceinline__ long long fix_f32(unsigned v, int sh, bool& inexact) {
  const int E = (v >> 23) & 0xff;
  unsigned long long M = v & 0x7fffffu;
  int e2;
  if (E == 0) {
    e2 = -149 + sh;
  } else {
    M |= 1ull << 23;
    e2 = E - 150 + sh;
  }
  long long mag;
  bool st = false;
  if (e2 >= 0) {
    mag = (long long)(M << e2);  // below 2^61 after the escape pre-check
  } else {
    const int r = -e2;
    if (r >= 64) {
      st = M != 0;
      mag = 0;
    } else {
      st = (M & ((1ull << r) - 1ull)) != 0;
      mag = (long long)(M >> r);
    }
  }
  inexact |= st;
  if (v >> 31) return -mag - (st ? 1 : 0);
  return mag;
}

// binary exponent E of a positive finite double: d in [2^(E-1), 2^E)
__device__ __forceinline__ int exponent_of(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int E = (int)(u >> 52) & 0x7ff;
  if (E) return E - 1022;
  return (63 - __clzll((long long)u)) - 1073;  // subnormal
}

// Per-histogram constants of the integer quantizer.
struct QConst {
  double dl;  // Delta = 2^k
  float dl_f;
  int k;
  int F;    // fractional bits of the fixed-point values (units of Delta)
  int FX;   // fractional bits of x' in the moment sums
  int thr;  // |xhat| >= 2^thr certainly escapes
  long long half, mask;
};

__device__ __forceinline__ bool make_qconst(double tau, double s, double alpha, int xbits,
                                            QConst& c) {
  c.dl = bin_width(tau, s, alpha);
  if (!(c.dl > 0.0) || !isfinite(c.dl)) return false;
  c.k = exponent_of(c.dl) - 1;
  const int IBx = exponent_of(s) - c.k;  // s / Delta < 2^IBx
  const int IB = (IBx > 15 ? IBx : 15) + 2;
  c.F = 62 - IB;
  c.FX = xbits - IBx;
  c.thr = c.k + IB - 1;
  c.half = 1ll << (c.F - 1);
  c.mask = (1ll << c.F) - 1;
  // float copies: Delta and the scale factors of the moment sums must be
  // normal floats (moments are scaled by vol Delta 2^-30 and vol Delta 2^-FX)
  const bool ok = c.F >= 31 && c.FX >= 1 && c.F - c.FX >= 1 && IBx >= 1 &&
                  c.k - 64 >= -100 && c.k + 20 <= 100;
  c.dl_f = ok ? exp2i(c.k) : 0.f;
  return ok;
}

struct PointQ {
  int code;
  int rho32;  // round((x - x') / Delta * 2^30)
  long long xpw;  // round(x' / Delta * 2^FX)
  float xpf;  // x' (float)
};

// Exact quantizer decision for one point (x finite, x >= 0).
__device__ __forceinline__ PointQ quant_point_int(double x, float xh, const QConst& c) {
  PointQ o;
  const unsigned long long u =
      (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned v = __float_as_uint(xh);
  const int Eh = (v >> 23) & 0xff;
  const int sh = c.F - c.k;
  bool inex = false;
  const long long X = fix_f64(u, sh, inex);
  long long rho_fix = 0, xp_fix;
  bool hard = false;
  if (Eh == 255 || Eh - 127 >= c.thr) {  // non-finite or certainly |q| > 32766
    o.code = AEQC_CODE_ESCAPE;
    xp_fix = X;
  } else {
    const long long Xh = fix_f32(v, sh, inex);
    const long long D = X - Xh;
    const long long m = D >> c.F;
    const long long frac = D & c.mask;
    long long q = 0;
    if (frac < c.half) q = m;
    else if (frac > c.half) q = m + 1;
    else if (inex) hard = true;
    else q = m + (m & 1);
    if (!hard) {
      if (q > AEQC_CODE_MAX || q < -AEQC_CODE_MAX) {
        o.code = AEQC_CODE_ESCAPE;
        xp_fix = X;
      } else {
        const long long G = Xh + q * (1ll << c.F);
        int zero;
        if (G <= -1) {
          zero = 1;
        } else {
          const long long A = G - 2 * X;
          if (A >= 2) zero = 1;
          else if (A <= -1) zero = 0;
          else if (inex) {
            zero = 0;
            hard = true;
          } else zero = A > 0;
        }
        if (!hard) {
          if (zero) {
            o.code = AEQC_CODE_ZERO;
            rho_fix = X;
            xp_fix = 0;
          } else {
            o.code = (int)q;
            rho_fix = D - q * (1ll << c.F);
            xp_fix = G;
          }
        }
      }
    }
  }
  if (hard) {
    double xpd;
    o.code = quant_point_fp64(x, (double)xh, c.dl, &xpd);
    const double rd = __ddiv_rn(__dsub_rn(x, xpd), c.dl);
    o.rho32 = __double2int_rn(ldexp(rd, 30));
    o.xpw = __double2ll_rn(ldexp(__ddiv_rn(xpd, c.dl), c.FX));
    o.xpf = (float)xpd;
    return o;
  }
  // round to nearest: a floor would bias every cell the same way, and the
  // high-order weights (v^4 up to 256) would turn that into a systematic error
  o.rho32 = (int)((rho_fix + (1ll << (c.F - 31))) >> (c.F - 30));
  o.xpw = (xp_fix + (1ll << (c.F - c.FX - 1))) >> (c.F - c.FX);
  if (o.code == AEQC_CODE_ESCAPE) o.xpf = ldexpf((float)o.xpw, -c.FX) * c.dl_f;
  else if (o.code == AEQC_CODE_ZERO) o.xpf = 0.f;
  else o.xpf = fmaf((float)o.code, c.dl_f, xh);
  return o;
}

// The lambda-independent moments of one quantization level, double-float.
struct Moments {
  df R[4];       // sum vol phi_k (x - x')
  df M[10];      // upper triangle of sum vol phi phi^T x' (m00 m01 m02 m03 m11 ...)
  float S[4];    // sum vol |phi_k| x'
  unsigned flags;  // CODE_ESCAPE / AE_EXACT
};

// Quantize the histogram (row xb, decoded row xhb) into shared memory and
// accumulate its moments.
__device__ void phase_a(const GridK& g, const FastGridK& fg, const double* xb,
                        const float* xhb, const QConst& c, FastWS& w, Moments& mo, int lane) {
  long long U[4] = {0, 0, 0, 0};
  long long T[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // T00 T10 T20 T30 T40 T01 T11 T21 T02
  float s1 = 0.f;
  int esc = 0, nonzero = 0;
  const float b_f = (float)fg.b, c0_f = (float)fg.c0;
  PointIter it(lane, g.n_par);
  for (; it.p < g.P; it.next()) {
    const double x = __ldg(xb + it.p);
    const float xh = __ldg(xhb + it.p);
    const PointQ o = quant_point_int(x, xh, c);
    w.codes[it.p] = (int16_t)o.code;
    w.xp[it.p] = o.xpf;
    w.rho[it.p] = ldexpf((float)o.rho32, -30);
    esc |= o.code == AEQC_CODE_ESCAPE;
    nonzero |= o.code != 0;
    const int ic = it.i - fg.i_c, j2 = it.j * it.j;
    const int ic2 = ic * ic;
    const long long r = o.rho32, X = o.xpw;
    U[0] += r;
    U[1] += r * ic;
    U[2] += r * ic2;
    U[3] += r * j2;
    T[0] += X;
    T[1] += X * ic;
    T[2] += X * ic2;
    T[3] += X * (ic2 * ic);
    T[4] += X * (ic2 * ic2);
    T[5] += X * j2;
    T[6] += X * (ic * j2);
    T[7] += X * (ic2 * j2);
    T[8] += X * (j2 * j2);
    s1 = fmaf(o.xpf, fabsf(fmaf(b_f, (float)ic, c0_f)), s1);
  }
  __syncwarp();
  // per-lane sums stay below 2^60; convert, then add across the warp exactly
  df u[4], t[9];
#pragma unroll
  for (int q = 0; q < 4; ++q) u[q] = df_wsum(df_from_ll(U[q]));
#pragma unroll
  for (int q = 0; q < 9; ++q) t[q] = df_wsum(df_from_ll(T[q]));
  const float S1 = df_wsum(df{s1, 0.f}).hi;
  const df vol = {fg.vol_h, fg.vol_l};
  const df sr = df_ldexp(vol, c.k - 30), sm = df_ldexp(vol, c.k - c.FX);
  const df b = {fg.coef_h[1][1], fg.coef_l[1][1]};   // C(1,1) b = b
  const df c0 = {fg.coef_h[1][0], fg.coef_l[1][0]};  // C(1,0) c0 = c0
  const df d2 = {fg.d2q_h[1], fg.d2q_l[1]};
  // R_k = vol Delta 2^-30 sum phi_k rho32, phi = (1, v, w, v^2), v = b ic + c0
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
  // m(p, q) = vol Delta 2^-FX d2^q sum_r C(p,r) b^r c0^(p-r) T[r][q]
  const df* Tq0 = t;      // T[r][0], r = 0..4
  const df Tq1[3] = {t[5], t[6], t[7]};
  auto mom = [&](int p, int q) {
    df acc = {0.f, 0.f};
    for (int r = 0; r <= p; ++r) {
      const df tr = q == 0 ? Tq0[r] : (q == 1 ? Tq1[r] : t[8]);
      acc = df_add(acc, df_mul(df{fg.coef_h[p][r], fg.coef_l[p][r]}, tr));
    }
    return df_mul(sm, df_mul(df{fg.d2q_h[q], fg.d2q_l[q]}, acc));
  };
  const df m00 = mom(0, 0), m10 = mom(1, 0), m20 = mom(2, 0), m30 = mom(3, 0),
           m40 = mom(4, 0), m01 = mom(0, 1), m11 = mom(1, 1), m21 = mom(2, 1),
           m02 = mom(0, 2);
  mo.M[0] = m00; mo.M[1] = m10; mo.M[2] = m01; mo.M[3] = m20;
  mo.M[4] = m20; mo.M[5] = m11; mo.M[6] = m30;
  mo.M[7] = m02; mo.M[8] = m21;
  mo.M[9] = m40;
  mo.S[0] = m00.hi;
  mo.S[1] = fg.vol_h * S1;
  mo.S[2] = m01.hi;
  mo.S[3] = m20.hi;
  mo.flags = 0;
  if (__any_sync(FULL, esc)) mo.flags |= AEQC_ST_CODE_ESCAPE;
  if (!__any_sync(FULL, nonzero)) mo.flags |= AEQC_ST_AE_EXACT;
}

struct PassOut {
  df H[4];
  float Habs[4];  // bounds on the sums of |terms| (for the FP32 rounding bound)
  float tmax;
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
template <bool EXACT>
__device__ void pass_warp(const GridK& g, const FastGridK& fg, const FastWS& w,
                          const QConst& c, const TCoef& tc, float e_lo, float e_hi, PassOut& o,
                          int lane) {
  df a[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // sums of y, y ic, y ic^2, y j^2
  float ab1 = 0.f, tmax = 0.f;
  int viol = 0, unc = 0;
  // walk p = lane, lane + 32, ... keeping ic and j^2 as exact floats
  int i = lane % g.n_par, j = lane / g.n_par;
  float icf = (float)(i - fg.i_c), jf = (float)j, j2f = jf * jf;
  const float npf = (float)g.n_par;
  for (int p = lane; p < g.P;) {
    const float xp = w.xp[p];
    const float ic2f = icf * icf;
    const float th = fmaf(tc.h[3], ic2f, fmaf(tc.h[1], icf, fmaf(tc.h[2], j2f, tc.h[0])));
    const float tl = fmaf(tc.l[3], ic2f, fmaf(tc.l[1], icf, fmaf(tc.l[2], j2f, tc.l[0])));
    const float t = th + tl;
    const float h =
        t * t * fmaf(-t, fmaf(-t, fmaf(-t, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f);
    const float y = xp * h;
    const float yi = y * icf;
    if (EXACT) {
      a[0] = df_add_f(a[0], y);
      a[1] = df_add_f(a[1], yi);
      a[2] = df_add_f(a[2], yi * icf);
      a[3] = df_add_f(a[3], y * j2f);
    } else {
      a[0].hi += y;
      a[1].hi += yi;
      a[2].hi = fmaf(yi, icf, a[2].hi);
      a[3].hi = fmaf(y, j2f, a[3].hi);
    }
    ab1 += fabsf(yi);
    if (xp > 0.f) tmax = fmaxf(tmax, fabsf(t));
    const float err = fabsf(fmaf(xp, h - t, -c.dl_f * w.rho[p]));
    viol |= err > e_hi;
    unc |= err > e_lo;
    p += 32;
    i += 32;
    icf += 32.f;
    while (i >= g.n_par) {
      i -= g.n_par;
      icf -= npf;
      j2f = fmaf(2.f, jf, j2f + 1.f);  // (j + 1)^2
      jf += 1.f;
    }
  }
  df A[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) A[k] = df_wsum(a[k]);
  const float B1 = df_wsum(df{ab1, 0.f}).hi;
  const df vol = {fg.vol_h, fg.vol_l};
  const df c0 = {fg.coef_h[1][0], fg.coef_l[1][0]}, b = {fg.coef_h[1][1], fg.coef_l[1][1]};
  const df c00 = {fg.coef_h[2][0], fg.coef_l[2][0]}, c21 = {fg.coef_h[2][1], fg.coef_l[2][1]};
  const df bb = {fg.coef_h[2][2], fg.coef_l[2][2]}, d2 = {fg.d2q_h[1], fg.d2q_l[1]};
  // H_k = vol sum phi_k y with phi = (1, v, w, v^2), v = b ic + c0, w = d2 j^2
  o.H[0] = df_mul(vol, A[0]);
  o.H[1] = df_mul(vol, df_add(df_mul(b, A[1]), df_mul(c0, A[0])));
  o.H[2] = df_mul(vol, df_mul(d2, A[3]));
  o.H[3] = df_mul(vol, df_add(df_add(df_mul(bb, A[2]), df_mul(c21, A[1])), df_mul(c00, A[0])));
  // y >= 0 (h >= 0, x' >= 0), so A0, A2, A3 are sums of non-negative terms
  const float vh = fg.vol_h;
  o.Habs[0] = vh * fabsf(A[0].hi);
  o.Habs[1] = vh * (fabsf(b.hi) * B1 + fabsf(c0.hi) * fabsf(A[0].hi));
  o.Habs[2] = vh * d2.hi * fabsf(A[3].hi);
  o.Habs[3] = vh * (bb.hi * fabsf(A[2].hi) + fabsf(c21.hi) * B1 + c00.hi * fabsf(A[0].hi));
  float tm = tmax;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) tm = fmaxf(tm, __shfl_xor_sync(FULL, tm, s));
  o.tmax = tm;
  o.viol = __any_sync(FULL, viol);
  o.uncertain = __any_sync(FULL, unc);
}

// FP32 Cholesky of the unit-diagonal scaling of M (the chord Jacobian).
struct Chol {
  float L[4][4];
  float d[4];  // 1 / sqrt(M_kk)
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
        ch.L[k][k] = s > 0.f ? sqrtf(s) : 1.f;
      } else {
        ch.L[k][l] = s / ch.L[l][l];
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
    y[k] = s / ch.L[k][k];
  }
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    float s = y[k];
#pragma unroll
    for (int q = k + 1; q < 4; ++q) s = fmaf(-ch.L[q][k], z[q], s);
    z[k] = s / ch.L[k][k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) dlt[k] = z[k] * ch.d[k];
}

// (M v)_k in double-float for a float vector v
__device__ __forceinline__ void df_matvec_f(const df M[10], const float v[4], df out[4]) {
  const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    df acc = df_mul_f(M[idx[k][0]], v[0]);
#pragma unroll
    for (int l = 1; l < 4; ++l) acc = df_add(acc, df_mul_f(M[idx[k][l]], v[l]));
    out[k] = acc;
  }
}

// (M lambda)_k in double-float
__device__ __forceinline__ void df_matvec(const df M[10], const df lam[4], df out[4]) {
  const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    df acc = df_mul(M[idx[k][0]], lam[0]);
#pragma unroll
    for (int l = 1; l < 4; ++l) acc = df_add(acc, df_mul(M[idx[k][l]], lam[l]));
    out[k] = acc;
  }
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
  for (int it = 0;; ++it) {
    df H[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const bool zero_lam =
        lam[0].hi == 0.f && lam[1].hi == 0.f && lam[2].hi == 0.f && lam[3].hi == 0.f;
    int viol = 0, unc = 0;
    bool did_pass = false;
    float tmax = 0.f;
    auto do_pass = [&]() {
      const float tb = fabsf(lam[0].hi) + fabsf(lam[1].hi) * fg.vmax + fabsf(lam[2].hi) * fg.wmax +
                       fabsf(lam[3].hi) * fg.vmax * fg.vmax;
      // FP32 rounding of the check (x' e^{-t} - x evaluated as x'(h - t) - Delta rho)
      const float margin = 4e-7f * (s * tb + c.dl_f) + 1e-30f;
      PassOut po;
      const TCoef tc = make_tcoef(fg, lam);
      pass_warp<false>(g, fg, w, c, tc, e - margin, e + margin, po, lane);
      bool redo = false;
#pragma unroll
      for (int k = 0; k < 4; ++k)  // 48 FP32 additions per lane: |error| <= 48 u sum|terms|
        redo = redo || 3e-6f * po.Habs[k] > 1e-13f * mo.S[k];
      if (redo) pass_warp<true>(g, fg, w, c, tc, e - margin, e + margin, po, lane);
#pragma unroll
      for (int k = 0; k < 4; ++k) H[k] = po.H[k];
      viol = po.viol;
      unc = po.uncertain;
      did_pass = true;
      tmax = po.tmax;
    };
    if (!zero_lam) do_pass();
    df Ml[4];
    df_matvec(mo.M, lam, Ml);
    df gk[4];
    float res = 0.f;
    bool finite_ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gk[k] = df_add(df_neg(df_add(mo.R[k], Ml[k])), H[k]);
      const float den = mo.S[k] > 0.f ? mo.S[k] : 1e-30f;
      const float rk = fabsf(gk[k].hi) / den;
      finite_ok = finite_ok && isfinite(rk);
      ns.gres[k] = rk;
      res = fmaxf(res, rk);
    }
    if (it == 0) *r0 = res;
    *rlast = res;
    *iters = it;
    if (!finite_ok) return 0;
    if (tmax > 0.05f) return -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (fabsf(H[k].hi) > 1e-5f * mo.S[k]) return -1;
    if (res <= tol) {
      if (!did_pass) do_pass();  // lambda = 0 converged: still check every point
      if (unc && !viol) return -1;
      ns.check_viol = viol;
      return 1;
    }
    if (it == max_iter) return 0;
    // chord step with one refinement: delta = M^-1 g, then M^-1 (g - M delta)
    float r[4], d1[4], d2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = gk[k].hi;
    chol_solve(ch, r, d1);
    df Md[4];
    df_matvec_f(mo.M, d1, Md);
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = df_add(gk[k], df_neg(Md[k])).hi;
    chol_solve(ch, r, d2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      lam[k] = df_add_f(lam[k], step * d1[k]);
      lam[k] = df_add_f(lam[k], step * d2[k]);
    }
  }
}

__device__ void fast_histogram(const FusedArgs& a, FastWS& w, long long b, int lane) {
  const GridK& g = a.grid;
  const ParamsK& pr = a.prm;
  const FastGridK& fg = a.fg;
  const int P = g.P;
  const double* xb = a.x + b * (long long)P;
  const float* xhb = a.xhat + b * a.ldx;
  // max(x) and input validity, on the bit patterns (no FP64 compares)
  unsigned long long umax = 0;
  int bad = 0;
  for (int p = lane; p < P; p += 32) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(__ldg(xb + p));
    if (u <= 0x7FEFFFFFFFFFFFFFull) umax = u > umax ? u : umax;  // finite, >= +0
    else bad |= u != 0x8000000000000000ull;                      // -0 counts as 0
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
  bool done = false;
  const float s_f = (float)s;
  for (int level = 0; level < 2 && !defer && !done; ++level) {
    QConst c;
    if (!make_qconst(pr.tau, s, level ? pr.alpha * 0.25 : pr.alpha, fg.xbits, c)) {
      defer = true;
      break;
    }
    Moments mo;
    phase_a(g, fg, xb, xhb, c, w, mo, lane);
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
#pragma unroll
      for (int k = 0; k < 4; ++k)
        dfeat[k] = mo.S[k] > 0.f ? mo.R[k].hi / mo.S[k] : 0.f;
      if (a.use_mlp) {
        const int L = a.latent.L;
        double l0[4];
        mlp_eval_warp(
            a.mlp, [&](int k) { return k < L ? load_latent(a.latent, b, k) : dfeat[k - L]; },
            l0, lane);
        warm = 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float v = (float)l0[k];
          warm = warm && isfinite(v);
          lam[k] = df{isfinite(v) ? v : 0.f, 0.f};
        }
        if (!warm) st |= AEQC_ST_WARM_REJECTED;
      }
    }
    const float e = (float)(pr.tau * s);
    NewtonState ns;
    ns.check_viol = 0;
    int conv, it1 = 0, itw = 0;
    float r0 = 0.f, rw = 0.f, rd0, rd1;
    const float tol = (float)pr.tol, step = (float)pr.step_s;
    if (warm) {
      conv = round1_fast(g, fg, w, c, mo, ch, lam, pr.warm_iters, step, tol, e, s_f, &itw, &r0,
                         &rw, ns, lane);
      if (conv == 0) {
        if (!isfinite(rw) || !isfinite(r0) || rw > (float)pr.warm_reject || rw > r0) {
          st |= AEQC_ST_WARM_REJECTED;
#pragma unroll
          for (int k = 0; k < 4; ++k) lam[k] = df{0.f, 0.f};
          conv = round1_fast(g, fg, w, c, mo, ch, lam, pr.max_iter, step, tol, e, s_f, &it1,
                             &rd0, &rd1, ns, lane);
        } else {
          conv = round1_fast(g, fg, w, c, mo, ch, lam, pr.max_iter - pr.warm_iters, step, tol,
                             e, s_f, &it1, &rd0, &rd1, ns, lane);
        }
      }
    } else {
      conv = round1_fast(g, fg, w, c, mo, ch, lam, pr.max_iter, step, tol, e, s_f, &it1, &r0,
                         &rd1, ns, lane);
    }
    total_it += itw + it1;
    if (conv != 1) {  // round 2 and verbatim storage belong to the FP64 kernel
      defer = true;
      break;
    }
    st |= AEQC_ST_CONVERGED;
    bool qoi_ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) qoi_ok = qoi_ok && ns.gres[k] <= (float)pr.qoi_check;
    if (!ns.check_viol && qoi_ok) done = true;
    else if (level == 1) defer = true;  // verbatim after the retry: the FP64 kernel stores it
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
    lamd = (double)lk.hi + (double)lk.lo;
  }
  // outputs
  int16_t* cb = a.codes + b * (long long)P;
  for (int p = lane; p < P; p += 32) cb[p] = w.codes[p];
  if (a.f_out) {
    // f = x' exp(-lambda.phi) with the rounding of the decompression kernel
    double ld[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ld[k] = __shfl_sync(FULL, lamd, k);
    for (int i = lane; i < g.n_par; i += 32) w.ta[i] = corr_a(ld, g.vpar[i]);
    for (int j = lane; j < g.n_perp; j += 32) w.tb[j] = corr_b(ld, g.vperp2[j]);
    __syncwarp();
    const double dl =
        bin_width(pr.tau, s, (st & AEQC_ST_ALPHA_RETRY) ? pr.alpha * 0.25 : pr.alpha);
    double* fb = a.f_out + b * (long long)P;
    PointIter pi(lane, g.n_par);
    for (; pi.p < P; pi.next()) {
      const int code = w.codes[pi.p];
      double xpd;
      if (code == AEQC_CODE_ESCAPE) xpd = __ldg(xb + pi.p);
      else if (code == AEQC_CODE_ZERO) xpd = 0.0;
      else xpd = __dadd_rn((double)__ldg(xhb + pi.p), __dmul_rn((double)code, dl));
      fb[pi.p] = corr_kl(xpd, w.ta[pi.i], w.tb[pi.j]);
    }
  }
  if (a.out.count && (st & AEQC_ST_CODE_ESCAPE)) {
    if (append_outliers(a.out, w.codes, xb, P, a.row0 + b, lane)) st |= AEQC_ST_OUTLIER_OVERFLOW;
  }
  if (a.features) {
    float* fr = a.features + b * (long long)(a.latent.L + 4);
    for (int l = lane; l < a.latent.L; l += 32) fr[l] = load_latent(a.latent, b, l);
    if (lane < 4) fr[a.latent.L + lane] = dfeat[lane];
  }
  if (lane < 4) a.lambda[b * 4 + lane] = lamd;
  if (lane == 0) {
    a.scale[b] = s;
    a.iters[b] = (uint8_t)(total_it > 255 ? 255 : total_it);
    a.status[b] = (uint16_t)st;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(FW * 32) fused_fast_kernel(const FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FastWS& w = reinterpret_cast<FastWS*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * FW;
  for (long long b = (long long)blockIdx.x * FW + (threadIdx.x >> 5); b < a.n; b += nw)
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
  f.vmax = (float)vmax;
  f.wmax = (float)g.vperp2[g.n_perp - 1];
  // x' bits: the largest integer weight (|i - i_c|^4, j^4, |i - i_c|^2 j^2)
  // times the points of one lane must stay below 2^62
  {
    const long long icm = ic > g.n_par - 1 - ic ? ic : g.n_par - 1 - ic;
    const long long jm = g.n_perp - 1;
    long long wmaxi = icm * icm * icm * icm;
    if (jm * jm * jm * jm > wmaxi) wmaxi = jm * jm * jm * jm;
    if (icm * icm * jm * jm > wmaxi) wmaxi = icm * icm * jm * jm;
    int bw = 0;
    while ((1ll << bw) <= wmaxi) ++bw;
    const int per_lane = (g.n_par * g.n_perp + 31) / 32;
    int bn = 0;
    while ((1 << bn) < per_lane) ++bn;
    f.xbits = 62 - bw - bn;
  }
  *out = f;
  return AEQC_OK;
}

int launch_fused_fast(const FusedArgs& a_in, cudaStream_t s) {
  if (a_in.n <= 0) return AEQC_OK;
  FusedArgs a = a_in;
  if (!a.fg.ok || a.prm.loss != 0 || a.grid.has_vol) return launch_fused_fp64(a, s);
  AEQC_CUDA_TRY(cudaMemsetAsync(a.fb_count, 0, sizeof(int), s));
  const size_t smem = sizeof(FastWS) * FW;
  static bool attr = false;
  if (!attr) {
    AEQC_CUDA_TRY(cudaFuncSetAttribute(fused_fast_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (a.n + FW - 1) / FW;
  const long long cap = (long long)sms * 3;  // 3 CTAs of 4 warps fit per SM
  if (blocks > cap) blocks = cap;
  fused_fast_kernel<<<(unsigned)blocks, FW * 32, smem, s>>>(a);
  int rc = check_launch("fused_fast_kernel");
  if (rc) return rc;
  return launch_fused_fp64_list(a, a.fb_list, a.fb_count, s);
}

}  // namespace aeqc
