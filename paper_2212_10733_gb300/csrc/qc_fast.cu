// Residual quantization and QoI correction with the per-point work on the
// integer and FP32 pipes (GB300's FP64 pipe runs at a small fraction of its
// FP32 rate; the per-histogram 4x4 algebra stays in FP64).  One warp per
// histogram; the histogram's x' (float), residual (float) and codes stay in
// shared memory for the Newton passes.
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
// integer sums (for the affine grid v_par = b (i - i_c) + c0, v_perp^2 = d2 j^2
// every weight is a small integer polynomial).  H is second order (|H|/S below
// ~1e-7 in practice), so FP32 sums carry it to far below the 1e-12 tolerance.
// Newton steps use M as the Jacobian (a chord step: M is the exact Jacobian at
// lambda = 0, and the method converges at a rate ~|t|); each step after the
// first costs one FP32 pass over x'.  The end-to-end check runs in the same
// pass.  Histograms the fast path cannot certify (non-finite or negative input,
// large lambda, no convergence, an ambiguous check, verbatim storage) are
// appended to a list that the FP64 kernel completes.
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

// Per-histogram constants of the integer quantizer.
struct QConst {
  double dl;       // Delta
  float dl_f;
  int k;           // Delta = 2^k
  int F;           // fractional bits of the fixed-point values (units of Delta)
  int FX;          // fractional bits of x' in the moment sums
  int thr;         // |xhat| >= 2^thr certainly escapes
  long long half, mask;
};

__device__ __forceinline__ bool make_qconst(double tau, double s, double alpha, QConst& c) {
  c.dl = bin_width(tau, s, alpha);
  int E;
  (void)frexp(c.dl, &E);
  c.k = E - 1;
  int Es;
  (void)frexp(s, &Es);      // s in [2^(Es-1), 2^Es)
  const int IBx = Es - c.k;  // s / Delta < 2^IBx
  const int IB = (IBx > 15 ? IBx : 15) + 2;
  c.F = 62 - IB;
  c.FX = 30 - IBx;
  c.thr = c.k + IB - 1;
  c.half = 1ll << (c.F - 1);
  c.mask = (1ll << c.F) - 1;
  c.dl_f = (float)c.dl;
  // the float copies and the 30-bit residual scale need F >= 31; FX >= 1
  return c.F >= 31 && c.FX >= 1 && IBx >= 1 && isfinite(c.dl_f) && c.dl_f > 0.f;
}

struct PointQ {
  int code;
  int rho32;   // round((x - x') / Delta * 2^30)
  int xp32;    // floor(x' / Delta * 2^FX)
  float xpf;   // x' (float)
};

// Exact quantizer decision for one point (x finite, x >= 0).
__device__ __forceinline__ PointQ quant_point_int(double x, float xh, const QConst& c) {
  PointQ o;
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
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
          else if (inex) { zero = 0; hard = true; }
          else zero = A > 0;
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
    o.xp32 = __double2int_rz(ldexp(__ddiv_rn(xpd, c.dl), c.FX));
    o.xpf = (float)xpd;
    return o;
  }
  o.rho32 = (int)((rho_fix + (1ll << (c.F - 31))) >> (c.F - 30));
  o.xp32 = (int)(xp_fix >> (c.F - c.FX));
  if (o.code == AEQC_CODE_ESCAPE) o.xpf = ldexpf((float)o.xp32, -c.FX) * c.dl_f;
  else if (o.code == AEQC_CODE_ZERO) o.xpf = 0.f;
  else o.xpf = fmaf((float)o.code, c.dl_f, xh);
  return o;
}

// The lambda-independent moments of one quantization level.
struct Moments {
  double R[4];   // sum vol phi_k (x - x')
  double M[10];  // upper triangle of sum vol phi phi^T x'
  double S[4];   // sum vol |phi_k| x'
  unsigned flags;  // CODE_ESCAPE / AE_EXACT
};

// Quantize the histogram (row xb, decoded row xhb) into shared memory and
// accumulate its moments.
__device__ void phase_a(const GridK& g, const FastGridK& fg, const double* xb, const float* xhb,
                        const QConst& c, FastWS& w, Moments& mo, int lane) {
  long long U0 = 0, U1 = 0, U2 = 0, U3 = 0;
  long long T00 = 0, T10 = 0, T20 = 0, T30 = 0, T40 = 0, T01 = 0, T11 = 0, T21 = 0, T02 = 0;
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
    const long long r = o.rho32, X = o.xp32;
    U0 += r;
    U1 += r * ic;
    U2 += r * ic2;
    U3 += r * j2;
    T00 += X;
    T10 += X * ic;
    T20 += X * ic2;
    T30 += X * (ic2 * ic);
    T40 += X * (ic2 * ic2);
    T01 += X * j2;
    T11 += X * (ic * j2);
    T21 += X * (ic2 * j2);
    T02 += X * (j2 * j2);
    s1 = fmaf(o.xpf, fabsf(fmaf(b_f, (float)ic, c0_f)), s1);
  }
  __syncwarp();
  const double u0 = wsum((double)U0), u1 = wsum((double)U1), u2 = wsum((double)U2),
               u3 = wsum((double)U3);
  double T[5][3];
  T[0][0] = wsum((double)T00); T[1][0] = wsum((double)T10); T[2][0] = wsum((double)T20);
  T[3][0] = wsum((double)T30); T[4][0] = wsum((double)T40);
  T[0][1] = wsum((double)T01); T[1][1] = wsum((double)T11); T[2][1] = wsum((double)T21);
  T[0][2] = wsum((double)T02);
  const double S1 = wsum((double)s1);
  const double vol = g.vol_uniform, b = fg.b, c0 = fg.c0, d2 = fg.d2;
  const double sr = vol * ldexp(c.dl, -30), sm = vol * ldexp(c.dl, -c.FX);
  mo.R[0] = sr * u0;
  mo.R[1] = sr * (b * u1 + c0 * u0);
  mo.R[2] = sr * (d2 * u3);
  mo.R[3] = sr * (b * b * u2 + 2.0 * b * c0 * u1 + c0 * c0 * u0);
  // m(p, q) = sum x' v^p w^q, v = b ic + c0, w = d2 j^2 (binomial expansion in ic)
  auto mom = [&](int p, int q) {
    const double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0},
                                {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    double acc = 0.0, bp = 1.0;
    for (int r = 0; r <= p; ++r) {
      double cp = 1.0;
      for (int e = 0; e < p - r; ++e) cp *= c0;
      acc += binom[p][r] * bp * cp * T[r][q];
      bp *= b;
    }
    double wq = 1.0;
    for (int e = 0; e < q; ++e) wq *= d2;
    return sm * wq * acc;
  };
  const double m00 = mom(0, 0), m10 = mom(1, 0), m20 = mom(2, 0), m30 = mom(3, 0),
               m40 = mom(4, 0), m01 = mom(0, 1), m11 = mom(1, 1), m21 = mom(2, 1),
               m02 = mom(0, 2);
  mo.M[0] = m00; mo.M[1] = m10; mo.M[2] = m01; mo.M[3] = m20;
  mo.M[4] = m20; mo.M[5] = m11; mo.M[6] = m30;
  mo.M[7] = m02; mo.M[8] = m21;
  mo.M[9] = m40;
  mo.S[0] = m00;
  mo.S[1] = vol * S1;
  mo.S[2] = m01;
  mo.S[3] = m20;
  mo.flags = 0;
  if (__any_sync(FULL, esc)) mo.flags |= AEQC_ST_CODE_ESCAPE;
  if (!__any_sync(FULL, nonzero)) mo.flags |= AEQC_ST_AE_EXACT;
}

struct PassOut {
  double H[4];
  float tmax;
  int viol, uncertain;
};

// One FP32 pass at lambda: H(lambda) and the end-to-end check.
__device__ void pass_warp(const GridK& g, const FastGridK& fg, const FastWS& w, const QConst& c,
                          const double lam[4], float e_lo, float e_hi, PassOut& o, int lane) {
  const float l0 = (float)lam[0], l1 = (float)lam[1], l2 = (float)lam[2], l3 = (float)lam[3];
  const float b_f = (float)fg.b, c0_f = (float)fg.c0, d2_f = (float)fg.d2;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, tmax = 0.f;
  int viol = 0, unc = 0;
  PointIter it(lane, g.n_par);
  for (; it.p < g.P; it.next()) {
    const float xp = w.xp[it.p];
    const float v = fmaf(b_f, (float)(it.i - fg.i_c), c0_f);
    const float wq = d2_f * (float)(it.j * it.j);
    const float t = fmaf(fmaf(l3, v, l1), v, fmaf(l2, wq, l0));
    const float h = t * t * fmaf(-t, fmaf(-t, fmaf(-t, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f);
    const float y = xp * h;
    a0 += y;
    const float yv = y * v;
    a1 += yv;
    a2 = fmaf(y, wq, a2);
    a3 = fmaf(yv, v, a3);
    if (xp > 0.f) tmax = fmaxf(tmax, fabsf(t));
    const float err = fabsf(fmaf(xp, h - t, -c.dl_f * w.rho[it.p]));
    viol |= err > e_hi;
    unc |= err > e_lo;
  }
  const double vol = g.vol_uniform;
  o.H[0] = vol * wsum((double)a0);
  o.H[1] = vol * wsum((double)a1);
  o.H[2] = vol * wsum((double)a2);
  o.H[3] = vol * wsum((double)a3);
  float tm = tmax;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) tm = fmaxf(tm, __shfl_xor_sync(FULL, tm, s));
  o.tmax = tm;
  o.viol = __any_sync(FULL, viol);
  o.uncertain = __any_sync(FULL, unc);
}

enum { FAST_OK = 0, FAST_DEFER = 1, FAST_CHECK_FAILED = 2, FAST_NOT_CONVERGED = 3 };

struct NewtonState {
  double lam[4];
  int iters;
  int check_viol;  // end-to-end violation at the final lambda (valid when converged)
  double g[4];
};

// Bound on |t| = |lambda.phi| over the grid (for the check's rounding margin).
__device__ __forceinline__ double t_bound(const double lam[4], double vmax, double wmax) {
  return fabs(lam[0]) + fabs(lam[1]) * vmax + fabs(lam[2]) * wmax + fabs(lam[3]) * vmax * vmax;
}

// Round 1 of Eq. (6) with the chord Jacobian M from lam (in/out).
// Returns 1 converged, 0 not converged, -1 defer (precision guards).
__device__ int round1_fast(const GridK& g, const FastGridK& fg, const FastWS& w,
                           const QConst& c, const Moments& mo, double lam[4], int max_iter,
                           double step, double tol, double e, double s, double vmax,
                           double wmax, int* iters, double* r0, double* rlast, NewtonState& ns,
                           int lane) {
  for (int it = 0;; ++it) {
    double H[4] = {0.0, 0.0, 0.0, 0.0};
    const bool zero_lam = lam[0] == 0.0 && lam[1] == 0.0 && lam[2] == 0.0 && lam[3] == 0.0;
    int viol = 0, unc = 0;
    // pass (also needed at lambda = 0 for the end-to-end check once converged)
    bool did_pass = false;
    auto do_pass = [&]() {
      const double tb = t_bound(lam, vmax, wmax);
      const double margin = 4e-7 * (s * tb + c.dl) + 1e-30;
      PassOut po;
      pass_warp(g, fg, w, c, lam, (float)(e - margin), (float)(e + margin), po, lane);
#pragma unroll
      for (int k = 0; k < 4; ++k) H[k] = po.H[k];
      viol = po.viol;
      unc = po.uncertain;
      did_pass = true;
      return po.tmax;
    };
    float tmax = 0.f;
    if (!zero_lam) tmax = do_pass();
    double gk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double* Mr = mo.M;
      double ml;
      switch (k) {
        case 0: ml = Mr[0] * lam[0] + Mr[1] * lam[1] + Mr[2] * lam[2] + Mr[3] * lam[3]; break;
        case 1: ml = Mr[1] * lam[0] + Mr[4] * lam[1] + Mr[5] * lam[2] + Mr[6] * lam[3]; break;
        case 2: ml = Mr[2] * lam[0] + Mr[5] * lam[1] + Mr[7] * lam[2] + Mr[8] * lam[3]; break;
        default: ml = Mr[3] * lam[0] + Mr[6] * lam[1] + Mr[8] * lam[2] + Mr[9] * lam[3]; break;
      }
      gk[k] = -mo.R[k] - ml + H[k];
    }
    const double res = scaled_residual(gk, mo.S);
    if (it == 0) *r0 = res;
    *rlast = res;
    *iters = it;
    if (!isfinite(res)) return 0;
    if (tmax > 0.05f) return -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (fabs(H[k]) > 1e-5 * mo.S[k]) return -1;
    if (res <= tol) {
      if (!did_pass) do_pass();  // lambda = 0 converged: still check every point
      if (unc && !viol) return -1;
      ns.check_viol = viol;
#pragma unroll
      for (int k = 0; k < 4; ++k) ns.g[k] = gk[k];
      return 1;
    }
    if (it == max_iter) return 0;
    double d[4];
    if (chol_solve4(mo.M, gk, d) != 0) return 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] += step * d[k];
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
  bool defer = bad || s == 0.0;

  // v_par and v_perp^2 extents for the check margin
  const double vmax = fabs(fg.b) * (double)((fg.i_c > g.n_par - 1 - fg.i_c) ? fg.i_c
                                                                            : g.n_par - 1 - fg.i_c) +
                      fabs(fg.c0);
  const double wmax = fg.d2 * (double)((g.n_perp - 1) * (g.n_perp - 1));
  unsigned st = 0;
  double lam[4] = {0.0, 0.0, 0.0, 0.0};
  int total_it = 0;
  double dfeat[4] = {0.0, 0.0, 0.0, 0.0};
  bool done = false;
  for (int level = 0; level < 2 && !defer && !done; ++level) {
    QConst c;
    if (!make_qconst(pr.tau, s, level ? pr.alpha * 0.25 : pr.alpha, c)) {
      defer = true;
      break;
    }
    Moments mo;
    phase_a(g, fg, xb, xhb, c, w, mo, lane);
    st = mo.flags | (level ? AEQC_ST_ALPHA_RETRY : 0u) | (st & AEQC_ST_WARM_REJECTED);
    int warm = 0;
    if (level == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double den = mo.S[k] > 0.0 ? mo.S[k] : 1e-300;
        dfeat[k] = mo.R[k] / den;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] = 0.0;
      if (a.use_mlp) {
        const int L = a.latent.L;
        mlp_eval_warp(
            a.mlp,
            [&](int k) { return k < L ? load_latent(a.latent, b, k) : (float)dfeat[k - L]; },
            lam, lane);
        warm = 1;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) ok = ok && isfinite(lam[k]);
        if (!ok) {
#pragma unroll
          for (int k = 0; k < 4; ++k) lam[k] = 0.0;
          warm = 0;
          st |= AEQC_ST_WARM_REJECTED;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] = 0.0;
    }
    const double e = pr.tau * s;
    NewtonState ns;
    ns.check_viol = 0;
    int conv, it1 = 0, itw = 0;
    double r0 = 0.0, rw = 0.0, rdummy, rdummy2;
    if (warm) {
      conv = round1_fast(g, fg, w, c, mo, lam, pr.warm_iters, pr.step_s, pr.tol, e, s, vmax,
                         wmax, &itw, &r0, &rw, ns, lane);
      if (conv == 0) {
        if (!isfinite(rw) || !isfinite(r0) || rw > pr.warm_reject || rw > r0) {
          st |= AEQC_ST_WARM_REJECTED;
#pragma unroll
          for (int k = 0; k < 4; ++k) lam[k] = 0.0;
          conv = round1_fast(g, fg, w, c, mo, lam, pr.max_iter, pr.step_s, pr.tol, e, s, vmax,
                             wmax, &it1, &rdummy, &rdummy2, ns, lane);
        } else {
          conv = round1_fast(g, fg, w, c, mo, lam, pr.max_iter - pr.warm_iters, pr.step_s,
                             pr.tol, e, s, vmax, wmax, &it1, &rdummy, &rdummy2, ns, lane);
        }
      }
    } else {
      conv = round1_fast(g, fg, w, c, mo, lam, pr.max_iter, pr.step_s, pr.tol, e, s, vmax,
                         wmax, &it1, &r0, &rdummy2, ns, lane);
    }
    total_it += itw + it1;
    if (conv != 1) {  // round 2 and verbatim storage belong to the FP64 kernel
      defer = true;
      break;
    }
    st |= AEQC_ST_CONVERGED;
    bool qoi_ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double den = mo.S[k] > 0.0 ? mo.S[k] : 1e-300;
      qoi_ok = qoi_ok && fabs(ns.g[k]) / den <= pr.qoi_check;
    }
    if (!ns.check_viol && qoi_ok) {
      done = true;
    } else if (level == 1) {
      defer = true;  // verbatim after the retry: the FP64 kernel stores it
    }
  }
  if (defer || !done) {
    if (lane == 0) {
      const int slot = atomicAdd(a.fb_count, 1);
      a.fb_list[slot] = (int)b;
    }
    __syncwarp();
    return;
  }
  // outputs
  int16_t* cb = a.codes + b * (long long)P;
  for (int p = lane; p < P; p += 32) cb[p] = w.codes[p];
  if (a.f_out) {
    // f = x' exp(-lambda.phi) with the rounding of the decompression kernel
    for (int i = lane; i < g.n_par; i += 32) w.ta[i] = corr_a(lam, g.vpar[i]);
    for (int j = lane; j < g.n_perp; j += 32) w.tb[j] = corr_b(lam, g.vperp2[j]);
    __syncwarp();
    const double dl = bin_width(pr.tau, s, (st & AEQC_ST_ALPHA_RETRY) ? pr.alpha * 0.25
                                                                     : pr.alpha);
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
    if (lane < 4) fr[a.latent.L + lane] = (float)dfeat[lane];
  }
  if (lane == 0) {
    a.scale[b] = s;
    a.iters[b] = (uint8_t)(total_it > 255 ? 255 : total_it);
    a.status[b] = (uint16_t)st;
#pragma unroll
    for (int k = 0; k < 4; ++k) a.lambda[b * 4 + k] = lam[k];
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

}  // namespace

int make_fast_grid(const GridK& g, FastGridK* out) {
  FastGridK f;
  f.ok = 0;
  f.i_c = 0;
  f.b = f.c0 = f.d2 = 0.0;
  *out = f;
  if (g.has_vol || g.n_par < 2 || g.n_perp < 2) return AEQC_OK;
  const double b = (g.vpar[g.n_par - 1] - g.vpar[0]) / (double)(g.n_par - 1);
  if (!(b > 0.0)) return AEQC_OK;
  double vmax = 0.0;
  for (int i = 0; i < g.n_par; ++i) vmax = fmax(vmax, fabs(g.vpar[i]));
  // index nearest to v_par = 0
  int ic = (int)llround(-g.vpar[0] / b);
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
