// Residual quantization and QoI correction with the per-point work in native
// FP64: one warp per histogram, the histogram staged in shared memory.  This
// is the plain form of Stages 4-5 and the GPU reference for the fast kernel.
//
//   targets   Q_k = sum vol phi_k x, phi = (1, v_par, v_perp^2, v_par^2),
//             the moments behind n, u_par, T_perp, T_par (Eq. (1)-(4));
//   quantizer Delta = 2^floor(log2(2 alpha tau max x)), exact round-half-even
//             codes with a zero level and escapes (Stage 4);
//   Newton    lambda <- lambda + s M^-1 g on the dual (Eq. (6)), the exponent
//             separated as exp(-lambda.phi) = a_i(lambda0, lambda1, lambda3)
//             b_j(lambda2), so each step takes n_par + n_perp exponentials;
//   fallback  round 2 (damped Newton from 0), end-to-end check, one retry with
//             alpha/4, verbatim (Stage 5 and the paper's parameter study).
#include "qc_common.cuh"

namespace aeqc {
namespace {

using namespace dev;

constexpr int WPC = 4;  // warps per CTA

struct WS {
  double xs[AEQC_MAX_P];  // x
  double xp[AEQC_MAX_P];  // x'
  double ta[AEQC_MAX_NPAR];
  double tb[AEQC_MAX_NPERP];
  int16_t codes[AEQC_MAX_P];
};

__device__ __forceinline__ double vol_of(const GridK& g, int p) {
  return g.has_vol ? __ldg(g.vol + p) : g.vol_uniform;
}

// Q_k(x) and S_k(x) = sum vol |phi_k| |x| for the histogram in xs.
__device__ void moments_warp(const GridK& g, const double* xs, double Q[4], double S[4],
                             int lane) {
  double q0 = 0, q1 = 0, q2 = 0, q3 = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  PointIter it(lane, g.n_par);
  for (; it.p < g.P; it.next()) {
    double v = g.vpar[it.i], v2 = g.vperp2[it.j];
    double w = vol_of(g, it.p) * xs[it.p];
    double aw = fabs(w);
    q0 += w;
    q1 += w * v;
    q2 += w * v2;
    q3 += w * v * v;
    s0 += aw;
    s1 += aw * fabs(v);
    s2 += aw * v2;
    s3 += aw * v * v;
  }
  Q[0] = wsum(q0); Q[1] = wsum(q1); Q[2] = wsum(q2); Q[3] = wsum(q3);
  S[0] = wsum(s0); S[1] = wsum(s1); S[2] = wsum(s2); S[3] = wsum(s3);
}

struct Eval {
  double A[4];   // sum vol phi_k f
  double S[4];   // sum vol |phi_k| |f|
  double M[10];  // upper triangle of sum vol phi phi^T w (w = f for KL, 1 for L2)
  double res;    // max_k |A_k - Q_k| / S_k
};

// One pass over the histogram at lambda: f, A, S, (M).  For the KL loss the
// exponential tables ta, tb are left for lambda in shared memory.
__device__ void eval_warp(const GridK& g, WS& w, const double lam[4], const double Q[4],
                          int loss, bool want_M, Eval& r, int lane) {
  if (loss == 0) {
    for (int i = lane; i < g.n_par; i += 32) w.ta[i] = corr_a(lam, g.vpar[i]);
    for (int j = lane; j < g.n_perp; j += 32) w.tb[j] = corr_b(lam, g.vperp2[j]);
    __syncwarp();
  }
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  double m00 = 0, m01 = 0, m02 = 0, m03 = 0, m12 = 0, m13 = 0, m22 = 0, m23 = 0, m33 = 0;
  PointIter it(lane, g.n_par);
  for (; it.p < g.P; it.next()) {
    double v = g.vpar[it.i], v2 = g.vperp2[it.j];
    double vol = vol_of(g, it.p);
    double f, wm;
    if (loss == 0) {
      f = corr_kl(w.xp[it.p], w.ta[it.i], w.tb[it.j]);
      wm = f * vol;
    } else {
      f = corr_l2(w.xp[it.p], lam, v, v2);
      wm = vol;
    }
    double fv = f * vol, af = fabs(fv);
    a0 += fv;
    a1 += fv * v;
    a2 += fv * v2;
    a3 += fv * v * v;
    s0 += af;
    s1 += af * fabs(v);
    s2 += af * v2;
    s3 += af * v * v;
    if (want_M) {
      double wv = wm * v;
      m00 += wm;
      m01 += wv;
      m02 += wm * v2;
      m03 += wv * v;
      m12 += wv * v2;
      m13 += wv * v * v;
      m22 += wm * v2 * v2;
      m23 += wv * v * v2;
      m33 += wv * v * v * v;
    }
  }
  r.A[0] = wsum(a0); r.A[1] = wsum(a1); r.A[2] = wsum(a2); r.A[3] = wsum(a3);
  r.S[0] = wsum(s0); r.S[1] = wsum(s1); r.S[2] = wsum(s2); r.S[3] = wsum(s3);
  if (want_M) {
    r.M[0] = wsum(m00); r.M[1] = wsum(m01); r.M[2] = wsum(m02); r.M[3] = wsum(m03);
    r.M[4] = r.M[3];  // sum w v^2 == m03
    r.M[5] = wsum(m12); r.M[6] = wsum(m13); r.M[7] = wsum(m22); r.M[8] = wsum(m23);
    r.M[9] = wsum(m33);
  }
  double gk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) gk[k] = r.A[k] - Q[k];
  r.res = scaled_residual(gk, r.S);
}

// Round 1: plain steps of Eq. (6) from lam; returns 1 if converged.  r0 is the
// scaled residual at the starting point, e the last evaluation.
__device__ int round1_warp(const GridK& g, WS& w, const double Q[4], double lam[4],
                           int max_iter, double step, double tol, int loss, int* iters,
                           double* r0, Eval& e, int lane) {
  for (int it = 0;; ++it) {
    eval_warp(g, w, lam, Q, loss, true, e, lane);
    if (it == 0) *r0 = e.res;
    *iters = it;
    if (!isfinite(e.res)) return 0;
    if (e.res <= tol) return 1;
    if (it == max_iter) return 0;
    double gk[4], d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gk[k] = e.A[k] - Q[k];
    if (chol_solve4(e.M, gk, d) != 0) return 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] += step * d[k];
  }
}

// Round 2: damped Newton from 0.  A step t in {1, 1/2, ...} is accepted when
// it lowers psi = sum vol f + lambda.Q by the Armijo amount, or, where that
// decrease is below psi's rounding (near the solution), when psi stays within
// 1e-12 of its scale sum vol |f| + sum |lambda_k Q_k| and the scaled residual
// falls by the factor (1 - t/2).  A step that raises psi beyond its rounding
// is never taken: one that blows f up also blows up S, the residual's scale.
__device__ int round2_warp(const GridK& g, WS& w, const double Q[4], double lam[4],
                           int max_iter, double tol, int loss, int* iters, Eval& e,
                           int lane) {
#pragma unroll
  for (int k = 0; k < 4; ++k) lam[k] = 0.0;
  for (int it = 0;; ++it) {
    eval_warp(g, w, lam, Q, loss, true, e, lane);
    *iters = it;
    if (!isfinite(e.res)) return 0;
    if (e.res <= tol) return 1;
    if (it == max_iter) return 0;
    double gk[4], d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gk[k] = e.A[k] - Q[k];
    if (chol_solve4(e.M, gk, d) != 0) return 0;
    double psi0 = e.A[0] + lam[0] * Q[0] + lam[1] * Q[1] + lam[2] * Q[2] + lam[3] * Q[3];
    double sc0 = e.S[0] + fabs(lam[0] * Q[0]) + fabs(lam[1] * Q[1]) + fabs(lam[2] * Q[2]) +
                 fabs(lam[3] * Q[3]);
    double slope = gk[0] * d[0] + gk[1] * d[1] + gk[2] * d[2] + gk[3] * d[3];
    double r = e.res, t = 1.0;
    int accepted = 0;
    for (int h = 0; h < 40; ++h, t *= 0.5) {
      double lt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) lt[k] = lam[k] + t * d[k];
      Eval et;
      eval_warp(g, w, lt, Q, loss, false, et, lane);
      if (!isfinite(et.res)) continue;
      double psit = et.A[0] + lt[0] * Q[0] + lt[1] * Q[1] + lt[2] * Q[2] + lt[3] * Q[3];
      double flat = 1e-12 * (sc0 + et.S[0] + fabs(lt[0] * Q[0]) + fabs(lt[1] * Q[1]) +
                             fabs(lt[2] * Q[2]) + fabs(lt[3] * Q[3]));
      if (psit <= psi0 - 1e-4 * t * slope ||
          (psit <= psi0 + flat && et.res <= (1.0 - 0.5 * t) * r)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) lam[k] = lt[k];
        accepted = 1;
        break;
      }
    }
    if (!accepted) return 0;
  }
}

constexpr unsigned NOT_CONVERGED = 0x8000u;

// Newton driver (rounds 1-2 and the warm-start probation).  Leaves the tables
// of the final lambda in shared memory and its evaluation in e.
__device__ unsigned newton_warp(const GridK& g, WS& w, const double Q[4], double lam[4],
                                int warm, const ParamsK& pr, int* iters, Eval& e,
                                int lane) {
  unsigned st = 0;
  int it1 = 0, it2 = 0, itw = 0, conv;
  double r0 = 0.0, rdummy;
  if (warm) {
    conv = round1_warp(g, w, Q, lam, pr.warm_iters, pr.step_s, pr.tol, pr.loss, &itw, &r0,
                       e, lane);
    if (conv) {
      *iters = itw;
      return AEQC_ST_CONVERGED;
    }
    double rw = e.res;
    if (!isfinite(rw) || !isfinite(r0) || rw > pr.warm_reject || rw > r0) {
      st |= AEQC_ST_WARM_REJECTED;
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] = 0.0;
      conv = round1_warp(g, w, Q, lam, pr.max_iter, pr.step_s, pr.tol, pr.loss, &it1,
                         &rdummy, e, lane);
    } else {
      conv = round1_warp(g, w, Q, lam, pr.max_iter - pr.warm_iters, pr.step_s, pr.tol,
                         pr.loss, &it1, &rdummy, e, lane);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] = 0.0;
    conv = round1_warp(g, w, Q, lam, pr.max_iter, pr.step_s, pr.tol, pr.loss, &it1, &r0, e,
                       lane);
  }
  if (conv) {
    *iters = itw + it1;
    return st | AEQC_ST_CONVERGED;
  }
  conv = round2_warp(g, w, Q, lam, pr.r2_max_iter, pr.tol, pr.loss, &it2, e, lane);
  *iters = itw + it1 + it2;
  if (conv) return st | AEQC_ST_ROUND2;
  return st | AEQC_ST_ROUND2 | NOT_CONVERGED;
}

// Quantize the histogram in xs against xhat row xh into w.codes / w.xp.
// Returns status bits CODE_ESCAPE / AE_EXACT.
__device__ unsigned quantize_warp(const GridK& g, WS& w, const float* xh, double dl,
                                  int lane) {
  int esc = 0, nonzero = 0;
  for (int p = lane; p < g.P; p += 32) {
    double xp;
    int c = quant_point_fp64(w.xs[p], (double)__ldg(xh + p), dl, &xp);
    w.codes[p] = (int16_t)c;
    w.xp[p] = xp;
    esc |= c == AEQC_CODE_ESCAPE;
    nonzero |= c != 0;
  }
  __syncwarp();
  unsigned st = 0;
  if (__any_sync(FULL, esc)) st |= AEQC_ST_CODE_ESCAPE;
  if (!__any_sync(FULL, nonzero)) st |= AEQC_ST_AE_EXACT;
  return st;
}

__device__ void process_fp64(const FusedArgs& a, WS& w, long long b, int lane) {
  const GridK& g = a.grid;
  const ParamsK& pr = a.prm;
  const int P = g.P;
  const double* xb = a.x + b * (long long)P;
  double s = 0.0;
  int bad = 0;
  for (int p = lane; p < P; p += 32) {
    double v = __ldg(xb + p);
    w.xs[p] = v;
    if (!isfinite(v) || v < 0.0) bad = 1;
    else if (v > s) s = v;
  }
  s = wmax(s);
  bad = __any_sync(FULL, bad);
  __syncwarp();

  unsigned st = 0;
  double lam[4] = {0.0, 0.0, 0.0, 0.0};
  int total_it = 0;
  double dfeat[4] = {0.0, 0.0, 0.0, 0.0};
  bool verbatim = false, zero = false;
  if (bad) {
    st = AEQC_ST_NONFINITE_INPUT | AEQC_ST_VERBATIM;
    verbatim = true;
  } else if (s == 0.0) {
    st = AEQC_ST_ZERO_IMAGE;
    zero = true;
    for (int p = lane; p < P; p += 32) {
      w.codes[p] = 0;
      w.xp[p] = 0.0;
    }
  } else {
    double Q[4], Sx[4];
    moments_warp(g, w.xs, Q, Sx, lane);
    bool done = false;
    for (int level = 0; level < 2 && !done; ++level) {
      double alpha = level ? pr.alpha * 0.25 : pr.alpha;
      double dl = bin_width(pr.tau, s, alpha);
      unsigned qs = quantize_warp(g, w, a.xhat + b * a.ldx, dl, lane);
      st = qs | (level ? AEQC_ST_ALPHA_RETRY : 0u) | (st & AEQC_ST_WARM_REJECTED);
      Eval e;
      int warm = 0;
      if (level == 0 && (a.features || a.use_mlp)) {
        eval_warp(g, w, lam, Q, pr.loss, false, e, lane);  // lam == 0 here
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          double den = e.S[k] > 0.0 ? e.S[k] : 1e-300;
          dfeat[k] = (Q[k] - e.A[k]) / den;
        }
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
            for (int k = 0; k < 4; ++k) lam[k] = 1e300;  // rejected by the probation
          }
        }
      }
      int it = 0;
      unsigned ns = newton_warp(g, w, Q, lam, warm, pr, &it, e, lane);
      total_it += it;
      st |= ns & 0x7fffu;
      if (ns & NOT_CONVERGED) break;
      // end-to-end check: |f - x| <= e at every point, moments within qoi_check
      double ebound = __dmul_rn(pr.tau, s);
      int viol = 0;
      PointIter pi(lane, g.n_par);
      for (; pi.p < P; pi.next()) {
        double f = pr.loss == 0 ? corr_kl(w.xp[pi.p], w.ta[pi.i], w.tb[pi.j])
                                : corr_l2(w.xp[pi.p], lam, g.vpar[pi.i], g.vperp2[pi.j]);
        viol |= !(fabs(f - w.xs[pi.p]) <= ebound);
      }
      bool ok = !__any_sync(FULL, viol);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double den = Sx[k] > 0.0 ? Sx[k] : 1e-300;
        ok = ok && (fabs(e.A[k] - Q[k]) / den <= pr.qoi_check);
      }
      if (ok) done = true;
    }
    if (!done) {
      st = (st & AEQC_ST_WARM_REJECTED) | AEQC_ST_VERBATIM | (st & AEQC_ST_ALPHA_RETRY) |
           (st & AEQC_ST_ROUND2);
      verbatim = true;
    }
  }
  if (verbatim) {
    for (int p = lane; p < P; p += 32) {
      w.codes[p] = AEQC_CODE_ESCAPE;
      w.xp[p] = w.xs[p];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] = 0.0;
  }
  __syncwarp();
  // outputs
  int16_t* cb = a.codes + b * (long long)P;
  for (int p = lane; p < P; p += 32) cb[p] = w.codes[p];
  if (a.f_out) {
    double* fb = a.f_out + b * (long long)P;
    PointIter pi(lane, g.n_par);
    for (; pi.p < P; pi.next()) {
      double f;
      if (verbatim) f = w.xs[pi.p];
      else if (zero) f = 0.0;
      else if (pr.loss == 0) f = corr_kl(w.xp[pi.p], w.ta[pi.i], w.tb[pi.j]);
      else f = corr_l2(w.xp[pi.p], lam, g.vpar[pi.i], g.vperp2[pi.j]);
      fb[pi.p] = f;
    }
  }
  if (a.out.count && (verbatim || (st & AEQC_ST_CODE_ESCAPE))) {
    if (append_outliers(a.out, w.codes, w.xs, P, a.row0 + b, lane))
      st |= AEQC_ST_OUTLIER_OVERFLOW;
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

__global__ void __launch_bounds__(WPC * 32) fused_fp64_kernel(const FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WS& w = reinterpret_cast<WS*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * WPC;
  for (long long b = (long long)blockIdx.x * WPC + (threadIdx.x >> 5); b < a.n; b += nw)
    process_fp64(a, w, b, lane);
}

// The same per-histogram work for the histograms listed by the fast kernel
// (list[0 .. *count)); a launch with an empty list returns at once.
__global__ void __launch_bounds__(WPC * 32) fused_fp64_list_kernel(const FusedArgs a,
                                                                   const int* list,
                                                                   const int* count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WS& w = reinterpret_cast<WS*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long cnt = *count;
  const long long nw = (long long)gridDim.x * WPC;
  for (long long t = (long long)blockIdx.x * WPC + (threadIdx.x >> 5); t < cnt; t += nw)
    process_fp64(a, w, list[t], lane);
}

// ---- single-stage kernels for the separate C-ABI calls ---------------------

__global__ void __launch_bounds__(128) moments_kernel(const GridK g, const double* x,
                                                      long long n, double* Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* xs = reinterpret_cast<double*>(smem_raw) + (threadIdx.x >> 5) * AEQC_MAX_P;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * 4;
  for (long long b = (long long)blockIdx.x * 4 + (threadIdx.x >> 5); b < n; b += nw) {
    for (int p = lane; p < g.P; p += 32) xs[p] = __ldg(x + b * g.P + p);
    __syncwarp();
    double q[4], sabs[4];
    moments_warp(g, xs, q, sabs, lane);
    if (lane < 4) Q[b * 4 + lane] = q[lane];
    __syncwarp();
  }
}

struct QuantArgs {
  const double* x;
  const float* xhat;
  long long ld, n;
  int P;
  ParamsK prm;
  int16_t* codes;
  double* scale;
  uint16_t* status;
  OutliersK out;
  double* xrec;
};

__global__ void __launch_bounds__(128) quantize_kernel(const QuantArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  int16_t* codes_s = reinterpret_cast<int16_t*>(smem_raw) + (threadIdx.x >> 5) * AEQC_MAX_P;
  double* raw = reinterpret_cast<double*>(smem_raw + 4 * AEQC_MAX_P * sizeof(int16_t)) +
                (threadIdx.x >> 5) * AEQC_MAX_P;
  const long long nw = (long long)gridDim.x * 4;
  for (long long b = (long long)blockIdx.x * 4 + (threadIdx.x >> 5); b < a.n; b += nw) {
    const double* xb = a.x + b * a.P;
    double s = 0.0;
    int bad = 0;
    for (int p = lane; p < a.P; p += 32) {
      double v = __ldg(xb + p);
      raw[p] = v;
      if (!isfinite(v) || v < 0.0) bad = 1;
      else if (v > s) s = v;
    }
    s = wmax(s);
    bad = __any_sync(FULL, bad);
    __syncwarp();
    unsigned st = 0;
    if (bad) {
      st = AEQC_ST_NONFINITE_INPUT | AEQC_ST_VERBATIM;
      for (int p = lane; p < a.P; p += 32) codes_s[p] = AEQC_CODE_ESCAPE;
      if (a.xrec)
        for (int p = lane; p < a.P; p += 32) a.xrec[b * a.P + p] = raw[p];
    } else if (s == 0.0) {
      st = AEQC_ST_ZERO_IMAGE;
      for (int p = lane; p < a.P; p += 32) {
        codes_s[p] = 0;
        if (a.xrec) a.xrec[b * a.P + p] = 0.0;
      }
    } else {
      double dl = bin_width(a.prm.tau, s, a.prm.alpha);
      int esc = 0, nonzero = 0;
      for (int p = lane; p < a.P; p += 32) {
        double xp;
        int c = quant_point_fp64(raw[p], (double)__ldg(a.xhat + b * a.ld + p), dl, &xp);
        codes_s[p] = (int16_t)c;
        if (a.xrec) a.xrec[b * a.P + p] = xp;
        esc |= c == AEQC_CODE_ESCAPE;
        nonzero |= c != 0;
      }
      if (__any_sync(FULL, esc)) st |= AEQC_ST_CODE_ESCAPE;
      if (!__any_sync(FULL, nonzero)) st |= AEQC_ST_AE_EXACT;
    }
    __syncwarp();
    for (int p = lane; p < a.P; p += 32) a.codes[b * a.P + p] = codes_s[p];
    if (a.out.count && (st & (AEQC_ST_CODE_ESCAPE | AEQC_ST_VERBATIM))) {
      if (append_outliers(a.out, codes_s, raw, a.P, b, lane)) st |= AEQC_ST_OUTLIER_OVERFLOW;
    }
    if (lane == 0) {
      a.scale[b] = s;
      a.status[b] = (uint16_t)st;
    }
    __syncwarp();
  }
}

// x' from codes (thread per value); escapes are filled by scatter_raw_kernel.
__global__ void dequantize_kernel(const float* xhat, long long ld, const int16_t* codes,
                                  const double* scale, const uint16_t* status, long long n,
                                  int P, ParamsK prm, double* xrec) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = n * (long long)P;
  for (; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long b = t / P;
    int p = (int)(t - b * P);
    unsigned st = status[b];
    int c = codes[t];
    double v;
    if (st & AEQC_ST_ZERO_IMAGE) v = 0.0;
    else if (c == AEQC_CODE_ESCAPE) continue;
    else if (c == AEQC_CODE_ZERO) v = 0.0;
    else {
      double alpha = (st & AEQC_ST_ALPHA_RETRY) ? prm.alpha * 0.25 : prm.alpha;
      double dl = bin_width(prm.tau, scale[b], alpha);
      v = __dadd_rn((double)xhat[b * ld + p], __dmul_rn((double)c, dl));
    }
    xrec[t] = v;
  }
}

__global__ void scatter_raw_kernel(const OutliersK o, long long total, double* xrec) {
  long long cnt = *o.count;
  if (cnt > o.capacity) cnt = o.capacity;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    long long i = o.index[t];
    if (i >= 0 && i < total) xrec[i] = o.value[t];
  }
}

struct NewtonArgs {
  GridK g;
  const double* xrec;
  const double* Q;
  long long n;
  ParamsK prm;
  int use_warm;
  double* lambda;
  double* f_out;
  uint8_t* iters;
  uint16_t* status;
};

__global__ void __launch_bounds__(WPC * 32) newton_kernel(const NewtonArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WS& w = reinterpret_cast<WS*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const GridK& g = a.g;
  const long long nw = (long long)gridDim.x * WPC;
  for (long long b = (long long)blockIdx.x * WPC + (threadIdx.x >> 5); b < a.n; b += nw) {
    for (int p = lane; p < g.P; p += 32) w.xp[p] = __ldg(a.xrec + b * g.P + p);
    __syncwarp();
    double Q[4], lam[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Q[k] = a.Q[b * 4 + k];
      lam[k] = a.use_warm ? a.lambda[b * 4 + k] : 0.0;
    }
    Eval e;
    int it = 0;
    unsigned st = newton_warp(g, w, Q, lam, a.use_warm, a.prm, &it, e, lane);
    if (a.f_out) {
      PointIter pi(lane, g.n_par);
      for (; pi.p < g.P; pi.next()) {
        double f = a.prm.loss == 0 ? corr_kl(w.xp[pi.p], w.ta[pi.i], w.tb[pi.j])
                                   : corr_l2(w.xp[pi.p], lam, g.vpar[pi.i], g.vperp2[pi.j]);
        a.f_out[b * g.P + pi.p] = f;
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a.lambda[b * 4 + k] = lam[k];
      a.iters[b] = (uint8_t)(it > 255 ? 255 : it);
      a.status[b] = (uint16_t)(st & 0x7fffu);
    }
    __syncwarp();
  }
}

// Decompression: f = x' exp(-lambda.phi) per value (warp per histogram for the
// exponential tables); escapes are written by scatter_corrected_kernel.
struct ApplyArgs {
  GridK g;
  const float* xhat;
  long long ld;
  const int16_t* codes;
  const double* scale;
  const double* lambda;
  const uint16_t* status;
  long long n;
  ParamsK prm;
  double* f;
};

__global__ void __launch_bounds__(128) apply_kernel(const ApplyArgs a) {
  __shared__ double ta[4][AEQC_MAX_NPAR], tb[4][AEQC_MAX_NPERP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GridK& g = a.g;
  const long long nw = (long long)gridDim.x * 4;
  for (long long b = (long long)blockIdx.x * 4 + warp; b < a.n; b += nw) {
    unsigned st = a.status[b];
    double lam[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] = a.lambda[b * 4 + k];
    if (a.prm.loss == 0) {
      for (int i = lane; i < g.n_par; i += 32) ta[warp][i] = corr_a(lam, g.vpar[i]);
      for (int j = lane; j < g.n_perp; j += 32) tb[warp][j] = corr_b(lam, g.vperp2[j]);
    }
    __syncwarp();
    double alpha = (st & AEQC_ST_ALPHA_RETRY) ? a.prm.alpha * 0.25 : a.prm.alpha;
    double dl = (st & (AEQC_ST_ZERO_IMAGE | AEQC_ST_VERBATIM))
                    ? 0.0
                    : bin_width(a.prm.tau, a.scale[b], alpha);
    PointIter pi(lane, g.n_par);
    for (; pi.p < g.P; pi.next()) {
      int c = a.codes[b * g.P + pi.p];
      if (c == AEQC_CODE_ESCAPE && !(st & AEQC_ST_ZERO_IMAGE)) continue;
      double xp;
      if ((st & AEQC_ST_ZERO_IMAGE) || c == AEQC_CODE_ZERO) xp = 0.0;
      else xp = __dadd_rn((double)a.xhat[b * a.ld + pi.p], __dmul_rn((double)c, dl));
      a.f[b * g.P + pi.p] = a.prm.loss == 0 ? corr_kl(xp, ta[warp][pi.i], tb[warp][pi.j])
                                            : corr_l2(xp, lam, g.vpar[pi.i], g.vperp2[pi.j]);
    }
    __syncwarp();
  }
}

struct ScatterArgs {
  GridK g;
  OutliersK o;
  const double* lambda;
  long long row0, n;
  int loss;
  double* f;
};

// raw values at escape points, with the histogram's correction applied
__global__ void scatter_corrected_kernel(const ScatterArgs a) {
  long long cnt = *a.o.count;
  if (cnt > a.o.capacity) cnt = a.o.capacity;
  const int P = a.g.P;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    long long idx = a.o.index[t] - a.row0 * P;
    if (idx < 0 || idx >= a.n * P) continue;
    long long b = idx / P;
    int p = (int)(idx - b * P);
    int j = p / a.g.n_par, i = p - j * a.g.n_par;
    double l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) l[k] = a.lambda[b * 4 + k];
    a.f[idx] = a.loss == 0 ? corr_kl(a.o.value[t], corr_a(l, a.g.vpar[i]),
                                     corr_b(l, a.g.vperp2[j]))
                           : corr_l2(a.o.value[t], l, a.g.vpar[i], a.g.vperp2[j]);
  }
}

int grid_for(long long warps, int sm_mult = 8) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (warps + 3) / 4;
  long long cap = (long long)sms * sm_mult;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

int launch_fused_fp64(const FusedArgs& a, cudaStream_t s) {
  if (a.n <= 0) return AEQC_OK;
  size_t smem = sizeof(WS) * WPC;
  {
    const int rc_attr = raise_smem_limit((const void*)fused_fp64_kernel, (int)smem);
    if (rc_attr) return rc_attr;
  }
  fused_fp64_kernel<<<grid_for(a.n, 2), WPC * 32, smem, s>>>(a);
  return check_launch("fused_fp64_kernel");
}

int launch_fused_fp64_list(const FusedArgs& a, const int* list, const int* count,
                           cudaStream_t s) {
  if (a.n <= 0) return AEQC_OK;
  size_t smem = sizeof(WS) * WPC;
  {
    const int rc_attr = raise_smem_limit((const void*)fused_fp64_list_kernel, (int)smem);
    if (rc_attr) return rc_attr;
  }
  // sized for a few percent of the batch; the grid-stride loop covers any count
  long long warps = a.n / 16 + 1;
  fused_fp64_list_kernel<<<grid_for(warps, 2), WPC * 32, smem, s>>>(a, list, count);
  return check_launch("fused_fp64_list_kernel");
}

int launch_moments(const GridK& g, const double* x, long long n, double* Q, cudaStream_t s) {
  if (n <= 0) return AEQC_OK;
  size_t smem = 4 * AEQC_MAX_P * sizeof(double);
  {
    const int rc_attr = raise_smem_limit((const void*)moments_kernel, (int)smem);
    if (rc_attr) return rc_attr;
  }
  moments_kernel<<<grid_for(n, 4), 128, smem, s>>>(g, x, n, Q);
  return check_launch("moments_kernel");
}

int launch_quantize(const double* x, const float* xhat, long long ld, long long n, int P,
                    const ParamsK& prm, int16_t* codes, double* scale, uint16_t* status,
                    const OutliersK& out, double* xrec, cudaStream_t s) {
  if (n <= 0) return AEQC_OK;
  if (out.count) AEQC_CUDA_TRY(cudaMemsetAsync(out.count, 0, sizeof(long long), s));
  QuantArgs a{x, xhat, ld, n, P, prm, codes, scale, status, out, xrec};
  size_t smem = 4 * AEQC_MAX_P * (sizeof(int16_t) + sizeof(double));
  {
    const int rc_attr = raise_smem_limit((const void*)quantize_kernel, (int)smem);
    if (rc_attr) return rc_attr;
  }
  quantize_kernel<<<grid_for(n, 4), 128, smem, s>>>(a);
  return check_launch("quantize_kernel");
}

int launch_dequantize(const float* xhat, long long ld, const int16_t* codes,
                      const OutliersK* out, const double* scale, const uint16_t* status,
                      long long n, int P, const ParamsK& prm, double* xrec, cudaStream_t s) {
  if (n <= 0) return AEQC_OK;
  long long total = n * (long long)P;
  long long blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  dequantize_kernel<<<(int)blocks, 256, 0, s>>>(xhat, ld, codes, scale, status, n, P, prm,
                                                xrec);
  int rc = check_launch("dequantize_kernel");
  if (rc != AEQC_OK) return rc;
  if (out && out->count) {
    scatter_raw_kernel<<<1024, 256, 0, s>>>(*out, total, xrec);
    rc = check_launch("scatter_raw_kernel");
  }
  return rc;
}

int launch_newton(const GridK& g, const double* xrec, const double* Q, long long n,
                  const ParamsK& prm, int use_warm, double* lambda, double* f_out,
                  uint8_t* iters, uint16_t* status, cudaStream_t s) {
  if (n <= 0) return AEQC_OK;
  NewtonArgs a{g, xrec, Q, n, prm, use_warm, lambda, f_out, iters, status};
  size_t smem = sizeof(WS) * WPC;
  {
    const int rc_attr = raise_smem_limit((const void*)newton_kernel, (int)smem);
    if (rc_attr) return rc_attr;
  }
  newton_kernel<<<grid_for(n, 2), WPC * 32, smem, s>>>(a);
  return check_launch("newton_kernel");
}

int launch_apply(const GridK& g, const float* xhat, long long ld, const int16_t* codes,
                 const OutliersK* out, const double* scale, const double* lambda,
                 const uint16_t* status, long long n, long long row0, const ParamsK& prm,
                 double* f, cudaStream_t s) {
  if (n <= 0) return AEQC_OK;
  ApplyArgs a{g, xhat, ld, codes, scale, lambda, status, n, prm, f};
  apply_kernel<<<grid_for(n, 8), 128, 0, s>>>(a);
  int rc = check_launch("apply_kernel");
  if (rc != AEQC_OK) return rc;
  if (out && out->count) {
    ScatterArgs sa{g, *out, lambda, row0, n, prm.loss, f};
    scatter_corrected_kernel<<<1024, 256, 0, s>>>(sa);
    rc = check_launch("scatter_corrected_kernel");
  }
  return rc;
}

}  // namespace aeqc
