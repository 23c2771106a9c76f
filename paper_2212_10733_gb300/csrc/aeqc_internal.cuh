// Internal declarations shared by the libaeqc translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/aeqc.h"

namespace aeqc {

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
void clear_error();

#define AEQC_CUDA_TRY(expr)                                                    \
  do {                                                                         \
    cudaError_t err__ = (expr);                                                \
    if (err__ != cudaSuccess)                                                  \
      return ::aeqc::set_error(AEQC_ECUDA, "%s failed: %s (%s:%d)", #expr,     \
                               cudaGetErrorString(err__), __FILE__, __LINE__); \
  } while (0)

#define AEQC_CHECK_ARG(cond, ...)                                  \
  do {                                                             \
    if (!(cond)) return ::aeqc::set_error(AEQC_EINVAL, __VA_ARGS__); \
  } while (0)

// launch check after a kernel launch
int check_launch(const char* what);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute is per device, so the raised value is kept
// per (kernel, device ordinal); thread-safe; a no-op once raised (so a call
// inside a stream capture after the first launch on that device does nothing).
int raise_smem_limit(const void* func, int bytes);

// ---------------------------------------------------------------------------
// kernel-side parameter blocks (passed by value)
// ---------------------------------------------------------------------------
struct GridK {
  int n_par, n_perp, P;
  int has_vol;
  const double* vol;   // device [P] or null
  double vol_uniform;
  double vpar[AEQC_MAX_NPAR];
  double vperp2[AEQC_MAX_NPERP];  // v_perp^2
};

struct ParamsK {
  double tau, alpha, step_s, tol, warm_reject, qoi_check;
  int max_iter, r2_max_iter, loss, warm_iters;
  // float copies for the fast kernel (no per-histogram conversions)
  double alpha4;  // alpha / 4 (the retry level)
  float tau_f, step_f, tol_f, warm_reject_f, qoi_check_f;
  // bin width on the integer pipe (fast kernel): set when tau is a normal
  // double and 2 alpha and 2 alpha / 4 are powers of two, 2^a2_e[level];
  // tau = tau_m 2^(tau_e - 52) with tau_m in [2^52, 2^53)
  int bw_int;
  int tau_e, a2_e[2];
  unsigned long long tau_m;
};

// Build kernel blocks from the public structs (validates; returns AEQC_*).
int make_grid(const aeqc_grid* g, GridK* out);
int make_params(const aeqc_params* p, ParamsK* out);

struct OutliersK {
  long long capacity;
  long long* count;
  long long* index;
  double* value;
};

inline OutliersK make_outliers(const aeqc_outliers* o) {
  OutliersK k;
  if (o) {
    k.capacity = o->capacity;
    k.count = reinterpret_cast<long long*>(o->count);
    k.index = reinterpret_cast<long long*>(o->index);
    k.value = o->value;
  } else {
    k.capacity = 0;
    k.count = nullptr;
    k.index = nullptr;
    k.value = nullptr;
  }
  return k;
}

// Warm-start MLP weights as the correction kernels read them (FP32, device).
struct MlpK {
  const float* W1;  // [nin][nh]
  const float* b1;
  const float* W2;  // [nh][nh]
  const float* b2;
  const float* W3;  // [nh][4]
  const float* b3;
  const float* in_mu;
  const float* in_sd;
  const float* out_mu;
  const float* out_sd;
  int nin, nh;
};

// Latent source for the in-kernel warm start features.
struct LatentK {
  const void* ptr;
  int L;
  int bf16;  // 1: __nv_bfloat16 elements, 0: float
};

// Affine form of a uniform grid for the fast correction kernel:
// v_par_i = b (i - i_c) + c0 and v_perp_j^2 = d2 j^2 (v_perp_0 = 0), so every
// moment weight is a polynomial in the integers (i - i_c) and j.
struct FastGridK {
  int ok;  // 0: the grid is not of this form (the fast kernel defers to FP64)
  int i_c;
  double b, c0, d2;
  // the same constants as float pairs (hi + lo) for double-float arithmetic:
  // vol, d2^q (q = 0..2), and coef[p][r] = C(p,r) b^r c0^(p-r) (p, r <= 4)
  float vol_h, vol_l;
  float d2q_h[3], d2q_l[3];
  float coef_h[5][5], coef_l[5][5];
  float b_f, c0_f;   // b and c0 as floats
  float vmax, wmax;  // max |v_par| and max v_perp^2 on the grid
  float wk[4];       // vol sum |phi_k| over the grid (bounds of per-point rounding)
  // lane segments of the column walk (no integer division on the device):
  // rw columns past the first 32 are cut into seg_nchunk chunks of seg_rpc
  // rows; lane l takes chunk (l * seg_mul) >> 16 = l / rw
  int seg_nchunk, seg_rpc, seg_mul;
};
int make_fast_grid(const GridK& g, FastGridK* out);

// ---------------------------------------------------------------------------
// correction kernels (qc_fp64.cu, qc_fast.cu)
// ---------------------------------------------------------------------------
struct FusedArgs {
  const double* x;
  const float* xhat;
  long long ldx;
  long long n;
  long long row0;         // global row of x[0] (for outlier indices)
  GridK grid;
  ParamsK prm;
  int16_t* codes;
  double* scale;
  double* lambda;
  uint8_t* iters;
  uint16_t* status;
  OutliersK out;
  float* features;        // [n][L+4] or null
  LatentK latent;         // for features / warm start
  int use_mlp;
  MlpK mlp;
  double* f_out;          // [n][P] or null
  FastGridK fg;           // fast kernel only
  int* fb_list;           // fast kernel: histograms deferred to the FP64 kernel
  int* fb_count;
};

int launch_fused_fp64(const FusedArgs& a, cudaStream_t s);
int launch_fused_fp64_list(const FusedArgs& a, const int* list, const int* count,
                           cudaStream_t s);
// fast kernel + FP64 kernel over its deferred list; fb_list [n] and fb_count
// are scratch in device memory
int launch_fused_fast(const FusedArgs& a, cudaStream_t s, int warps_per_sm = 0);

int launch_moments(const GridK& g, const double* x, long long n, double* Q, cudaStream_t s);
int launch_quantize(const double* x, const float* xhat, long long ld, long long n, int P,
                    const ParamsK& prm, int16_t* codes, double* scale, uint16_t* status,
                    const OutliersK& out, double* xrec, cudaStream_t s);
int launch_dequantize(const float* xhat, long long ld, const int16_t* codes,
                      const OutliersK* out, const double* scale, const uint16_t* status,
                      long long n, int P, const ParamsK& prm, double* xrec,
                      cudaStream_t s);
int launch_newton(const GridK& g, const double* xrec, const double* Q, long long n,
                  const ParamsK& prm, int use_warm, double* lambda, double* f_out,
                  uint8_t* iters, uint16_t* status, cudaStream_t s);
int launch_apply(const GridK& g, const float* xhat, long long ld, const int16_t* codes,
                 const OutliersK* out, const double* scale, const double* lambda,
                 const uint16_t* status, long long n, long long row0, const ParamsK& prm,
                 double* f, cudaStream_t s);

}  // namespace aeqc
