// NRMSE of decompressed data (Sec. IV-A, Eq. (7)) and the search for the
// largest error bound that meets an NRMSE target (the paper's automatic
// error-bound mode for its residual compressor, Sec. III Stage 4 and
// Sec. V; here the bound is tau of the pointwise guarantee).
//
// nrmse_batch: one warp per histogram sums (f - x)^2 and takes min/max of x
// in a fixed order; a single block folds the per-histogram partials in row
// order, so the batch value is deterministic.
// aeqc_bound_search: bisection on log(tau) between tau_lo and tau_hi; each
// probe compresses and decompresses the batch with the library's calls and
// reads the batch NRMSE back (a synchronisation per probe).  The result is
// the largest probed tau whose NRMSE does not exceed the target.
#include <math.h>
#include <string.h>

#include "model.cuh"
#include "workspace.cuh"

namespace aeqc {
namespace {

struct NPart {
  double ss, mn, mx;
};

__global__ void nrmse_rows_kernel(const double* x, const double* f, long long n, int P,
                                  double* per_hist, NPart* part) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < n;
       b += nw) {
    const double* xb = x + b * P;
    const double* fb = f + b * P;
    double ss = 0.0, mn = INFINITY, mx = -INFINITY;
    for (int p = lane; p < P; p += 32) {
      const double xv = xb[p], d = xv - fb[p];
      ss = fma(d, d, ss);
      mn = fmin(mn, xv);
      mx = fmax(mx, xv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      if (per_hist) per_hist[b] = sqrt(ss / P) / (mx - mn);
      part[b] = NPart{ss, mn, mx};
    }
  }
}

// one block: fixed-order fold of the partials (thread t takes rows t, t + T,
// ...; the threads' results are then folded in thread order)
__global__ void nrmse_fold_kernel(const NPart* part, long long n, int P, double* batch) {
  __shared__ double s_ss[256], s_mn[256], s_mx[256];
  double ss = 0.0, mn = INFINITY, mx = -INFINITY;
  for (long long b = threadIdx.x; b < n; b += blockDim.x) {
    ss += part[b].ss;
    mn = fmin(mn, part[b].mn);
    mx = fmax(mx, part[b].mx);
  }
  s_ss[threadIdx.x] = ss;
  s_mn[threadIdx.x] = mn;
  s_mx[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      a += s_ss[t];
      lo = fmin(lo, s_mn[t]);
      hi = fmax(hi, s_mx[t]);
    }
    *batch = sqrt(a / ((double)n * P)) / (hi - lo);
  }
}

int run_nrmse(const double* x, const double* f, long long n, int P, double* per_hist,
              double* batch, NPart* part, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 7) / 8;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  nrmse_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, f, n, P, per_hist, part);
  nrmse_fold_kernel<<<1, 256, 0, s>>>(part, n, P, batch);
  return check_launch("nrmse");
}

}  // namespace
}  // namespace aeqc

using namespace aeqc;

extern "C" size_t nrmse_workspace_size(int64_t n) {
  if (n <= 0) return 0;
  WsSize w;
  w.add<NPart>((size_t)n);
  return w.bytes;
}

extern "C" int nrmse_batch(const double* x, const double* f, int64_t n, int32_t P,
                           double* per_hist, double* batch, void* workspace,
                           size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(n >= 1 && P >= 1, "nrmse_batch: n=%lld P=%d", (long long)n, P);
  AEQC_CHECK_ARG(x && f && batch && workspace, "nrmse_batch: null pointer");
  AEQC_CHECK_ARG(workspace_bytes >= nrmse_workspace_size(n), "nrmse_batch: workspace too small");
  WsCarver c(static_cast<char*>(workspace), workspace_bytes);
  NPart* part = c.take<NPart>((size_t)n);
  AEQC_CHECK_ARG(c.ok(), "nrmse_batch: workspace not 256-byte aligned");
  return run_nrmse(x, f, n, P, per_hist, batch, part, static_cast<cudaStream_t>(stream));
}

namespace {
struct SearchLayout {
  void* latent;
  double *scale, *lambda, *f, *batch;
  int16_t* codes;
  uint8_t* iters;
  uint16_t* status;
  long long *count, *oidx;
  double* oval;
  NPart* part;
  char* cws;
  size_t cws_bytes;
};

size_t search_layout(const aeqc_model* m, int64_t n, int64_t cap, char* base, size_t bytes,
                     SearchLayout* L) {
  const int P = m->d.P, Ld = m->d.L;
  const size_t esz = m->d.dtype == AEQC_DTYPE_BF16 ? 2 : 4;
  const size_t cws = compress_batch_workspace_size(m, n), dws = decompress_batch_workspace_size(m, n);
  WsSize w;
  w.add<char>((size_t)n * Ld * esz);
  w.add<double>((size_t)n);
  w.add<double>((size_t)n * 4);
  w.add<double>((size_t)n * P);
  w.add<double>(1);
  w.add<int16_t>((size_t)n * P);
  w.add<uint8_t>((size_t)n);
  w.add<uint16_t>((size_t)n);
  w.add<long long>(1);
  w.add<long long>((size_t)cap);
  w.add<double>((size_t)cap);
  w.add<NPart>((size_t)n);
  w.add<char>(cws > dws ? cws : dws);
  if (!base) return w.bytes;
  WsCarver c(base, bytes);
  L->latent = c.take<char>((size_t)n * Ld * esz);
  L->scale = c.take<double>((size_t)n);
  L->lambda = c.take<double>((size_t)n * 4);
  L->f = c.take<double>((size_t)n * P);
  L->batch = c.take<double>(1);
  L->codes = c.take<int16_t>((size_t)n * P);
  L->iters = c.take<uint8_t>((size_t)n);
  L->status = c.take<uint16_t>((size_t)n);
  L->count = c.take<long long>(1);
  L->oidx = c.take<long long>((size_t)cap);
  L->oval = c.take<double>((size_t)cap);
  L->part = c.take<NPart>((size_t)n);
  L->cws_bytes = cws > dws ? cws : dws;
  L->cws = c.take<char>(L->cws_bytes);
  return c.ok() ? w.bytes : 0;
}
}  // namespace

extern "C" size_t aeqc_bound_search_workspace_size(const aeqc_model* m, int64_t n,
                                                   int64_t outlier_capacity) {
  if (!m || n <= 0 || outlier_capacity < 1) return 0;
  return search_layout(m, n, outlier_capacity, nullptr, 0, nullptr);
}

extern "C" int aeqc_bound_search(aeqc_model* m, const aeqc_grid* grid, const double* x, int64_t n,
                                 const int64_t* group_offsets, const aeqc_params* base,
                                 double target, double tau_lo, double tau_hi, int32_t probes,
                                 int64_t outlier_capacity, double* tau_out, double* nrmse_out,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  AEQC_CHECK_ARG(m && grid && x && base && tau_out && nrmse_out && workspace,
                 "aeqc_bound_search: null argument");
  AEQC_CHECK_ARG(n >= 1 && outlier_capacity >= 1, "aeqc_bound_search: n=%lld", (long long)n);
  AEQC_CHECK_ARG(target > 0.0 && tau_lo > 0.0 && tau_hi > tau_lo && probes >= 1 && probes <= 64,
                 "aeqc_bound_search: target %g, tau in [%g, %g], %d probes", target, tau_lo,
                 tau_hi, probes);
  AEQC_CHECK_ARG(workspace_bytes >= aeqc_bound_search_workspace_size(m, n, outlier_capacity),
                 "aeqc_bound_search: workspace too small");
  SearchLayout L;
  AEQC_CHECK_ARG(search_layout(m, n, outlier_capacity, static_cast<char*>(workspace),
                               workspace_bytes, &L),
                 "aeqc_bound_search: workspace not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  aeqc_compressed out;
  memset(&out, 0, sizeof(out));
  out.latent = L.latent;
  out.scale = L.scale;
  out.codes = L.codes;
  out.lambda = L.lambda;
  out.iters = L.iters;
  out.status = L.status;
  out.outliers.capacity = outlier_capacity;
  out.outliers.count = reinterpret_cast<int64_t*>(L.count);
  out.outliers.index = reinterpret_cast<int64_t*>(L.oidx);
  out.outliers.value = L.oval;
  aeqc_params p = *base;
  double lo = log(tau_lo), hi = log(tau_hi), best_tau = 0.0, best_e = 0.0;
  int rc;
  for (int it = 0; it < probes; ++it) {
    const double t = it == 0 ? tau_lo : exp(0.5 * (lo + hi));  // the lower end first
    p.tau = t;
    if ((rc = compress_batch(m, nullptr, grid, x, n, group_offsets, &p, &out, L.cws, L.cws_bytes,
                             stream)))
      return rc;
    long long cnt = 0;
    AEQC_CUDA_TRY(cudaMemcpyAsync(&cnt, L.count, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    AEQC_CUDA_TRY(cudaStreamSynchronize(s));
    if (cnt > outlier_capacity)  // escaped values were dropped: no faithful decompression
      return set_error(AEQC_EUNSUPPORTED,
                       "aeqc_bound_search: %lld escaped values at tau = %g exceed the outlier "
                       "capacity %lld",
                       cnt, t, (long long)outlier_capacity);
    if ((rc = decompress_batch(m, grid, &out, n, group_offsets, &p, L.f, L.cws, L.cws_bytes,
                               stream)))
      return rc;
    if ((rc = run_nrmse(x, L.f, n, m->d.P, nullptr, L.batch, L.part, s))) return rc;
    double e = 0.0;
    AEQC_CUDA_TRY(cudaMemcpyAsync(&e, L.batch, sizeof(double), cudaMemcpyDeviceToHost, s));
    AEQC_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(e <= target)) {
      if (it == 0) break;  // even the lower end misses the target
      hi = log(t);
    } else {
      if (t > best_tau) {
        best_tau = t;
        best_e = e;
      }
      if (it > 0) lo = log(t);
    }
  }
  if (best_tau == 0.0)
    return set_error(AEQC_EUNSUPPORTED, "aeqc_bound_search: NRMSE at tau_lo already above %g",
                     target);
  *tau_out = best_tau;
  *nrmse_out = best_e;
  return AEQC_OK;
}
