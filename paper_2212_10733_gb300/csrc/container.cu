// Host-side serialisation: model and MLP checkpoints (weights, normalisation,
// Adam state and step counts) and the compressed-batch container (the codes,
// latents and multipliers a decompressor needs, Sec. III end of Stage 5).
// Little-endian blobs with a versioned header; every header is validated on
// the host before anything is copied (AEQC_ECORRUPT on any inconsistency).
#include <stddef.h>
#include <string.h>

#include <string>
#include <vector>

#include "model.cuh"

using namespace aeqc;

namespace {

constexpr char kModelMagic[8] = {'A', 'E', 'Q', 'C', 'M', 'D', 'L', '1'};
constexpr char kMlpMagic[8] = {'A', 'E', 'Q', 'C', 'M', 'L', 'P', '1'};
constexpr char kBatchMagic[8] = {'A', 'E', 'Q', 'C', 'B', 'A', 'T', '1'};
constexpr uint32_t kVersion = 1;

struct ModelHeader {  // 64 bytes
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  aeqc_model_desc desc;  // 32 bytes
  uint64_t n_group;      // floats of one group's parameters (with mu, sigma)
  uint64_t n_train;      // floats of one group's trainable parameters (Adam moments)
};
static_assert(sizeof(ModelHeader) == 64, "model header layout");

struct MlpHeader {  // 40 bytes
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int32_t n_in, n_hidden;
  uint64_t n_all, n_train;
};
static_assert(sizeof(MlpHeader) == 40, "mlp header layout");

constexpr int kSections = 8;  // latent scale codes lambda iters status out_index out_value
struct BatchHeader {          // 192 bytes
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n;
  int32_t P, L, latent_dtype, reserved;
  int64_t outliers;
  uint64_t total_bytes;
  uint64_t off[kSections];
  uint64_t len[kSections];
  uint64_t pad;
};
static_assert(sizeof(BatchHeader) == 192, "batch header layout");

size_t model_blob_bytes(const aeqc_model* m) {
  const size_t G = (size_t)m->d.n_groups;
  return sizeof(ModelHeader) + sizeof(float) * (G * m->n_group + 2 * G * m->n_train) +
         sizeof(int32_t) * G;
}

size_t mlp_blob_bytes(const aeqc_mlp* m) {
  return sizeof(MlpHeader) + sizeof(float) * (size_t)(m->n_all + 2 * m->n_train) +
         sizeof(int32_t);
}

size_t align16(size_t v) { return (v + 15) / 16 * 16; }

// section lengths of a batch
void batch_lens(int64_t n, int32_t P, int32_t L, int32_t dt, int64_t outl, uint64_t len[]) {
  const uint64_t esz = dt == AEQC_DTYPE_BF16 ? 2 : 4;
  len[0] = (uint64_t)n * L * esz;
  len[1] = (uint64_t)n * 8;
  len[2] = (uint64_t)n * P * 2;
  len[3] = (uint64_t)n * 32;
  len[4] = (uint64_t)n;
  len[5] = (uint64_t)n * 2;
  len[6] = (uint64_t)outl * 8;
  len[7] = (uint64_t)outl * 8;
}

uint64_t batch_layout(int64_t n, int32_t P, int32_t L, int32_t dt, int64_t outl, uint64_t off[],
                      uint64_t len[]) {
  batch_lens(n, P, L, dt, outl, len);
  uint64_t o = sizeof(BatchHeader);
  for (int k = 0; k < kSections; ++k) {
    off[k] = o;
    o = align16(o + len[k]);
  }
  return o;
}

// Validates a batch header against the blob size; AEQC_OK or AEQC_ECORRUPT.
int check_batch(const void* blob, size_t bytes, BatchHeader* out) {
  AEQC_CHECK_ARG(blob, "batch container: null blob");
  if (bytes < sizeof(BatchHeader))
    return set_error(AEQC_ECORRUPT, "batch container: %zu bytes, shorter than its header", bytes);
  BatchHeader h;
  memcpy(&h, blob, sizeof(h));
  if (memcmp(h.magic, kBatchMagic, 8) != 0)
    return set_error(AEQC_ECORRUPT, "batch container: bad magic");
  if (h.version != kVersion || h.header_bytes != sizeof(BatchHeader))
    return set_error(AEQC_ECORRUPT, "batch container: version %u / header %u not supported",
                     h.version, h.header_bytes);
  if (h.n < 0 || h.n > (int64_t)1 << 40 || h.P <= 0 || h.P > AEQC_MAX_P || h.L <= 0 ||
      h.L > 256 || (h.latent_dtype != AEQC_DTYPE_F32 && h.latent_dtype != AEQC_DTYPE_BF16) ||
      h.outliers < 0 || h.outliers > h.n * (int64_t)h.P)
    return set_error(AEQC_ECORRUPT, "batch container: counts out of range (n=%lld P=%d L=%d "
                     "outliers=%lld)", (long long)h.n, h.P, h.L, (long long)h.outliers);
  uint64_t len[kSections];
  batch_lens(h.n, h.P, h.L, h.latent_dtype, h.outliers, len);
  uint64_t prev_end = sizeof(BatchHeader);
  for (int k = 0; k < kSections; ++k) {
    if (h.len[k] != len[k])
      return set_error(AEQC_ECORRUPT, "batch container: section %d has %llu bytes, %llu expected",
                       k, (unsigned long long)h.len[k], (unsigned long long)len[k]);
    if (h.off[k] < prev_end || h.off[k] % 16 != 0 || h.off[k] > h.total_bytes ||
        h.len[k] > h.total_bytes - h.off[k])
      return set_error(AEQC_ECORRUPT, "batch container: section %d at %llu+%llu outside or "
                       "overlapping", k, (unsigned long long)h.off[k],
                       (unsigned long long)h.len[k]);
    prev_end = h.off[k] + h.len[k];
  }
  if (h.total_bytes != bytes)
    return set_error(AEQC_ECORRUPT, "batch container: header says %llu bytes, blob has %zu",
                     (unsigned long long)h.total_bytes, bytes);
  *out = h;
  return AEQC_OK;
}

}  // namespace

// ---- model checkpoints ----------------------------------------------------------

extern "C" size_t aeqc_model_save_size(const aeqc_model* m) { return m ? model_blob_bytes(m) : 0; }

extern "C" int aeqc_model_save(const aeqc_model* m, void* blob, size_t bytes) {
  clear_error();
  AEQC_CHECK_ARG(m && blob, "aeqc_model_save: null argument");
  const size_t need = model_blob_bytes(m);
  AEQC_CHECK_ARG(bytes >= need, "aeqc_model_save: %zu bytes needed", need);
  ModelHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kModelMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(ModelHeader);
  h.desc = m->d;
  h.n_group = (uint64_t)m->n_group;
  h.n_train = (uint64_t)m->n_train;
  char* p = static_cast<char*>(blob);
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t G = (size_t)m->d.n_groups;
  const size_t fb = sizeof(float) * (G * m->n_group + 2 * G * m->n_train);
  // params, adam_m and adam_v are contiguous in the model's device block
  AEQC_CUDA_TRY(cudaDeviceSynchronize());
  AEQC_CUDA_TRY(cudaMemcpy(p, m->params, fb, cudaMemcpyDeviceToHost));
  p += fb;
  for (size_t g = 0; g < G; ++g) {
    const int32_t st = m->step[g];
    memcpy(p + 4 * g, &st, 4);
  }
  return AEQC_OK;
}

extern "C" int aeqc_model_load(const void* blob, size_t bytes, aeqc_model** out) {
  clear_error();
  AEQC_CHECK_ARG(blob && out, "aeqc_model_load: null argument");
  if (bytes < sizeof(ModelHeader))
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: %zu bytes, shorter than the header", bytes);
  ModelHeader h;
  memcpy(&h, blob, sizeof(h));
  if (memcmp(h.magic, kModelMagic, 8) != 0)
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: bad magic");
  if (h.version != kVersion || h.header_bytes != sizeof(ModelHeader))
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: version %u / header %u not supported",
                     h.version, h.header_bytes);
  const uint64_t G0 = (uint64_t)h.desc.n_groups;
  if (h.desc.n_groups <= 0 || G0 > (1u << 20) || h.n_group == 0 || h.n_group > (1ull << 32) ||
      h.n_train > h.n_group ||
      (uint64_t)bytes != sizeof(ModelHeader) + 4 * G0 * (h.n_group + 2 * h.n_train) + 4 * G0)
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: header sizes do not match the blob");
  aeqc_model* m = nullptr;
  int rc = aeqc_model_create(&h.desc, &m);  // validates the descriptor
  if (rc == AEQC_EINVAL || rc == AEQC_EUNSUPPORTED) {
    const std::string why = aeqc_last_error();
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: %s", why.c_str());
  }
  if (rc) return rc;
  if ((uint64_t)m->n_group != h.n_group || (uint64_t)m->n_train != h.n_train ||
      bytes != model_blob_bytes(m)) {
    aeqc_model_destroy(m);
    return set_error(AEQC_ECORRUPT, "aeqc_model_load: sizes do not match the descriptor");
  }
  const char* p = static_cast<const char*>(blob) + sizeof(h);
  const size_t G = (size_t)h.desc.n_groups;
  const size_t fb = sizeof(float) * (G * m->n_group + 2 * G * m->n_train);
  if (cudaMemcpy(m->params, p, fb, cudaMemcpyHostToDevice) != cudaSuccess) {
    aeqc_model_destroy(m);
    return set_error(AEQC_ECUDA, "aeqc_model_load: copy failed");
  }
  p += fb;
  for (size_t g = 0; g < G; ++g) {
    int32_t st;
    memcpy(&st, p + 4 * g, 4);
    m->step[g] = st;
  }
  m->dirty = true;
  *out = m;
  return AEQC_OK;
}

// ---- MLP checkpoints ----------------------------------------------------------------

extern "C" size_t aeqc_mlp_save_size(const aeqc_mlp* m) { return m ? mlp_blob_bytes(m) : 0; }

extern "C" int aeqc_mlp_save(const aeqc_mlp* m, void* blob, size_t bytes) {
  clear_error();
  AEQC_CHECK_ARG(m && blob, "aeqc_mlp_save: null argument");
  AEQC_CHECK_ARG(bytes >= mlp_blob_bytes(m), "aeqc_mlp_save: %zu bytes needed", mlp_blob_bytes(m));
  MlpHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMlpMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(MlpHeader);
  h.n_in = m->nin;
  h.n_hidden = m->nh;
  h.n_all = (uint64_t)m->n_all;
  h.n_train = (uint64_t)m->n_train;
  char* p = static_cast<char*>(blob);
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t fb = sizeof(float) * (size_t)(m->n_all + 2 * m->n_train);
  AEQC_CUDA_TRY(cudaDeviceSynchronize());
  AEQC_CUDA_TRY(cudaMemcpy(p, m->params, fb, cudaMemcpyDeviceToHost));
  const int32_t st = m->step;
  memcpy(p + fb, &st, 4);
  return AEQC_OK;
}

extern "C" int aeqc_mlp_load(const void* blob, size_t bytes, aeqc_mlp** out) {
  clear_error();
  AEQC_CHECK_ARG(blob && out, "aeqc_mlp_load: null argument");
  if (bytes < sizeof(MlpHeader))
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: %zu bytes, shorter than the header", bytes);
  MlpHeader h;
  memcpy(&h, blob, sizeof(h));
  if (memcmp(h.magic, kMlpMagic, 8) != 0)
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: bad magic");
  if (h.version != kVersion || h.header_bytes != sizeof(MlpHeader))
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: version %u / header %u not supported",
                     h.version, h.header_bytes);
  if (h.n_all == 0 || h.n_all > (1ull << 32) || h.n_train > h.n_all ||
      (uint64_t)bytes != sizeof(MlpHeader) + 4 * (h.n_all + 2 * h.n_train) + 4)
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: header sizes do not match the blob");
  aeqc_mlp* m = nullptr;
  int rc = aeqc_mlp_create(h.n_in, h.n_hidden, &m);
  if (rc == AEQC_EINVAL || rc == AEQC_EUNSUPPORTED) {
    const std::string why = aeqc_last_error();
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: %s", why.c_str());
  }
  if (rc) return rc;
  if ((uint64_t)m->n_all != h.n_all || (uint64_t)m->n_train != h.n_train ||
      bytes != mlp_blob_bytes(m)) {
    aeqc_mlp_destroy(m);
    return set_error(AEQC_ECORRUPT, "aeqc_mlp_load: sizes do not match the header");
  }
  const char* p = static_cast<const char*>(blob) + sizeof(h);
  const size_t fb = sizeof(float) * (size_t)(m->n_all + 2 * m->n_train);
  if (cudaMemcpy(m->params, p, fb, cudaMemcpyHostToDevice) != cudaSuccess) {
    aeqc_mlp_destroy(m);
    return set_error(AEQC_ECUDA, "aeqc_mlp_load: copy failed");
  }
  int32_t st;
  memcpy(&st, p + fb, 4);
  m->step = st;
  *out = m;
  return AEQC_OK;
}

// ---- compressed-batch container --------------------------------------------------------

extern "C" size_t aeqc_batch_pack_size(int64_t n, int32_t P, int32_t L, int32_t latent_dtype,
                                       int64_t outliers) {
  if (n < 0 || P <= 0 || L <= 0 || outliers < 0) return 0;
  uint64_t off[kSections], len[kSections];
  return (size_t)batch_layout(n, P, L, latent_dtype, outliers, off, len);
}

extern "C" int aeqc_batch_pack(const aeqc_compressed* in, int64_t n, int32_t P, int32_t L,
                               int32_t latent_dtype, void* blob, size_t bytes, size_t* written,
                               void* stream) {
  clear_error();
  AEQC_CHECK_ARG(in && blob && written, "aeqc_batch_pack: null argument");
  AEQC_CHECK_ARG(n >= 0 && P > 0 && P <= AEQC_MAX_P && L > 0 && L <= 256,
                 "aeqc_batch_pack: bad sizes");
  AEQC_CHECK_ARG(latent_dtype == AEQC_DTYPE_F32 || latent_dtype == AEQC_DTYPE_BF16,
                 "aeqc_batch_pack: bad latent dtype");
  AEQC_CHECK_ARG(in->latent && in->scale && in->codes && in->lambda && in->iters && in->status &&
                     in->outliers.count,
                 "aeqc_batch_pack: null array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t cnt = 0;
  AEQC_CUDA_TRY(cudaMemcpyAsync(&cnt, in->outliers.count, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  AEQC_CUDA_TRY(cudaStreamSynchronize(s));
  if (cnt > in->outliers.capacity) cnt = in->outliers.capacity;  // dropped entries are flagged
  if (cnt < 0) cnt = 0;
  BatchHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kBatchMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(BatchHeader);
  h.n = n;
  h.P = P;
  h.L = L;
  h.latent_dtype = latent_dtype;
  h.outliers = cnt;
  h.total_bytes = batch_layout(n, P, L, latent_dtype, cnt, h.off, h.len);
  AEQC_CHECK_ARG(bytes >= h.total_bytes, "aeqc_batch_pack: %llu bytes needed",
                 (unsigned long long)h.total_bytes);
  char* b = static_cast<char*>(blob);
  memset(b, 0, (size_t)h.total_bytes);
  memcpy(b, &h, sizeof(h));
  const void* src[kSections] = {in->latent, in->scale, in->codes, in->lambda,
                                in->iters,  in->status, in->outliers.index, in->outliers.value};
  for (int k = 0; k < kSections; ++k)
    if (h.len[k])
      AEQC_CUDA_TRY(cudaMemcpyAsync(b + h.off[k], src[k], h.len[k], cudaMemcpyDeviceToHost, s));
  AEQC_CUDA_TRY(cudaStreamSynchronize(s));
  *written = (size_t)h.total_bytes;
  return AEQC_OK;
}

extern "C" int aeqc_batch_peek(const void* blob, size_t bytes, int64_t* n, int32_t* P, int32_t* L,
                               int32_t* latent_dtype, int64_t* outliers) {
  clear_error();
  BatchHeader h;
  int rc = check_batch(blob, bytes, &h);
  if (rc) return rc;
  if (n) *n = h.n;
  if (P) *P = h.P;
  if (L) *L = h.L;
  if (latent_dtype) *latent_dtype = h.latent_dtype;
  if (outliers) *outliers = h.outliers;
  return AEQC_OK;
}

extern "C" int aeqc_batch_unpack(const void* blob, size_t bytes, aeqc_compressed* out,
                                 void* stream) {
  clear_error();
  BatchHeader h;
  int rc = check_batch(blob, bytes, &h);
  if (rc) return rc;
  AEQC_CHECK_ARG(out && out->latent && out->scale && out->codes && out->lambda && out->iters &&
                     out->status && out->outliers.count,
                 "aeqc_batch_unpack: null output array");
  AEQC_CHECK_ARG(h.outliers <= out->outliers.capacity &&
                     (h.outliers == 0 || (out->outliers.index && out->outliers.value)),
                 "aeqc_batch_unpack: %lld outliers, capacity %lld", (long long)h.outliers,
                 (long long)out->outliers.capacity);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* b = static_cast<const char*>(blob);
  void* dst[kSections] = {out->latent, out->scale, out->codes, out->lambda,
                          out->iters,  out->status, out->outliers.index, out->outliers.value};
  for (int k = 0; k < kSections; ++k)
    if (h.len[k])
      AEQC_CUDA_TRY(cudaMemcpyAsync(dst[k], b + h.off[k], h.len[k], cudaMemcpyHostToDevice, s));
  AEQC_CUDA_TRY(cudaMemcpyAsync(out->outliers.count, b + offsetof(BatchHeader, outliers),
                                sizeof(int64_t), cudaMemcpyHostToDevice, s));
  AEQC_CUDA_TRY(cudaStreamSynchronize(s));
  return AEQC_OK;
}
