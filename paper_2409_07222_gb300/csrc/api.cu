// api.cu -- the C ABI of liblabs.so: context, argument validation, dispatch to the kernels.
#include <cstdlib>
#include <cstring>
#include <new>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {

void* ws_get(labs_ctx* ctx, int slot, size_t bytes) {
  if (slot < 0 || slot >= 8) return nullptr;
  if (ctx->ws_bytes[slot] >= bytes && ctx->ws[slot]) return ctx->ws[slot];
  if (ctx->ws[slot]) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws[slot]);
    ctx->ws[slot] = nullptr;
    ctx->ws_bytes[slot] = 0;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) return nullptr;
  ctx->ws[slot] = p;
  ctx->ws_bytes[slot] = want;
  return p;
}

}  // namespace labsg

namespace {

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

int set_device(labs_ctx* ctx) { return cudaSetDevice(ctx->device) == cudaSuccess ? LABS_OK : LABS_ERR_CUDA; }

}  // namespace

extern "C" {

int labs_abi_version(void) { return 1; }

const char* labs_status_string(int status) {
  switch (status) {
    case LABS_OK: return "ok";
    case LABS_ERR_INVALID_ARG: return "invalid argument";
    case LABS_ERR_CAPACITY: return "capacity exceeded";
    case LABS_ERR_TIMEOUT: return "device wait timed out";
    case LABS_ERR_CUDA: return "CUDA error";
    case LABS_ERR_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

int labs_ctx_create(labs_ctx** out, int device) {
  if (!out) return LABS_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LABS_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return LABS_ERR_CUDA;
  labs_ctx* c = new (std::nothrow) labs_ctx();
  if (!c) return LABS_ERR_NOMEM;
  std::memset(c, 0, sizeof(*c));
  c->device = device;
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->num_sms = sms > 0 ? sms : 1;
  c->smem_optin = (size_t)optin;
  *out = c;
  return LABS_OK;
}

void labs_ctx_destroy(labs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (int i = 0; i < 8; i++)
    if (ctx->ws[i]) cudaFree(ctx->ws[i]);
  delete ctx;
}

int labs_energy_batch(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out,
                      void* stream) {
  LABS_TRACE("labs_energy_batch");
  if (!ctx || L < 2 || L > LABS_MAX_L || n < 0) return LABS_ERR_INVALID_ARG;
  if (n > 0 && (!seqs || !E_out || !aligned8(seqs) || !aligned4(E_out) || (C_out && !aligned4(C_out))))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_energy_batch(ctx, seqs, L, n, E_out, C_out, (cudaStream_t)stream);
}

int labs_flip_deltas(labs_ctx* ctx, const uint64_t* seqs, const int32_t* C, int L, int64_t n, int skew, int p,
                     int32_t* dE_out, void* stream) {
  LABS_TRACE("labs_flip_deltas");
  if (!ctx || L < 2 || L > LABS_MAX_L || n < 0 || (skew != 0 && skew != 1) || p < 0) return LABS_ERR_INVALID_ARG;
  if (skew && (L % 2 == 0 || L < 3 || p > (L - 1) / 2)) return LABS_ERR_INVALID_ARG;
  if (!skew && p >= L) return LABS_ERR_INVALID_ARG;
  if (n > 0 && (!seqs || !dE_out || !aligned8(seqs) || !aligned4(dE_out) || (C && !aligned4(C))))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_flip_deltas(ctx, seqs, C, L, n, skew, p, dE_out, (cudaStream_t)stream);
}

int labs_sample_threshold(labs_ctx* ctx, int L, int skew, int p, const uint64_t* prefixes, int n_prefix,
                          uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr_out, int32_t* E_samples,
                          void* stream) {
  LABS_TRACE("labs_sample_threshold");
  if (!ctx) return LABS_ERR_INVALID_ARG;
  int s = labsg::check_walk_shape(L, skew, p, n_prefix, prefixes);
  if (s != LABS_OK) return s;
  if (n_samples < 1 || rank < 0 || rank >= n_samples || !E_thr_out || !aligned4(E_thr_out) ||
      (E_samples && !aligned4(E_samples)))
    return LABS_ERR_INVALID_ARG;
  s = set_device(ctx);
  if (s != LABS_OK) return s;
  int pw = p > 0 ? (p + 63) / 64 : 1;
  return labsg::launch_sample_threshold(ctx, L, skew, p, prefixes, n_prefix, pw, seed, n_samples, rank, E_thr_out,
                                       E_samples, (cudaStream_t)stream);
}

int labs_skew_search(labs_ctx* ctx, const labs_walk_cfg* cfg, const uint64_t* prefixes, int n_prefix,
                     labs_candidate* out, int64_t* walk_stats, labs_walk_stats* stats, void* stream) {
  LABS_TRACE("labs_skew_search");
  if (!ctx || !cfg) return LABS_ERR_INVALID_ARG;
  int s = labsg::check_walk_shape(cfg->L, cfg->skew, cfg->p, n_prefix, prefixes);
  if (s != LABS_OK) return s;
  if (cfg->n_walks < 0 || cfg->walk_begin < 0 || cfg->flip_budget < 0 || cfg->R < 1 || cfg->R > labsg::kMaxR ||
      cfg->bloom_log2 < 5 || cfg->bloom_log2 > 15 || cfg->bloom_k < 1 || cfg->bloom_k > 8)
    return LABS_ERR_INVALID_ARG;
  if (cfg->walk_begin + cfg->n_walks > 0xffffffffLL) return LABS_ERR_INVALID_ARG;  // walk ids are stored as u32
  if (cfg->flip_budget > 0xffffffffLL) return LABS_ERR_INVALID_ARG;               // steps are stored as u32
  if (cfg->tile_m != 0 && cfg->tile_m != 8 && cfg->tile_m != 12 && cfg->tile_m != 16)
    return LABS_ERR_INVALID_ARG;
  if (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 12) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk != 0 && cfg->lanes_per_walk != 16 && cfg->lanes_per_walk != 32) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk == 32 && cfg->warps_per_cta > 8) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk == 16 && cfg->R > 16) return LABS_ERR_INVALID_ARG;
  if (cfg->E_thr_dev && !aligned4(cfg->E_thr_dev)) return LABS_ERR_INVALID_ARG;
  if (!cfg->E_thr_dev && cfg->E_thr == LABS_AUTO_THRESHOLD &&
      (cfg->n_thresh_samples < 1 || cfg->thresh_rank < 0 || cfg->thresh_rank >= cfg->n_thresh_samples))
    return LABS_ERR_INVALID_ARG;
  if (!stats || !aligned8(stats) || (cfg->n_walks > 0 && (!out || !aligned8(out))) ||
      (walk_stats && !aligned8(walk_stats)))
    return LABS_ERR_INVALID_ARG;
  s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_skew_search(ctx, cfg, prefixes, n_prefix, out, walk_stats, stats, (cudaStream_t)stream);
}

int labs_batched_search(labs_ctx* ctx, const labs_batch_cfg* cfg, const int32_t* lengths, const int64_t* walks,
                        const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                        int32_t* E_thr_out, labs_walk_stats* stats, void* stream) {
  LABS_TRACE("labs_batched_search");
  if (!ctx || !cfg || !lengths || !walks || cfg->n_len < 1 || cfg->n_len > 96) return LABS_ERR_INVALID_ARG;
  int64_t total = 0;
  int min_odd = LABS_MAX_L + 1;
  for (int i = 0; i < cfg->n_len; i++) {
    if (lengths[i] < 3 || lengths[i] > LABS_MAX_L || walks[i] < 0) return LABS_ERR_INVALID_ARG;
    if (lengths[i] & 1) min_odd = lengths[i] < min_odd ? lengths[i] : min_odd;
    total += walks[i];
  }
  if (cfg->p < 0 || (min_odd <= LABS_MAX_L && cfg->p > (min_odd - 1) / 2)) return LABS_ERR_INVALID_ARG;
  if (n_prefix < 1 || !prefixes || !aligned8(prefixes)) return LABS_ERR_INVALID_ARG;
  if (total > 0xffffffffLL || cfg->flip_budget < 0 || cfg->flip_budget > 0xffffffffLL) return LABS_ERR_INVALID_ARG;
  if (cfg->R < 1 || cfg->R > labsg::kMaxR || cfg->bloom_log2 < 5 || cfg->bloom_log2 > 15 || cfg->bloom_k < 1 ||
      cfg->bloom_k > 8)
    return LABS_ERR_INVALID_ARG;
  if (cfg->n_thresh_samples < 1 || cfg->n_thresh_samples > 0x7fffffffLL || cfg->thresh_rank < 0 ||
      cfg->thresh_rank >= cfg->n_thresh_samples)
    return LABS_ERR_INVALID_ARG;
  if (cfg->tile_m != 0 && cfg->tile_m != 8 && cfg->tile_m != 12 && cfg->tile_m != 16) return LABS_ERR_INVALID_ARG;
  if (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 8) return LABS_ERR_INVALID_ARG;
  if (!stats || !aligned8(stats) || (total > 0 && (!out || !aligned8(out))) || (walk_stats && !aligned8(walk_stats)) ||
      (E_thr_out && !aligned4(E_thr_out)))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_batched_search(ctx, cfg, lengths, walks, prefixes, n_prefix, out, walk_stats, E_thr_out, stats,
                                      (cudaStream_t)stream);
}

int labs_chunked_search(labs_ctx* ctx, const labs_walk_cfg* cfg, labs_policy* policy, float lambda, int chunk,
                        const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                        labs_walk_stats* stats, float* logits_log, uint64_t* state_log, int32_t* move_log,
                        void* stream) {
  LABS_TRACE("labs_chunked_search");
  if (!ctx || !cfg || chunk < 1 || !(lambda == lambda)) return LABS_ERR_INVALID_ARG;
  int s = labsg::check_walk_shape(cfg->L, cfg->skew, cfg->p, n_prefix, prefixes);
  if (s != LABS_OK) return s;
  if (cfg->n_walks < 0 || cfg->walk_begin < 0 || cfg->flip_budget < 0 || cfg->R < 1 || cfg->R > labsg::kMaxR ||
      cfg->bloom_log2 < 5 || cfg->bloom_log2 > 15 || cfg->bloom_k < 1 || cfg->bloom_k > 8)
    return LABS_ERR_INVALID_ARG;
  if (cfg->walk_begin + cfg->n_walks > 0xffffffffLL || cfg->flip_budget > 0x7fffffffLL) return LABS_ERR_INVALID_ARG;
  if (cfg->tile_m != 0 && cfg->tile_m != 8 && cfg->tile_m != 12 && cfg->tile_m != 16) return LABS_ERR_INVALID_ARG;
  if (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 12) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk != 0 && cfg->lanes_per_walk != 16 && cfg->lanes_per_walk != 32) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk == 32 && cfg->warps_per_cta > 8) return LABS_ERR_INVALID_ARG;
  if (cfg->lanes_per_walk == 16 && cfg->R > 16) return LABS_ERR_INVALID_ARG;
  if (!cfg->E_thr_dev && cfg->E_thr == LABS_AUTO_THRESHOLD &&
      (cfg->n_thresh_samples < 1 || cfg->thresh_rank < 0 || cfg->thresh_rank >= cfg->n_thresh_samples))
    return LABS_ERR_INVALID_ARG;
  if (!stats || !aligned8(stats) || (cfg->n_walks > 0 && (!out || !aligned8(out))))
    return LABS_ERR_INVALID_ARG;
  if (policy && labsg::policy_length(policy) != cfg->L) return LABS_ERR_INVALID_ARG;
  s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_chunked_search(ctx, cfg, policy, lambda, chunk, prefixes, n_prefix, out, walk_stats, stats,
                                      logits_log, state_log, move_log, (cudaStream_t)stream);
}

int labs_pq_refine(labs_ctx* ctx, const labs_pq_cfg* cfg, const uint64_t* seeds, int n_seeds, uint64_t* best_seq,
                   int32_t* best_E, labs_pq_stats* stats, void* stream) {
  LABS_TRACE("labs_pq_refine");
  if (!ctx || !cfg || cfg->L < 2 || cfg->L > LABS_MAX_L || cfg->B < 1 || cfg->B > 8192 || cfg->cap < 1 ||
      cfg->cap > (1ll << 24) || cfg->H_log2 < 10 || cfg->H_log2 > 31 || cfg->T_r < 0 || cfg->T_r > 64 || 2 * cfg->T_r >= cfg->L || cfg->max_expansions < 0 ||
      n_seeds < 1)
    return LABS_ERR_INVALID_ARG;
  if (!seeds || !aligned8(seeds) || !best_seq || !aligned8(best_seq) || !best_E || !aligned4(best_E) || !stats ||
      !aligned8(stats))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_pq_refine(ctx, cfg, seeds, n_seeds, best_seq, best_E, stats, (cudaStream_t)stream);
}

int labs_sequence_operators(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, uint64_t* grow, int32_t* E_grow,
                            uint64_t* shrink, int32_t* E_shrink, void* stream) {
  LABS_TRACE("labs_sequence_operators");
  if (!ctx || L < 3 || L > LABS_MAX_L - 1 || n < 0) return LABS_ERR_INVALID_ARG;
  if (n > 0 && (!seqs || !aligned8(seqs) || (grow && !aligned8(grow)) || (shrink && !aligned8(shrink)) ||
                (E_grow && !aligned4(E_grow)) || (E_shrink && !aligned4(E_shrink))))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_sequence_operators(ctx, seqs, L, n, grow, E_grow, shrink, E_shrink, (cudaStream_t)stream);
}

int labs_legendre_family(int L, double r_lo, double r_hi, double t_max, int32_t* params, int64_t max_n,
                         int64_t* n_out) {
  if (L < 3 || L > LABS_MAX_L || !(r_lo >= 0.0) || !(r_hi >= r_lo) || !(t_max >= 0.0) || !n_out || max_n < 0)
    return LABS_ERR_INVALID_ARG;
  return labsg::legendre_family(L, r_lo, r_hi, t_max, params, max_n, n_out);
}

int labs_legendre_construct(labs_ctx* ctx, int L, const int32_t* params, int64_t n, uint64_t* seqs, int32_t* E_out,
                            void* stream) {
  LABS_TRACE("labs_legendre_construct");
  if (!ctx || L < 3 || L > LABS_MAX_L || n < 0) return LABS_ERR_INVALID_ARG;
  if (n > 0 && (!params || !aligned4(params) || (seqs && !aligned8(seqs)) || (E_out && !aligned4(E_out))))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_legendre(ctx, L, params, n, seqs, E_out, (cudaStream_t)stream);
}

int labs_pq_independent(labs_ctx* ctx, const labs_pq_indep_cfg* cfg, const uint64_t* seeds, int n, uint64_t* best_seqs,
                        int32_t* best_E, labs_pq_stats* stats, void* stream) {
  LABS_TRACE("labs_pq_independent");
  if (!ctx || !cfg || cfg->L < 2 || cfg->L > LABS_MAX_L || cfg->T_r < 0 || cfg->T_r > 64 || 2 * cfg->T_r >= cfg->L ||
      cfg->H_log2 < 10 || cfg->H_log2 > 30 || cfg->max_expansions < 1 || cfg->max_expansions >= (1ll << 21) ||
      cfg->max_workspace_bytes < 0 || n < 0)
    return LABS_ERR_INVALID_ARG;
  if (n > 0 && (!seeds || !aligned8(seeds) || !best_seqs || !aligned8(best_seqs) || !best_E || !aligned4(best_E) ||
                !stats || !aligned8(stats)))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_pq_independent(ctx, cfg, seeds, n, best_seqs, best_E, stats, (cudaStream_t)stream);
}

// Hexadecimal coding of a sequence (Section 4, the results' table): the hex digits, most significant
// first, spell 4 * ceil(L/4) bits whose first 4 * ceil(L/4) - L are zero pads; the remaining bits are
// s_1 .. s_L in order, a 1 standing for +1 and a 0 for -1.  Host memory only; no device work.
int labs_seq_to_hex(const uint64_t* seq, int L, char* hex, size_t hex_size) {
  if (!seq || !hex || L < 1 || L > LABS_MAX_L) return LABS_ERR_INVALID_ARG;
  const int nd = (L + 3) / 4, pad = 4 * nd - L;
  if (hex_size < (size_t)nd + 1) return LABS_ERR_CAPACITY;
  for (int d = 0; d < nd; d++) {
    int v = 0;
    for (int b = 0; b < 4; b++) {
      const int i = 4 * d + b - pad + 1;  // position carried by this bit; i < 1 is a pad
      const int bit = i >= 1 ? (int)((seq[(i - 1) >> 6] >> ((i - 1) & 63)) & 1u) : 0;
      v = 2 * v + bit;
    }
    hex[d] = "0123456789ABCDEF"[v];
  }
  hex[nd] = '\0';
  return LABS_OK;
}

int labs_hex_to_seq(const char* hex, int L, uint64_t* seq) {
  if (!hex || !seq || L < 1 || L > LABS_MAX_L) return LABS_ERR_INVALID_ARG;
  const int nd = (L + 3) / 4, pad = 4 * nd - L;
  if (std::strlen(hex) != (size_t)nd) return LABS_ERR_INVALID_ARG;
  uint64_t w[LABS_MAX_W] = {0};
  for (int d = 0; d < nd; d++) {
    const char c = hex[d];
    int v;
    if (c >= '0' && c <= '9') v = c - '0';
    else if (c >= 'A' && c <= 'F') v = c - 'A' + 10;
    else if (c >= 'a' && c <= 'f') v = c - 'a' + 10;
    else return LABS_ERR_INVALID_ARG;
    for (int b = 0; b < 4; b++) {
      const int bit = (v >> (3 - b)) & 1;
      const int i = 4 * d + b - pad + 1;
      if (i < 1) {
        if (bit) return LABS_ERR_INVALID_ARG;  // a pad bit must be zero
        continue;
      }
      w[(i - 1) >> 6] |= (uint64_t)bit << ((i - 1) & 63);
    }
  }
  for (int t = 0; t < (L + 63) / 64; t++) seq[t] = w[t];
  return LABS_OK;
}

int labs_skew_exhaustive(labs_ctx* ctx, int L, int p, uint64_t prefix, int32_t* out_min_E, uint64_t* out_count,
                         uint64_t* out_argmin_free, uint64_t* out_argmin_seq, void* stream) {
  LABS_TRACE("labs_skew_exhaustive");
  if (!ctx || L < 3 || L > 127 || L % 2 == 0 || p < 0 || p > (L - 1) / 2) return LABS_ERR_INVALID_ARG;
  if ((L - 1) / 2 - p + 1 > 40 || p > 64) return LABS_ERR_INVALID_ARG;
  if (!out_min_E || !out_count || !out_argmin_free || !out_argmin_seq || !aligned4(out_min_E) ||
      !aligned8(out_count) || !aligned8(out_argmin_free) || !aligned8(out_argmin_seq))
    return LABS_ERR_INVALID_ARG;
  int s = set_device(ctx);
  if (s != LABS_OK) return s;
  return labsg::launch_skew_exhaustive(ctx, L, p, prefix, out_min_E, out_count, out_argmin_free, out_argmin_seq,
                                      (cudaStream_t)stream);
}

}  // extern "C"
