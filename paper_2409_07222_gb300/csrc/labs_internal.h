// labs_internal.h -- host-side declarations shared by the translation units of liblabs.so.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "labs.h"

// An NVTX range named after a C-ABI entry point, open while the call runs on the host (its kernels show
// under it in a profiler's timeline).  NVTX v3 is header-only; without an attached tool a range costs a
// branch.
struct LabsTraceRange {
  explicit LabsTraceRange(const char* name) { nvtxRangePushA(name); }
  ~LabsTraceRange() { nvtxRangePop(); }
  LabsTraceRange(const LabsTraceRange&) = delete;
  LabsTraceRange& operator=(const LabsTraceRange&) = delete;
};
#define LABS_TRACE(name) LabsTraceRange labs_trace_range_(name)

constexpr int kMaxTuned = 16;

struct labs_ctx {
  int device;
  int num_sms;
  size_t smem_optin;
  // growable device workspace, one region per purpose
  void* ws[8];
  size_t ws_bytes[8];
  // autotuner cache: (length-set key) -> tile M, lag ranges H, lanes per walk, warps per CTA
  int n_tuned;
  uint64_t tuned_key[kMaxTuned];
  int tuned[kMaxTuned][4];
  // captured batched step (one at a time) and the stream it was captured on
  cudaGraphExec_t graph_exec;
  uint64_t graph_key;
  cudaStream_t capture_stream;
};

namespace labsg {

enum WsSlot {
  kWsThreshSamples = 0,
  kWsThreshHist = 1,
  kWsWalkCounters = 2,
  kWsBatchThresholds = 3,
  kWsPq0 = 4,
  kWsChunkState = 5,
  kWsChunkIo = 6,
  kWsPqIndep = 7
};

// Returns a device region of at least `bytes` for `slot`, growing it if needed (not capturable).
void* ws_get(labs_ctx* ctx, int slot, size_t bytes);

int policy_length(const labs_policy* P);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? LABS_OK : LABS_ERR_CUDA; }

// Shape of a walk or a sieve sample (Algorithm 1): length, mode, prefix length (Eq. 3) and the prefix
// array.  Shared by every entry point that draws walk starts, so their validation cannot drift apart.
inline int check_walk_shape(int L, int skew, int p, int n_prefix, const uint64_t* prefixes) {
  if (L < 3 || L > LABS_MAX_L || (skew != 0 && skew != 1) || p < 0 || n_prefix < 1) return LABS_ERR_INVALID_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return LABS_ERR_INVALID_ARG;
  if (!skew && p >= L) return LABS_ERR_INVALID_ARG;
  if (p > 64 * LABS_MAX_W) return LABS_ERR_INVALID_ARG;
  if (!prefixes || (reinterpret_cast<uintptr_t>(prefixes) & 7u)) return LABS_ERR_INVALID_ARG;
  return LABS_OK;
}

// Host launchers (argument validation happens in the C-ABI layer).
int launch_energy_batch(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out,
                        cudaStream_t st);
int launch_flip_deltas(labs_ctx* ctx, const uint64_t* seqs, const int32_t* C, int L, int64_t n, int skew, int p,
                       int32_t* dE_out, cudaStream_t st);
int launch_sample_threshold(labs_ctx* ctx, int L, int skew, int p, const uint64_t* prefixes, int n_prefix,
                            int prefix_words, uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr_out,
                            int32_t* E_samples, cudaStream_t st);
int launch_skew_search(labs_ctx* ctx, const labs_walk_cfg* cfg, const uint64_t* prefixes, int n_prefix,
                       labs_candidate* out, int64_t* walk_stats, labs_walk_stats* stats, cudaStream_t st);
int launch_batched_search(labs_ctx* ctx, const labs_batch_cfg* cfg, const int32_t* lengths, const int64_t* walks,
                          const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                          int32_t* E_thr_out, labs_walk_stats* stats, cudaStream_t st);
int launch_chunked_search(labs_ctx* ctx, const labs_walk_cfg* cfg, labs_policy* policy, float lambda, int chunk,
                          const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                          labs_walk_stats* stats, float* logits_log, uint64_t* state_log, int32_t* move_log,
                          cudaStream_t st);
int launch_sequence_operators(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, uint64_t* grow, int32_t* E_grow,
                              uint64_t* shrink, int32_t* E_shrink, cudaStream_t st);
int legendre_family(int L, double r_lo, double r_hi, double t_max, int32_t* out, int64_t max_out, int64_t* n_out);
int launch_legendre(labs_ctx* ctx, int L, const int32_t* params, int64_t n, uint64_t* seqs, int32_t* E_out,
                    cudaStream_t st);
int launch_pq_independent(labs_ctx* ctx, const labs_pq_indep_cfg* cfg, const uint64_t* seeds, int n,
                          uint64_t* best_seqs, int32_t* best_E, labs_pq_stats* stats, cudaStream_t st);
int launch_pq_refine(labs_ctx* ctx, const labs_pq_cfg* cfg, const uint64_t* seeds, int n_seeds, uint64_t* best_seq,
                     int32_t* best_E, labs_pq_stats* stats, cudaStream_t st);
int launch_skew_exhaustive(labs_ctx* ctx, int L, int p, uint64_t prefix, int32_t* out_min_E, uint64_t* out_count,
                           uint64_t* out_argmin_free, uint64_t* out_argmin_seq, cudaStream_t st);

}  // namespace labsg
