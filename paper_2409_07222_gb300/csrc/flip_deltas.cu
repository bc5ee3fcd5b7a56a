// flip_deltas.cu -- labs_flip_deltas: exact Delta E of every single-flip neighbour (BEST_NEIGHBOUR of
// Algorithm 1, the neighbourhood loop of Algorithm 2), stand-alone.
//
// One warp per sequence.  The warp stages the sequence, builds (or loads) its correlation table,
// lays out the byte windows and runs the same tiled dp4a scan as the walk kernel; every lane owns a
// tile of M neighbours per pass.  Work per sequence: (#neighbours) x (#lags) multiply-adds.
#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kFdWarps = 4;
constexpr int kFdM = 8;

template <int M>
__global__ void __launch_bounds__(32 * kFdWarps) flip_deltas_kernel(const uint64_t* __restrict__ seqs,
                                                                     const int32_t* __restrict__ Cin, int L, int64_t n,
                                                                     int skew, int p, int32_t* __restrict__ dE) {
  __shared__ ScanSmem slabs[kFdWarps];
  __shared__ int16_t P_all[kFdWarps][kMaxL];
  __shared__ uint32_t xb_all[kFdWarps][kBitWords], rb_all[kFdWarps][kBitWords];
  ScanSmem& sm = slabs[threadIdx.x >> 5];
  int16_t* Pm = P_all[threadIdx.x >> 5];
  const int lane = lane_id();
  Layout ly;
  make_layout(ly, L, skew, p, M);  // validated by the host launcher
  const int W = (L + 63) >> 6;
  const int64_t warps_total = (int64_t)gridDim.x * kFdWarps;
  for (int64_t q = (int64_t)blockIdx.x * kFdWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    load_bits(sm, seqs + q * W, L);
    if (Cin) {
      for (int h = lane; h < kCLen; h += 32) {
        int g = h + 1;
        sm.C16[h] = (int16_t)((g <= ly.G) ? Cin[q * (L - 1) + (ly.lam * g - 1)] : 0);
      }
      __syncwarp();
    } else {
      build_table(sm, ly);
    }
    const bool fast = pack_c8(sm, ly);
    const int SC = table_sum(sm, ly);
    build_bytes(sm, ly);
    p_all(sm, ly, xb_all[threadIdx.x >> 5], rb_all[threadIdx.x >> 5], Pm, p + 1, ly.mlast);  // the neighbours only
    int32_t* out = dE + q * L;
    for (int i = lane; i < L; i += 32) out[i] = INT32_MAX;
    __syncwarp();
    for (int base = 0; base < ly.n_tiles; base += 32) {
      const int tau = base + lane;
      int cls = 0, q0 = 0;
      const bool has = tau < ly.n_tiles;
      if (has) tile_of(ly, tau, cls, q0);
      int acc[M];
      if (has) {
        if (fast)
          scan_tile<M, false>(sm, ly, cls, q0, acc);
        else
          scan_tile<M, true>(sm, ly, cls, q0, acc);
#pragma unroll
        for (int j = 0; j < M; j++) {
          SlotInfo si = slot_info(ly, cls, q0 + j);
          if (!si.active) continue;
          out[si.m - 1] = finish_delta(sm, ly, cls, q0 + j, si, acc[j], SC, Pm[si.m - 1]);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace

int launch_flip_deltas(labs_ctx* ctx, const uint64_t* seqs, const int32_t* C, int L, int64_t n, int skew, int p,
                       int32_t* dE_out, cudaStream_t st) {
  if (n == 0) return LABS_OK;
  Layout ly;
  if (!make_layout(ly, L, skew, p, kFdM)) return LABS_ERR_INVALID_ARG;
  int64_t blocks = (n + kFdWarps - 1) / kFdWarps;
  int64_t cap = (int64_t)ctx->num_sms * 32;
  if (blocks > cap) blocks = cap;
  flip_deltas_kernel<kFdM><<<(unsigned)blocks, 32 * kFdWarps, 0, st>>>(seqs, C, L, n, skew, p, dE_out);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
