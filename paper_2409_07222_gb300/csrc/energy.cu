// energy.cu -- labs_energy_batch: C_k and E = sum C_k^2 for a batch of bit-packed sequences
// (Section 1 definitions; ENERGY in Algorithms 1 and 2).
//
// One warp per sequence: the 64-bit words are staged in shared memory as 32-bit words, lanes split
// the lags, and each lag is a popcount of x XOR (x >> k) over ceil((L-k)/32) words.  The arithmetic
// is integer popcount work (about (L-1) * L / 64 popc per sequence); 8 B per word in, 4 B out.
#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kEnergyWarps = 8;

__global__ void __launch_bounds__(32 * kEnergyWarps) energy_batch_kernel(const uint64_t* __restrict__ seqs, int L,
                                                                          int64_t n, int32_t* __restrict__ E_out,
                                                                          int32_t* __restrict__ C_out) {
  __shared__ uint32_t bits_all[kEnergyWarps][kBitWords];
  uint32_t* bits = bits_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6;
  const int W32 = (L + 31) >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * kEnergyWarps;
  for (int64_t q = (int64_t)blockIdx.x * kEnergyWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    const uint64_t* src = seqs + q * W;
    if (lane < kBitWords) {
      uint32_t v = 0;
      if (lane < W32) {
        uint64_t x = src[lane >> 1];
        v = (lane & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
        int rem = L - 32 * lane;
        if (rem < 32) v &= (1u << rem) - 1u;
      }
      bits[lane] = v;
    }
    __syncwarp();
    int e = 0;
    for (int k = lane + 1; k < L; k += 32) {
      int c = corr_lag(bits, L, k);
      if (C_out) C_out[q * (L - 1) + (k - 1)] = c;
      e += c * c;
    }
    e = warp_sum_i32(e);
    if (lane == 0) E_out[q] = e;
    __syncwarp();
  }
}

}  // namespace

int launch_energy_batch(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out,
                        cudaStream_t st) {
  if (n == 0) return LABS_OK;
  int64_t blocks = (n + kEnergyWarps - 1) / kEnergyWarps;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (blocks > cap) blocks = cap;
  energy_batch_kernel<<<(unsigned)blocks, 32 * kEnergyWarps, 0, st>>>(seqs, L, n, E_out, C_out);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
