// energy.cu -- labs_energy_batch: C_k and E = sum C_k^2 for a batch of bit-packed sequences
// (Section 1 definitions; ENERGY in Algorithms 1 and 2).
//
// One warp per sequence, the sequence's W32 32-bit words held in registers by every lane
// (energy_words.cuh: one funnel shift, XOR, popcount and add per 32 products).  8 B per word in,
// 4 B out (plus the C_k when asked for).
#include "energy_words.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kEnergyWarps = 8;

template <int W32>
__global__ void __launch_bounds__(32 * kEnergyWarps) energy_batch_kernel(const uint64_t* __restrict__ seqs, int L,
                                                                          int64_t n, int32_t* __restrict__ E_out,
                                                                          int32_t* __restrict__ C_out) {
  __shared__ uint32_t bits_all[kEnergyWarps][W32 + 1];
  __shared__ int pre_all[kEnergyWarps][W32 + 1];
  uint32_t* sb = bits_all[threadIdx.x >> 5];
  int* pre = pre_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6;
  const int64_t warps_total = (int64_t)gridDim.x * kEnergyWarps;
  for (int64_t q = (int64_t)blockIdx.x * kEnergyWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    const uint64_t* src = seqs + q * W;
    __syncwarp();  // the previous sequence's readers of sb are done
    if (lane <= W32) {
      uint32_t v = 0;
      if (lane < W32) {
        const uint64_t x = src[lane >> 1];
        v = (lane & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
        const int rem = L - 32 * lane;
        if (rem < 32) v &= (1u << rem) - 1u;
      }
      sb[lane] = v;
    }
    __syncwarp();
    const int e = energy_words<W32>(sb, L, pre, C_out ? C_out + q * (L - 1) : nullptr);
    if (lane == 0) E_out[q] = e;
  }
}

template <int W32>
void launch_energy_w(const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out, unsigned blocks,
                     cudaStream_t st) {
  energy_batch_kernel<W32><<<blocks, 32 * kEnergyWarps, 0, st>>>(seqs, L, n, E_out, C_out);
}

}  // namespace

int launch_energy_batch(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out,
                        cudaStream_t st) {
  if (n == 0) return LABS_OK;
  int64_t blocks = (n + kEnergyWarps - 1) / kEnergyWarps;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (blocks > cap) blocks = cap;
  const unsigned nb = (unsigned)blocks;
  switch ((L + 31) >> 5) {
    case 1: launch_energy_w<1>(seqs, L, n, E_out, C_out, nb, st); break;
    case 2: launch_energy_w<2>(seqs, L, n, E_out, C_out, nb, st); break;
    case 3: launch_energy_w<3>(seqs, L, n, E_out, C_out, nb, st); break;
    case 4: launch_energy_w<4>(seqs, L, n, E_out, C_out, nb, st); break;
    case 5: launch_energy_w<5>(seqs, L, n, E_out, C_out, nb, st); break;
    case 6: launch_energy_w<6>(seqs, L, n, E_out, C_out, nb, st); break;
    case 7: launch_energy_w<7>(seqs, L, n, E_out, C_out, nb, st); break;
    case 8: launch_energy_w<8>(seqs, L, n, E_out, C_out, nb, st); break;
    case 9: launch_energy_w<9>(seqs, L, n, E_out, C_out, nb, st); break;
    case 10: launch_energy_w<10>(seqs, L, n, E_out, C_out, nb, st); break;
    case 11: launch_energy_w<11>(seqs, L, n, E_out, C_out, nb, st); break;
    case 12: launch_energy_w<12>(seqs, L, n, E_out, C_out, nb, st); break;
    case 13: launch_energy_w<13>(seqs, L, n, E_out, C_out, nb, st); break;
    case 14: launch_energy_w<14>(seqs, L, n, E_out, C_out, nb, st); break;
    case 15: launch_energy_w<15>(seqs, L, n, E_out, C_out, nb, st); break;
    case 16: launch_energy_w<16>(seqs, L, n, E_out, C_out, nb, st); break;
    case 17: launch_energy_w<17>(seqs, L, n, E_out, C_out, nb, st); break;
    case 18: launch_energy_w<18>(seqs, L, n, E_out, C_out, nb, st); break;
    default: return LABS_ERR_INVALID_ARG;
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
