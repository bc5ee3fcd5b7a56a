// operators.cu -- labs_sequence_operators: the end-element operators that move candidates to the
// neighbouring lengths (Section 3: appending or removing an element at either end gives sequences of
// length L+1 and L-1 with comparable merit factor, which re-enter step 2; the loop of Fig. 4).
//
// One warp per input sequence.  Lane w owns 32-bit word w of the sequence and of each variant: an append
// sets bit L, a prepend shifts every word up by one bit, a removal clears the last bit or shifts down by
// one.  Each variant's energy is then the Section 1 definition evaluated as in labs_energy_batch
// (energy_words.cuh: the variant held in registers, one popcount per 32 products).  Six variants per
// input: about 6 (L+-1)^2/64 popcounts.
#include "energy_words.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kOpWarps = 8;

// Writes the variant in vbits (length Lv) as packed 64-bit words.
__device__ __forceinline__ void store_words(const uint32_t* vbits, int Lv, uint64_t* dst) {
  const int lane = lane_id();
  const int W = (Lv + 63) >> 6;
  if (lane < W) dst[lane] = (uint64_t)vbits[2 * lane] | ((uint64_t)vbits[2 * lane + 1] << 32);
}

// NW: 32-bit words of the longer variants (L + 1 bits), so every variant fits with a zero word after it.
template <int NW>
__global__ void __launch_bounds__(32 * kOpWarps) operators_kernel(const uint64_t* __restrict__ seqs, int L, int64_t n,
                                                                  uint64_t* __restrict__ grow, int32_t* __restrict__ E_grow,
                                                                  uint64_t* __restrict__ shrink,
                                                                  int32_t* __restrict__ E_shrink) {
  __shared__ uint32_t sb[kOpWarps][kBitWords];
  __shared__ uint32_t vb[kOpWarps][kBitWords];
  __shared__ int pre_all[kOpWarps][kBitWords + 1];
  uint32_t* bits = sb[threadIdx.x >> 5];
  uint32_t* v = vb[threadIdx.x >> 5];
  int* pre = pre_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6, Wg = (L + 64) >> 6, Ws = (L + 62) >> 6;
  const int W32 = (L + 31) >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * kOpWarps;
  for (int64_t q = (int64_t)blockIdx.x * kOpWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    if (lane < kBitWords) {
      uint32_t x = 0;
      if (lane < W32) {
        const uint64_t w = seqs[q * W + (lane >> 1)];
        x = (lane & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
        const int rem = L - 32 * lane;
        if (rem < 32) x &= (1u << rem) - 1u;
      }
      bits[lane] = x;
    }
    __syncwarp();
    // grow: v = 0, 1 append +1 / -1 (bit L), v = 2, 3 prepend +1 / -1 (shift up, bit 0)
    for (int var = 0; var < 4; var++) {
      const uint32_t x = (var & 1) ? 0u : 1u;  // bit value of the new element (1 = +1)
      if (lane < kBitWords) {
        uint32_t w;
        if (var < 2) {
          w = bits[lane];
          if (lane == (L >> 5)) w |= x << (L & 31);
        } else {
          w = (bits[lane] << 1) | (lane ? bits[lane - 1] >> 31 : x);
        }
        v[lane] = w;
      }
      __syncwarp();
      const int E = energy_words<NW>(v, L + 1, pre, nullptr);
      if (grow) store_words(v, L + 1, grow + (q * 4 + var) * Wg);
      if (E_grow && lane == 0) E_grow[q * 4 + var] = E;
      __syncwarp();
    }
    // shrink: v = 0 drops the last element (clear bit L-1), v = 1 drops the first (shift down)
    for (int var = 0; var < 2; var++) {
      if (lane < kBitWords) {
        uint32_t w;
        if (var == 0) {
          w = bits[lane];
          if (lane == ((L - 1) >> 5)) w &= ~(1u << ((L - 1) & 31));
        } else {
          w = (bits[lane] >> 1) | (lane + 1 < kBitWords ? bits[lane + 1] << 31 : 0u);
        }
        v[lane] = w;
      }
      __syncwarp();
      const int E = energy_words<NW>(v, L - 1, pre, nullptr);
      if (shrink) store_words(v, L - 1, shrink + (q * 2 + var) * Ws);
      if (E_shrink && lane == 0) E_shrink[q * 2 + var] = E;
      __syncwarp();
    }
  }
}

}  // namespace

int launch_sequence_operators(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, uint64_t* grow, int32_t* E_grow,
                              uint64_t* shrink, int32_t* E_shrink, cudaStream_t st) {
  if (n == 0) return LABS_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + kOpWarps - 1) / kOpWarps, (int64_t)ctx->num_sms * 32);
#define LABS_OPS_CASE(NWC)                                                                                   \
  case NWC:                                                                                                \
    operators_kernel<NWC><<<blocks, 32 * kOpWarps, 0, st>>>(seqs, L, n, grow, E_grow, shrink, E_shrink); \
    break;
  switch ((L + 32) >> 5) {  // words of L + 1 bits
    LABS_OPS_CASE(1) LABS_OPS_CASE(2) LABS_OPS_CASE(3) LABS_OPS_CASE(4) LABS_OPS_CASE(5) LABS_OPS_CASE(6)
    LABS_OPS_CASE(7) LABS_OPS_CASE(8) LABS_OPS_CASE(9) LABS_OPS_CASE(10) LABS_OPS_CASE(11) LABS_OPS_CASE(12)
    LABS_OPS_CASE(13) LABS_OPS_CASE(14) LABS_OPS_CASE(15) LABS_OPS_CASE(16) LABS_OPS_CASE(17) LABS_OPS_CASE(18)
    LABS_OPS_CASE(19)
    default: return LABS_ERR_INVALID_ARG;
  }
#undef LABS_OPS_CASE
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
