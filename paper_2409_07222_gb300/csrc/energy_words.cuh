// energy_words.cuh -- E = sum_k C_k^2 (Section 1) of one bit-packed sequence by one warp, the sequence
// held in registers.
//
// Lane l takes the lags k = 32 j + l (j = 0 .. NW - 1): for a given j every lane's word offset is j and its
// bit shift is l, so with NW a compile-time constant the loops over j and the words unroll, and each 32
// products cost one funnel shift, one XOR, one popcount and one add.  C_k = (L - k) - 2 d, d counting the
// disagreeing pairs (s_i != s_{i+k}, i < L - k): the popcounts run over whole words, and the positions
// past L - k (where the shifted word is zero) are taken out with prefix popcounts of the words.
#pragma once

#include "labs_core.cuh"

namespace labsg {

// sb: the sequence's NW 32-bit words in shared memory followed by one zero word (sb[NW] = 0), bits at and
// above L zero, L <= 32 NW; pre: per-warp scratch of NW + 1 ints.  Returns E on every lane; C_out, when not
// null, receives C_k at C_out[k - 1] for k = 1 .. L-1.
template <int NW>
__device__ __forceinline__ int energy_words(const uint32_t* sb, int L, int* pre, int32_t* C_out) {
  const int lane = lane_id();
  int c1 = __popc(lane < NW ? sb[lane] : 0u);  // inclusive prefix of the words' popcounts
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, c1, o);
    if (lane >= o) c1 += t;
  }
  __syncwarp();  // an earlier call's readers of pre are done
  if (lane < NW) pre[lane + 1] = c1;
  if (lane == 0) pre[0] = 0;
  __syncwarp();
  uint32_t b[NW + 1];
#pragma unroll
  for (int w = 0; w <= NW; w++) b[w] = sb[w];
  int e = 0;
#pragma unroll
  for (int j = 0; j < NW; j++) {
    const int k = 32 * j + lane;
    int d = 0;
#pragma unroll
    for (int w = 0; w + j < NW; w++) d += __popc(b[w] ^ __funnelshift_r(b[w + j], b[w + j + 1], lane));
    if (k >= 1 && k < L) {
      // the words cover positions [0, 32 (NW - j)); past t = L - k the shifted word is zero, so the
      // popcount also counted the ones of s there
      const int t = L - k;
      const int pt = pre[t >> 5] + __popc(sb[t >> 5] & ((1u << (t & 31)) - 1u));
      d -= pre[NW - j] - pt;
      const int c = t - 2 * d;
      if (C_out) C_out[k - 1] = c;
      e += c * c;
    }
  }
  return warp_sum_i32(e);
}

}  // namespace labsg
