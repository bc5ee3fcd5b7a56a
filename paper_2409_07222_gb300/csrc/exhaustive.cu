// exhaustive.cu -- labs_skew_exhaustive: every skew-symmetric sequence (Eq. 2) of odd length L <= 127
// behind a fixed prefix (Eq. 3).  One thread per assignment of the k-p+1 free elements; the sequence
// fits two 64-bit words (one for L <= 64, a path of its own), so the table is computed directly with
// 64-bit popcounts.  Two passes over the
// assignment space (minimum, then count + smallest argmin) keep the result exact and independent of
// the order in which threads finish; the outputs themselves hold the running reductions.
#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

struct Seq128 {
  uint64_t lo, hi;
};

// The sequence of free assignment a, built with word operations: the left half (positions 1..c) is the
// prefix followed by the free elements (bit j of a set means element p+1+j is -1); the right half follows
// from Eq. 2, position c + j mirroring c - j with the sign (-1)^j: the bit-reversed left half without the
// centre, XOR an alternating mask.
__device__ __forceinline__ Seq128 assignment_seq(int L, int p, uint64_t prefix, uint64_t a) {
  const int c = (L + 1) / 2, k = c - 1, nfree = c - p;  // 1 <= k <= 63 for 3 <= L <= 127
  const uint64_t pmask = p >= 64 ? ~0ull : (1ull << p) - 1ull;
  const uint64_t fmask = nfree >= 64 ? ~0ull : (1ull << nfree) - 1ull;
  const uint64_t left = (prefix & pmask) | (p < 64 ? ((~a & fmask) << p) : 0ull);
  const uint64_t kmask = (1ull << k) - 1ull;
  const uint64_t right = (__brevll(left & kmask) >> (64 - k)) ^ (0x5555555555555555ull & kmask);
  Seq128 x;
  if (c >= 64) {
    x.lo = left;
    x.hi = right;
  } else {
    x.lo = left | (right << c);
    x.hi = right >> (64 - c);
  }
  return x;
}

// Energy of a skew-symmetric sequence of L <= 64 positions (one word): one 64-bit popcount per even lag.
__device__ __forceinline__ int energy64(uint64_t x, int L) {
  int E = 0;
  for (int k = 2; k < L; k += 2) {  // odd lags vanish for skew-symmetric sequences (Eq. 2)
    const int n = L - k;
    const int dis = __popcll((x ^ (x >> k)) & (n >= 64 ? ~0ull : ((1ull << n) - 1ull)));
    const int cval = n - 2 * dis;
    E += cval * cval;
  }
  return E;
}

// NW = 1: the sequence fits one word (L <= 64) and the high word is never touched.
template <int NW>
__device__ __forceinline__ int energy_nw(const Seq128& x, int L);
template <>
__device__ __forceinline__ int energy_nw<1>(const Seq128& x, int L) { return energy64(x.lo, L); }

__device__ __forceinline__ int energy128(const Seq128& x, int L) {
  int E = 0;
  for (int k = 2; k < L; k += 2) {  // odd lags vanish for skew-symmetric sequences (Eq. 2)
    // y = x >> k
    uint64_t ylo = k < 64 ? ((x.lo >> k) | (k ? (x.hi << (64 - k)) : 0ull)) : (x.hi >> (k - 64));
    uint64_t yhi = k < 64 ? (x.hi >> k) : 0ull;
    int n = L - k;
    uint64_t mlo = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    uint64_t mhi = n > 64 ? ((n - 64) >= 64 ? ~0ull : ((1ull << (n - 64)) - 1ull)) : 0ull;
    int dis = __popcll((x.lo ^ ylo) & mlo) + __popcll((x.hi ^ yhi) & mhi);
    int cval = n - 2 * dis;
    E += cval * cval;
  }
  return E;
}
template <>
__device__ __forceinline__ int energy_nw<2>(const Seq128& x, int L) { return energy128(x, L); }

__global__ void exh_init_kernel(int32_t* minE, uint64_t* count, uint64_t* argmin) {
  *minE = INT32_MAX;
  *count = 0;
  *argmin = ~0ull;
}

template <int NW>
__global__ void exh_min_kernel(int L, int p, uint64_t prefix, uint64_t total, int32_t* minE) {
  int best = INT32_MAX;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += (uint64_t)gridDim.x * blockDim.x)
    best = min(best, energy_nw<NW>(assignment_seq(L, p, prefix, a), L));
  best = warp_min_i32(best);
  if (lane_id() == 0) atomicMin(minE, best);
}

template <int NW>
__global__ void exh_count_kernel(int L, int p, uint64_t prefix, uint64_t total, const int32_t* minE, uint64_t* count,
                                 uint64_t* argmin) {
  const int target = *minE;
  unsigned long long cnt = 0, arg = ~0ull;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += (uint64_t)gridDim.x * blockDim.x)
    if (energy_nw<NW>(assignment_seq(L, p, prefix, a), L) == target) {
      cnt++;
      arg = min(arg, (unsigned long long)a);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(kFull, cnt, o);
    arg = min(arg, (unsigned long long)__shfl_xor_sync(kFull, arg, o));
  }
  if (lane_id() == 0) {
    if (cnt) atomicAdd(reinterpret_cast<unsigned long long*>(count), cnt);
    atomicMin(reinterpret_cast<unsigned long long*>(argmin), arg);
  }
}

__global__ void exh_seq_kernel(int L, int p, uint64_t prefix, const uint64_t* argmin, uint64_t* seq) {
  Seq128 x = assignment_seq(L, p, prefix, *argmin);
  seq[0] = x.lo;
  if (L > 64) seq[1] = x.hi;
}

}  // namespace

int launch_skew_exhaustive(labs_ctx* ctx, int L, int p, uint64_t prefix, int32_t* out_min_E, uint64_t* out_count,
                           uint64_t* out_argmin_free, uint64_t* out_argmin_seq, cudaStream_t st) {
  const int k = (L - 1) / 2;
  const int nfree = k - p + 1;
  const uint64_t total = 1ull << nfree;
  uint64_t blocks = (total + 255) / 256;
  uint64_t cap = (uint64_t)ctx->num_sms * 16;
  if (blocks > cap) blocks = cap;
  exh_init_kernel<<<1, 1, 0, st>>>(out_min_E, out_count, out_argmin_free);
  if (L <= 64) {  // one word: no popcount of an empty high word
    exh_min_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(L, p, prefix, total, out_min_E);
    exh_count_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(L, p, prefix, total, out_min_E, out_count, out_argmin_free);
  } else {
    exh_min_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(L, p, prefix, total, out_min_E);
    exh_count_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(L, p, prefix, total, out_min_E, out_count, out_argmin_free);
  }
  exh_seq_kernel<<<1, 1, 0, st>>>(L, p, prefix, out_argmin_free, out_argmin_seq);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
