// legendre.cu -- Legendre-sequence seeds for step 2 (Section 4, Table 2): a Legendre sequence of prime
// length p rotated by `off` elements with its first L - p elements appended, i.e. the periodic extension
//   s_i = chi((i + off) mod p),  i = 0 .. L-1,
// chi(j) = +1 if j is a non-zero quadratic residue mod p, -1 otherwise (j = 0 included), with the exact
// energy of each.  labs_legendre_family enumerates the parameter family on the host; the device builds
// the sequences (one warp each: the non-zero squares k^2 mod p, k <= (p-1)/2, marked in a shared-memory
// bitmap, then one bitmap test per position and ballots into words) and their energies as in
// labs_energy_batch (energy_words.cuh).
#include "energy_words.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kLegWarps = 8;

// Primality of 0 .. 32 kPrimeWords - 1 as a bitmap, filled on the host and passed by value.
constexpr int kPrimeWords = 19;  // covers every p <= L <= 576
struct PrimeBits {
  uint32_t w[kPrimeWords];
};

// x mod p for 0 <= x < 2^24, 2 <= p < 2^10, through a float reciprocal: the quotient estimate is off by at
// most one either way, which the two corrections take out.
__device__ __forceinline__ int mod_small(int x, int p, float rp) {
  const int q = (int)((float)x * rp);
  int r = x - q * p;
  if (r < 0) r += p;
  if (r >= p) r -= p;
  return r;
}

// NW: 32-bit words of L bits.
template <int NW>
__global__ void __launch_bounds__(32 * kLegWarps) legendre_kernel(int L, const int32_t* __restrict__ params, int64_t n,
                                                                 uint64_t* __restrict__ seqs, int32_t* __restrict__ E_out,
                                                                 const __grid_constant__ PrimeBits primes) {
  __shared__ int pre_all[kLegWarps][kBitWords + 1];
  __shared__ uint32_t bits_all[kLegWarps][kBitWords];
  __shared__ uint32_t qr_all[kLegWarps][kBitWords];  // bit j: j is a non-zero square mod p
  uint32_t* bits = bits_all[threadIdx.x >> 5];
  uint32_t* qr = qr_all[threadIdx.x >> 5];
  int* pre = pre_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6;
  const int64_t warps_total = (int64_t)gridDim.x * kLegWarps;
  for (int64_t q = (int64_t)blockIdx.x * kLegWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    const int p = params[2 * q], off = params[2 * q + 1];
    if (p < 2 || p > L || off < 0 || off >= p || !((primes.w[p >> 5] >> (p & 31)) & 1u)) {  // not a seed: E = INT32_MAX
      if (seqs && lane < W) seqs[q * W + lane] = 0;
      if (E_out && lane == 0) E_out[q] = INT32_MAX;
      continue;
    }
    if (lane < kBitWords) qr[lane] = 0u;
    const float rp = __frcp_rn((float)p);
    __syncwarp();
    for (int k = lane + 1; 2 * k <= p - 1; k += 32) {  // the squares of 1..(p-1)/2 cover every residue
      const int r = mod_small(k * k, p, rp);
      atomicOr(&qr[r >> 5], 1u << (r & 31));
    }
    __syncwarp();
    int j = (lane + off) % p;           // (32 w + lane + off) mod p, stepped by 32 mod p
    const int step = 32 % p;
    for (int w = 0; w < kBitWords; w++) {
      const int i = 32 * w + lane;
      const int bit = (i < L && j != 0) ? (int)((qr[j >> 5] >> (j & 31)) & 1u) : 0;  // chi(0) = -1
      const unsigned word = __ballot_sync(kFull, bit);
      if (lane == 0) bits[w] = word;
      j += step;
      if (j >= p) j -= p;
    }
    __syncwarp();
    const int e = energy_words<NW>(bits, L, pre, nullptr);
    if (seqs && lane < W) seqs[q * W + lane] = (uint64_t)bits[2 * lane] | ((uint64_t)bits[2 * lane + 1] << 32);
    if (E_out && lane == 0) E_out[q] = e;
    __syncwarp();
  }
}

bool is_prime(int v) {
  if (v < 2) return false;
  for (int d = 2; d * d <= v; d++)
    if (v % d == 0) return false;
  return true;
}

}  // namespace

int legendre_family(int L, double r_lo, double r_hi, double t_max, int32_t* out, int64_t max_out, int64_t* n_out) {
  int64_t n = 0;
  for (int p = 3; p <= L; p++) {
    if (!is_prime(p)) continue;
    const int t = L - p;
    if ((double)t > t_max * (double)p) continue;
    for (int off = 0; off < p; off++) {
      const double r = (double)off / (double)L;
      if (r < r_lo || r > r_hi) continue;
      if (out && n < max_out) {
        out[2 * n] = p;
        out[2 * n + 1] = off;
      }
      n++;
    }
  }
  *n_out = n;
  return (out && n > max_out) ? LABS_ERR_CAPACITY : LABS_OK;
}

int launch_legendre(labs_ctx* ctx, int L, const int32_t* params, int64_t n, uint64_t* seqs, int32_t* E_out,
                    cudaStream_t st) {
  if (n == 0) return LABS_OK;
  const int64_t blocks = std::min<int64_t>((n + kLegWarps - 1) / kLegWarps, (int64_t)ctx->num_sms * 32);
  const unsigned nb = (unsigned)blocks;
  PrimeBits pb{};
  for (int v = 0; v < 32 * kPrimeWords; v++)
    if (is_prime(v)) pb.w[v >> 5] |= 1u << (v & 31);
#define LABS_LEG_CASE(NWC)                                                             \
  case NWC:                                                                          \
    legendre_kernel<NWC><<<nb, 32 * kLegWarps, 0, st>>>(L, params, n, seqs, E_out, pb); \
    break;
  switch ((L + 31) >> 5) {
    LABS_LEG_CASE(1) LABS_LEG_CASE(2) LABS_LEG_CASE(3) LABS_LEG_CASE(4) LABS_LEG_CASE(5) LABS_LEG_CASE(6)
    LABS_LEG_CASE(7) LABS_LEG_CASE(8) LABS_LEG_CASE(9) LABS_LEG_CASE(10) LABS_LEG_CASE(11) LABS_LEG_CASE(12)
    LABS_LEG_CASE(13) LABS_LEG_CASE(14) LABS_LEG_CASE(15) LABS_LEG_CASE(16) LABS_LEG_CASE(17) LABS_LEG_CASE(18)
    default: return LABS_ERR_INVALID_ARG;
  }
#undef LABS_LEG_CASE
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
