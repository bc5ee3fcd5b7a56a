// legendre.cu -- Legendre-sequence seeds for step 2 (Section 4, Table 2): a Legendre sequence of prime
// length p rotated by `off` elements with its first L - p elements appended, i.e. the periodic extension
//   s_i = chi((i + off) mod p),  i = 0 .. L-1,
// chi(j) = +1 if j is a non-zero quadratic residue mod p, -1 otherwise (j = 0 included), with the exact
// energy of each.  labs_legendre_family enumerates the parameter family on the host; the device builds
// the sequences (one warp each: the non-zero squares k^2 mod p, k <= (p-1)/2, marked in a shared-memory
// bitmap, then one bitmap test per position and ballots into words) and their energies like
// labs_energy_batch.
#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kLegWarps = 8;

__device__ __forceinline__ bool prime_dev(int v) {
  if (v < 2) return false;
  for (int d = 2; d * d <= v; d++)
    if (v % d == 0) return false;
  return true;
}


__global__ void __launch_bounds__(32 * kLegWarps) legendre_kernel(int L, const int32_t* __restrict__ params, int64_t n,
                                                                 uint64_t* __restrict__ seqs, int32_t* __restrict__ E_out) {
  __shared__ uint32_t bits_all[kLegWarps][kBitWords];
  __shared__ uint32_t qr_all[kLegWarps][kBitWords];  // bit j: j is a non-zero square mod p
  uint32_t* bits = bits_all[threadIdx.x >> 5];
  uint32_t* qr = qr_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6;
  const int64_t warps_total = (int64_t)gridDim.x * kLegWarps;
  for (int64_t q = (int64_t)blockIdx.x * kLegWarps + (threadIdx.x >> 5); q < n; q += warps_total) {
    const int p = params[2 * q], off = params[2 * q + 1];
    if (p < 2 || p > L || off < 0 || off >= p || !prime_dev(p)) {  // not a seed of this length: E = INT32_MAX
      if (seqs && lane < W) seqs[q * W + lane] = 0;
      if (E_out && lane == 0) E_out[q] = INT32_MAX;
      continue;
    }
    if (lane < kBitWords) qr[lane] = 0u;
    __syncwarp();
    for (int k = lane + 1; 2 * k <= p - 1; k += 32) {  // the squares of 1..(p-1)/2 cover every residue
      const int r = (k * k) % p;
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
    int e = 0;
    for (int k = lane + 1; k < L; k += 32) {
      const int c = corr_lag(bits, L, k);
      e += c * c;
    }
    e = warp_sum_i32(e);
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
  legendre_kernel<<<(unsigned)blocks, 32 * kLegWarps, 0, st>>>(L, params, n, seqs, E_out);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
