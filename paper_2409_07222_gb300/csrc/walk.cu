// walk.cu -- step 1 of the dual-step search: Algorithm 1's self-avoiding walks (labs_skew_search)
// and the sieve bound E_l (labs_sample_threshold).
//
// GB300 mapping.  The paper runs one walk per thread block with a shared-memory reduction (Fig. 3);
// here one walk is one warp (shuffle/redux reductions, no block barriers) and a persistent grid pulls
// walk ids from a device counter, so long and short walks balance across the 152 SMs.  Each warp's
// state (sequence bits, byte windows, correlation table, Bloom filter of 2^bloom_log2 bits) lives in
// its shared-memory slab; a step is
//   scan   -- Delta E of every free neighbour (tiled dp4a loop, labs_core.cuh),
//   select -- warp argmin of (Delta E, m); Bloom test of the winner's fingerprint; on a hit the owner
//             lane excludes that neighbour and the argmin repeats (same result as testing them all),
//   apply  -- O(L) table update, byte/bit flips, fingerprint, Bloom insert,
//   sieve  -- the walk's R best distinct (E, fp) states with E <= E_thr, one per lane.
#include <algorithm>
#include <mutex>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

struct WalkSmem {
  ScanSmem s;
  uint32_t bloom[1024];  // up to 2^15 bits
};

struct WalkParams {
  Layout ly;  // computed on the host; read from the kernel's parameter space
  int L, skew, p, T_i, R, bloom_log2, bloom_k, prefix_words, n_prefix, M;
  int64_t n_walks, walk_begin, flip_budget;
  uint64_t seed;
  const uint64_t* prefixes;
  const int32_t* E_thr_ptr;  // nullable: use E_thr_value
  int32_t E_thr_value;
  int32_t E_target;
  labs_candidate* out;
  int64_t* walk_stats;
  labs_walk_stats* stats;
  unsigned long long* counter;
};

__device__ __forceinline__ uint32_t bloom_idx(uint64_t fp, int j, uint32_t mask) {
  uint32_t lo = (uint32_t)fp, hi = (uint32_t)(fp >> 32);
  return (lo + (uint32_t)j * (hi | 1u)) & mask;
}

// Every lane returns whether all K probes of fp are set.
__device__ __forceinline__ bool bloom_test(const uint32_t* bloom, uint64_t fp, int K, uint32_t mask) {
  const int lane = lane_id();
  bool hit = true;
  if (lane < K) {
    uint32_t b = bloom_idx(fp, lane, mask);
    hit = (bloom[b >> 5] >> (b & 31)) & 1u;
  }
  return __all_sync(kFull, hit);
}

__device__ __forceinline__ void bloom_add(uint32_t* bloom, uint64_t fp, int K, uint32_t mask) {
  const int lane = lane_id();
  if (lane < K) {
    uint32_t b = bloom_idx(fp, lane, mask);
    atomicOr(&bloom[b >> 5], 1u << (b & 31));
  }
  __syncwarp();
}

__device__ __forceinline__ bool key_less(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}

// Per-slot constants derived from the position m: alpha, the excluded lag gd, the sign relation
// s_{m'} = sigma s_m (Eq. 2) and K0 = alpha^2 (n_f + n_b - pair).
struct SlotConst {
  int alpha, gd, sigma, K0, gmax;
};

// Closed forms: skew walks (L = 2c - 1, m <= c): n_f + n_b = G - 1 + (m & 1), n_b <= n_f, the excluded
// lag of the pair (m, m') is g = c - m and s_{m'} = (-1)^{c-m} s_m (Eq. 2).  Unrestricted walks:
// n_f + n_b = L - 1.
__device__ __forceinline__ SlotConst slot_const(const Layout& ly, int m) {
  SlotConst k;
  if (ly.skew) {
    const int pair = m != ly.c;
    k.alpha = pair ? 4 : 2;
    k.gd = ly.c - m;
    k.sigma = (k.gd & 1) ? -1 : 1;
    k.K0 = k.alpha * k.alpha * (ly.G - 1 + (m & 1) - pair);
    k.gmax = (m - 1) >> 1;
  } else {
    k.alpha = 2;
    k.gd = 0;
    k.sigma = 1;
    k.K0 = 4 * (ly.L - 1);
    k.gmax = min(ly.L - m, m - 1);
  }
  return k;
}

// P bookkeeping of one slot (class index q) when position f (class cf, class index qf, pre-flip value
// sf) flips: the product s_{m - lambda g} s_{m + lambda g} with g = |q - qf| loses its sign unless g is
// outside 1..gmax, is the excluded pair lag, or the product's other end flips too (the skew centre
// when a pair flips).  The other end has class index 2q - qf.
__device__ __forceinline__ int p_step(const ScanSmem& sm, int cls, int q, const SlotConst& k, int P, int cf, int qf,
                                      int sf) {
  const int d = q - qf;
  const int g = d < 0 ? -d : d;
  if (cls == cf && (unsigned)(g - 1) < (unsigned)k.gmax && g != k.gd) {
    const uint8_t* F = reinterpret_cast<const uint8_t*>(sm.fwd + cls_words(cls));
    P -= 2 * sf * ((int)F[q + d] - 1);
  }
  return P;
}

template <int M, int H, int NP>
__global__ void __launch_bounds__(256, 2) walk_kernel(WalkParams P) {
  constexpr int MH = M / H;   // slots owned by a lane per pass
  constexpr int S = NP * MH;  // slots owned by a lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  WalkSmem& ws = reinterpret_cast<WalkSmem*>(smem_raw)[wid];
  uint64_t* ztab = reinterpret_cast<uint64_t*>(smem_raw + sizeof(WalkSmem) * nwarps);
  ScanSmem& sm = ws.s;
  const int lane = lane_id();
  const Layout& ly = P.ly;
  const uint64_t zkey = stream_key(0, kPurposeZobrist, (uint64_t)P.L, 0);
  const int32_t E_thr = P.E_thr_ptr ? *P.E_thr_ptr : P.E_thr_value;
  const uint32_t bmask = (1u << P.bloom_log2) - 1u;
  const int bwords = 1 << (P.bloom_log2 - 5);
  const int W = (P.L + 63) >> 6;
  const int R = P.R;
  // Zobrist keys of this length, shared by the block (index i-1 for position i)
  for (int i = threadIdx.x; i < P.L; i += blockDim.x) ztab[i] = zobrist(zkey, i + 1);
  __syncthreads();

  // this lane's task per pass: tile (class, q0) and lag range h; its slots are tile positions
  // h*MH .. h*MH+MH-1 (after the partial sums of the H lanes of a tile are combined)
  int tcls[NP], tq0[NP], th[NP];
  bool thas[NP];
  int slot_m[S];  // position of each owned slot, 0 if none
#pragma unroll
  for (int ps = 0; ps < NP; ps++) {
    const int task = ps * 32 + lane;
    thas[ps] = task < ly.n_tasks;
    th[ps] = H == 2 ? (task & 1) : 0;
    tcls[ps] = 0;
    tq0[ps] = 0;
    const int tile = H == 2 ? (task >> 1) : task;
    if (tile < ly.n_tiles) tile_of(ly, tile, tcls[ps], tq0[ps]);
#pragma unroll
    for (int k = 0; k < MH; k++) {
      const int m = q_pos(ly, tcls[ps], tq0[ps] + th[ps] * MH + k);
      slot_m[ps * MH + k] = (thas[ps] && m >= ly.p + 1 && m <= ly.mlast) ? m : 0;
    }
  }

  long long agg_flips = 0, agg_segs = 0, agg_skips = 0, agg_dead = 0;
  int agg_best = INT32_MAX;

  while (true) {
    unsigned long long wrel = 0;
    if (lane == 0) wrel = atomicAdd(P.counter, 1ull);
    wrel = __shfl_sync(kFull, wrel, 0);
    if ((long long)wrel >= P.n_walks) break;
    const int64_t w = P.walk_begin + (int64_t)wrel;
    const uint64_t* prefix = P.prefixes + (w % P.n_prefix) * P.prefix_words;
    labs_candidate* rec = P.out + (int64_t)wrel * R;

    // empty sieve slots
    for (int r = lane; r < R; r += 32) {
      rec[r].E = INT32_MAX;
      rec[r].walk = 0;
      rec[r].step = 0;
      rec[r].pad = 0;
      rec[r].fp = ~0ull;
#pragma unroll
      for (int t = 0; t < LABS_MAX_W; t++) rec[r].seq[t] = 0;
    }
    int cE = INT32_MAX;
    uint64_t cfp = ~0ull;
    int wE = INT32_MAX;
    uint64_t wfp = ~0ull;
    int wlane = 0;

    // flip_budget < 2^32 is checked by the host, so the per-walk counters fit 32 bits (skips: 64)
    unsigned flips = 0, segs = 0, dead = 0;
    long long skips = 0;
    int first_hit = -1;
    int bestE = INT32_MAX;
    int slot_P[S], slot_ms[S];  // P_m and s_m * m

    const unsigned budget = (unsigned)P.flip_budget;
    while (flips < budget) {
      for (int t = lane; t < bwords; t += 32) ws.bloom[t] = 0u;
      build_start(sm, ly, prefix, stream_key(P.seed, kPurposeWalk, (uint64_t)w, (uint64_t)segs));
      segs++;
      uint64_t fp = fingerprint(sm, P.L, zkey);
      bloom_add(ws.bloom, fp, P.bloom_k, bmask);
      int E = build_table(sm, ly);
      int SC = table_sum(sm);
      bool fast = pack_c8(sm);
      build_bytes(sm, ly);
#pragma unroll
      for (int t = 0; t < S; t++) {
        slot_P[t] = 0;
        const int m = slot_m[t];
        slot_ms[t] = m;
        if (m) {
          SlotInfo si = slot_info(ly, pos_cls(ly, m), pos_q(ly, m));
          slot_P[t] = p_from_scratch(sm, ly, pos_cls(ly, m), pos_q(ly, m), si);
          slot_ms[t] = s_at(sm, ly, m) * m;
        }
      }

      int it = 0;
      int mprev = 0;  // free position flipped by the previous move of this segment
      while (it < P.T_i && flips < budget) {
        it++;
        // ---- scan; each lane keeps its best (Delta E, m)
        int bd = INT32_MAX, bm = INT32_MAX;
        int dprev = INT32_MAX;  // this lane's Delta E of the move back (only its owner sets it)
        int slot_d[S];
#pragma unroll
        for (int ps = 0; ps < NP; ps++) {
          int acc[M];
#pragma unroll
          for (int j = 0; j < M; j++) acc[j] = 0;
          if (thas[ps]) {
            const int u_begin = th[ps] ? ly.NGh : 0;
            const int u_end = th[ps] ? ly.NGend : ly.NGh;
            if (fast)
              scan_range<M, false>(sm, ly, tcls[ps], tq0[ps], u_begin, u_end, acc);
            else
              scan_range<M, true>(sm, ly, tcls[ps], tq0[ps], u_begin, u_end, acc);
          }
          if (H == 2) {
#pragma unroll
            for (int j = 0; j < M; j++) acc[j] += __shfl_xor_sync(kFull, acc[j], 1);
          }
#pragma unroll
          for (int k = 0; k < MH; k++) {
            const int t = ps * MH + k;
            const int ms = slot_ms[t];
            const int m = ms < 0 ? -ms : ms;
            const int a = (H == 2 && th[ps]) ? acc[MH + k] : acc[k];
            int d = INT32_MAX;
            if (m) {
              const SlotConst kc = slot_const(ly, m);
              const int s_m = ms < 0 ? -1 : 1;
              d = -2 * kc.alpha * s_m * (a - 2 * SC) + kc.K0 + 2 * kc.alpha * kc.alpha * slot_P[t];
              if (kc.alpha == 4) d += 8 * kc.sigma * (int)sm.C16[kc.gd - 1];
              if (m == mprev) {
                dprev = d;  // the state just left: certainly in the Bloom filter
                d = INT32_MAX;
              } else if (d < bd || (d == bd && m < bm)) {
                bd = d;
                bm = m;
              }
            }
            slot_d[t] = d;
          }
        }
        // ---- select: smallest (Delta E, m) whose neighbour is not in the Bloom filter
        int mstar = -1, dstar = 0;
        uint64_t nfp = 0;
        for (int guard = 0; guard <= S * 32; guard++) {
          int dmin = warp_min_i32(bd);
          if (dmin == INT32_MAX) break;
          int mm = (int)warp_min_u32(bd == dmin ? (unsigned)bm : 0xffffffffu);
          uint64_t cand = fp ^ ztab[mm - 1];
          if (ly.skew && mm != ly.c) cand ^= ztab[ly.L - mm];
          if (!bloom_test(ws.bloom, cand, P.bloom_k, bmask)) {
            mstar = mm;
            dstar = dmin;
            nfp = cand;
            break;
          }
          skips++;
          if (bd == dmin && bm == mm) {
            // the owner lane's next best: smallest key ranked after (dmin, mm); keys ranked ahead were
            // excluded earlier in this step
            bd = INT32_MAX;
            int nbm = INT32_MAX;
#pragma unroll
            for (int t = 0; t < S; t++) {
              const int d = slot_d[t], m = slot_ms[t] < 0 ? -slot_ms[t] : slot_ms[t];
              if (d == INT32_MAX) continue;
              if (d < dmin || (d == dmin && m <= mm)) continue;
              if (d < bd || (d == bd && m < nbm)) {
                bd = d;
                nbm = m;
              }
            }
            bm = nbm;
          }
        }
        // the move back ranked ahead of the chosen move: count it as a Bloom skip
        if (__any_sync(kFull, dprev != INT32_MAX && (mstar < 0 || dprev < dstar || (dprev == dstar && mprev < mstar))))
          skips++;
        if (mstar < 0) {
          dead++;
          break;
        }
        // ---- apply
        const int f1 = (ly.skew && mstar != ly.c) ? ly.L + 1 - mstar : 0;
        const int c0 = pos_cls(ly, mstar), q0f = pos_q(ly, mstar);
        const int s0 = s_at(sm, ly, mstar);
        const int q1f = f1 ? pos_q(ly, f1) : 0;  // the mirror has the class of m*
        const int s1 = f1 ? s_at(sm, ly, f1) : 0;
#pragma unroll
        for (int t = 0; t < S; t++) {
          const int m = slot_ms[t] < 0 ? -slot_ms[t] : slot_ms[t];
          if (m) {
            const SlotConst kc = slot_const(ly, m);
            const int cls = pos_cls(ly, m), q = pos_q(ly, m);
            if (!(f1 && m == ly.c)) {  // the centre's products (c - g, c + g) flip at both ends
              slot_P[t] = p_step(sm, cls, q, kc, slot_P[t], c0, q0f, s0);
              if (f1) slot_P[t] = p_step(sm, cls, q, kc, slot_P[t], c0, q1f, s1);
            }
            if (m == mstar) slot_ms[t] = -slot_ms[t];
          }
        }
        mprev = mstar;
        SC += table_update(sm, ly, mstar, &fast);
        if (lane == 0) flip_position(sm, ly, mstar);
        if (lane == 1 && f1) flip_position(sm, ly, f1);
        __syncwarp();
        E += dstar;
        fp = nfp;
        bloom_add(ws.bloom, fp, P.bloom_k, bmask);
        flips++;
        if (E < bestE) bestE = E;
        if (first_hit < 0 && E <= P.E_target) first_hit = (int)flips;
        // ---- sieve
        if (E <= E_thr && key_less(E, fp, wE, wfp)) {
          bool dup = __any_sync(kFull, lane < R && cE != INT32_MAX && cfp == fp);
          if (!dup) {
            if (lane == wlane) {
              cE = E;
              cfp = fp;
            }
            labs_candidate* rr = rec + wlane;
            if (lane == 0) {
              rr->E = E;
              rr->walk = (uint32_t)w;
              rr->step = (uint32_t)flips;
              rr->fp = fp;
            }
            if (lane < W) rr->seq[lane] = (uint64_t)sm.bits[2 * lane] | ((uint64_t)sm.bits[2 * lane + 1] << 32);
            // new worst slot: largest (E, fp), lowest lane among equals
            int mE = warp_max_i32(lane < R ? cE : INT32_MIN);
            uint64_t mf = (lane < R && cE == mE) ? cfp : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              uint64_t other = __shfl_xor_sync(kFull, mf, o);
              mf = other > mf ? other : mf;
            }
            unsigned who = __ballot_sync(kFull, lane < R && cE == mE && cfp == mf);
            wE = mE;
            wfp = mf;
            wlane = __ffs(who) - 1;
          }
        }
      }
    }

    // ---- final: sort the R slots by (E, fp) (ties between empty slots by lane) and rewrite in place
    int rank = 0;
    for (int r = 0; r < R; r++) {
      int oE = __shfl_sync(kFull, cE, r);
      uint64_t of = __shfl_sync(kFull, cfp, r);
      if (key_less(oE, of, cE, cfp) || (oE == cE && of == cfp && r < lane)) rank++;
    }
    __syncwarp();
    labs_candidate mine;
    if (lane < R) mine = rec[lane];
    __syncwarp();
    if (lane < R) rec[rank] = mine;
    __syncwarp();
    if (P.walk_stats && lane == 0) {
      int64_t* st = P.walk_stats + (int64_t)wrel * 6;
      st[0] = (int64_t)flips;
      st[1] = (int64_t)segs;
      st[2] = skips;
      st[3] = (int64_t)dead;
      st[4] = bestE;
      st[5] = first_hit;
    }
    agg_flips += flips;
    agg_segs += segs;
    agg_skips += skips;
    agg_dead += dead;
    agg_best = min(agg_best, bestE);
  }
  if (lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->flips), (unsigned long long)agg_flips);
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->segments), (unsigned long long)agg_segs);
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->bloom_skips), (unsigned long long)agg_skips);
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->dead_ends), (unsigned long long)agg_dead);
    atomicMin(&P.stats->best_E, agg_best);
  }
}

__global__ void walk_init_kernel(labs_walk_stats* stats, const int32_t* E_thr_ptr, int32_t E_thr_value,
                                 unsigned long long* counter) {
  stats->flips = 0;
  stats->segments = 0;
  stats->bloom_skips = 0;
  stats->dead_ends = 0;
  stats->E_thr = E_thr_ptr ? *E_thr_ptr : E_thr_value;
  stats->best_E = INT32_MAX;
  stats->status = LABS_OK;
  stats->reserved = 0;
  *counter = 0ull;
}

// ---------------------------------------------------------------------------------------------
// Sieve bound: sample energies, then an exact two-level radix select (13 + 13 bits; E < 2^26).
// ---------------------------------------------------------------------------------------------
constexpr int kSampleWarps = 8;
constexpr int kHistBins = 8192;

__global__ void __launch_bounds__(32 * kSampleWarps) sample_kernel(int L, int skew, int p,
                                                                    const uint64_t* __restrict__ prefixes, int n_prefix,
                                                                    int prefix_words, uint64_t seed, int64_t n,
                                                                    int32_t* __restrict__ E_out,
                                                                    unsigned* __restrict__ hist) {
  __shared__ ScanSmem slabs[kSampleWarps];
  ScanSmem& sm = slabs[threadIdx.x >> 5];
  Layout ly;
  make_layout(ly, L, skew, p, 8);
  const int64_t warps_total = (int64_t)gridDim.x * kSampleWarps;
  for (int64_t i = (int64_t)blockIdx.x * kSampleWarps + (threadIdx.x >> 5); i < n; i += warps_total) {
    build_start(sm, ly, prefixes + (i % n_prefix) * prefix_words, stream_key(seed, kPurposeThresh, (uint64_t)i, 0));
    int E;
    if (skew) {
      E = build_table(sm, ly);
    } else {
      int e = 0;
      for (int k = lane_id() + 1; k < L; k += 32) {
        int c = corr_lag(sm.bits, L, k);
        e += c * c;
      }
      E = warp_sum_i32(e);
    }
    if (lane_id() == 0) {
      E_out[i] = E;
      atomicAdd(&hist[E >> 13], 1u);
    }
    __syncwarp();
  }
}

// One block: finds the bin holding `rank` in hist (kHistBins bins); sel[0] = bin, sel[1] = rank inside.
__global__ void select_bin_kernel(const unsigned* __restrict__ hist, int64_t rank, long long* sel) {
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;  // 1024 threads, 8 bins each
  unsigned long long s = 0;
  for (int b = 0; b < 8; b++) s += hist[t * 8 + b];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long acc = 0;
    int chunk = 0;
    while (chunk < 1024 && acc + part[chunk] <= (unsigned long long)rank) acc += part[chunk++];
    int bin = chunk * 8;
    while (bin < chunk * 8 + 7 && acc + hist[bin] <= (unsigned long long)rank) acc += hist[bin++];
    sel[0] = bin;
    sel[1] = (long long)rank - (long long)acc;
  }
}

__global__ void hist_low_kernel(const int32_t* __restrict__ E, int64_t n, const long long* sel,
                                unsigned* __restrict__ hist2) {
  const int bin = (int)sel[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int e = E[i];
    if ((e >> 13) == bin) atomicAdd(&hist2[e & 8191], 1u);
  }
}

__global__ void finish_select_kernel(const unsigned* __restrict__ hist2, long long* sel, int32_t* E_thr_out) {
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;
  unsigned long long s = 0;
  for (int b = 0; b < 8; b++) s += hist2[t * 8 + b];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long rank = (unsigned long long)sel[1], acc = 0;
    int chunk = 0;
    while (chunk < 1024 && acc + part[chunk] <= rank) acc += part[chunk++];
    int low = chunk * 8;
    while (low < chunk * 8 + 7 && acc + hist2[low] <= rank) acc += hist2[low++];
    *E_thr_out = (int32_t)((sel[0] << 13) | low);
  }
}

template <int M, int H, int NP>
int launch_walk_t(labs_ctx* ctx, const WalkParams& P, int warps, cudaStream_t st) {
  size_t smem = sizeof(WalkSmem) * (size_t)warps + sizeof(uint64_t) * LABS_MAX_L;
  auto kern = walk_kernel<M, H, NP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return LABS_ERR_CUDA;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
  if (e != cudaSuccess || per_sm < 1) return LABS_ERR_CUDA;
  long long blocks = (long long)per_sm * ctx->num_sms;
  long long need = (P.n_walks + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, 32 * warps, smem, st>>>(P);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int launch_sample_threshold(labs_ctx* ctx, int L, int skew, int p, const uint64_t* prefixes, int n_prefix,
                            int prefix_words, uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr_out,
                            int32_t* E_samples, cudaStream_t st) {
  int32_t* Es = E_samples;
  if (!Es) {
    Es = static_cast<int32_t*>(ws_get(ctx, kWsThreshSamples, sizeof(int32_t) * (size_t)n_samples));
    if (!Es) return LABS_ERR_NOMEM;
  }
  unsigned* hist = static_cast<unsigned*>(ws_get(ctx, kWsThreshHist, sizeof(unsigned) * 2 * kHistBins + 64));
  if (!hist) return LABS_ERR_NOMEM;
  long long* sel = reinterpret_cast<long long*>(hist + 2 * kHistBins);
  if (cudaMemsetAsync(hist, 0, sizeof(unsigned) * 2 * kHistBins, st) != cudaSuccess) return LABS_ERR_CUDA;
  int64_t blocks = std::min<int64_t>((n_samples + kSampleWarps - 1) / kSampleWarps, (int64_t)ctx->num_sms * 8);
  sample_kernel<<<(unsigned)blocks, 32 * kSampleWarps, 0, st>>>(L, skew, p, prefixes, n_prefix, prefix_words, seed,
                                                                 n_samples, Es, hist);
  select_bin_kernel<<<1, 1024, 0, st>>>(hist, rank, sel);
  int64_t hb = std::min<int64_t>((n_samples + 255) / 256, (int64_t)ctx->num_sms * 8);
  hist_low_kernel<<<(unsigned)hb, 256, 0, st>>>(Es, n_samples, sel, hist + kHistBins);
  finish_select_kernel<<<1, 1024, 0, st>>>(hist + kHistBins, sel, E_thr_out);
  return cuda_status(cudaGetLastError());
}

// Walk-kernel variants: (tile M, lag ranges H, passes NP).  The chooser takes the variant with the
// least per-lane scan work NP * M / H (ties: more lanes per tile, then the larger tile).
struct Variant {
  int M, H, NP;
};
static const Variant kVariants[] = {{8, 1, 1},  {8, 1, 2},  {8, 1, 3},  {12, 1, 1}, {12, 1, 2}, {12, 2, 1},
                                    {12, 2, 2}, {16, 1, 1}, {16, 1, 2}, {16, 2, 1}, {16, 2, 2}, {16, 2, 3}};

static bool choose_variant(int L, int skew, int p, int req_m, Variant* out) {
  bool found = false;
  Variant best{0, 0, 0};
  for (const Variant& v : kVariants) {
    if (req_m && v.M != req_m) continue;
    Layout ly;
    if (!make_layout(ly, L, skew, p, v.M, v.H)) continue;
    int np = (ly.n_tasks + 31) / 32;
    if (np < 1) np = 1;
    if (np != v.NP) continue;
    int cost = v.NP * v.M / v.H, bcost = found ? best.NP * best.M / best.H : 0;
    if (!found || cost < bcost || (cost == bcost && (v.H > best.H || (v.H == best.H && v.M > best.M)))) {
      best = v;
      found = true;
    }
  }
  *out = best;
  return found;
}

int launch_skew_search(labs_ctx* ctx, const labs_walk_cfg* cfg, const uint64_t* prefixes, int n_prefix,
                       labs_candidate* out, int64_t* walk_stats, labs_walk_stats* stats, cudaStream_t st) {
  WalkParams P{};
  P.L = cfg->L;
  P.skew = cfg->skew;
  P.p = cfg->p;
  P.T_i = cfg->T_i > 0 ? cfg->T_i : 4 * (cfg->L + 1);
  P.R = cfg->R;
  P.bloom_log2 = cfg->bloom_log2;
  P.bloom_k = cfg->bloom_k;
  P.prefix_words = cfg->p > 0 ? (cfg->p + 63) / 64 : 1;
  P.n_prefix = n_prefix;
  P.n_walks = cfg->n_walks;
  P.walk_begin = cfg->walk_begin;
  P.flip_budget = cfg->flip_budget;
  P.seed = cfg->seed;
  P.prefixes = prefixes;
  P.E_target = cfg->E_target;
  P.out = out;
  P.walk_stats = walk_stats;
  P.stats = stats;
  Variant v;
  if (!choose_variant(P.L, P.skew, P.p, cfg->tile_m, &v)) return LABS_ERR_INVALID_ARG;
  P.M = v.M;
  make_layout(P.ly, P.L, P.skew, P.p, v.M, v.H);

  char* w = static_cast<char*>(ws_get(ctx, kWsWalkCounters, 256));
  if (!w) return LABS_ERR_NOMEM;
  P.counter = reinterpret_cast<unsigned long long*>(w);
  int32_t* thr = reinterpret_cast<int32_t*>(w + 64);
  if (cfg->E_thr_dev) {
    P.E_thr_ptr = cfg->E_thr_dev;
  } else if (cfg->E_thr == LABS_AUTO_THRESHOLD) {
    int s = launch_sample_threshold(ctx, P.L, P.skew, P.p, prefixes, n_prefix, P.prefix_words, P.seed,
                                    cfg->n_thresh_samples, cfg->thresh_rank, thr, nullptr, st);
    if (s != LABS_OK) return s;
    P.E_thr_ptr = thr;
  } else {
    P.E_thr_ptr = nullptr;
    P.E_thr_value = cfg->E_thr;
  }
  walk_init_kernel<<<1, 1, 0, st>>>(stats, P.E_thr_ptr, P.E_thr_value, P.counter);
  if (P.n_walks == 0) return cuda_status(cudaGetLastError());
  int warps = cfg->warps_per_cta > 0 ? cfg->warps_per_cta : 8;
  switch (v.M * 100 + v.H * 10 + v.NP) {
    case 811: return launch_walk_t<8, 1, 1>(ctx, P, warps, st);
    case 812: return launch_walk_t<8, 1, 2>(ctx, P, warps, st);
    case 813: return launch_walk_t<8, 1, 3>(ctx, P, warps, st);
    case 1621: return launch_walk_t<16, 2, 1>(ctx, P, warps, st);
    case 1622: return launch_walk_t<16, 2, 2>(ctx, P, warps, st);
    case 1623: return launch_walk_t<16, 2, 3>(ctx, P, warps, st);
    case 1211: return launch_walk_t<12, 1, 1>(ctx, P, warps, st);
    case 1212: return launch_walk_t<12, 1, 2>(ctx, P, warps, st);
    case 1221: return launch_walk_t<12, 2, 1>(ctx, P, warps, st);
    case 1222: return launch_walk_t<12, 2, 2>(ctx, P, warps, st);
    case 1611: return launch_walk_t<16, 1, 1>(ctx, P, warps, st);
    case 1612: return launch_walk_t<16, 1, 2>(ctx, P, warps, st);
    default: return LABS_ERR_INVALID_ARG;
  }
}

}  // namespace labsg

// ---------------------------------------------------------------------------------------------
// Sieve bound without any allocation (labs_sample_threshold_noalloc).
//
// Some callers cannot allocate device memory while they run this library.  An application whose
// allocator owns every device byte (a framework memory pool, a fixed arena sized at start-up) forbids
// direct cudaMalloc; latency-sensitive callers avoid it because it can synchronise the device; and no
// library context (which grows workspace on demand) may exist at all.  For them this entry point runs the
// same kernels as labs_sample_threshold with its scratch -- the sampled energies, both histograms and the
// selected bin -- in one file-scope device array of fixed size, loaded with the library.
// ---------------------------------------------------------------------------------------------
namespace labsg {
namespace {

constexpr int64_t kNoAllocMaxSamples = int64_t(1) << 20;  // 1,048,576 samples (>= the 10^6 sieve sample)
constexpr size_t kNoAllocSamplesBytes = sizeof(int32_t) * (size_t)kNoAllocMaxSamples;
constexpr size_t kNoAllocHistBytes = sizeof(unsigned) * 2 * kHistBins;
constexpr size_t kNoAllocBytes = kNoAllocSamplesBytes + kNoAllocHistBytes + 256;  // + the selected bin

// Every GPU that loads the library holds these 4.26 MB until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_threshold_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kNoAllocMaxDevices];  // device address of g_threshold_scratch per device

// Set-up, once per device, with that device current: the host-side name of the array is not a device
// address, so ask the runtime for it.
int threshold_scratch(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_threshold_scratch) != cudaSuccess || !p) return LABS_ERR_CUDA;
    g_scratch_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return LABS_OK;
}

}  // namespace
}  // namespace labsg

extern "C" int labs_sample_threshold_noalloc(int L, int skew, int p, const uint64_t* prefixes, int n_prefix,
                                             uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr_out,
                                             void* stream) {
  using namespace labsg;
  if (L < 3 || L > LABS_MAX_L || (skew != 0 && skew != 1) || p < 0 || n_prefix < 1) return LABS_ERR_INVALID_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return LABS_ERR_INVALID_ARG;
  if (!skew && p >= L) return LABS_ERR_INVALID_ARG;
  if (!prefixes || (reinterpret_cast<uintptr_t>(prefixes) & 7u) || !E_thr_out ||
      (reinterpret_cast<uintptr_t>(E_thr_out) & 3u))
    return LABS_ERR_INVALID_ARG;
  if (n_samples < 1 || rank < 0 || rank >= n_samples) return LABS_ERR_INVALID_ARG;
  if (n_samples > kNoAllocMaxSamples) return LABS_ERR_CAPACITY;  // beyond the fixed scratch
  int device = 0, sms = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kNoAllocMaxDevices) return LABS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return LABS_ERR_CUDA;
  unsigned char* base = nullptr;
  int s = threshold_scratch(device, &base);
  if (s != LABS_OK) return s;
  int32_t* Es = reinterpret_cast<int32_t*>(base);
  unsigned* hist = reinterpret_cast<unsigned*>(base + kNoAllocSamplesBytes);
  long long* sel = reinterpret_cast<long long*>(base + kNoAllocSamplesBytes + kNoAllocHistBytes);
  cudaStream_t st = (cudaStream_t)stream;
  const int prefix_words = p > 0 ? (p + 63) / 64 : 1;
  // the histograms keep the previous call's counts: clear them first
  if (cudaMemsetAsync(hist, 0, kNoAllocHistBytes, st) != cudaSuccess) return LABS_ERR_CUDA;
  int64_t blocks = std::min<int64_t>((n_samples + kSampleWarps - 1) / kSampleWarps, (int64_t)sms * 8);
  sample_kernel<<<(unsigned)blocks, 32 * kSampleWarps, 0, st>>>(L, skew, p, prefixes, n_prefix, prefix_words, seed,
                                                                 n_samples, Es, hist);
  select_bin_kernel<<<1, 1024, 0, st>>>(hist, rank, sel);
  int64_t hb = std::min<int64_t>((n_samples + 255) / 256, (int64_t)sms * 8);
  hist_low_kernel<<<(unsigned)hb, 256, 0, st>>>(Es, n_samples, sel, hist + kHistBins);
  finish_select_kernel<<<1, 1024, 0, st>>>(hist + kHistBins, sel, E_thr_out);
  return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ERR_CUDA;
}
