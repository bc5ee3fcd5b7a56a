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

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

struct WalkSmem {
  ScanSmem s;
  uint32_t bloom[1024];  // up to 2^15 bits
};

struct WalkParams {
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

// Per-slot state lives in shared memory, lane-major ([slot][lane], conflict-free): packed slot info,
// P_m and the latest Delta E.  Keeping it out of registers leaves the scan its registers.
template <int S>
struct SlotSmem {
  uint32_t info[S][32];  // m | nf << 10 | nb << 20 | active << 30 | pair << 31
  int pm[S][32];
  int de[S][32];
};

__device__ __forceinline__ uint32_t pack_info(const SlotInfo& si) {
  return (uint32_t)si.m | ((uint32_t)si.nf << 10) | ((uint32_t)si.nb << 20) | ((uint32_t)si.active << 30) |
         ((uint32_t)si.pair << 31);
}

__device__ __forceinline__ SlotInfo unpack_info(const Layout& ly, uint32_t v) {
  SlotInfo si;
  si.m = (int)(v & 1023u);
  si.nf = (int)((v >> 10) & 1023u);
  si.nb = (int)((v >> 20) & 1023u);
  si.active = (int)((v >> 30) & 1u);
  si.pair = (int)(v >> 31);
  si.gd = si.pair ? (ly.L + 1 - 2 * si.m) / 2 : 0;
  return si;
}

template <int M, int NP>
__global__ void __launch_bounds__(256, 2) walk_kernel(WalkParams P) {
  constexpr int S = M * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5;
  WalkSmem& ws = reinterpret_cast<WalkSmem*>(smem_raw)[wid];
  SlotSmem<S>& ss = reinterpret_cast<SlotSmem<S>*>(smem_raw + sizeof(WalkSmem) * (blockDim.x >> 5))[wid];
  ScanSmem& sm = ws.s;
  const int lane = lane_id();
  Layout ly;
  make_layout(ly, P.L, P.skew, P.p, M);
  const uint64_t zkey = stream_key(0, kPurposeZobrist, (uint64_t)P.L, 0);
  const int32_t E_thr = P.E_thr_ptr ? *P.E_thr_ptr : P.E_thr_value;
  const uint32_t bmask = (1u << P.bloom_log2) - 1u;
  const int bwords = 1 << (P.bloom_log2 - 5);
  const int W = (P.L + 63) >> 6;
  const int R = P.R;

  // this lane's tiles (one per pass) and slot info
  int tcls[NP], tq0[NP];
  bool thas[NP];
#pragma unroll
  for (int ps = 0; ps < NP; ps++) {
    int tau = ps * 32 + lane;
    thas[ps] = tau < ly.n_tiles;
    tcls[ps] = 0;
    tq0[ps] = 0;
    if (thas[ps]) tile_of(ly, tau, tcls[ps], tq0[ps]);
#pragma unroll
    for (int j = 0; j < M; j++) {
      SlotInfo si = slot_info(ly, tcls[ps], tq0[ps] + j);
      if (!thas[ps]) si.active = 0;
      ss.info[ps * M + j][lane] = pack_info(si);
    }
  }
  __syncwarp();

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

    long long flips = 0, segs = 0, skips = 0, dead = 0, first_hit = -1;
    int bestE = INT32_MAX;

    while (flips < P.flip_budget) {
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
      for (int ps = 0; ps < NP; ps++)
#pragma unroll
        for (int j = 0; j < M; j++) {
          SlotInfo si = unpack_info(ly, ss.info[ps * M + j][lane]);
          ss.pm[ps * M + j][lane] = p_from_scratch(sm, ly, tcls[ps], tq0[ps] + j, si);
        }

      int it = 0;
      while (it < P.T_i && flips < P.flip_budget) {
        it++;
        // ---- scan; each lane keeps its best (Delta E, m)
        int bd = INT32_MAX, bm = INT32_MAX;
#pragma unroll
        for (int ps = 0; ps < NP; ps++) {
          if (thas[ps]) {
            int acc[M];
            if (fast)
              scan_tile<M, false>(sm, ly, tcls[ps], tq0[ps], acc);
            else
              scan_tile<M, true>(sm, ly, tcls[ps], tq0[ps], acc);
#pragma unroll
            for (int j = 0; j < M; j++) {
              SlotInfo si = unpack_info(ly, ss.info[ps * M + j][lane]);
              int d = INT32_MAX;
              if (si.active) {
                d = finish_delta(sm, ly, tcls[ps], tq0[ps] + j, si, acc[j], SC, ss.pm[ps * M + j][lane]);
                if (d < bd || (d == bd && si.m < bm)) {
                  bd = d;
                  bm = si.m;
                }
              }
              ss.de[ps * M + j][lane] = d;
            }
          } else {
#pragma unroll
            for (int j = 0; j < M; j++) ss.de[ps * M + j][lane] = INT32_MAX;  // read by the exclusion rescan
          }
        }
        // ---- select: smallest (Delta E, m) whose neighbour is not in the Bloom filter
        int mstar = -1, dstar = 0;
        uint64_t nfp = 0;
        for (int guard = 0; guard <= S * 32; guard++) {
          int dmin = warp_min_i32(bd);
          if (dmin == INT32_MAX) break;
          int mm = (int)warp_min_u32(bd == dmin ? (unsigned)bm : 0xffffffffu);
          uint64_t cand = fp ^ zobrist(zkey, mm);
          if (ly.skew && mm != ly.c) cand ^= zobrist(zkey, ly.L + 1 - mm);
          if (!bloom_test(ws.bloom, cand, P.bloom_k, bmask)) {
            mstar = mm;
            dstar = dmin;
            nfp = cand;
            break;
          }
          skips++;
          if (bd == dmin && bm == mm) {
            // the owner lane drops that neighbour and recomputes its best from the stored deltas
            bd = INT32_MAX;
            int nbm = INT32_MAX;
#pragma unroll
            for (int s = 0; s < S; s++) {
              int d = ss.de[s][lane];
              int m = (int)(ss.info[s][lane] & 1023u);
              if (d == INT32_MAX) continue;
              if (m == mm) {
                ss.de[s][lane] = INT32_MAX;
                continue;
              }
              if (d < dmin || (d == dmin && m <= mm)) continue;  // already ranked ahead, hence excluded
              if (d < bd || (d == bd && m < nbm)) {
                bd = d;
                nbm = m;
              }
            }
            bm = nbm;
          }
        }
        if (mstar < 0) {
          dead++;
          break;
        }
        // ---- apply
        const int f1 = (ly.skew && mstar != ly.c) ? ly.L + 1 - mstar : 0;
#pragma unroll
        for (int s = 0; s < S; s++) {
          SlotInfo si = unpack_info(ly, ss.info[s][lane]);
          ss.pm[s][lane] = p_update(sm, ly, si, ss.pm[s][lane], mstar, f1);
        }
        SC += table_update(sm, ly, mstar, &fast);
        if (lane == 0) {
          flip_position(sm, ly, mstar);
          if (f1) flip_position(sm, ly, f1);
        }
        __syncwarp();
        E += dstar;
        fp = nfp;
        bloom_add(ws.bloom, fp, P.bloom_k, bmask);
        flips++;
        if (E < bestE) bestE = E;
        if (first_hit < 0 && E <= P.E_target) first_hit = flips;
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
      st[0] = flips;
      st[1] = segs;
      st[2] = skips;
      st[3] = dead;
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

template <int M, int NP>
int launch_walk_t(labs_ctx* ctx, const WalkParams& P, int warps, cudaStream_t st) {
  size_t smem = (sizeof(WalkSmem) + sizeof(SlotSmem<M * NP>)) * (size_t)warps;
  auto kern = walk_kernel<M, NP>;
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

// Picks the tile size M and pass count NP: least per-lane scan work NP * M, ties to the larger tile
// (fewer window loads per multiply-add).  NP <= 3 (<= 2 for M = 16).
static void choose_tiles(int L, int skew, int p, int req_m, int* M, int* NP) {
  const int cand[4] = {4, 8, 12, 16};
  int bestM = 0, bestNP = 0;
  for (int a = 0; a < 4; a++) {
    int m = cand[a];
    if (req_m && m != req_m) continue;
    Layout ly;
    if (!make_layout(ly, L, skew, p, m)) continue;
    int np = (ly.n_tiles + 31) / 32;
    if (np < 1) np = 1;
    if (np > (m == 16 ? 2 : 3)) continue;
    if (bestM == 0 || np * m < bestNP * bestM || (np * m == bestNP * bestM && m > bestM)) {
      bestM = m;
      bestNP = np;
    }
  }
  *M = bestM;
  *NP = bestNP;
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
  int M = 0, NP = 0;
  choose_tiles(P.L, P.skew, P.p, cfg->tile_m, &M, &NP);
  if (M == 0) return LABS_ERR_INVALID_ARG;
  P.M = M;

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
  switch (M * 10 + NP) {
    case 41: return launch_walk_t<4, 1>(ctx, P, warps, st);
    case 42: return launch_walk_t<4, 2>(ctx, P, warps, st);
    case 43: return launch_walk_t<4, 3>(ctx, P, warps, st);
    case 81: return launch_walk_t<8, 1>(ctx, P, warps, st);
    case 82: return launch_walk_t<8, 2>(ctx, P, warps, st);
    case 83: return launch_walk_t<8, 3>(ctx, P, warps, st);
    case 121: return launch_walk_t<12, 1>(ctx, P, warps, st);
    case 122: return launch_walk_t<12, 2>(ctx, P, warps, st);
    case 123: return launch_walk_t<12, 3>(ctx, P, warps, st);
    case 161: return launch_walk_t<16, 1>(ctx, P, warps, st);
    case 162: return launch_walk_t<16, 2>(ctx, P, warps, st);
    default: return LABS_ERR_INVALID_ARG;
  }
}

}  // namespace labsg
