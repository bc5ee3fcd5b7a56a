// pq_indep.cu -- step 2 with one independent priority queue per candidate (labs_pq_independent): the
// paper's own parallelisation of Algorithm 2 (every candidate refined on its own, Section 3), with the
// queue unbounded as in the listing (nothing is evicted) and B = 1 pops per step.
//
// GB300 mapping.  One warp per candidate; a candidate's state lives in HBM:
//   arena  -- every pushed node as a 16-byte record (E, link, fp); the survivors of one pop are appended
//             as one run sorted by (E, fp, column), so the arena is a set of sorted runs;
//   runs   -- a binary heap over the runs' current heads keyed by (E, fp): its top is the queue minimum,
//             a pop advances that run's head (one sift-down), a new run is one sift-up;
//   pivots -- the sequence of every popped node (a node is stored as its pivot and column, and is made
//             into a sequence only when popped);
//   H      -- the candidate's visited set (open addressing, cleared per candidate).
// A pop scans all L single flips (the dp4a tiles of labs_core.cuh) and, with T_r > 0, the pivot's 2 T_r
// rotations; survivors are sorted in shared memory (bitonic, one warp) and pushed as one run.  Memory per
// resident warp is about max_expansions x (L + 2 T_r) x 16 B + 2^H_log2 x 8 B: HBM capacity, not
// bandwidth, is what this design spends.
#include <algorithm>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kIWarps = 4;
constexpr int kIM = 8;
constexpr int kSortN = 1024;  // most survivors of one pop, padded to a power of two: L + 2 T_r <= 576 + 128
constexpr uint64_t kEmpty = ~0ull;
constexpr int kProbeLimit = 1 << 20;
constexpr int kInsBatch = 4;  // visited-set inserts in flight per lane
constexpr int kMaxTr = 64;    // rotations per side (the library's bound on T_r)

struct Node {  // one queue record: 16 bytes
  int32_t E;
  int32_t link;  // pivot * 1024 + column (column < L: flip, else rotation column - L); -1: the seed
  uint64_t fp;
};

struct RunHead {  // heap element: the run's current head key and its remaining range in the arena
  int32_t E;
  int32_t cur;
  uint64_t fp;
  int32_t end;
  int32_t pad;
};

struct IndepArgs {
  int L, W, Tr, width, H_log2;
  long long max_exp, T_u;
  long long arena_cap, heap_cap;
  long long n;
  const uint64_t* seeds;
  uint64_t* best_seqs;
  int32_t* best_E;
  labs_pq_stats* stats;
  // per-slot workspaces (slot = resident warp)
  Node* arena;
  RunHead* heap;
  uint64_t* pivots;
  uint64_t* H;
  const uint64_t* ztab;
  unsigned long long* counter;
  int smem_stride;  // bytes of shared memory per warp: IndepSmem + the sort buffer
};

__device__ __forceinline__ bool kless(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}

// Visited set of one slot (open addressing, linear probing); *err set on an exhausted probe sequence.
// The first probe of several keys is issued by the caller, all at once, so that their latencies
// overlap; these continue a key's probe sequence after a first slot that held another key.
__device__ __forceinline__ uint64_t hs_home(uint64_t fp, int log2) { return (fp * kGamma) >> (64 - log2); }
__device__ __forceinline__ bool hs_contains_from(const uint64_t* H, int log2, uint64_t fp, uint64_t s, int* err) {
  const uint64_t mask = (1ull << log2) - 1;
  for (int it = 1; it < kProbeLimit; it++) {
    s = (s + 1) & mask;
    const uint64_t v = H[s];
    if (v == fp) return true;
    if (v == kEmpty) return false;
  }
  *err = 1;
  return true;
}
__device__ __forceinline__ void hs_insert_from(uint64_t* H, int log2, uint64_t fp, uint64_t s, int* err) {
  const uint64_t mask = (1ull << log2) - 1;
  for (int it = 1; it < kProbeLimit; it++) {
    s = (s + 1) & mask;
    const unsigned long long old =
        atomicCAS(reinterpret_cast<unsigned long long*>(&H[s]), (unsigned long long)kEmpty, fp);
    if (old == kEmpty || old == fp) return;
  }
  *err = 1;
}
__device__ __forceinline__ bool hs_contains(const uint64_t* H, int log2, uint64_t fp, bool has_empty, int* err) {
  if (fp == kEmpty) return has_empty;
  const uint64_t s = hs_home(fp, log2);
  const uint64_t v = H[s];
  if (v == fp) return true;
  if (v == kEmpty) return false;
  return hs_contains_from(H, log2, fp, s, err);
}
__device__ __forceinline__ void hs_insert(uint64_t* H, int log2, uint64_t fp, int* err) {
  const uint64_t s = hs_home(fp, log2);
  const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(&H[s]), (unsigned long long)kEmpty, fp);
  if (old == kEmpty || old == fp) return;
  hs_insert_from(H, log2, fp, s, err);
}

// Left shift of rotation code c: c < Tr moves the first c + 1 elements to the end, c >= Tr the last
// c - Tr + 1 to the start.
__device__ __forceinline__ int rshift(int L, int Tr, int c) {
  const int r = c < Tr ? c + 1 : L - ((c - Tr + 1) % L);
  return r % L;
}

// bits (32-bit words in shared memory) of src with position col + 1 flipped.
__device__ __forceinline__ void flip_bits(const uint32_t* src, int col, uint32_t* dst) {
  const int lane = lane_id();
  if (lane < kBitWords) dst[lane] = src[lane] ^ (lane == (col >> 5) ? 1u << (col & 31) : 0u);
  __syncwarp();
}

__device__ __forceinline__ void rotate_bits(const uint32_t* src, int L, int r, uint32_t* dst) {
  const int lane = lane_id();
  for (int w = 0; w < kBitWords; w++) {
    const int i = 32 * w + lane;
    int bit = 0;
    if (i < L) {
      int j = i + r;
      if (j >= L) j -= L;
      bit = (src[j >> 5] >> (j & 31)) & 1u;
    }
    const unsigned word = __ballot_sync(kFull, bit);
    if (lane == 0) dst[w] = word;
  }
  __syncwarp();
}

__device__ __forceinline__ void words_to_bits(const uint64_t* src, int L, uint32_t* dst) {
  const int lane = lane_id();
  if (lane < kBitWords) {
    const int W32 = (L + 31) >> 5;
    uint32_t v = 0;
    if (lane < W32) {
      const uint64_t x = src[lane >> 1];
      v = (lane & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
      const int rem = L - 32 * lane;
      if (rem < 32) v &= (1u << rem) - 1u;
    }
    dst[lane] = v;
  }
  __syncwarp();
}

__device__ __forceinline__ void bits_to_words(const uint32_t* src, int L, uint64_t* dst) {
  const int lane = lane_id();
  if (lane < ((L + 63) >> 6)) dst[lane] = (uint64_t)src[2 * lane] | ((uint64_t)src[2 * lane + 1] << 32);
}

__device__ __forceinline__ int energy_bits(const uint32_t* bits, int L) {
  int e = 0;
  for (int k = lane_id() + 1; k < L; k += 32) {
    const int c = corr_lag(bits, L, k);
    e += c * c;
  }
  return warp_sum_i32(e);
}

__device__ __forceinline__ uint64_t fp_bits(const uint32_t* bits, int L, const uint64_t* ztab) {
  uint64_t h = 0;
  for (int i = lane_id(); i < L; i += 32)
    if (!((bits[i >> 5] >> (i & 31)) & 1u)) h ^= ztab[i];
  return warp_xor_u64(h);
}

// A survivor of one pop as one 64-bit key: E (26 bits: E < L^3 / 3 < 2^26 for L <= 576), the top 28
// bits of its fingerprint, its column (10 bits).  Unsigned order is (E, fp >> 36, column); runs of equal
// (E, fp >> 36) are then put in (fp, column) order, so the survivors end in (E, fp, column) order.  The
// fingerprint itself is the pivot's with the column's key (a flip) or the rotation's, kept aside.
constexpr uint64_t kPadKey = ~0ull;
__device__ __forceinline__ uint64_t pack_key(int E, uint64_t fp, int col) {
  return ((uint64_t)(uint32_t)E << 38) | ((fp >> 36) << 10) | (uint64_t)col;
}
__device__ __forceinline__ int key_E(uint64_t k) { return (int)(k >> 38); }
__device__ __forceinline__ int key_col(uint64_t k) { return (int)(k & 1023u); }

// Per-warp shared memory: this fixed part, then the survivors' sort buffer of np2 keys (the next power
// of two of L + 2 T_r, at most kSortN), so that shorter queues leave room for more resident warps.
struct __align__(16) IndepSmem {
  ScanSmem s;
  uint64_t rfp[2 * kMaxTr];   // fingerprints of the pivot's rotations (columns L ..)
  uint32_t pbits[kBitWords];  // the pivot
  uint32_t cbits[kBitWords];  // a child
  int16_t P[kMaxL];  // P_m of the pivot's neighbours
  uint32_t xb[kBitWords];
  int n_surv;
};

__global__ void __launch_bounds__(32 * kIWarps) pq_indep_kernel(IndepArgs a, Layout ly) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* wbase = smem_raw + (size_t)(threadIdx.x >> 5) * a.smem_stride;
  IndepSmem& S = *reinterpret_cast<IndepSmem*>(wbase);
  uint64_t* keys = reinterpret_cast<uint64_t*>(wbase + sizeof(IndepSmem));
  ScanSmem& sm = S.s;
  const int lane = lane_id();
  const long long slot = (long long)blockIdx.x * kIWarps + (threadIdx.x >> 5);
  Node* arena = a.arena + slot * a.arena_cap;
  RunHead* heap = a.heap + slot * a.heap_cap;
  uint64_t* pivots = a.pivots + slot * a.max_exp * a.W;
  uint64_t* H = a.H + slot * (1ll << a.H_log2);
  const long long hslots = 1ll << a.H_log2;

  while (true) {
    unsigned long long cand = 0;
    if (lane == 0) cand = atomicAdd(a.counter, 1ull);
    cand = __shfl_sync(kFull, cand, 0);
    if ((long long)cand >= a.n) break;
    int err = 0;
    // ---- reset the visited set, seed the queue
    for (long long t = lane; t < hslots; t += 32) H[t] = kEmpty;
    __threadfence_block();
    __syncwarp();
    words_to_bits(a.seeds + cand * a.W, a.L, S.pbits);
    int bestE = energy_bits(S.pbits, a.L);
    uint64_t bestfp = fp_bits(S.pbits, a.L, a.ztab);
    bool has_empty = bestfp == kEmpty;
    if (lane == 0) {
      if (!has_empty) hs_insert(H, a.H_log2, bestfp, &err);
      arena[0] = Node{bestE, -1, bestfp};
      heap[0] = RunHead{bestE, 0, bestfp, 1, 0};
    }
    bits_to_words(S.pbits, a.L, a.best_seqs + cand * a.W);
    __syncwarp();
    long long heap_n = 1, top = 1, exps = 0, u = 0, surv = 0, improvements = 0, h_size = 1;
    int stop = 0;
    while (true) {
      if (exps >= a.max_exp) stop = 1;
      else if (heap_n == 0) stop = 2;
      else if (a.T_u > 0 && u >= a.T_u) stop = 3;
      if (stop || err) break;
      // ---- pop: the top run's head; advance the run, sift down (lane 0)
      int pE = 0, plink = 0;
      unsigned long long pfp = 0;
      if (lane == 0) {
        RunHead h = heap[0];
        const Node nd = arena[h.cur];
        pE = nd.E;
        plink = nd.link;
        pfp = nd.fp;
        h.cur++;
        if (h.cur < h.end) {
          const Node nx = arena[h.cur];
          h.E = nx.E;
          h.fp = nx.fp;
        } else {
          heap_n--;
          h = heap[heap_n];
        }
        if (heap_n > 0) {
          long long i = 0;
          while (true) {
            const long long l = 2 * i + 1, r = l + 1;
            if (l >= heap_n) break;
            long long c = l;
            if (r < heap_n && kless(heap[r].E, heap[r].fp, heap[l].E, heap[l].fp)) c = r;
            if (!kless(heap[c].E, heap[c].fp, h.E, h.fp)) break;
            heap[i] = heap[c];
            i = c;
          }
          heap[i] = h;
        }
      }
      heap_n = __shfl_sync(kFull, heap_n, 0);
      pE = __shfl_sync(kFull, pE, 0);
      plink = __shfl_sync(kFull, plink, 0);
      pfp = __shfl_sync(kFull, pfp, 0);
      // ---- the pivot's sequence: the seed, or the child `col` of an earlier pivot
      if (plink < 0) {
        words_to_bits(a.seeds + cand * a.W, a.L, S.pbits);
      } else {
        words_to_bits(pivots + (long long)(plink >> 10) * a.W, a.L, S.cbits);
        const int col = plink & 1023;
        if (col < a.L)
          flip_bits(S.cbits, col, S.pbits);
        else
          rotate_bits(S.cbits, a.L, rshift(a.L, a.Tr, col - a.L), S.pbits);
      }
      bits_to_words(S.pbits, a.L, pivots + exps * a.W);
      // ---- expand: every single flip (dp4a tiles), then the rotations
      if (lane == 0) S.n_surv = 0;
      for (int w = lane; w < kBitWords; w += 32) sm.bits[w] = S.pbits[w];
      __syncwarp();
      build_table(sm, ly);
      const bool fast = pack_c8(sm);
      const int SC = table_sum(sm);
      build_bytes(sm, ly);
      p_all(sm, ly, S.xb, S.cbits, S.P);
      for (int base = 0; base < ly.n_tiles; base += 32) {
        const int tau = base + lane;
        if (tau < ly.n_tiles) {
          int cls, q0;
          tile_of(ly, tau, cls, q0);
          int acc[kIM];
          if (fast)
            scan_tile<kIM, false>(sm, ly, cls, q0, acc);
          else
            scan_tile<kIM, true>(sm, ly, cls, q0, acc);
          // the tile's Delta E and fingerprints, then the first visited-set probe of all of them at
          // once (independent loads), then the rare longer probe sequences
          int dv[kIM], mv[kIM];
          uint64_t fv[kIM], hv[kIM];
#pragma unroll
          for (int j = 0; j < kIM; j++) {
            const SlotInfo si = slot_info(ly, cls, q0 + j);
            mv[j] = si.active ? si.m : 0;
            dv[j] = si.active ? finish_delta(sm, ly, cls, q0 + j, si, acc[j], SC, S.P[si.m - 1]) : 0;
            fv[j] = si.active ? pfp ^ a.ztab[si.m - 1] : kEmpty;
          }
#pragma unroll
          for (int j = 0; j < kIM; j++) hv[j] = (mv[j] && fv[j] != kEmpty) ? H[hs_home(fv[j], a.H_log2)] : kEmpty;
#pragma unroll
          for (int j = 0; j < kIM; j++) {
            if (!mv[j]) continue;
            bool seen;
            if (fv[j] == kEmpty)
              seen = has_empty;
            else if (hv[j] == fv[j] || hv[j] == kEmpty)
              seen = hv[j] == fv[j];
            else
              seen = hs_contains_from(H, a.H_log2, fv[j], hs_home(fv[j], a.H_log2), &err);
            if (!seen) {
              const int k = atomicAdd(&S.n_surv, 1);
              keys[k] = pack_key(pE + dv[j], fv[j], mv[j] - 1);
            }
          }
        }
      }
      __syncwarp();
      for (int c = 0; c < 2 * a.Tr; c++) {
        rotate_bits(S.pbits, a.L, rshift(a.L, a.Tr, c), S.cbits);
        const int e = energy_bits(S.cbits, a.L);
        const uint64_t h = fp_bits(S.cbits, a.L, a.ztab);
        if (lane == 0) {
          S.rfp[c] = h;
          if (!hs_contains(H, a.H_log2, h, has_empty, &err)) keys[S.n_surv++] = pack_key(e, h, a.L + c);
        }
        __syncwarp();
      }
      err = __reduce_or_sync(kFull, err);
      const int ns = S.n_surv;
      // ---- sort the survivors by (E, fp, column): bitonic over the next power of two on the packed keys
      auto fp_of = [&](int col) -> uint64_t { return col < a.L ? pfp ^ a.ztab[col] : S.rfp[col - a.L]; };
      int np2 = 1;
      while (np2 < ns) np2 <<= 1;
      for (int i = ns + lane; i < np2; i += 32) keys[i] = kPadKey;
      __syncwarp();
      // every substage compares np2 / 2 disjoint pairs (i, i + j), i with bit j clear: pair p maps to i
      // by inserting a zero at bit j, so every lane has a pair in every iteration
      for (int k = 2; k <= np2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int pr = lane; pr < (np2 >> 1); pr += 32) {
            const int i = ((pr & ~(j - 1)) << 1) | (pr & (j - 1));
            const int l = i | j;
            const uint64_t x = keys[i], y = keys[l];
            const bool up = (i & k) == 0;
            if (up ? y < x : x < y) {
              keys[i] = y;
              keys[l] = x;
            }
          }
          __syncwarp();
        }
      // runs of equal (E, fp >> 36), if any, into (fp, column) order (one lane; such runs are rare)
      bool tie = false;
      for (int i = lane; i + 1 < ns; i += 32) tie |= (keys[i] >> 10) == (keys[i + 1] >> 10);
      if (__any_sync(kFull, tie)) {
        if (lane == 0)
          for (int i = 1; i < ns; i++) {
            const uint64_t kx = keys[i];
            const uint64_t fx = fp_of(key_col(kx));
            int c = i;
            while (c > 0 && (keys[c - 1] >> 10) == (kx >> 10)) {
              const uint64_t fy = fp_of(key_col(keys[c - 1]));
              if (fy < fx || (fy == fx && key_col(keys[c - 1]) < key_col(kx))) break;
              keys[c] = keys[c - 1];
              c--;
            }
            keys[c] = kx;
          }
        __syncwarp();
      }
      // ---- distinct survivors (equal (E, fp): the same sequence) become one run; H receives them
      int nu = 0;
      int carryE = 0;  // the element before this lane-0's: last lane's of the previous 32
      uint64_t carryF = 0;
      for (int i0 = 0; i0 < ns; i0 += 32 * kInsBatch) {
        // kInsBatch keys per lane: their first compare-and-swap all in flight at once
        bool ins[kInsBatch];
        uint64_t fk[kInsBatch];
        unsigned long long old[kInsBatch];
#pragma unroll
        for (int r = 0; r < kInsBatch; r++) {
          const int i = i0 + 32 * r + lane;
          int xE = 0, xc = 0;
          uint64_t xf = 0;
          if (i < ns) {
            const uint64_t kx = keys[i];
            xE = key_E(kx);
            xc = key_col(kx);
            xf = fp_of(xc);
          }
          int pE = __shfl_up_sync(kFull, xE, 1);
          uint64_t pf = __shfl_up_sync(kFull, xf, 1);
          if (lane == 0) {
            pE = carryE;
            pf = carryF;
          }
          carryE = __shfl_sync(kFull, xE, 31);
          carryF = __shfl_sync(kFull, xf, 31);
          const bool keep = i < ns && (i == 0 || pE != xE || pf != xf);
          const unsigned m = __ballot_sync(kFull, keep);
          if (keep) {
            const int o = nu + __popc(m & ((1u << lane) - 1u));
            arena[top + o] = Node{xE, (int)(exps << 10) | xc, xf};
            if (xf == kEmpty) has_empty = true;
          }
          nu += __popc(m);
          ins[r] = keep && xf != kEmpty;
          fk[r] = xf;
        }
#pragma unroll
        for (int r = 0; r < kInsBatch; r++)
          old[r] = ins[r] ? atomicCAS(reinterpret_cast<unsigned long long*>(&H[hs_home(fk[r], a.H_log2)]),
                                      (unsigned long long)kEmpty, fk[r])
                          : (unsigned long long)kEmpty;
#pragma unroll
        for (int r = 0; r < kInsBatch; r++)
          if (ins[r] && old[r] != kEmpty && old[r] != fk[r]) hs_insert_from(H, a.H_log2, fk[r], hs_home(fk[r], a.H_log2), &err);
      }
      has_empty = __any_sync(kFull, has_empty);
      err = __reduce_or_sync(kFull, err);
      __syncwarp();
      // ---- best, statistics, the new run
      const int E0 = nu > 0 ? key_E(keys[0]) : INT32_MAX, col0 = nu > 0 ? key_col(keys[0]) : 0;
      const uint64_t fp0 = nu > 0 ? fp_of(col0) : 0;
      if (nu > 0 && E0 < bestE) {
        bestE = E0;
        bestfp = fp0;
        const int col = col0;
        if (col < a.L)
          flip_bits(S.pbits, col, S.cbits);
        else
          rotate_bits(S.pbits, a.L, rshift(a.L, a.Tr, col - a.L), S.cbits);
        bits_to_words(S.cbits, a.L, a.best_seqs + cand * a.W);
        improvements++;
        u = 0;
      } else {
        u++;
      }
      if (nu > 0 && lane == 0) {  // push the run: sift up
        RunHead h{E0, (int)top, fp0, (int)(top + nu), 0};
        long long i = heap_n;
        while (i > 0) {
          const long long p = (i - 1) >> 1;
          if (!kless(h.E, h.fp, heap[p].E, heap[p].fp)) break;
          heap[i] = heap[p];
          i = p;
        }
        heap[i] = h;
      }
      if (nu > 0) heap_n++;
      top += nu;
      surv += nu;
      h_size += nu;
      exps++;
      __syncwarp();
      if (h_size * 4 > hslots * 3) err = 1;  // keep the visited set below 3/4 load
    }
    if (lane == 0) {
      a.best_E[cand] = bestE;
      labs_pq_stats st{};
      st.expansions = exps;
      st.rounds = exps;
      st.survivors = surv;
      st.admitted = surv;
      st.evicted = 0;
      st.h_size = h_size;
      st.improvements = improvements;
      st.best_fp = bestfp;
      st.stop_reason = err ? 0 : stop;
      st.status = err ? LABS_ERR_CAPACITY : LABS_OK;
      a.stats[cand] = st;
    }
    __syncwarp();
  }
}

__global__ void indep_ztab_kernel(uint64_t* ztab, int L) {
  const uint64_t zk = stream_key(0, kPurposeZobrist, (uint64_t)L, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) ztab[i] = zobrist(zk, i + 1);
}

}  // namespace

int launch_pq_independent(labs_ctx* ctx, const labs_pq_indep_cfg* cfg, const uint64_t* seeds, int n,
                          uint64_t* best_seqs, int32_t* best_E, labs_pq_stats* stats, cudaStream_t st) {
  if (n == 0) return LABS_OK;
  const int L = cfg->L, W = (L + 63) / 64;
  Layout ly;
  if (!make_layout(ly, L, 0, 0, kIM)) return LABS_ERR_INVALID_ARG;
  IndepArgs a{};
  a.L = L;
  a.W = W;
  a.Tr = cfg->T_r;
  a.width = L + 2 * cfg->T_r;
  a.H_log2 = cfg->H_log2;
  a.max_exp = cfg->max_expansions;
  a.T_u = cfg->T_u;
  a.arena_cap = 1 + a.max_exp * a.width;
  a.heap_cap = a.max_exp + 1;
  a.n = n;
  a.seeds = seeds;
  a.best_seqs = best_seqs;
  a.best_E = best_E;
  a.stats = stats;
  // resident warps: as many slots as the memory budget allows, at most one per candidate
  const size_t per_slot = (size_t)a.arena_cap * sizeof(Node) + (size_t)a.heap_cap * sizeof(RunHead) +
                          (size_t)a.max_exp * W * 8 + (8ull << a.H_log2);
  int np2max = 1;  // a pop's survivors (at most width) are sorted over the next power of two
  while (np2max < a.width) np2max <<= 1;
  if (np2max > kSortN || cfg->T_r > kMaxTr) return LABS_ERR_INVALID_ARG;
  a.smem_stride = (int)((sizeof(IndepSmem) + sizeof(uint64_t) * np2max + 15) & ~size_t(15));
  const size_t smem = (size_t)a.smem_stride * kIWarps;
  if (cudaFuncSetAttribute(pq_indep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return LABS_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pq_indep_kernel, 32 * kIWarps, smem) != cudaSuccess ||
      per_sm < 1)
    return LABS_ERR_CUDA;
  long long blocks = std::min<long long>((long long)per_sm * ctx->num_sms, ((long long)n + kIWarps - 1) / kIWarps);
  const size_t budget = cfg->max_workspace_bytes > 0 ? (size_t)cfg->max_workspace_bytes : ((size_t)64 << 30);
  blocks = std::min<long long>(blocks, (long long)(budget / (per_slot * kIWarps)));
  if (blocks < 1) return LABS_ERR_NOMEM;
  const size_t slots = (size_t)blocks * kIWarps;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t oA = take(slots * (size_t)a.arena_cap * sizeof(Node)), oHp = take(slots * (size_t)a.heap_cap * sizeof(RunHead));
  const size_t oP = take(slots * (size_t)a.max_exp * W * 8), oH = take(slots * (8ull << a.H_log2));
  const size_t oZ = take(8 * (size_t)L), oC = take(8);
  char* base = static_cast<char*>(ws_get(ctx, kWsPqIndep, off));
  if (!base) return LABS_ERR_NOMEM;
  a.arena = reinterpret_cast<Node*>(base + oA);
  a.heap = reinterpret_cast<RunHead*>(base + oHp);
  a.pivots = reinterpret_cast<uint64_t*>(base + oP);
  a.H = reinterpret_cast<uint64_t*>(base + oH);
  a.ztab = reinterpret_cast<uint64_t*>(base + oZ);
  a.counter = reinterpret_cast<unsigned long long*>(base + oC);
  indep_ztab_kernel<<<(L + 255) / 256, 256, 0, st>>>(reinterpret_cast<uint64_t*>(base + oZ), L);
  if (cudaMemsetAsync(a.counter, 0, 8, st) != cudaSuccess) return LABS_ERR_CUDA;
  pq_indep_kernel<<<(unsigned)blocks, 32 * kIWarps, smem, st>>>(a, ly);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
