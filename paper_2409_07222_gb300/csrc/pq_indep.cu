// pq_indep.cu -- step 2 with one independent priority queue per candidate (labs_pq_independent): the
// paper's own parallelisation of Algorithm 2 (every candidate refined on its own, Section 3), with the
// queue unbounded as in the listing (nothing is evicted) and B = 1 pops per step.
//
// GB300 mapping.  One warp per candidate; a candidate's state lives in HBM:
//   arena  -- every pushed node as a 16-byte record (E, link, fp); the survivors of one pop are appended
//             as one run, in no particular order;
//   runs   -- a binary heap over the runs keyed by each run's smallest (E, fp): its top is the queue
//             minimum.  A pop takes that node out of its run (the run's last node fills the gap), finds
//             the run's new smallest by one warp-wide rescan (at most L + 2 T_r records) and sifts down;
//             a new run is one sift-up.  Keys (E, fp) are distinct in a queue (the visited set admits a
//             sequence once), so the pop order is that of the sequential definition;
//   pivots -- the sequence of every popped node (a node is stored as its pivot and column, and is made
//             into a sequence only when popped), with its correlation table and P_m, so that a flip
//             child starts from its parent's by one O(L) update;
//   H      -- the candidate's visited set (open addressing, cleared per candidate).
// A pop scans all L single flips (the dp4a tiles of labs_core.cuh); each neighbour is one
// insert-if-absent into H, a survivor being one whose key was absent.  With T_r > 0 the pivot's 2 T_r
// rotations follow the flips (a rotation equal to a flip child or to an earlier rotation finds its key in
// H and is dropped, as the ordered dedup keeps the smaller column).  Memory per resident warp is about
// max_expansions x ((L + 2 T_r) x 16 B + 4 L B) + 2^H_log2 x 8 B: HBM capacity, not bandwidth, is what
// this design spends.
#include <algorithm>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kIWarps = 4;
constexpr int kIM = 8;
constexpr uint64_t kEmpty = ~0ull;
constexpr int kProbeLimit = 1 << 20;
constexpr int kMaxTr = 64;  // rotations per side (the library's bound on T_r)

struct Node {  // one queue record: 16 bytes
  int32_t E;
  int32_t link;  // pivot * 1024 + column (column < L: flip, else rotation column - L); -1: the seed
  uint64_t fp;
};

struct RunHead {  // heap element: the run's smallest key, where it is, and the run's live range
  int32_t E;
  int32_t cur;  // arena index of the smallest node
  uint64_t fp;
  int32_t end;    // live nodes are [begin, end)
  int32_t begin;
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
  uint32_t* tables;  // per popped pivot: its C table (2 NG words of int16 pairs) and P_m (ceil(L/2) words)
  int tab_words;
  uint64_t* H;
  const uint64_t* ztab;
  unsigned long long* counter;
};

__device__ __forceinline__ bool kless(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}

// Visited set of one slot (open addressing, linear probing); *err set on an exhausted probe sequence.
// The first compare-and-swap of several keys is issued by the caller, all at once, so that their
// latencies overlap; the _from forms continue a key's probe sequence after a first slot that held
// another key.
__device__ __forceinline__ uint64_t hs_home(uint64_t fp, int log2) { return (fp * kGamma) >> (64 - log2); }
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
__device__ __forceinline__ void hs_insert(uint64_t* H, int log2, uint64_t fp, int* err) {
  const uint64_t s = hs_home(fp, log2);
  const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(&H[s]), (unsigned long long)kEmpty, fp);
  if (old == kEmpty || old == fp) return;
  hs_insert_from(H, log2, fp, s, err);
}
// Insert-if-absent, continuing after slot s (whose key was another one): true when fp was inserted.
__device__ __forceinline__ bool hs_add_from(uint64_t* H, int log2, uint64_t fp, uint64_t s, int* err) {
  const uint64_t mask = (1ull << log2) - 1;
  for (int it = 1; it < kProbeLimit; it++) {
    s = (s + 1) & mask;
    const unsigned long long old =
        atomicCAS(reinterpret_cast<unsigned long long*>(&H[s]), (unsigned long long)kEmpty, fp);
    if (old == kEmpty) return true;
    if (old == fp) return false;
  }
  *err = 1;
  return false;
}
// Insert-if-absent (the key ~0 by the flag has_empty): true when fp was inserted.
__device__ __forceinline__ bool hs_add(uint64_t* H, int log2, uint64_t fp, bool& has_empty, int* err) {
  if (fp == kEmpty) {
    const bool fresh = !has_empty;
    has_empty = true;
    return fresh;
  }
  const uint64_t s = hs_home(fp, log2);
  const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(&H[s]), (unsigned long long)kEmpty, fp);
  if (old == kEmpty) return true;
  if (old == fp) return false;
  return hs_add_from(H, log2, fp, s, err);
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

// The warp's smallest (E, fp) over the lanes' candidates (bi >= 0; keys distinct) and its index, on every
// lane.
__device__ __forceinline__ void warp_argmin(int bE, uint64_t bf, int bi, int& E, uint64_t& fp, int& idx) {
  const int mE = __reduce_min_sync(kFull, bE);
  const unsigned mhi = __reduce_min_sync(kFull, bE == mE ? (unsigned)(bf >> 32) : 0xffffffffu);
  const bool on = bE == mE && (unsigned)(bf >> 32) == mhi;
  const unsigned mlo = __reduce_min_sync(kFull, on ? (unsigned)bf : 0xffffffffu);
  const unsigned who = __ballot_sync(kFull, on && (unsigned)bf == mlo && bi >= 0);
  E = mE;
  fp = ((uint64_t)mhi << 32) | mlo;
  idx = __shfl_sync(kFull, bi, __ffs(who) - 1);
}

// Smallest (E, fp) of arena nodes [begin, end) (non-empty, keys distinct) and its index, on every lane.
__device__ __forceinline__ void run_min(const Node* arena, int begin, int end, int& E, uint64_t& fp, int& idx) {
  int bE = INT32_MAX, bi = -1;
  uint64_t bf = ~0ull;
  for (int i = begin + lane_id(); i < end; i += 32) {
    const Node x = arena[i];
    if (kless(x.E, x.fp, bE, bf)) {
      bE = x.E;
      bf = x.fp;
      bi = i;
    }
  }
  warp_argmin(bE, bf, bi, E, fp, idx);
}

// Per-warp shared memory.
struct __align__(16) IndepSmem {
  ScanSmem s;
  uint32_t pbits[kBitWords];  // the pivot
  uint32_t cbits[kBitWords];  // a child
  int16_t P[kMaxL];  // P_m of the pivot's neighbours
  uint32_t xb[kBitWords];
  int n_surv;
};

__global__ void __launch_bounds__(32 * kIWarps) pq_indep_kernel(IndepArgs a, Layout ly) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  IndepSmem& S = reinterpret_cast<IndepSmem*>(smem_raw)[threadIdx.x >> 5];
  ScanSmem& sm = S.s;
  const int lane = lane_id();
  const long long slot = (long long)blockIdx.x * kIWarps + (threadIdx.x >> 5);
  Node* arena = a.arena + slot * a.arena_cap;
  RunHead* heap = a.heap + slot * a.heap_cap;
  uint64_t* pivots = a.pivots + slot * a.max_exp * a.W;
  uint32_t* tables = a.tables + slot * a.max_exp * a.tab_words;
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
      // ---- pop: the top run's smallest node; the run's last node fills its place, the run's new
      //      smallest by a rescan (warp), then the sift-down (lane 0)
      RunHead h = heap[0];
      const Node nd = arena[h.cur];
      const int pE = nd.E, plink = nd.link;
      const uint64_t pfp = nd.fp;
      __syncwarp();
      if (lane == 0 && h.cur != h.end - 1) arena[h.cur] = arena[h.end - 1];
      __syncwarp();
      h.end--;
      const bool alive = h.end > h.begin;
      if (alive) run_min(arena, h.begin, h.end, h.E, h.fp, h.cur);
      if (lane == 0) {
        if (!alive) {
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
      // ---- the pivot's correlation table and P_m: a flip child's from its parent's (kept with every
      //      popped pivot) by one O(L) update, the seed's and a rotation's from scratch
      if (lane == 0) S.n_surv = 0;
      bool fast;
      uint32_t* ptab = tables + exps * a.tab_words;
      const int pcol = plink & 1023;
      if (plink >= 0 && pcol < a.L) {
        const uint32_t* par = tables + (long long)(plink >> 10) * a.tab_words;
        uint32_t* C16w = reinterpret_cast<uint32_t*>(sm.C16);
        uint32_t* Pw = reinterpret_cast<uint32_t*>(S.P);
        for (int w = lane; w < 2 * ly.NG; w += 32) C16w[w] = par[w];
        for (int w = lane; w < (a.L + 1) / 2; w += 32) Pw[w] = par[2 * ly.NG + w];
        for (int w = lane; w < kBitWords; w += 32) sm.bits[w] = S.cbits[w];  // the parent
        __syncwarp();
        build_bytes(sm, ly);
        // P_m of the child: flipping f changes the product s_f s_{2m-f} of every m != f (pads: 0)
        const int f = pcol + 1;
        const uint8_t* Fc = reinterpret_cast<const uint8_t*>(sm.fwd);
        const int qf = pos_q(ly, f), sf = (int)Fc[qf] - 1;
        for (int m = lane + 1; m <= a.L; m += 32)
          if (m != f) S.P[m - 1] = (int16_t)(S.P[m - 1] - 2 * sf * ((int)Fc[max(2 * pos_q(ly, m) - qf, 0)] - 1));
        __syncwarp();
        table_update(sm, ly, f, &fast);
        if (lane == 0) flip_position(sm, ly, f);
        __syncwarp();
      } else {
        for (int w = lane; w < kBitWords; w += 32) sm.bits[w] = S.pbits[w];
        __syncwarp();
        build_table(sm, ly);
        fast = pack_c8(sm, ly);
        build_bytes(sm, ly);
        p_all(sm, ly, S.xb, S.cbits, S.P);
      }
      const int SC = table_sum(sm, ly);
      {
        const uint32_t* C16w = reinterpret_cast<const uint32_t*>(sm.C16);
        const uint32_t* Pw = reinterpret_cast<const uint32_t*>(S.P);
        for (int w = lane; w < 2 * ly.NG; w += 32) ptab[w] = C16w[w];
        for (int w = lane; w < (a.L + 1) / 2; w += 32) ptab[2 * ly.NG + w] = Pw[w];
      }
      Node* run = arena + top;
      const int link0 = (int)(exps << 10);
      int rE = INT32_MAX, ri = -1;  // this lane's smallest survivor (the run's head comes from these)
      uint64_t rf = ~0ull;
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
          // the tile's Delta E and fingerprints, then an insert-if-absent of each neighbour into the
          // visited set, the first compare-and-swap of all of them in flight at once: a neighbour is a
          // survivor when its key was absent.  Inserting while other neighbours are still tested changes
          // none of their answers: their keys differ, and inserts only fill empty slots, which no probe
          // sequence of a present key crosses.
          int dv[kIM], mv[kIM];
          uint64_t fv[kIM];
          unsigned long long hv[kIM];
#pragma unroll
          for (int j = 0; j < kIM; j++) {
            const SlotInfo si = slot_info(ly, cls, q0 + j);
            mv[j] = si.active ? si.m : 0;
            dv[j] = si.active ? finish_delta(sm, ly, cls, q0 + j, si, acc[j], SC, S.P[si.m - 1]) : 0;
            fv[j] = si.active ? pfp ^ a.ztab[si.m - 1] : kEmpty;
          }
#pragma unroll
          for (int j = 0; j < kIM; j++)
            hv[j] = (mv[j] && fv[j] != kEmpty)
                        ? atomicCAS(reinterpret_cast<unsigned long long*>(&H[hs_home(fv[j], a.H_log2)]),
                                    (unsigned long long)kEmpty, fv[j])
                        : (unsigned long long)kEmpty;
#pragma unroll
          for (int j = 0; j < kIM; j++) {
            if (!mv[j]) continue;
            bool fresh;
            if (fv[j] == kEmpty) {
              fresh = !has_empty;
              has_empty = true;
            } else if (hv[j] == kEmpty || hv[j] == fv[j]) {
              fresh = hv[j] == kEmpty;
            } else {
              fresh = hs_add_from(H, a.H_log2, fv[j], hs_home(fv[j], a.H_log2), &err);
            }
            if (fresh) {
              const int k = atomicAdd(&S.n_surv, 1);
              run[k] = Node{pE + dv[j], link0 | (mv[j] - 1), fv[j]};
              if (kless(pE + dv[j], fv[j], rE, rf)) {
                rE = pE + dv[j];
                rf = fv[j];
                ri = (int)top + k;
              }
            }
          }
        }
      }
      has_empty = __any_sync(kFull, has_empty);
      // ---- the rotations, after the flips: one equal to a flip child or to an earlier rotation finds
      //      its key in the visited set (the same sequence; the smaller column is kept)
      for (int c = 0; c < 2 * a.Tr; c++) {
        rotate_bits(S.pbits, a.L, rshift(a.L, a.Tr, c), S.cbits);
        const int e = energy_bits(S.cbits, a.L);
        const uint64_t hf = fp_bits(S.cbits, a.L, a.ztab);
        if (lane == 0) {
          if (hs_add(H, a.H_log2, hf, has_empty, &err)) {
            const int k = S.n_surv++;
            run[k] = Node{e, link0 | (a.L + c), hf};
            if (kless(e, hf, rE, rf)) {
              rE = e;
              rf = hf;
              ri = (int)top + k;
            }
          }
        }
        __syncwarp();
      }
      has_empty = __any_sync(kFull, has_empty);
      err = __reduce_or_sync(kFull, err);
      const int nu = S.n_surv;
      // ---- best, statistics, the new run
      int E0 = INT32_MAX, i0 = 0;
      uint64_t fp0 = 0;
      if (nu > 0) warp_argmin(rE, rf, ri, E0, fp0, i0);
      if (nu > 0 && E0 < bestE) {
        bestE = E0;
        bestfp = fp0;
        const int col = arena[i0].link & 1023;
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
        const RunHead nh{E0, i0, fp0, (int)(top + nu), (int)top};
        long long i = heap_n;
        while (i > 0) {
          const long long pp = (i - 1) >> 1;
          if (!kless(nh.E, nh.fp, heap[pp].E, heap[pp].fp)) break;
          heap[i] = heap[pp];
          i = pp;
        }
        heap[i] = nh;
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
  a.tab_words = 2 * ly.NG + (L + 1) / 2;
  const size_t per_slot = (size_t)a.arena_cap * sizeof(Node) + (size_t)a.heap_cap * sizeof(RunHead) +
                          (size_t)a.max_exp * W * 8 + (size_t)a.max_exp * a.tab_words * 4 + (8ull << a.H_log2);
  if (cfg->T_r > kMaxTr) return LABS_ERR_INVALID_ARG;
  const size_t smem = sizeof(IndepSmem) * kIWarps;
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
  const size_t oT = take(slots * (size_t)a.max_exp * a.tab_words * 4);
  const size_t oZ = take(8 * (size_t)L), oC = take(8);
  char* base = static_cast<char*>(ws_get(ctx, kWsPqIndep, off));
  if (!base) return LABS_ERR_NOMEM;
  a.arena = reinterpret_cast<Node*>(base + oA);
  a.heap = reinterpret_cast<RunHead*>(base + oHp);
  a.pivots = reinterpret_cast<uint64_t*>(base + oP);
  a.H = reinterpret_cast<uint64_t*>(base + oH);
  a.tables = reinterpret_cast<uint32_t*>(base + oT);
  a.ztab = reinterpret_cast<uint64_t*>(base + oZ);
  a.counter = reinterpret_cast<unsigned long long*>(base + oC);
  indep_ztab_kernel<<<(L + 255) / 256, 256, 0, st>>>(reinterpret_cast<uint64_t*>(base + oZ), L);
  if (cudaMemsetAsync(a.counter, 0, 8, st) != cudaSuccess) return LABS_ERR_CUDA;
  pq_indep_kernel<<<(unsigned)blocks, 32 * kIWarps, smem, st>>>(a, ly);
  return cuda_status(cudaGetLastError());
}

}  // namespace labsg
