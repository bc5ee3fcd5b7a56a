// walk.cu -- step 1 of the dual-step search: Algorithm 1's self-avoiding walks (labs_skew_search,
// labs_batched_search) and the sieve bound E_l (labs_sample_threshold).
//
// GB300 mapping.  The paper runs one walk per thread block with a shared-memory reduction (Fig. 3);
// here one walk is one warp (shuffle/redux reductions, no block barriers) and a persistent grid pulls
// work items (length, walk) from a device counter, so walks of different lengths and lengths of
// different cost balance across the 152 SMs in one launch.  Each warp's state (sequence bits, byte
// windows, correlation table, Bloom filter of 2^bloom_log2 bits, per-neighbour slots) lives in its
// shared-memory slab; a step is
//   scan   -- Delta E of every free neighbour (tiled dp4a loop, labs_core.cuh),
//   select -- group argmin of (Delta E, m); Bloom test of the winner's fingerprint; on a hit the owner
//             lane puts its second best in its place and the argmin repeats (same result as testing
//             them all),
//   apply  -- O(L) table update, O(1)-per-neighbour P update, byte/bit flips, fingerprint, Bloom insert,
//   sieve  -- the walk's R best distinct (E, fp) states with E <= E_thr, one per lane.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kMaxLens = 96;    // lengths in one launch (kernel parameter table)
constexpr int kMaxPasses = 3;   // lane passes over the tasks of one walk
// per slot and lane: slot word and choice key (int32 each), plus Delta E when the choice is biased
__host__ __device__ constexpr int slot_bytes(bool biased) { return biased ? 12 : 8; }
// threads per block the kernels are compiled for: whole-warp walks run two 8-warp blocks per SM (128
// registers a thread); half-warp walks run one block of up to 12 warps (24 walks), whose register budget,
// 65536 / 384 threads, holds the whole step without spills
__host__ __device__ constexpr int walk_block_threads(int GL) { return GL == 32 ? 256 : 384; }
__host__ __device__ constexpr int walk_min_blocks(int GL) { return GL == 32 ? 2 : 1; }

// Shared-memory slab of one walk, sized per launch for its lengths (byte offsets, 16-byte aligned):
// the sequence bits at 0, the tables, the byte-window arrays, the Bloom filter and the per-slot words
// ([slot][lane of the group]).
struct SlabPlan {
  int off_C16, off_C8, off_fwd, off_bwd, off_bloom, off_slots, bytes;
};

// Per-length entry of a launch: the layout (tiles, windows) and where its walks sit among the items.
struct LenEntry {
  Layout ly;
  int T_i;
  int32_t E_thr_value;  // used when WalkParams::E_thr_dev is null
  int64_t item_begin;   // first work item of this length
  int64_t walk_begin;   // global walk id of its first walk
};

struct WalkParams {
  int n_len, R, bloom_log2, bloom_k, prefix_words, n_prefix, slot_stride;
  int32_t E_target;
  int64_t n_items, flip_budget;
  uint64_t seed;
  const uint64_t* prefixes;
  const int32_t* E_thr_dev;  // nullable: per-length sieve bounds in device memory
  labs_candidate* out;       // [n_items][R]
  int64_t* walk_stats;       // nullable: [n_items][6]
  labs_walk_stats* stats;
  unsigned long long* counter;
  // resumable chunks (learned proposal); all nullable / zero for a plain run to the end
  unsigned char* state;  // [n_items][state_stride] walk states between launches
  int state_stride;
  int chunk;             // > 0: at most `chunk` accepted flips per walk and launch; < 0: set-up only
  const float* bias;     // [n_items][L] proposal logits biasing the choice (null: plain walk)
  float lambda;
  uint64_t* seq_out;     // [n_items][W]: the walk's sequence when the launch leaves it
  int32_t* move_log;     // [n_items][2]: first move of the launch (position, Delta E), (-1, 0) if none
  SlabPlan slab;
  LenEntry len[kMaxLens];
};

// Header of a saved walk state; followed by the sequence bits, the int16 table and the Bloom filter.
struct WalkStateHdr {
  unsigned long long fp;
  long long skips;
  int E, flips, segs, dead, it, mprev, first_hit, bestE, need_start, started, done, pad[5];
};
constexpr int kStateBits = sizeof(WalkStateHdr);
constexpr int kStateC = kStateBits + 4 * kBitWords;
constexpr int kStateBloom = kStateC + 2 * kCLen;
constexpr int kStateBytes = kStateBloom + 4 * 1024;

// Order-preserving int32 image of a float (-0 folded onto +0 first).
__device__ __forceinline__ int float_key(float f) {
  const int i = __float_as_int(f + 0.0f);
  return i ^ ((i >> 31) & 0x7fffffff);
}

__device__ __forceinline__ uint32_t bloom_idx(uint64_t fp, int j, uint32_t mask) {
  uint32_t lo = (uint32_t)fp, hi = (uint32_t)(fp >> 32);
  return (lo + (uint32_t)j * (hi | 1u)) & mask;
}

// Every lane of the group returns whether all K probes of fp are set.
template <int GL>
__device__ __forceinline__ bool bloom_test(const uint32_t* bloom, uint64_t fp, int K, uint32_t mask) {
  const int lane = glane<GL>();
  bool hit = true;
  if (lane < K) {
    uint32_t b = bloom_idx(fp, lane, mask);
    hit = (bloom[b >> 5] >> (b & 31)) & 1u;
  }
  return gall<GL>(hit);
}

template <int GL>
__device__ __forceinline__ void bloom_add(uint32_t* bloom, uint64_t fp, int K, uint32_t mask) {
  const int lane = glane<GL>();
  if (lane < K) {
    uint32_t b = bloom_idx(fp, lane, mask);
    atomicOr(&bloom[b >> 5], 1u << (b & 31));
  }
  gsync<GL>();
}

__device__ __forceinline__ bool key_less(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}

// Slot word of one neighbour: high half the signed position s_m * m (0: no neighbour in this slot), low
// half alpha^2 Q_m, where Q_m = sum of y_kappa^2 over the valid lags = n_f + n_b - [pair] + 2 P_m.  It is
// a sum of squares, so 0 <= alpha^2 Q_m <= 16 * 4 * 287 < 2^16 for every L <= 576.
__device__ __forceinline__ int slot_pack(int sm_m, int Pt) { return (int)(((unsigned)sm_m << 16) | (unsigned)Pt); }
__device__ __forceinline__ int slot_pos(int word) { return word >> 16; }  // s_m * m
__device__ __forceinline__ int slot_Pt(int word) { return word & 0xffff; }

// Delta E of a neighbour from its accumulator a = sum_g C8/C16 (y + 2) and the table sum SC:
//   Delta E = base - 2 alpha s_m (a - 2 SC),   base = alpha^2 Q_m + 2 alpha sigma C_{gd} [pair],
// alpha = 4 for a skew pair (m, m'), 2 otherwise; the pair's own product at lag gd = c - m is removed
// with s_{m'} = sigma s_m, sigma = (-1)^{c-m} (Eq. 2).  base depends only on the table and the slot
// word, so it is formed before the scan (prep_code).

// The last accepted move, not yet folded into the slot words: its flipped positions f0 (and the mirror
// f1 of a skew pair), their class and class indices, and their values before the flip.  Flipping f
// changes the product s_{2m-f} s_f of every neighbour m of f's class by -2 s_f s_{2m-f}; the byte at
// class index 2q - q_f gives s_{2m-f}, and the pads (s = 0) drop products with an end outside 1..L.
// That byte is never one of the flipped positions for the neighbours that change, so the update may be
// applied after the flip, when the next step reads the slot anyway.  Excluded: the flipped neighbour
// itself (its products do not contain s_m; its sign changes), the skew centre when a pair flips (both
// ends of each of its products flip), and the pair product (m, m') of m, whose end m' is 2m - f0 when
// 3 q - q_f0 = c + 6 - b (b = 1 for odd positions, 2 for even).
struct PendingFlip {
  bool on, pair;
  int cls, q0f, q1f, s0, s1, qmir;
};

// Folds the pending move into the slot words of its class.  The class's (task, k) slots are spread over
// the group's lanes, task fastest, so that neighbouring lanes touch different banks.
template <int M, int H, int GL, class S>
__device__ __forceinline__ void fold_flip(const S& sm, const Layout& ly, const PendingFlip& pf, int* sl_w) {
  constexpr int MH = M / H;
  const uint8_t* Fc = reinterpret_cast<const uint8_t*>(sm.fwd + cls_words(ly, pf.cls));
  const int pmul = ly.skew ? -64 : -16;  // -4 alpha^2 for the neighbours that change
  const int qc = (pf.pair && pos_cls(ly, ly.c) == pf.cls) ? pos_q(ly, ly.c) : -1;  // the centre
  const int m3 = ly.skew ? pf.qmir + pf.q0f : -1;                                  // 3 q of the pair-product
  const int qm = (m3 >= 0 && m3 % 3 == 0) ? m3 / 3 : -1;                           // exclusion
  const int q1f = pf.pair ? pf.q1f : (1 << 20);  // single flip: the f1 term reads a pad
  const int nt = ly.ntiles[pf.cls] * H;          // tasks of the class
  const int task0 = (pf.cls ? ly.ntiles[0] : 0) * H;
  const int qt = ly.tile_first[pf.cls];
  const int mg = ly.fold_magic[pf.cls];
  const int lane = glane<GL>();
  int k = (lane * mg) >> 16, tl = lane - k * nt;
  const int step_k = (GL * mg) >> 16, step_t = GL - step_k * nt;
  for (; k < MH;) {
    const int task = task0 + tl;
    const int q = qt + (tl / H) * M + (tl % H) * MH + k;
    const int idx = ((task / GL) * MH + k) * GL + (task % GL);
    int wv = sl_w[idx];
    const int ms = slot_pos(wv);
    int v = ((int)Fc[max(2 * q - pf.q0f, 0)] - 1) * pf.s0;
    if (q == qm) v = 0;
    v += ((int)Fc[max(2 * q - q1f, 0)] - 1) * pf.s1;
    if (ms != 0 && q != pf.q0f && q != qc) wv += pmul * v;
    if (ms != 0 && q == pf.q0f) wv = slot_pack(-ms, slot_Pt(wv));
    sl_w[idx] = wv;
    tl += step_t;
    k += step_k;
    if (tl >= nt) {
      tl -= nt;
      k++;
    }
  }
  gsync<GL>();
}

// Finish code of a slot, formed by prep: base * 32 + code, where base is the constant part of the
// neighbour's Delta E and code = 2 alpha s_m + 8 (0, 4, 12 or 16), plus 1 for the neighbour
// the last move flipped (the state just left), or 31 for no neighbour.  Branch-free: a slot without a
// pair term reads the table's last entry, which is always zero (lags beyond G).
constexpr int kNoSlot = 31;
template <class S>
__device__ __forceinline__ int prep_code(const S& sm, const Layout& ly, int word, bool back) {
  const int ms = slot_pos(word);
  const int m = ms < 0 ? -ms : ms;
  const bool pair = ly.skew && m != ly.c && m != 0;
  const int gd = pair ? ly.c - m : ly.cl;
  const int cg = 8 * (int)sm.C16[gd - 1];
  const int base = slot_Pt(word) + ((gd & 1) ? -cg : cg);
  const int a2 = pair ? 8 : 4;
  const int code = (ms < 0 ? 8 - a2 : 8 + a2) + (back ? 1 : 0);
  return ms == 0 ? kNoSlot : base * 32 + code;
}

// Task of group lane `lane` in pass `ps`: tile (class, q0), lag range h, whether it exists.
template <int GL>
__device__ __forceinline__ bool lane_task(const Layout& ly, int H, int ps, int lane, int& cls, int& q0, int& h) {
  const int task = ps * GL + lane;
  h = H == 2 ? (task & 1) : 0;
  cls = 0;
  q0 = 0;
  if (task >= ly.n_tasks) return false;
  tile_of(ly, H == 2 ? (task >> 1) : task, cls, q0);
  return true;
}

// One walk-step kernel for every length of the launch.  Template: tile size M and lag ranges per tile H
// (the autotuned "words per thread"), lanes per walk GL (32: one walk per warp; 16: one per half-warp,
// two walks sharing every instruction of the step's serial phases); the number of lane passes is per
// length (<= kMaxPasses).  Per-slot state sits in the walk's slab, lane-major ([slot][lane], conflict
// free): the slot word, the step's choice key and, for biased walks, its Delta E.  With `state` the walk
// runs in chunks of accepted flips and is saved between launches (bits, table, Bloom filter, counters);
// the sieve slots stay in the output records meanwhile.
// ONE: a single-length launch -- the length's entry is read at a fixed parameter offset and its
// Zobrist keys are tabulated once per block in shared memory.  BIASED: the choice key is the proposal
// score of WalkParams::bias (single-length launches only).
template <int M, int H, bool ONE, bool BIASED, int GL>
__global__ void __launch_bounds__(walk_block_threads(GL), walk_min_blocks(GL))
    walk_kernel(const __grid_constant__ WalkParams P) {
  constexpr int MH = M / H;  // slots owned by a lane per pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gid = threadIdx.x / GL;  // walk slot of this group in the block
  const int ngroups = blockDim.x / GL;
  unsigned char* slab = smem_raw + (size_t)gid * P.slab.bytes;
  ScanView sm;
  sm.bits = reinterpret_cast<uint32_t*>(slab);
  sm.C16 = reinterpret_cast<int16_t*>(slab + P.slab.off_C16);
  sm.C8 = reinterpret_cast<int8_t*>(slab + P.slab.off_C8);
  sm.fwd = reinterpret_cast<uint32_t*>(slab + P.slab.off_fwd);
  sm.bwd = reinterpret_cast<uint32_t*>(slab + P.slab.off_bwd);
  uint32_t* bloom = reinterpret_cast<uint32_t*>(slab + P.slab.off_bloom);
  uint64_t* ztab = reinterpret_cast<uint64_t*>(smem_raw + (size_t)P.slab.bytes * ngroups);
  if (ONE) {
    const uint64_t zk = stream_key(0, kPurposeZobrist, (uint64_t)P.len[0].ly.L, 0);
    for (int i = threadIdx.x; i < P.len[0].ly.L; i += blockDim.x) ztab[i] = zobrist(zk, i + 1);
    __syncthreads();
  }
  int* sl_w = reinterpret_cast<int*>(slab + P.slab.off_slots);  // slot words
  int* sl_k = sl_w + P.slot_stride * GL;                         // choice keys of the step
  int* sl_d = sl_k + P.slot_stride * GL;                         // Delta E of the step (BIASED only; else = key)
  const int lane = glane<GL>();
  const uint32_t bmask = (1u << P.bloom_log2) - 1u;
  const int bwords = 1 << (P.bloom_log2 - 5);
  const int R = P.R;
  const unsigned budget = (unsigned)P.flip_budget;  // < 2^32, checked by the host

  long long agg_flips = 0, agg_segs = 0, agg_skips = 0, agg_dead = 0;
  int agg_best = INT32_MAX;

  while (true) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(P.counter, 1ull);
    item = gshfl<GL>(item, 0);
    if ((long long)item >= P.n_items) break;
    int li = 0;
    if (!ONE)
      while (li + 1 < P.n_len && P.len[li + 1].item_begin <= (long long)item) li++;
    const LenEntry& le = ONE ? P.len[0] : P.len[li];
    const Layout& ly = le.ly;
    const int64_t w = le.walk_begin + ((long long)item - le.item_begin);
    const uint64_t* prefix = P.prefixes + (w % P.n_prefix) * P.prefix_words;
    const uint64_t zkey = stream_key(0, kPurposeZobrist, (uint64_t)ly.L, 0);
    const int32_t E_thr = P.E_thr_dev ? P.E_thr_dev[li] : le.E_thr_value;
    const int W = (ly.L + 63) >> 6;
    const int NP = (ly.n_tasks + GL - 1) / GL;
    const int S = NP * MH;
    labs_candidate* rec = P.out + (int64_t)item * R;
    const float* bias = BIASED ? P.bias + (long long)item * ly.L : nullptr;
    WalkStateHdr* gh = P.state ? reinterpret_cast<WalkStateHdr*>(P.state + (size_t)item * P.state_stride) : nullptr;
    if (gh && gh->done) continue;
    const bool resumed = gh && gh->started;

    // slot positions of this length
    for (int ps = 0; ps < NP; ps++) {
      int cls, q0, h;
      const bool has = lane_task<GL>(ly, H, ps, lane, cls, q0, h);
#pragma unroll
      for (int k = 0; k < MH; k++) {
        const int m = q_pos(ly, cls, q0 + h * MH + k);
        sl_w[(ps * MH + k) * GL + lane] = slot_pack((has && m >= ly.p + 1 && m <= ly.mlast) ? m : 0, 0);
      }
    }
    int cE = INT32_MAX;
    uint64_t cfp = ~0ull;
    int wE = INT32_MAX;
    uint64_t wfp = ~0ull;
    int wlane = 0;
    unsigned flips = 0, segs = 0, dead = 0;
    long long skips = 0;
    int first_hit = -1;
    int bestE = INT32_MAX;
    int E = 0, SC = 0, it = 0;
    int mprev = 0;  // free position flipped by the previous move of this segment
    uint64_t fp = 0;
    bool fast = true, need_start = true;
    PendingFlip pend;
    pend.on = false;

    // rebuilds everything derived from the bits and the table: windows, int8 table, slot P and signs
    auto derive = [&]() {
      SC = table_sum<GL>(sm, ly);
      fast = pack_c8<GL>(sm, ly);
      build_bytes<GL>(sm, ly);
      for (int t = 0; t < S; t++) {
        int m = slot_pos(sl_w[t * GL + lane]);
        m = m < 0 ? -m : m;
        int word = 0;
        if (m) {
          const SlotInfo si = slot_info(ly, pos_cls(ly, m), pos_q(ly, m));
          const int Pm = p_from_scratch(sm, ly, pos_cls(ly, m), pos_q(ly, m), si);
          const int a2 = si.pair ? 16 : 4;
          word = slot_pack(s_at(sm, ly, m) * m, a2 * (si.nf + si.nb - si.pair + 2 * Pm));
        }
        sl_w[t * GL + lane] = word;
      }
      pend.on = false;
    };
    // INIT_PARTITIONED_SEQUENCE of a new segment (Algorithm 1)
    auto start_segment = [&]() {
      for (int t = lane; t < bwords; t += GL) bloom[t] = 0u;
      build_start<GL>(sm, ly, prefix, stream_key(P.seed, kPurposeWalk, (uint64_t)w, (uint64_t)segs));
      segs++;
      fp = fingerprint<GL>(sm, ly.L, zkey);
      bloom_add<GL>(bloom, fp, P.bloom_k, bmask);
      E = build_table<GL>(sm, ly);
      derive();
      it = 0;
      mprev = 0;
      need_start = false;
    };
    // new worst sieve slot: largest (E, fp), lowest lane among equals
    auto find_worst = [&]() {
      int mE = gmax<GL>(lane < R ? cE : INT32_MIN);
      uint64_t mf = (lane < R && cE == mE) ? cfp : 0ull;
#pragma unroll
      for (int o = GL / 2; o > 0; o >>= 1) {
        uint64_t other = gshfl_xor<GL>(mf, o);
        mf = other > mf ? other : mf;
      }
      unsigned who = gballot<GL>(lane < R && cE == mE && cfp == mf);
      wE = mE;
      wfp = mf;
      wlane = __ffs(who) - 1;
    };

    if (!resumed) {
      for (int r = lane; r < R; r += GL) {  // empty sieve slots
        rec[r].E = INT32_MAX;
        rec[r].walk = 0;
        rec[r].step = 0;
        rec[r].pad = 0;
        rec[r].fp = ~0ull;
#pragma unroll
        for (int t = 0; t < LABS_MAX_W; t++) rec[r].seq[t] = 0;
      }
    } else {
      flips = gh->flips;
      segs = gh->segs;
      dead = gh->dead;
      skips = gh->skips;
      first_hit = gh->first_hit;
      bestE = gh->bestE;
      need_start = gh->need_start;
      it = gh->it;
      mprev = gh->mprev;
      E = gh->E;
      fp = gh->fp;
      if (lane < R) {
        cE = rec[lane].E;
        cfp = rec[lane].fp;
      }
      find_worst();
      if (!need_start) {
        const unsigned char* gb = reinterpret_cast<const unsigned char*>(gh);
        for (int t = lane; t < kBitWords; t += GL) sm.bits[t] = reinterpret_cast<const uint32_t*>(gb + kStateBits)[t];
        for (int t = lane; t < ly.cl / 2; t += GL)
          reinterpret_cast<uint32_t*>(sm.C16)[t] = reinterpret_cast<const uint32_t*>(gb + kStateC)[t];
        for (int t = lane; t < bwords; t += GL) bloom[t] = reinterpret_cast<const uint32_t*>(gb + kStateBloom)[t];
        gsync<GL>();
        derive();
      }
    }
    const unsigned flips0 = flips, segs0 = segs, dead0 = dead;
    const long long skips0 = skips;
    const unsigned chunk = P.chunk > 0 ? (unsigned)P.chunk : (P.chunk < 0 ? 0u : 0xffffffffu);
    if (P.chunk < 0 && need_start && flips < budget) start_segment();  // set-up launch: first state only
    unsigned taken = 0;

    while (flips < budget && taken < chunk) {
      if (need_start) start_segment();
      it++;
      if (pend.on) {  // the last move's P bookkeeping
        fold_flip<M, H, GL>(sm, ly, pend, sl_w);
        pend.on = false;
      }
      // ---- scan; each lane keeps its two best (key, m), where key orders the choice: Delta E, or the
      //      biased score Delta E - lambda * logit[m] mapped to an order-preserving integer (a Bloom hit on
      //      its best then hands over the second without a rescan of the lane's slots)
      int bk = INT32_MAX, bm = INT32_MAX, bdE = 0;
      int bk2 = INT32_MAX, bm2 = INT32_MAX, bd2 = 0;
      bool have2 = true;
      int kprev = INT32_MAX;  // this lane's key of the move back (only its owner sets it)
      for (int ps = 0; ps < NP; ps++) {
        int cls, q0, h;
        const bool has = lane_task<GL>(ly, H, ps, lane, cls, q0, h);
        const int q_first = q0 + h * MH;
        {
          // prep, while no accumulator is live: park each neighbour's Delta E base with its finish code
          // in the key array
          int wv[MH];
#pragma unroll
          for (int k = 0; k < MH; k++) wv[k] = sl_w[(ps * MH + k) * GL + lane];
          // the move back: the neighbour flipped by the previous move of this segment
          const int kback = (mprev && pos_cls(ly, mprev) == cls) ? pos_q(ly, mprev) - q_first : -1;
#pragma unroll
          for (int k = 0; k < MH; k++)
            sl_k[(ps * MH + k) * GL + lane] = prep_code(sm, ly, wv[k], k == kback);
        }
        int acc[M];
#pragma unroll
        for (int j = 0; j < M; j++) acc[j] = 0;
        if (has) {
          // one lag range per tile: only the groups that hold lags (the layout pads the range to whole
          // ring turns and the table is zero beyond G); two ranges keep their padded turns, since the
          // two lanes of a tile run in step and the longer range sets the time anyway
          const int u_begin = h ? ly.NGh : 0;
          const int u_end = H == 1 ? min(ly.NGh, ly.NG) : (h ? ly.NGend : ly.NGh);
          if (fast)
            scan_range<M, false>(sm, ly, cls, q0, u_begin, u_end, acc);
          else
            scan_range<M, true>(sm, ly, cls, q0, u_begin, u_end, acc);
        }
        // H = 2: the two lanes of a tile hold partial sums over the two lag ranges, and each needs the
        // totals of its own MH slots only: it sends the partner's half and adds what it receives
        if (H == 2) {
#pragma unroll
          for (int k = 0; k < MH; k++) {
            const int send = h ? acc[k] : acc[MH + k];
            const int keep = h ? acc[MH + k] : acc[k];
            acc[k] = keep + gshfl_xor<GL>(send, 1);
          }
        }
        // finish: keys of this pass's neighbours, then their two smallest (below)
        const int m_first = q_pos(ly, cls, q_first);
        int kv[MH], mv[MH], dv[MH];
#pragma unroll
        for (int k = 0; k < MH; k++) {
          const int t = ps * MH + k;
          const int pk = sl_k[t * GL + lane];
          const int code = pk & 31;
          const int m = m_first + ly.lam * k;
          const int a = acc[k];
          const int d = (pk >> 5) - ((code & 30) - 8) * (a - 2 * SC);
          int key = d;
          if (BIASED) {
            float l = bias[min(max(m, 1), ly.L) - 1];
            if (!isfinite(l)) l = 0.f;  // a missing or broken proposal falls back to the plain choice
            key = float_key(fmaf(-P.lambda, l, (float)d));
          }
          if (code == kNoSlot) {
            key = INT32_MAX;
          } else if (code & 1) {
            kprev = key;  // the state just left: certainly in the Bloom filter
            key = INT32_MAX;
          }
          sl_k[t * GL + lane] = key;
          if (BIASED) sl_d[t * GL + lane] = d;
          kv[k] = key;
          mv[k] = m;
          dv[k] = d;
        }
        // the pass's two smallest (key, m): slots come in increasing m, so strict comparisons keep the
        // smaller m ahead among equal keys
        int p1 = INT32_MAX, q1 = INT32_MAX, e1 = 0, p2 = INT32_MAX, q2 = INT32_MAX, e2 = 0;
#pragma unroll
        for (int k = 0; k < MH; k++) {
          const bool lt1 = kv[k] < p1, lt2 = kv[k] < p2;
          p2 = lt1 ? p1 : (lt2 ? kv[k] : p2);
          q2 = lt1 ? q1 : (lt2 ? mv[k] : q2);
          if (BIASED) e2 = lt1 ? e1 : (lt2 ? dv[k] : e2);
          p1 = lt1 ? kv[k] : p1;
          q1 = lt1 ? mv[k] : q1;
          if (BIASED) e1 = lt1 ? dv[k] : e1;
        }
        if (!BIASED) {
          e1 = p1;
          e2 = p2;
        }
        // merge with the earlier passes' two (a later pass may hold smaller m only in another class)
        auto before = [](int ka, int ma, int kb, int mb) { return ka < kb || (ka == kb && ka != INT32_MAX && ma < mb); };
        if (before(p1, q1, bk, bm)) {
          const bool sec = before(bk, bm, p2, q2);  // the old best stays second unless the pass's second is smaller
          bk2 = sec ? bk : p2;
          bm2 = sec ? bm : q2;
          bd2 = sec ? bdE : e2;
          bk = p1;
          bm = q1;
          bdE = e1;
        } else if (before(p1, q1, bk2, bm2)) {
          bk2 = p1;
          bm2 = q1;
          bd2 = e1;
        }
      }
      // ---- select: smallest (key, m) whose neighbour is not in the Bloom filter
      int mstar = -1, kstar = 0, dstar = 0;
      uint64_t nfp = 0;
      for (int guard = 0; guard <= S * GL; guard++) {
        int kmin, mm;
        if (!BIASED) {
          // one reduction on (key, m) while the minimum key is inside the 22-bit window: a key clamped to
          // the window's edge can only tie with the minimum when the minimum is at that edge itself
          constexpr int kHalf = 1 << 21;
          const unsigned comp = bk == INT32_MAX ? 0xffffffffu
                                                : ((unsigned)(min(max(bk, -kHalf), kHalf - 1) + kHalf) << 10) | (unsigned)bm;
          const unsigned cmin = gminu<GL>(comp);
          if (cmin == 0xffffffffu) break;
          kmin = (int)(cmin >> 10) - kHalf;
          mm = (int)(cmin & 1023u);
          if (kmin == -kHalf || kmin == kHalf - 1) {
            kmin = gmin<GL>(bk);
            mm = (int)gminu<GL>(bk == kmin ? (unsigned)bm : 0xffffffffu);
          }
        } else {
          kmin = gmin<GL>(bk);
          if (kmin == INT32_MAX) break;
          mm = (int)gminu<GL>(bk == kmin ? (unsigned)bm : 0xffffffffu);
        }
        const bool mine = bk == kmin && bm == mm;
        int dmm = kmin;  // the plain choice key is Delta E itself
        if (BIASED) dmm = gshfl<GL>(bdE, __ffs(gballot<GL>(mine)) - 1);
        uint64_t cand = fp ^ (ONE ? ztab[mm - 1] : zobrist(zkey, mm));
        if (ly.skew && mm != ly.c) cand ^= ONE ? ztab[ly.L - mm] : zobrist(zkey, ly.L + 1 - mm);
        if (!bloom_test<GL>(bloom, cand, P.bloom_k, bmask)) {
          mstar = mm;
          kstar = kmin;
          dstar = dmm;
          nfp = cand;
          break;
        }
        skips++;
        if (mine && have2) {
          // the owner lane's next best is its second
          bk = bk2;
          bm = bm2;
          bdE = bd2;
          have2 = false;
        } else if (mine) {
          // the owner lane's next best: smallest key ranked after (kmin, mm); keys ranked ahead were
          // dropped earlier in this step
          bk = INT32_MAX;
          int nbm = INT32_MAX, nbd = 0;
          for (int t = 0; t < S; t++) {
            const int key = sl_k[t * GL + lane];
            const int ms = slot_pos(sl_w[t * GL + lane]);
            const int m = ms < 0 ? -ms : ms;
            if (key == INT32_MAX) continue;
            if (key < kmin || (key == kmin && m <= mm)) continue;
            if (key < bk || (key == bk && m < nbm)) {
              bk = key;
              nbm = m;
              nbd = BIASED ? sl_d[t * GL + lane] : key;
            }
          }
          bm = nbm;
          bdE = nbd;
        }
      }
      // the move back ranked ahead of the chosen move: count it as a Bloom skip
      if (gany<GL>(kprev != INT32_MAX && (mstar < 0 || kprev < kstar || (kprev == kstar && mprev < mstar))))
        skips++;
      if (mstar < 0) {
        dead++;
        need_start = true;
        continue;
      }
      // ---- apply; the slot words take the move at the next scan (fold_flip)
      pend.on = true;
      pend.pair = ly.skew && mstar != ly.c;
      pend.cls = pos_cls(ly, mstar);
      pend.q0f = pos_q(ly, mstar);
      pend.s0 = s_at(sm, ly, mstar);
      pend.q1f = pend.pair ? pos_q(ly, ly.L + 1 - mstar) : 0;  // the mirror has the class of m*
      pend.s1 = pend.pair ? s_at(sm, ly, ly.L + 1 - mstar) : 0;
      pend.qmir = ly.c + 6 - (pend.cls ? 1 : 2);
      mprev = mstar;
      SC += table_update<GL>(sm, ly, mstar, &fast);
      if (lane == 0) flip_position(sm, ly, mstar);
      if (lane == 1 && pend.pair) flip_position(sm, ly, ly.L + 1 - mstar);
      gsync<GL>();
      E += dstar;
      fp = nfp;
      bloom_add<GL>(bloom, fp, P.bloom_k, bmask);
      flips++;
      taken++;
      if (taken == 1 && P.move_log && lane == 0) {
        P.move_log[2 * item] = mstar;
        P.move_log[2 * item + 1] = dstar;
      }
      if (E < bestE) bestE = E;
      if (first_hit < 0 && E <= P.E_target) first_hit = (int)flips;
      // ---- sieve
      if (E <= E_thr && key_less(E, fp, wE, wfp)) {
        bool dup = gany<GL>(lane < R && cE != INT32_MAX && cfp == fp);
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
          find_worst();
        }
      }
      if (it >= le.T_i) need_start = true;
    }
    if (P.move_log && taken == 0 && lane == 0) {
      P.move_log[2 * item] = -1;
      P.move_log[2 * item + 1] = 0;
    }
    if (P.seq_out && lane < W)
      P.seq_out[(size_t)item * W + lane] = (uint64_t)sm.bits[2 * lane] | ((uint64_t)sm.bits[2 * lane + 1] << 32);

    if (flips < budget) {
      // ---- leave the walk for the next launch
      if (gh) {
        unsigned char* gb = reinterpret_cast<unsigned char*>(gh);
        for (int t = lane; t < kBitWords; t += GL) reinterpret_cast<uint32_t*>(gb + kStateBits)[t] = sm.bits[t];
        for (int t = lane; t < ly.cl / 2; t += GL)
          reinterpret_cast<uint32_t*>(gb + kStateC)[t] = reinterpret_cast<const uint32_t*>(sm.C16)[t];
        for (int t = lane; t < bwords; t += GL) reinterpret_cast<uint32_t*>(gb + kStateBloom)[t] = bloom[t];
        if (lane == 0) {
          gh->fp = fp;
          gh->skips = skips;
          gh->E = E;
          gh->flips = (int)flips;
          gh->segs = (int)segs;
          gh->dead = (int)dead;
          gh->it = it;
          gh->mprev = mprev;
          gh->first_hit = first_hit;
          gh->bestE = bestE;
          gh->need_start = need_start ? 1 : 0;
          gh->started = 1;
          gh->done = 0;
        }
      }
    } else {
      // ---- final: sort the R slots by (E, fp) (ties between empty slots by lane) and rewrite in place
      int rank = 0;
      for (int r = 0; r < R; r++) {
        int oE = gshfl<GL>(cE, r);
        uint64_t of = gshfl<GL>(cfp, r);
        if (key_less(oE, of, cE, cfp) || (oE == cE && of == cfp && r < lane)) rank++;
      }
      gsync<GL>();
      labs_candidate mine;
      if (lane < R) mine = rec[lane];
      gsync<GL>();
      if (lane < R) rec[rank] = mine;
      gsync<GL>();
      if (P.walk_stats && lane == 0) {
        int64_t* st = P.walk_stats + (int64_t)item * 6;
        st[0] = (int64_t)flips;
        st[1] = (int64_t)segs;
        st[2] = skips;
        st[3] = (int64_t)dead;
        st[4] = bestE;
        st[5] = first_hit;
      }
      if (gh && lane == 0) {
        gh->done = 1;
        gh->started = 1;
      }
    }
    gsync<GL>();
    agg_flips += flips - flips0;
    agg_segs += segs - segs0;
    agg_skips += skips - skips0;
    agg_dead += dead - dead0;
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

// Zeroes the aggregates and the work counter; E_thr reports the first length's sieve bound.
__global__ void walk_init_kernel(labs_walk_stats* stats, const int32_t* E_thr_dev, int32_t E_thr_value,
                                 unsigned long long* counter) {
  stats->flips = 0;
  stats->segments = 0;
  stats->bloom_skips = 0;
  stats->dead_ends = 0;
  stats->E_thr = E_thr_dev ? E_thr_dev[0] : E_thr_value;
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

struct Variant {
  int M, H, GL;  // tile, lag ranges per tile, lanes per walk
};
static const Variant kVariants[] = {{8, 1, 32}, {12, 1, 32}, {16, 1, 32}, {16, 2, 32},
                                    {8, 1, 16}, {12, 1, 16}, {16, 1, 16}, {16, 2, 16}};

// Passes a length needs with variant v (0 if the layout does not fit).
static int passes_for(int L, int skew, int p, const Variant& v) {
  Layout ly;
  if (!make_layout(ly, L, skew, p, v.M, v.H)) return 0;
  int np = (ly.n_tasks + v.GL - 1) / v.GL;
  return np < 1 ? 1 : np;
}

// Bytes of a launch's dynamic shared memory: the walks' slabs and, for single-length launches, the
// Zobrist table.
static size_t walk_smem(const WalkParams& P, int walks_per_block) {
  return (size_t)P.slab.bytes * (size_t)walks_per_block + (P.n_len == 1 ? sizeof(uint64_t) * (size_t)P.len[0].ly.L : 0);
}

template <int M, int H, int GL>
int walk_t(labs_ctx* ctx, const WalkParams& P, int warps, cudaStream_t st, bool configure, long long* blocks) {
  const bool one = P.n_len == 1, biased = P.bias != nullptr;
  if (biased && !one) return LABS_ERR_INVALID_ARG;
  if (32 * warps > walk_block_threads(GL)) return LABS_ERR_INVALID_ARG;
  const size_t smem = walk_smem(P, warps * (32 / GL));
  auto kern = !one ? walk_kernel<M, H, false, false, GL>
                   : biased ? walk_kernel<M, H, true, true, GL> : walk_kernel<M, H, true, false, GL>;
  if (configure) {
    if (smem > ctx->smem_optin) return LABS_ERR_INVALID_ARG;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return LABS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem) != cudaSuccess || per_sm < 1)
      return LABS_ERR_CUDA;
    long long b = (long long)per_sm * ctx->num_sms;
    const long long walks_per_block = (long long)warps * (32 / GL);
    const long long need = (P.n_items + walks_per_block - 1) / walks_per_block;
    if (b > need) b = need;
    *blocks = b < 1 ? 1 : b;
    return LABS_OK;
  }
  kern<<<(unsigned)*blocks, 32 * warps, smem, st>>>(P);
  return cuda_status(cudaGetLastError());
}

// configure = true: sets the kernel's shared-memory limit and sizes the persistent grid (*blocks);
// configure = false: launches with that grid (no runtime call besides the launch itself).
static int walk_variant(labs_ctx* ctx, const WalkParams& P, const Variant& v, int warps, cudaStream_t st,
                        bool configure, long long* blocks) {
  switch (v.M * 1000 + v.H * 100 + v.GL) {
    case 8132: return walk_t<8, 1, 32>(ctx, P, warps, st, configure, blocks);
    case 12132: return walk_t<12, 1, 32>(ctx, P, warps, st, configure, blocks);
    case 16132: return walk_t<16, 1, 32>(ctx, P, warps, st, configure, blocks);
    case 16232: return walk_t<16, 2, 32>(ctx, P, warps, st, configure, blocks);
    case 8116: return walk_t<8, 1, 16>(ctx, P, warps, st, configure, blocks);
    case 12116: return walk_t<12, 1, 16>(ctx, P, warps, st, configure, blocks);
    case 16116: return walk_t<16, 1, 16>(ctx, P, warps, st, configure, blocks);
    case 16216: return walk_t<16, 2, 16>(ctx, P, warps, st, configure, blocks);
    default: return LABS_ERR_INVALID_ARG;
  }
}

// Warps per block of a launch: the requested count, else 8 for whole-warp walks and, for half-warp
// walks, as many (up to the block limit) as fit one block's slabs in the shared memory of an SM.
static int warps_for(const labs_ctx* ctx, const WalkParams& P, const Variant& v, int requested) {
  if (requested > 0) return requested;
  if (v.GL == 32) return 8;
  int w = walk_block_threads(16) / 32;
  while (w > 1 && walk_smem(P, 2 * w) > ctx->smem_optin) w--;
  return w;
}

static int launch_walk(labs_ctx* ctx, const WalkParams& P, const Variant& v, int warps, cudaStream_t st) {
  long long blocks = 0;
  int s = walk_variant(ctx, P, v, warps, st, true, &blocks);
  return s == LABS_OK ? walk_variant(ctx, P, v, warps, st, false, &blocks) : s;
}

// One launch's lengths.
struct LenSpec {
  int L, skew, p, T_i;
  int64_t walks, walk_begin;
};

// Fills the per-length table, the slot stride and the slab plan for variant v; false if some length does
// not fit.  Every length's arrays are shrunk to what it needs (compact_layout) and the slab takes the
// largest of each piece over the launch's lengths.
static bool fill_params(WalkParams& P, const std::vector<LenSpec>& lens, const Variant& v, int R, bool biased,
                        int bloom_log2) {
  P.n_len = (int)lens.size();
  int64_t item = 0;
  int maxnp = 1, fwd_bytes = 16, cl = 8;
  for (size_t i = 0; i < lens.size(); i++) {
    LenEntry& e = P.len[i];
    if (!make_layout(e.ly, lens[i].L, lens[i].skew, lens[i].p, v.M, v.H)) return false;
    compact_layout(e.ly);
    int np = (e.ly.n_tasks + v.GL - 1) / v.GL;
    if (np > kMaxPasses) return false;
    maxnp = std::max(maxnp, np);
    fwd_bytes = std::max(fwd_bytes, 4 * e.ly.cw * e.ly.ncls);
    cl = std::max(cl, e.ly.cl);
    e.T_i = lens[i].T_i > 0 ? lens[i].T_i : 4 * (lens[i].L + 1);
    e.E_thr_value = INT32_MAX;
    e.item_begin = item;
    e.walk_begin = lens[i].walk_begin;
    item += lens[i].walks;
  }
  if (R > v.GL) return false;  // one sieve slot per lane
  P.n_items = item;
  P.slot_stride = maxnp * (v.M / v.H);
  auto up16 = [](int b) { return (b + 15) & ~15; };
  SlabPlan& sp = P.slab;
  int off = up16(4 * kBitWords);
  sp.off_C16 = off;
  off += up16(2 * cl);
  sp.off_C8 = off;
  off += up16(cl);
  sp.off_fwd = off;
  off += up16(fwd_bytes);
  sp.off_bwd = off;
  off += up16(fwd_bytes);
  sp.off_bloom = off;
  off += up16(std::max(4, (1 << bloom_log2) / 8));
  sp.off_slots = off;
  off += up16(P.slot_stride * v.GL * slot_bytes(biased));
  // slab stride = 8 (mod 128) bytes: the two walks of a half-warp launch then sit two banks apart, so
  // their lanes' window loads (tiles four words apart, all multiples of four banks) do not collide
  // (every slab access is at most 4 bytes wide, so 8-byte alignment of a slab suffices)
  sp.bytes = off + (136 - off % 128) % 128;
  return true;
}

// Heuristic choice: least total per-warp scan work, sum(walks * NP * M / H * GL / 32) (a half-warp walk
// shares its warp's instructions with another walk); ties to fewer lanes per walk (the two walks of a
// warp then share every instruction of the serial phases), then to fewer lane passes (each pass repeats
// the per-slot phases), then to more lanes per tile, then the larger tile.
// req_m / req_gl: 0 or the tile size / lanes per walk the caller fixed; R: sieve slots per walk.
static bool choose_variant(const std::vector<LenSpec>& lens, int req_m, int req_gl, int R, Variant* out) {
  bool found = false;
  long double best_cost = 0;
  int best_np = 0;
  Variant best{0, 0, 0};
  for (const Variant& v : kVariants) {
    if (req_m && v.M != req_m) continue;
    if (req_gl && v.GL != req_gl) continue;
    if (R > v.GL) continue;
    long double cost = 0;
    int max_np = 0;
    bool ok = true;
    for (const LenSpec& s : lens) {
      int np = passes_for(s.L, s.skew, s.p, v);
      if (np == 0 || np > kMaxPasses) {
        ok = false;
        break;
      }
      max_np = std::max(max_np, np);
      cost += (long double)std::max<int64_t>(s.walks, 1) * np * v.M / v.H * v.GL / 32;
    }
    if (!ok) continue;
    const bool better =
        !found || cost < best_cost ||
        (cost == best_cost &&
         (v.GL < best.GL ||
          (v.GL == best.GL && (max_np < best_np || (max_np == best_np && (v.H > best.H || (v.H == best.H && v.M > best.M)))))));
    if (better) {
      best = v;
      best_cost = cost;
      best_np = max_np;
      found = true;
    }
  }
  *out = best;
  return found;
}

static void base_params(WalkParams& P, int R, int bloom_log2, int bloom_k, int p, int n_prefix, int64_t flip_budget,
                        uint64_t seed, int32_t E_target, const uint64_t* prefixes, labs_candidate* out,
                        int64_t* walk_stats, labs_walk_stats* stats, unsigned long long* counter) {
  P.R = R;
  P.bloom_log2 = bloom_log2;
  P.bloom_k = bloom_k;
  P.prefix_words = p > 0 ? (p + 63) / 64 : 1;
  P.n_prefix = n_prefix;
  P.flip_budget = flip_budget;
  P.seed = seed;
  P.E_target = E_target;
  P.prefixes = prefixes;
  P.out = out;
  P.walk_stats = walk_stats;
  P.stats = stats;
  P.counter = counter;
  P.E_thr_dev = nullptr;
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

int launch_skew_search(labs_ctx* ctx, const labs_walk_cfg* cfg, const uint64_t* prefixes, int n_prefix,
                       labs_candidate* out, int64_t* walk_stats, labs_walk_stats* stats, cudaStream_t st) {
  std::vector<LenSpec> lens{{cfg->L, cfg->skew, cfg->p, cfg->T_i, cfg->n_walks, cfg->walk_begin}};
  Variant v;
  if (!choose_variant(lens, cfg->tile_m, cfg->lanes_per_walk, cfg->R, &v)) return LABS_ERR_INVALID_ARG;
  WalkParams* P = new (std::nothrow) WalkParams();
  if (!P) return LABS_ERR_NOMEM;
  char* w = static_cast<char*>(ws_get(ctx, kWsWalkCounters, 256));
  if (!w) {
    delete P;
    return LABS_ERR_NOMEM;
  }
  base_params(*P, cfg->R, cfg->bloom_log2, cfg->bloom_k, cfg->p, n_prefix, cfg->flip_budget, cfg->seed,
              cfg->E_target, prefixes, out, walk_stats, stats, reinterpret_cast<unsigned long long*>(w));
  if (!fill_params(*P, lens, v, cfg->R, false, cfg->bloom_log2)) {
    delete P;
    return LABS_ERR_INVALID_ARG;
  }
  int32_t* thr = reinterpret_cast<int32_t*>(w + 64);
  int s = LABS_OK;
  if (cfg->E_thr_dev) {
    P->E_thr_dev = cfg->E_thr_dev;
  } else if (cfg->E_thr == LABS_AUTO_THRESHOLD) {
    s = launch_sample_threshold(ctx, cfg->L, cfg->skew, cfg->p, prefixes, n_prefix, P->prefix_words, cfg->seed,
                                cfg->n_thresh_samples, cfg->thresh_rank, thr, nullptr, st);
    P->E_thr_dev = thr;
  } else {
    P->len[0].E_thr_value = cfg->E_thr;
  }
  if (s == LABS_OK) {
    walk_init_kernel<<<1, 1, 0, st>>>(stats, P->E_thr_dev, P->len[0].E_thr_value, P->counter);
    s = cuda_status(cudaGetLastError());
  }
  if (s == LABS_OK && P->n_items > 0) s = launch_walk(ctx, *P, v, warps_for(ctx, *P, v, cfg->warps_per_cta), st);
  delete P;
  return s;
}

// ---------------------------------------------------------------------------------------------
// Chunked walks: the same Algorithm 1 walks run `chunk` accepted flips per launch and are saved in
// between, so a proposal network can score every walk's current state before each chunk (learned mode).
// Without a network the results equal labs_skew_search's.
// ---------------------------------------------------------------------------------------------
int launch_chunked_search(labs_ctx* ctx, const labs_walk_cfg* cfg, labs_policy* policy, float lambda, int chunk,
                          const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                          labs_walk_stats* stats, float* logits_log, uint64_t* state_log, int32_t* move_log,
                          cudaStream_t st) {
  std::vector<LenSpec> lens{{cfg->L, cfg->skew, cfg->p, cfg->T_i, cfg->n_walks, cfg->walk_begin}};
  Variant v;
  if (!choose_variant(lens, cfg->tile_m, cfg->lanes_per_walk, cfg->R, &v)) return LABS_ERR_INVALID_ARG;
  const long long n = cfg->n_walks;
  const int L = cfg->L, W = (L + 63) / 64;
  const long long n_chunks = (cfg->flip_budget + chunk - 1) / chunk;
  char* w = static_cast<char*>(ws_get(ctx, kWsWalkCounters, 256));
  unsigned char* state = static_cast<unsigned char*>(ws_get(ctx, kWsChunkState, (size_t)kStateBytes * (size_t)n));
  char* io = static_cast<char*>(ws_get(ctx, kWsChunkIo, (size_t)n * (8 * W + 4 * L) + 256));
  if (!w || !state || !io) return LABS_ERR_NOMEM;
  uint64_t* seqbuf = reinterpret_cast<uint64_t*>(io);
  float* logits = reinterpret_cast<float*>(io + (((size_t)n * 8 * W + 255) & ~size_t(255)));
  WalkParams* P = new (std::nothrow) WalkParams();
  if (!P) return LABS_ERR_NOMEM;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(w);
  base_params(*P, cfg->R, cfg->bloom_log2, cfg->bloom_k, cfg->p, n_prefix, cfg->flip_budget, cfg->seed, cfg->E_target,
              prefixes, out, walk_stats, stats, counter);
  if (!fill_params(*P, lens, v, cfg->R, policy != nullptr, cfg->bloom_log2)) {  // one slab plan for the plain and biased launches
    delete P;
    return LABS_ERR_INVALID_ARG;
  }
  int32_t* thr = reinterpret_cast<int32_t*>(w + 64);
  int s = LABS_OK;
  if (cfg->E_thr_dev) {
    P->E_thr_dev = cfg->E_thr_dev;
  } else if (cfg->E_thr == LABS_AUTO_THRESHOLD) {
    s = launch_sample_threshold(ctx, cfg->L, cfg->skew, cfg->p, prefixes, n_prefix, P->prefix_words, cfg->seed,
                                cfg->n_thresh_samples, cfg->thresh_rank, thr, nullptr, st);
    P->E_thr_dev = thr;
  } else {
    P->len[0].E_thr_value = cfg->E_thr;
  }
  const int warps = warps_for(ctx, *P, v, cfg->warps_per_cta);
  long long blocks = 0, blocks_biased = 0;
  if (s == LABS_OK) s = walk_variant(ctx, *P, v, warps, st, true, &blocks);
  if (s == LABS_OK && policy) {  // the chunks run the biased instantiation: configure it as well
    P->bias = logits;
    s = walk_variant(ctx, *P, v, warps, st, true, &blocks_biased);
    P->bias = nullptr;
  }
  if (s == LABS_OK && cudaMemsetAsync(state, 0, (size_t)kStateBytes * (size_t)n, st) != cudaSuccess) s = LABS_ERR_CUDA;
  if (s == LABS_OK) {
    walk_init_kernel<<<1, 1, 0, st>>>(stats, P->E_thr_dev, P->len[0].E_thr_value, counter);
    s = cuda_status(cudaGetLastError());
  }
  P->state = state;
  P->state_stride = kStateBytes;
  P->seq_out = seqbuf;
  // set-up launch: every walk's first state
  P->chunk = -1;
  if (s == LABS_OK && n > 0) s = walk_variant(ctx, *P, v, warps, st, false, &blocks);
  for (long long c = 0; c < n_chunks && s == LABS_OK && n > 0; c++) {
    if (policy) {
      s = labs_policy_forward(policy, seqbuf, n, logits, st);
      if (s != LABS_OK) break;
      P->bias = logits;
      P->lambda = lambda;
      if (logits_log && cudaMemcpyAsync(logits_log + (size_t)c * n * L, logits, sizeof(float) * (size_t)n * L,
                                        cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        s = LABS_ERR_CUDA;
        break;
      }
    }
    if (state_log && cudaMemcpyAsync(state_log + (size_t)c * n * W, seqbuf, 8 * (size_t)n * W,
                                     cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      s = LABS_ERR_CUDA;
      break;
    }
    P->chunk = chunk;
    P->move_log = move_log ? move_log + (size_t)c * n * 2 : nullptr;
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st) != cudaSuccess) {
      s = LABS_ERR_CUDA;
      break;
    }
    s = walk_variant(ctx, *P, v, warps, st, false, policy ? &blocks_biased : &blocks);
  }
  delete P;
  if (policy) {  // the network's tensor-core waits: a failure makes the logits of that chunk invalid
    const int ps = labs_policy_sync_status(policy, st);
    if (s == LABS_OK) s = ps;
  }
  return s;
}

// ---------------------------------------------------------------------------------------------
// Batched mixed-length search: every length's sieve bound, then one persistent walk launch over all
// (length, walk) items; the sequence is captured once into a CUDA graph and replayed.  The tile variant
// (words per thread) and the walks per CTA come from a timing autotuner cached per (length set, SMs).
// ---------------------------------------------------------------------------------------------
namespace {

uint64_t mix_key(uint64_t h, uint64_t v) { return sm64_at(h ^ v, 0x5EED); }

// Issues the whole batched step on `st`.  blocks > 0: the walk grid was sized beforehand, so nothing
// but stream work is issued (capturable); blocks == 0: the walk kernel is configured here.
int issue_batch(labs_ctx* ctx, const labs_batch_cfg* cfg, const std::vector<LenSpec>& lens, const Variant& v,
                int warps, const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                int32_t* thr, labs_walk_stats* stats, unsigned long long* counter, int64_t flip_budget,
                bool thresholds, long long blocks, cudaStream_t st) {
  WalkParams* P = new (std::nothrow) WalkParams();
  if (!P) return LABS_ERR_NOMEM;
  base_params(*P, cfg->R, cfg->bloom_log2, cfg->bloom_k, cfg->p, n_prefix, flip_budget, cfg->seed, cfg->E_target,
              prefixes, out, walk_stats, stats, counter);
  if (!fill_params(*P, lens, v, cfg->R, false, cfg->bloom_log2)) {
    delete P;
    return LABS_ERR_INVALID_ARG;
  }
  P->E_thr_dev = thr;
  int s = LABS_OK;
  if (thresholds) {
    for (size_t i = 0; i < lens.size() && s == LABS_OK; i++)
      s = launch_sample_threshold(ctx, lens[i].L, lens[i].skew, lens[i].p, prefixes, n_prefix, P->prefix_words,
                                  cfg->seed, cfg->n_thresh_samples, cfg->thresh_rank, thr + i, nullptr, st);
  }
  if (s == LABS_OK) {
    walk_init_kernel<<<1, 1, 0, st>>>(stats, thr, 0, counter);
    s = cuda_status(cudaGetLastError());
  }
  if (s == LABS_OK && P->n_items > 0) {
    if (blocks > 0)
      s = walk_variant(ctx, *P, v, warps, st, false, &blocks);
    else
      s = launch_walk(ctx, *P, v, warps, st);
  }
  delete P;
  return s;
}

}  // namespace

int launch_batched_search(labs_ctx* ctx, const labs_batch_cfg* cfg, const int32_t* lengths, const int64_t* walks,
                          const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                          int32_t* E_thr_out, labs_walk_stats* stats, cudaStream_t st) {
  std::vector<LenSpec> lens;
  int64_t begin = 0;
  for (int i = 0; i < cfg->n_len; i++) {
    const int L = lengths[i];
    const int skew = L & 1;
    lens.push_back({L, skew, skew ? cfg->p : 0, cfg->T_i, walks[i], 0});
    begin += walks[i];
  }
  // workspace first (nothing below may allocate once a capture has begun)
  char* w = static_cast<char*>(ws_get(ctx, kWsWalkCounters, 256));
  int32_t* thr = E_thr_out ? E_thr_out : static_cast<int32_t*>(ws_get(ctx, kWsBatchThresholds, sizeof(int32_t) * kMaxLens));
  if (!w || !thr) return LABS_ERR_NOMEM;
  if (!ws_get(ctx, kWsThreshSamples, sizeof(int32_t) * (size_t)cfg->n_thresh_samples) ||
      !ws_get(ctx, kWsThreshHist, sizeof(unsigned) * 2 * kHistBins + 64))
    return LABS_ERR_NOMEM;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(w);

  // ---- variant and walks per CTA: given, or timed
  Variant v{0, 0, 0};
  int warps = cfg->warps_per_cta;
  uint64_t tkey = (uint64_t)ctx->num_sms;
  for (const LenSpec& s : lens) tkey = mix_key(tkey, ((uint64_t)s.L << 40) ^ (uint64_t)s.walks);
  tkey = mix_key(tkey, ((uint64_t)cfg->tile_m << 8) ^ (uint64_t)warps ^ ((uint64_t)cfg->R << 16) ^
                           ((uint64_t)cfg->bloom_log2 << 24));
  bool cached = false;
  for (int i = 0; i < ctx->n_tuned; i++)
    if (ctx->tuned_key[i] == tkey) {
      v = {ctx->tuned[i][0], ctx->tuned[i][1], ctx->tuned[i][2]};
      warps = ctx->tuned[i][3];
      cached = true;
    }
  // the (variant, warps per CTA) candidates: whole-warp walks try 4 and 8 warps, half-warp walks the
  // largest block whose slabs fit an SM
  WalkParams* Q = new (std::nothrow) WalkParams();
  if (!Q) return LABS_ERR_NOMEM;
  if (!cached) {
    std::vector<std::pair<Variant, int>> cands;
    for (const Variant& c : kVariants) {
      if (cfg->tile_m && c.M != cfg->tile_m) continue;
      if (!fill_params(*Q, lens, c, cfg->R, false, cfg->bloom_log2)) continue;
      if (warps > 0) {
        if (32 * warps <= walk_block_threads(c.GL)) cands.push_back({c, warps});
      } else if (c.GL == 32) {
        cands.push_back({c, 4});
        cands.push_back({c, 8});
      } else {
        cands.push_back({c, warps_for(ctx, *Q, c, 0)});
      }
    }
    if (cands.empty()) {
      delete Q;
      return LABS_ERR_INVALID_ARG;
    }
    if (cands.size() == 1) {
      v = cands[0].first;
      warps = cands[0].second;
    } else {
      // trial: every length with 1/16 of its walks (at least one), 512 flips each, thresholds off
      std::vector<LenSpec> trial = lens;
      for (LenSpec& s : trial) s.walks = std::max<int64_t>(1, s.walks / 16);
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best_ms = 0;
      for (const auto& cw : cands) {
        cudaEventRecord(e0, st);
        int s = issue_batch(ctx, cfg, trial, cw.first, cw.second, prefixes, n_prefix, out, nullptr, thr, stats,
                            counter, std::min<int64_t>(cfg->flip_budget, 512), false, 0, st);
        cudaEventRecord(e1, st);
        if (s != LABS_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (v.M == 0 || ms < best_ms) {
          best_ms = ms;
          v = cw.first;
          warps = cw.second;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (v.M == 0) {
        delete Q;
        return LABS_ERR_CUDA;
      }
    }
    if (ctx->n_tuned < kMaxTuned) {
      ctx->tuned_key[ctx->n_tuned] = tkey;
      ctx->tuned[ctx->n_tuned][0] = v.M;
      ctx->tuned[ctx->n_tuned][1] = v.H;
      ctx->tuned[ctx->n_tuned][2] = v.GL;
      ctx->tuned[ctx->n_tuned][3] = warps;
      ctx->n_tuned++;
    }
  }
  // kernel attributes and grid size before any capture
  long long blocks = 0;
  {
    int s = fill_params(*Q, lens, v, cfg->R, false, cfg->bloom_log2) ? LABS_OK : LABS_ERR_INVALID_ARG;
    Q->bloom_log2 = cfg->bloom_log2;
    if (s == LABS_OK) s = walk_variant(ctx, *Q, v, warps, st, true, &blocks);
    delete Q;
    if (s != LABS_OK) return s;
  }
  if (!cfg->use_graph)
    return issue_batch(ctx, cfg, lens, v, warps, prefixes, n_prefix, out, walk_stats, thr, stats, counter,
                       cfg->flip_budget, true, blocks, st);

  // ---- CUDA graph: capture once per (configuration, buffers), replay afterwards
  uint64_t gkey = tkey;
  gkey = mix_key(gkey, ((uint64_t)v.M << 32) ^ ((uint64_t)v.H << 16) ^ ((uint64_t)v.GL << 8) ^ (uint64_t)warps);
  gkey = mix_key(gkey, (uint64_t)cfg->flip_budget ^ ((uint64_t)cfg->R << 48));
  gkey = mix_key(gkey, cfg->seed);
  gkey = mix_key(gkey, ((uint64_t)cfg->p << 32) ^ ((uint64_t)cfg->bloom_log2 << 16) ^ (uint64_t)cfg->bloom_k);
  gkey = mix_key(gkey, ((uint64_t)cfg->T_i << 32) ^ (uint32_t)cfg->E_target);
  gkey = mix_key(gkey, (uint64_t)cfg->n_thresh_samples ^ ((uint64_t)cfg->thresh_rank << 40));
  const void* bufs[] = {prefixes, out, walk_stats, thr, stats, w, ctx->ws[kWsThreshSamples], ctx->ws[kWsThreshHist]};
  for (const void* ptr : bufs) gkey = mix_key(gkey, (uint64_t)(uintptr_t)ptr);
  gkey = mix_key(gkey, (uint64_t)n_prefix ^ ((uint64_t)blocks << 32));
  if (!ctx->graph_exec || ctx->graph_key != gkey) {
    if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
      return LABS_ERR_CUDA;
    if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return LABS_ERR_CUDA;
    int s = issue_batch(ctx, cfg, lens, v, warps, prefixes, n_prefix, out, walk_stats, thr, stats, counter,
                        cfg->flip_budget, true, blocks, ctx->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (s != LABS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return LABS_ERR_CUDA;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return LABS_ERR_CUDA;
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = ex;
    ctx->graph_key = gkey;
  }
  return cuda_status(cudaGraphLaunch(ctx->graph_exec, st));
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
  if (check_walk_shape(L, skew, p, n_prefix, prefixes) != LABS_OK) return LABS_ERR_INVALID_ARG;
  if (!E_thr_out || (reinterpret_cast<uintptr_t>(E_thr_out) & 3u)) return LABS_ERR_INVALID_ARG;
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
