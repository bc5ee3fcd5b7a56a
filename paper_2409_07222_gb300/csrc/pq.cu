// pq.cu -- step 2 of the dual-step search: Algorithm 2's priority-queue refinement over the unrestricted
// space, in batch-synchronous form (labs_pq_refine).
//
// GB300 mapping.  The paper runs one priority queue per candidate in Rust on CPU cores; here one open
// set of the cap smallest (E, fp) keys lives in HBM as an UNORDERED pool of entries (energy,
// fingerprint, sequence) with a free-slot stack, and beside it a histogram of the entries' energies
// (one bin per energy, clamped at both ends of a 2^17-bin window, and a coarse level of 256 bins per
// entry).  The B smallest keys, or the cap smallest, are then found without ordering the pool: the
// histogram's prefix sums give the bin where the count is reached, every entry below it is taken, and
// only the entries of that one boundary bin are ranked (a radix select on their full (E, fp) key, so a
// clamped bin holding several energies is still exact).  A round
//   pop      -- the b = min(B, open, budget left) smallest keys leave the pool (one pass over it), are
//               put in key order (one block) and become the round's pivots;
//   expand   -- one warp per pivot: its correlation table, the all-position dp4a scan and a visited-set
//               lookup per neighbour, written to a dense [pivot][column] survivor array;
//   dedup    -- survivors with equal (E', fp') (the same sequence) are kept once, through a hash table;
//               the one kept is the smallest (pivot, column), as in the sequential definition;
//   best     -- strict improvement test on the smallest survivor key;
//   cut      -- the cap smallest of (pool u survivors): entries of the pool above the cut are evicted,
//               survivors below it are admitted into free slots and into the visited set H;
// keeps every result identical to the sequential definition whatever order threads run in.  The seeds
// enter through the same survivor path.  With T_r > 0 every pivot also offers its 2 T_r rotations
// (MAKE_ROTATIONS) as survivor columns L .. L + 2 T_r - 1, after its L flips.
#include <algorithm>
#include <new>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr uint64_t kEmptyKey = ~0ull;  // free slot of the visited set (fp == ~0 is tracked by a flag)
constexpr int kPqWarps = 4;
constexpr int kPqM = 8;
constexpr int kMaxProbe = 1 << 20;
constexpr int kNB = 1 << 17;        // fine energy bins: bin = clamp(E - E_base, 0, kNB - 1)
constexpr int kCoarse = 256;        // fine bins per coarse bin
constexpr int kNC = kNB / kCoarse;  // coarse bins
constexpr int kColBits = 11;        // survivor column inside a representative: width <= 576 + 128 < 2^11
constexpr int kSortMax = 8192;      // pops per round (B <= 8192), put in key order by one block
constexpr int kSelThreads = 1024;   // threads of the single-block select, boundary and sort kernels

// Device-side state of one refinement (every round reads and writes it; the host only polls `stop`).
struct PqState {
  long long nP;  // open-set entries
  long long expansions, rounds, survivors, admitted, evicted, h_size, improvements, u;
  unsigned long long best_fp;
  long long free_top;   // free pool slots (the stack holds their ids)
  long long pop_cnt;    // entries gathered for popping this round
  long long cand_cnt;   // boundary-bin candidates gathered
  long long nU;         // unique survivors of the round
  long long sel_lt;     // entries below the boundary bin
  long long sel_need;   // entries taken from the boundary bin; 0: none; -1: no cut (everything kept)
  long long ev_round;   // evicted this round
  long long adm_round;  // admitted this round
  int b, stop, best_E, error, h_has_empty, E_base;
  int sel_bin;     // boundary fine bin
  int minE_round;  // smallest survivor energy of the round
  int sel_E, pad0;
  unsigned long long sel_fp;  // boundary key: a boundary-bin entry is taken iff (E, fp) <= (sel_E, sel_fp)
  unsigned long long minfp_round;
  unsigned best_rep_round, pad1;
};

struct PqBufs {
  int L, W, B, H_log2;
  int Tr, width;  // rotations per side (MAKE_ROTATIONS) and survivor columns per pivot: L flips + 2 Tr rotations
  long long cap, max_exp, T_u;
  int hs_log2;        // dedup hash table: 2^hs_log2 slots, at least twice the dense survivors
  long long cand_cap; // boundary candidate capacity (cap + dense survivors)
  int n_seeds;
  int32_t* pE;        // pool [cap]: energy, INT32_MAX for a free slot
  uint64_t* pFp;      // pool [cap]: fingerprint
  uint64_t* pSeq;     // pool [cap][W]
  int32_t* freeIds;   // free-slot stack [cap]
  unsigned* hP;       // histogram of the pool's energies: fine [kNB], coarse [kNC]
  unsigned* hP2;
  unsigned* hU;       // histogram of the round's unique survivors
  unsigned* hU2;
  int32_t* popId;     // pool ids gathered for popping [B]
  int32_t* pivE;      // pivots in key order [B]
  uint64_t* pivFp;
  uint64_t* pivSeq;   // [B][W]
  int32_t* candId;    // boundary candidates: pool id >= 0, or -(u + 1) for survivor u
  int32_t* dE;        // dense survivors [pivot][column]: energy, or INT32_MAX (visited)
  uint64_t* dFp;
  uint64_t* hkey;     // dedup hash table: mixed (E, fp) key, 0 = empty
  int32_t* hval;      // the unique survivor of a slot
  int32_t* uE;        // unique survivors
  uint64_t* uFp;
  unsigned* uRep;     // representative (pivot << kColBits | column): the smallest of equal keys
  int32_t* uSlot;     // dedup slot of the survivor
  uint64_t* H;        // visited set (open addressing)
  uint64_t* ztab;
  PqState* st;
  uint64_t* best_seq;
  const uint64_t* seeds;
};

// Left shift of rotation code c (MAKE_ROTATIONS): c < Tr moves the first c + 1 elements to the end,
// c >= Tr moves the last c - Tr + 1 elements to the start (a left shift by L - (c - Tr + 1)).
__host__ __device__ __forceinline__ int rot_shift(int L, int Tr, int c) {
  const int r = c < Tr ? c + 1 : L - ((c - Tr + 1) % L);
  return r % L;
}

// Survivor column col of a pivot (src, W words): col < L flips position col + 1, else rotation col - L.
// One thread; dst may be global memory.
__device__ __forceinline__ void pq_child(const uint64_t* src, const PqBufs& b, int col, uint64_t* dst) {
  uint64_t out[LABS_MAX_W];
  if (col < b.L) {
    for (int t = 0; t < b.W; t++) out[t] = src[t] ^ (t == (col >> 6) ? 1ull << (col & 63) : 0ull);
  } else {
    const int r = rot_shift(b.L, b.Tr, col - b.L);
    for (int t = 0; t < b.W; t++) out[t] = 0;
    for (int i = 0; i < b.L; i++) {
      int j = i + r;
      if (j >= b.L) j -= b.L;
      if ((src[j >> 6] >> (j & 63)) & 1ull) out[i >> 6] |= 1ull << (i & 63);
    }
  }
  for (int t = 0; t < b.W; t++) dst[t] = out[t];
}

__device__ __forceinline__ uint64_t h_slot(uint64_t fp, int log2) { return (fp * kGamma) >> (64 - log2); }

// Continues the probe sequence of fp after slot s, whose key was another one.
__device__ __forceinline__ bool h_contains_after(const PqBufs& b, uint64_t fp, uint64_t s) {
  const uint64_t mask = (1ull << b.H_log2) - 1;
  for (int it = 1; it < kMaxProbe; it++) {
    s = (s + 1) & mask;
    const uint64_t v = b.H[s];
    if (v == fp) return true;
    if (v == kEmptyKey) return false;
  }
  atomicExch(&b.st->error, 1);  // probe limit: the set is too full (reported as a capacity error)
  return true;
}

__device__ __forceinline__ bool h_contains(const PqBufs& b, uint64_t fp) {
  if (fp == kEmptyKey) return b.st->h_has_empty != 0;
  const uint64_t s = h_slot(fp, b.H_log2);
  const uint64_t v = b.H[s];
  if (v == fp) return true;
  if (v == kEmptyKey) return false;
  return h_contains_after(b, fp, s);
}

// Inserts fp; returns 1 when it was not there yet (the caller counts insertions into h_size in bulk).
__device__ __forceinline__ int h_insert(const PqBufs& b, uint64_t fp) {
  if (fp == kEmptyKey) return atomicExch(&b.st->h_has_empty, 1) == 0 ? 1 : 0;
  const uint64_t mask = (1ull << b.H_log2) - 1;
  uint64_t s = h_slot(fp, b.H_log2);
  for (int it = 0; it < kMaxProbe; it++) {
    const unsigned long long old =
        atomicCAS(reinterpret_cast<unsigned long long*>(&b.H[s]), (unsigned long long)kEmptyKey, fp);
    if (old == kEmptyKey) return 1;
    if (old == fp) return 0;
    s = (s + 1) & mask;
  }
  atomicExch(&b.st->error, 1);
  return 0;
}

__device__ __forceinline__ bool key_lt(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}
__device__ __forceinline__ bool key_le(int Ea, uint64_t fa, int Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa <= fb);
}

__device__ __forceinline__ int e_bin(int E, int E_base) {
  const int d = E - E_base;
  return d < 0 ? 0 : (d >= kNB ? kNB - 1 : d);
}

// Adds v to *ctr once per warp (every lane of the warp calls it with its own v).
__device__ __forceinline__ void warp_add(long long* ctr, int v) {
  const int s = __reduce_add_sync(kFull, v);
  if (lane_id() == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(ctr), (unsigned long long)(long long)s);
}

// Reserves one output index per lane with pred, one atomic per warp (every lane calls it); returns the
// lane's index, or -1.
__device__ __forceinline__ long long warp_append(long long* ctr, bool pred) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (!m) return -1;
  const int leader = __ffs(m) - 1;
  long long base = 0;
  if (lane_id() == leader)
    base = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(ctr), (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  return pred ? base + __popc(m & ((1u << lane_id()) - 1u)) : -1;
}

// Adds the insertions of a warp to h_size (every lane calls it).
__device__ __forceinline__ void h_count(const PqBufs& b, int inserted) { warp_add(&b.st->h_size, inserted); }

// Mixed key of (E, fp) for the dedup table; 0 marks an empty slot, so a mixed key of 0 becomes 1.
__device__ __forceinline__ uint64_t dedup_key(int E, uint64_t fp) {
  const uint64_t k = fp ^ ((uint64_t)(uint32_t)E * 0xD6E8FEB86659FD93ull);
  return k ? k : 1ull;
}

// Key of a boundary candidate (pool entry or survivor).
__device__ __forceinline__ void cand_key(const PqBufs& b, int32_t c, int& E, uint64_t& fp) {
  if (c >= 0) {
    E = b.pE[c];
    fp = b.pFp[c];
  } else {
    E = b.uE[-c - 1];
    fp = b.uFp[-c - 1];
  }
}

// ---------------------------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------------------------
__global__ void pq_ztab_kernel(uint64_t* ztab, int L) {
  const uint64_t zk = stream_key(0, kPurposeZobrist, (uint64_t)L, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) ztab[i] = zobrist(zk, i + 1);
}

// Every pool slot free (the stack holds them all), the state zeroed.
__global__ void pq_init_kernel(PqBufs b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < b.cap; i += (long long)gridDim.x * blockDim.x) {
    b.pE[i] = INT32_MAX;
    b.freeIds[i] = (int32_t)(b.cap - 1 - i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PqState z{};
    z.free_top = b.cap;
    z.best_E = INT32_MAX;
    z.best_fp = ~0ull;
    z.minE_round = INT32_MAX;
    z.minfp_round = ~0ull;
    z.best_rep_round = ~0u;
    *b.st = z;
  }
}

// One warp per seed: energy over all lags and the fingerprint, into the dense arrays (one column).
__global__ void __launch_bounds__(32 * kPqWarps) pq_seed_kernel(PqBufs b, int n_seeds) {
  __shared__ uint32_t bits_all[kPqWarps][kBitWords];
  uint32_t* bits = bits_all[threadIdx.x >> 5];
  const int lane = lane_id();
  for (int q = blockIdx.x * kPqWarps + (threadIdx.x >> 5); q < n_seeds; q += gridDim.x * kPqWarps) {
    const uint64_t* src = b.seeds + (size_t)q * b.W;
    if (lane < kBitWords) {
      const int W32 = (b.L + 31) >> 5;
      uint32_t v = 0;
      if (lane < W32) {
        uint64_t x = src[lane >> 1];
        v = (lane & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
        int rem = b.L - 32 * lane;
        if (rem < 32) v &= (1u << rem) - 1u;
      }
      bits[lane] = v;
    }
    __syncwarp();
    int e = 0;
    for (int k = lane + 1; k < b.L; k += 32) {
      const int c = corr_lag(bits, b.L, k);
      e += c * c;
    }
    e = warp_sum_i32(e);
    uint64_t h = 0;
    for (int i = lane + 1; i <= b.L; i += 32)
      if (!((bits[(i - 1) >> 5] >> ((i - 1) & 31)) & 1u)) h ^= b.ztab[i - 1];
    h = warp_xor_u64(h);
    if (lane == 0) {
      b.dE[q] = e;
      b.dFp[q] = h;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Round kernels.  SEED = true runs the survivor path on the seeds (dense = the seeds, one column each,
// representatives are seed indices; nothing is counted as a survivor or an admission).
// ---------------------------------------------------------------------------------------------
__global__ void pq_round_begin_kernel(PqBufs b) {
  PqState* st = b.st;
  if (!st->stop) {
    if (st->error)
      st->stop = 4;
    else if (st->expansions >= b.max_exp)
      st->stop = 1;
    else if (st->nP == 0)
      st->stop = 2;
    else if (b.T_u > 0 && st->u >= b.T_u)
      st->stop = 3;
  }
  st->pop_cnt = 0;
  st->cand_cnt = 0;
  st->nU = 0;
  st->ev_round = 0;
  st->adm_round = 0;
  st->minE_round = INT32_MAX;
  st->minfp_round = ~0ull;
  st->best_rep_round = ~0u;
  if (st->stop) {
    st->b = 0;
    return;
  }
  long long bb = min((long long)b.B, st->nP);
  bb = min(bb, b.max_exp - st->expansions);
  st->b = (int)bb;
}

// One block: the fine bin where the count of entries reaches the target (POP: b over the pool; else
// cap over the pool's rest and the survivors, or no cut when everything fits).  sel_lt = entries below
// that bin, sel_need = entries to take from it.
template <bool POP>
__global__ void __launch_bounds__(kSelThreads) pq_select_kernel(PqBufs b) {
  PqState* st = b.st;
  __shared__ unsigned long long part[kSelThreads];
  __shared__ long long s_target;
  __shared__ int s_cb;
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x;
  if (t == 0) {
    long long target;
    if (POP) {
      target = st->b;
    } else {
      st->cand_cnt = 0;  // the pop's candidates are done with
      const long long total = st->nP - st->b + st->nU;
      target = total > b.cap ? b.cap : -1;
    }
    s_target = target;
    if (target <= 0) {
      st->sel_need = target < 0 ? -1 : 0;
      st->sel_bin = kNB;
      st->sel_lt = 0;
    }
  }
  __syncthreads();
  const long long target = s_target;
  if (target <= 0) return;
  // coarse level
  unsigned long long c = 0;
  if (t < kNC) c = (unsigned long long)b.hP2[t] + (POP ? 0u : b.hU2[t]);
  part[t] = c;
  __syncthreads();
  for (int off = 1; off < kSelThreads; off <<= 1) {  // inclusive scan
    const unsigned long long v = t >= off ? part[t - off] : 0ull;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  if (t < kNC) {
    const unsigned long long before = t ? part[t - 1] : 0ull;
    if (before < (unsigned long long)target && part[t] >= (unsigned long long)target) {
      s_cb = t;
      s_before = before;
    }
  }
  __syncthreads();
  const int cb = s_cb;
  const unsigned long long cbefore = s_before;
  // fine level: the coarse bin's 256 bins
  unsigned long long f = 0;
  if (t < kCoarse) f = (unsigned long long)b.hP[cb * kCoarse + t] + (POP ? 0u : b.hU[cb * kCoarse + t]);
  __syncthreads();
  part[t] = f;
  __syncthreads();
  for (int off = 1; off < kCoarse; off <<= 1) {
    const unsigned long long v = (t < kCoarse && t >= off) ? part[t - off] : 0ull;
    __syncthreads();
    if (t < kCoarse) part[t] += v;
    __syncthreads();
  }
  if (t < kCoarse) {
    const unsigned long long before = cbefore + (t ? part[t - 1] : 0ull);
    if (before < (unsigned long long)target && cbefore + part[t] >= (unsigned long long)target) {
      st->sel_bin = cb * kCoarse + t;
      st->sel_lt = (long long)before;
      st->sel_need = target - (long long)before;
    }
  }
}

// Pass over the pool (U = false) or the survivors (U = true): POP gathers the pool entries below the
// boundary bin (popped) and those in it (candidates); the cut gathers the boundary bin's entries.
template <bool POP, bool U>
__global__ void __launch_bounds__(256) pq_gather_kernel(PqBufs b) {
  PqState* st = b.st;
  if (POP ? st->b == 0 : st->sel_need <= 0) return;
  const int sel = st->sel_bin, Eb = st->E_base;
  const long long n = U ? st->nU : b.cap;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    int bin = kNB;
    if (i < n) {
      const int E = U ? b.uE[i] : b.pE[i];
      if (E != INT32_MAX) bin = e_bin(E, Eb);
    }
    // the histogram bounds both counts (b entries below the boundary bin at most); a count beyond a
    // buffer can only come from an inconsistent state, which is reported instead of written
    if (POP) {
      const long long o = warp_append(&st->pop_cnt, bin < sel);
      if (o >= b.B) st->error = 1;
      else if (o >= 0) b.popId[o] = (int32_t)i;
    }
    const long long o2 = warp_append(&st->cand_cnt, bin == sel);
    if (o2 >= b.cand_cap) st->error = 1;
    else if (o2 >= 0) b.candId[o2] = U ? -(int32_t)i - 1 : (int32_t)i;
  }
}

// One block: the sel_need smallest (E, fp) keys among the boundary candidates, by a most-significant-
// digit-first radix select over the 96-bit key (four energy bytes, then eight fingerprint bytes); keys
// are distinct, so exactly sel_need candidates are <= the selected key.  POP appends them to the pops.
template <bool POP>
__global__ void __launch_bounds__(kSelThreads) pq_boundary_kernel(PqBufs b) {
  PqState* st = b.st;
  if (POP ? st->b == 0 : st->sel_need <= 0) return;
  const long long n = min(st->cand_cnt, b.cand_cap);
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_pre_e, s_pre_f;  // the digits fixed so far
  __shared__ long long s_k;
  const int t = threadIdx.x;
  if (t == 0) {
    s_pre_e = 0;
    s_pre_f = 0;
    s_k = st->sel_need;
  }
  __syncthreads();
  for (int d = 0; d < 12; d++) {
    if (t < 256) hist[t] = 0;
    __syncthreads();
    const unsigned long long pe = s_pre_e, pf = s_pre_f;
    for (long long i = t; i < n; i += kSelThreads) {
      int E;
      uint64_t fp;
      cand_key(b, b.candId[i], E, fp);
      const uint64_t ue = (uint32_t)E;
      bool match;
      unsigned digit;
      if (d < 4) {
        const int sh = 24 - 8 * d;
        match = d == 0 || (ue >> (sh + 8)) == (pe >> (sh + 8));
        digit = (unsigned)(ue >> sh) & 255u;
      } else {
        const int sh = 56 - 8 * (d - 4);
        match = ue == pe && (d == 4 || (fp >> (sh + 8)) == (pf >> (sh + 8)));
        digit = (unsigned)(fp >> sh) & 255u;
      }
      if (match) atomicAdd(&hist[digit], 1u);
    }
    __syncthreads();
    if (t == 0) {
      const long long k = s_k;
      long long acc = 0;
      int dg = 0;
      while (dg < 255 && acc + hist[dg] < k) acc += hist[dg++];
      s_k = k - acc;
      if (d < 4)
        s_pre_e = pe | ((unsigned long long)dg << (24 - 8 * d));
      else
        s_pre_f = pf | ((unsigned long long)dg << (56 - 8 * (d - 4)));
    }
    __syncthreads();
  }
  const int selE = (int)(uint32_t)s_pre_e;
  const uint64_t selF = s_pre_f;
  if (t == 0) {
    st->sel_E = selE;
    st->sel_fp = selF;
  }
  if (POP) {
    for (long long i = t; i < n; i += kSelThreads) {
      int E;
      uint64_t fp;
      const int32_t c = b.candId[i];
      cand_key(b, c, E, fp);
      if (key_le(E, fp, selE, selF)) {
        const long long o = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&st->pop_cnt), 1ull);
        if (o < b.B)
          b.popId[o] = c;
        else
          st->error = 1;
      }
    }
  }
}

// One block: the popped entries in key order (bitonic sort of (E, fp, id), padded to a power of two)
// become pivots 0..b-1; their pool slots are freed and leave the histogram.
__global__ void __launch_bounds__(kSelThreads) pq_pop_sort_kernel(PqBufs b) {
  PqState* st = b.st;
  const int nb = st->b;
  if (nb == 0) return;
  if (st->pop_cnt != nb || st->error) {  // an inconsistent pop: stop the search (capacity status)
    __syncthreads();
    if (threadIdx.x == 0) {
      st->error = 1;
      st->b = 0;
    }
    return;
  }
  extern __shared__ unsigned long long sm_pop[];
  unsigned long long* kf = sm_pop;                      // fingerprints
  int* ke = reinterpret_cast<int*>(sm_pop + kSortMax);  // energies
  int* ki = ke + kSortMax;                              // pool ids
  int n2 = 1;
  while (n2 < nb) n2 <<= 1;
  const int t = threadIdx.x;
  for (int i = t; i < n2; i += kSelThreads) {
    if (i < nb) {
      const int id = b.popId[i];
      kf[i] = b.pFp[id];
      ke[i] = b.pE[id];
      ki[i] = id;
    } else {
      kf[i] = ~0ull;
      ke[i] = INT32_MAX;
      ki[i] = -1;
    }
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = t; i < n2; i += kSelThreads) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const bool gt = key_lt(ke[j], kf[j], ke[i], kf[i]);  // a[i] > a[j]
          if (gt == up) {
            const unsigned long long f = kf[i];
            kf[i] = kf[j];
            kf[j] = f;
            const int e = ke[i];
            ke[i] = ke[j];
            ke[j] = e;
            const int d = ki[i];
            ki[i] = ki[j];
            ki[j] = d;
          }
        }
      }
      __syncthreads();
    }
  const int Eb = st->E_base;
  const long long top = st->free_top;
  for (int q = t; q < nb; q += kSelThreads) {
    const int id = ki[q];
    b.pivE[q] = ke[q];
    b.pivFp[q] = kf[q];
    for (int w = 0; w < b.W; w++) b.pivSeq[(size_t)q * b.W + w] = b.pSeq[(size_t)id * b.W + w];
    b.pE[id] = INT32_MAX;
    b.freeIds[top + q] = id;
    const int bin = e_bin(ke[q], Eb);
    atomicSub(&b.hP[bin], 1u);
    atomicSub(&b.hP2[bin / kCoarse], 1u);
  }
  __syncthreads();
  if (t == 0) st->free_top = top + nb;
}

// One warp per pivot: Delta E of all L single flips, visited-set test, dense survivor output.
__global__ void __launch_bounds__(32 * kPqWarps) pq_expand_kernel(PqBufs b, Layout ly) {
  __shared__ ScanSmem slabs[kPqWarps];
  __shared__ uint32_t rbits_all[kPqWarps][kBitWords];
  __shared__ int16_t P_all[kPqWarps][kMaxL];
  __shared__ uint32_t xbits_all[kPqWarps][kBitWords];
  ScanSmem& sm = slabs[threadIdx.x >> 5];
  uint32_t* rbits = rbits_all[threadIdx.x >> 5];
  int16_t* Pm = P_all[threadIdx.x >> 5];
  uint32_t* xbits = xbits_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const PqState* st = b.st;
  const int nb = st->b;
  for (int q = blockIdx.x * kPqWarps + (threadIdx.x >> 5); q < nb; q += gridDim.x * kPqWarps) {
    load_bits(sm, b.pivSeq + (size_t)q * b.W, b.L);
    build_table(sm, ly);
    const bool fast = pack_c8(sm, ly);
    const int SC = table_sum(sm, ly);
    build_bytes(sm, ly);
    p_all(sm, ly, xbits, rbits, Pm);
    const int E = b.pivE[q];
    const uint64_t fp = b.pivFp[q];
    for (int base = 0; base < ly.n_tiles; base += 32) {
      const int tau = base + lane;
      if (tau < ly.n_tiles) {
        int cls, q0;
        tile_of(ly, tau, cls, q0);
        int acc[kPqM];
        if (fast)
          scan_tile<kPqM, false>(sm, ly, cls, q0, acc);
        else
          scan_tile<kPqM, true>(sm, ly, cls, q0, acc);
        // the tile's Delta E and fingerprints, then the first visited-set probe of all of them at once
        // (independent loads), then the rare longer probe sequences
        int dv[kPqM], mv[kPqM];
        uint64_t fv[kPqM], hv[kPqM];
#pragma unroll
        for (int j = 0; j < kPqM; j++) {
          const SlotInfo si = slot_info(ly, cls, q0 + j);
          mv[j] = si.active ? si.m : 0;
          dv[j] = si.active ? finish_delta(sm, ly, cls, q0 + j, si, acc[j], SC, Pm[si.m - 1]) : 0;
          fv[j] = si.active ? fp ^ b.ztab[si.m - 1] : kEmptyKey;
        }
#pragma unroll
        for (int j = 0; j < kPqM; j++) hv[j] = (mv[j] && fv[j] != kEmptyKey) ? b.H[h_slot(fv[j], b.H_log2)] : kEmptyKey;
#pragma unroll
        for (int j = 0; j < kPqM; j++) {
          if (!mv[j]) continue;
          bool seen;
          if (fv[j] == kEmptyKey)
            seen = st->h_has_empty != 0;
          else if (hv[j] == fv[j] || hv[j] == kEmptyKey)
            seen = hv[j] == fv[j];
          else
            seen = h_contains_after(b, fv[j], h_slot(fv[j], b.H_log2));
          const size_t di = (size_t)q * b.width + (mv[j] - 1);
          b.dE[di] = seen ? INT32_MAX : E + dv[j];
          b.dFp[di] = fv[j];
        }
      }
    }
    // MAKE_ROTATIONS of the pivot: each rotation's energy and fingerprint from scratch
    for (int c = 0; c < 2 * b.Tr; c++) {
      const int r = rot_shift(b.L, b.Tr, c);
      for (int w = 0; w < kBitWords; w++) {
        const int i = 32 * w + lane;  // 0-based position of the rotated sequence
        int bit = 0;
        if (i < b.L) {
          int j = i + r;
          if (j >= b.L) j -= b.L;
          bit = seq_bit(sm, j + 1);
        }
        const unsigned word = __ballot_sync(kFull, bit);
        if (lane == 0) rbits[w] = word;
      }
      __syncwarp();
      int e = 0;
      for (int k = lane + 1; k < b.L; k += 32) {
        const int cv = corr_lag(rbits, b.L, k);
        e += cv * cv;
      }
      e = warp_sum_i32(e);
      uint64_t h = 0;
      for (int i = lane; i < b.L; i += 32)
        if (!((rbits[i >> 5] >> (i & 31)) & 1u)) h ^= b.ztab[i];
      h = warp_xor_u64(h);
      if (lane == 0) {
        const size_t di = (size_t)q * b.width + b.L + c;
        b.dE[di] = h_contains(b, h) ? INT32_MAX : e;
        b.dFp[di] = h;
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

// Dense survivors of the round: b pivots x width columns, or the seeds (one column each).
template <bool SEED>
__device__ __forceinline__ long long dense_n(const PqBufs& b, int n_seeds) {
  return SEED ? (long long)n_seeds : (long long)b.st->b * b.width;
}

// Dedup, first pass: every survivor inserts its (E, fp) key; the first inserter of a key creates the
// unique survivor (its representative is settled by the second pass).
template <bool SEED>
__global__ void __launch_bounds__(256) pq_dedup_insert_kernel(PqBufs b, int n_seeds) {
  const long long n = dense_n<SEED>(b, n_seeds);
  const uint64_t mask = (1ull << b.hs_log2) - 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    bool fresh = false;
    uint64_t slot = 0;
    int E = INT32_MAX;
    uint64_t fp = 0;
    if (i < n) {
      E = b.dE[i];
      fp = b.dFp[i];
    }
    if (E != INT32_MAX) {
      const uint64_t k = dedup_key(E, fp);
      uint64_t s = (k * kGamma) >> (64 - b.hs_log2);
      for (uint64_t it = 0; it <= mask; it++) {  // the table holds at most half its slots
        const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(&b.hkey[s]), 0ull, k);
        if (old == 0ull) {
          fresh = true;
          slot = s;
          break;
        }
        if (old == k) break;
        s = (s + 1) & mask;
      }
    }
    const long long u = warp_append(&b.st->nU, fresh);
    if (fresh) {
      b.uE[u] = E;
      b.uFp[u] = fp;
      b.uRep[u] = ~0u;
      b.uSlot[u] = (int32_t)slot;
      b.hval[slot] = (int32_t)u;
    }
  }
}

// Dedup, second pass: each survivor finds its key's slot and lowers the representative to the smallest
// (pivot, column) -- the pivots are in key order, so this is the sequential definition's first occurrence.
template <bool SEED>
__global__ void __launch_bounds__(256) pq_dedup_rep_kernel(PqBufs b, int n_seeds) {
  const long long n = dense_n<SEED>(b, n_seeds);
  const uint64_t mask = (1ull << b.hs_log2) - 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int E = b.dE[i];
    if (E == INT32_MAX) continue;
    const uint64_t k = dedup_key(E, b.dFp[i]);
    uint64_t s = (k * kGamma) >> (64 - b.hs_log2);
    for (uint64_t it = 0; it <= mask; it++) {
      if (b.hkey[s] == k) break;
      s = (s + 1) & mask;
    }
    const unsigned rep = SEED ? (unsigned)i << kColBits
                              : ((unsigned)(i / b.width) << kColBits) | (unsigned)(i % b.width);
    atomicMin(&b.uRep[b.hval[s]], rep);
  }
}

// The round's smallest survivor energy.
__global__ void __launch_bounds__(256) pq_u_min_kernel(PqBufs b) {
  const long long n = b.st->nU;
  int m = INT32_MAX;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
    m = min(m, b.uE[u]);
  m = __reduce_min_sync(kFull, m);
  if (lane_id() == 0 && m != INT32_MAX) atomicMin(&b.st->minE_round, m);
}

// The histogram's energy window, from the smallest seed energy (improvements stay far inside it).
__global__ void pq_set_window_kernel(PqBufs b) {
  PqState* st = b.st;
  st->E_base = st->minE_round == INT32_MAX ? 0 : max(0, st->minE_round - kNB / 2);
}

// Survivor histogram, and the smallest fingerprint among the smallest-energy survivors.
__global__ void __launch_bounds__(256) pq_u_hist_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->nU;
  const int Eb = st->E_base, mE = st->minE_round;
  uint64_t mf = ~0ull;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    const int E = b.uE[u];
    const int bin = e_bin(E, Eb);
    atomicAdd(&b.hU[bin], 1u);
    atomicAdd(&b.hU2[bin / kCoarse], 1u);
    if (E == mE) mf = min(mf, b.uFp[u]);
  }
  if (mf != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(&st->minfp_round), (unsigned long long)mf);
}

// The representative of the smallest survivor key (unique).
__global__ void __launch_bounds__(256) pq_u_best_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->nU;
  const int mE = st->minE_round;
  const uint64_t mf = st->minfp_round;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
    if (b.uE[u] == mE && b.uFp[u] == mf) st->best_rep_round = b.uRep[u];
}

// One thread: the best (a strict improvement, as in Algorithm 2; for the seeds, the smallest seed) and
// the round's counters.
template <bool SEED>
__global__ void pq_best_kernel(PqBufs b) {
  PqState* st = b.st;
  if (!SEED && st->b == 0) return;
  const unsigned rep = st->best_rep_round;
  if (SEED) {
    if (st->nU > 0 && (rep >> kColBits) < (unsigned)b.n_seeds) {
      st->best_E = st->minE_round;
      st->best_fp = st->minfp_round;
      const int q = (int)(rep >> kColBits);
      for (int t = 0; t < b.W; t++) b.best_seq[t] = b.seeds[(size_t)q * b.W + t];
    }
    return;
  }
  st->survivors += st->nU;
  if (st->nU > 0 && (rep >> kColBits) >= (unsigned)st->b) {  // every survivor has a representative
    st->error = 1;
    return;
  }
  if (st->nU > 0 && st->minE_round < st->best_E) {
    st->best_E = st->minE_round;
    st->best_fp = st->minfp_round;
    pq_child(b.pivSeq + (size_t)(rep >> kColBits) * b.W, b, (int)(rep & ((1u << kColBits) - 1u)), b.best_seq);
    st->improvements++;
    st->u = 0;
  } else {
    st->u += st->b;
  }
}

// Whether a key of bin `bin` is inside the cut.
__device__ __forceinline__ bool below_cut(const PqState* st, int bin, int E, uint64_t fp) {
  if (st->sel_need < 0) return true;  // no cut
  return bin < st->sel_bin || (bin == st->sel_bin && key_le(E, fp, st->sel_E, st->sel_fp));
}

// Pool pass: the entries beyond the cut are evicted (slot freed, histogram updated).
__global__ void __launch_bounds__(256) pq_evict_kernel(PqBufs b) {
  PqState* st = b.st;
  if (st->sel_need < 0) return;
  const int Eb = st->E_base;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < b.cap; base += stride) {
    const long long i = base + threadIdx.x;
    bool out = false;
    int bin = 0;
    if (i < b.cap) {
      const int E = b.pE[i];
      if (E != INT32_MAX) {
        bin = e_bin(E, Eb);
        out = !below_cut(st, bin, E, b.pFp[i]);
      }
    }
    const long long o = warp_append(&st->free_top, out);
    if (out) {
      b.freeIds[o] = (int32_t)i;
      b.pE[i] = INT32_MAX;
      atomicSub(&b.hP[bin], 1u);
      atomicSub(&b.hP2[bin / kCoarse], 1u);
    }
    warp_add(&st->ev_round, out ? 1 : 0);
  }
}

// Survivor pass: the survivors inside the cut take a free slot (the sequence built from the pivot, or
// copied from the seed) and enter the visited set; every survivor clears its dedup slot.
template <bool SEED>
__global__ void __launch_bounds__(256) pq_admit_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->nU;
  const int Eb = st->E_base;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long u = base + threadIdx.x;
    bool in = false;
    int E = 0, bin = 0;
    uint64_t fp = 0;
    if (u < n) {
      E = b.uE[u];
      fp = b.uFp[u];
      bin = e_bin(E, Eb);
      in = below_cut(st, bin, E, fp);
      b.hkey[b.uSlot[u]] = 0ull;
    }
    // free slots come off the top of the stack, one atomic per warp
    const unsigned m = __ballot_sync(kFull, in);
    long long top = 0;
    if (m) {
      const int leader = __ffs(m) - 1;
      if (lane_id() == leader)
        top = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&st->free_top),
                                   (unsigned long long)(-(long long)__popc(m)));
      top = __shfl_sync(kFull, top, leader);
    }
    int ins = 0;
    const long long o = top - 1 - __popc(m & ((1u << lane_id()) - 1u));
    if (in && o < 0) {  // more admissions than free slots: only an inconsistent state gets here
      st->error = 1;
      in = false;
    }
    const unsigned rep = in ? b.uRep[u] : 0u;
    if (in && (rep >> kColBits) >= (unsigned)(SEED ? b.n_seeds : st->b)) {  // every survivor has one (pass 2)
      st->error = 1;
      in = false;
    }
    if (in) {
      const int id = b.freeIds[o];
      b.pE[id] = E;
      b.pFp[id] = fp;
      if (SEED) {
        for (int t = 0; t < b.W; t++) b.pSeq[(size_t)id * b.W + t] = b.seeds[(size_t)(rep >> kColBits) * b.W + t];
      } else {
        pq_child(b.pivSeq + (size_t)(rep >> kColBits) * b.W, b, (int)(rep & ((1u << kColBits) - 1u)),
                 b.pSeq + (size_t)id * b.W);
      }
      atomicAdd(&b.hP[bin], 1u);
      atomicAdd(&b.hP2[bin / kCoarse], 1u);
      ins = h_insert(b, fp);
    }
    h_count(b, ins);
    warp_add(&st->adm_round, in ? 1 : 0);
  }
}

template <bool SEED>
__global__ void pq_round_end_kernel(PqBufs b) {
  PqState* st = b.st;
  if (SEED) {
    st->nP = st->adm_round;
  } else {
    if (st->b == 0) return;
    st->nP = st->nP - st->b - st->ev_round + st->adm_round;
    st->admitted += st->adm_round;
    st->evicted += st->ev_round;
    st->expansions += st->b;
    st->rounds++;
  }
  const long long slots = 1ll << b.H_log2;
  if (st->h_size * 4 > slots * 3) st->error = 1;
}

__global__ void pq_write_stats_kernel(PqBufs b, int32_t* best_E, labs_pq_stats* out) {
  const PqState* st = b.st;
  *best_E = st->best_E;
  out->expansions = st->expansions;
  out->rounds = st->rounds;
  out->survivors = st->survivors;
  out->admitted = st->admitted;
  out->evicted = st->evicted;
  out->h_size = st->h_size;
  out->improvements = st->improvements;
  out->best_fp = st->best_fp;
  out->stop_reason = st->stop == 4 ? 0 : st->stop;
  out->status = st->error ? LABS_ERR_CAPACITY : LABS_OK;
}

}  // namespace

int launch_pq_refine(labs_ctx* ctx, const labs_pq_cfg* cfg, const uint64_t* seeds, int n_seeds, uint64_t* best_seq,
                     int32_t* best_E, labs_pq_stats* stats, cudaStream_t st) {
  const int L = cfg->L, W = (L + 63) / 64;
  if (cfg->B > kSortMax) return LABS_ERR_INVALID_ARG;
  Layout ly;
  if (!make_layout(ly, L, 0, 0, kPqM)) return LABS_ERR_INVALID_ARG;
  const int width = L + 2 * cfg->T_r;
  const long long n_dense = std::max<long long>((long long)cfg->B * width, n_seeds);
  int hs_log2 = 10;
  while ((1ll << hs_log2) < 2 * n_dense) hs_log2++;
  const long long cap = cfg->cap;
  // workspace layout (one region, 256-byte aligned pieces)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t opE = take(4 * cap), opF = take(8 * cap), opS = take(8 * cap * W), ofree = take(4 * cap);
  const size_t ohP = take(4 * kNB), ohP2 = take(4 * kNC), ohU = take(4 * kNB), ohU2 = take(4 * kNC);
  const size_t opop = take(4 * (size_t)cfg->B), opivE = take(4 * (size_t)cfg->B), opivF = take(8 * (size_t)cfg->B);
  const size_t opivS = take(8 * (size_t)cfg->B * W);
  const size_t ocand = take(4 * (size_t)(cap + n_dense));
  const size_t odE = take(4 * n_dense), odF = take(8 * n_dense);
  const size_t ohk = take(8ull << hs_log2), ohv = take(4ull << hs_log2);
  const size_t ouE = take(4 * n_dense), ouF = take(8 * n_dense), ouR = take(4 * n_dense), ouS = take(4 * n_dense);
  const size_t ozt = take(8 * L), ost = take(sizeof(PqState)), obest = take(8 * W);
  const size_t oH = take(8ull << cfg->H_log2);
  char* base = static_cast<char*>(ws_get(ctx, kWsPq0, off));
  if (!base) return LABS_ERR_NOMEM;
  PqBufs b{};
  b.L = L;
  b.W = W;
  b.B = cfg->B;
  b.Tr = cfg->T_r;
  b.width = width;
  b.H_log2 = cfg->H_log2;
  b.cap = cap;
  b.max_exp = cfg->max_expansions;
  b.T_u = cfg->T_u;
  b.hs_log2 = hs_log2;
  b.cand_cap = cap + n_dense;
  b.n_seeds = n_seeds;
  b.pE = reinterpret_cast<int32_t*>(base + opE);
  b.pFp = reinterpret_cast<uint64_t*>(base + opF);
  b.pSeq = reinterpret_cast<uint64_t*>(base + opS);
  b.freeIds = reinterpret_cast<int32_t*>(base + ofree);
  b.hP = reinterpret_cast<unsigned*>(base + ohP);
  b.hP2 = reinterpret_cast<unsigned*>(base + ohP2);
  b.hU = reinterpret_cast<unsigned*>(base + ohU);
  b.hU2 = reinterpret_cast<unsigned*>(base + ohU2);
  b.popId = reinterpret_cast<int32_t*>(base + opop);
  b.pivE = reinterpret_cast<int32_t*>(base + opivE);
  b.pivFp = reinterpret_cast<uint64_t*>(base + opivF);
  b.pivSeq = reinterpret_cast<uint64_t*>(base + opivS);
  b.candId = reinterpret_cast<int32_t*>(base + ocand);
  b.dE = reinterpret_cast<int32_t*>(base + odE);
  b.dFp = reinterpret_cast<uint64_t*>(base + odF);
  b.hkey = reinterpret_cast<uint64_t*>(base + ohk);
  b.hval = reinterpret_cast<int32_t*>(base + ohv);
  b.uE = reinterpret_cast<int32_t*>(base + ouE);
  b.uFp = reinterpret_cast<uint64_t*>(base + ouF);
  b.uRep = reinterpret_cast<unsigned*>(base + ouR);
  b.uSlot = reinterpret_cast<int32_t*>(base + ouS);
  b.ztab = reinterpret_cast<uint64_t*>(base + ozt);
  b.st = reinterpret_cast<PqState*>(base + ost);
  b.best_seq = reinterpret_cast<uint64_t*>(base + obest);
  b.H = reinterpret_cast<uint64_t*>(base + oH);
  b.seeds = seeds;

  const unsigned g_pool = (unsigned)std::max(1ll, std::min<long long>((cap + 255) / 256, (long long)ctx->num_sms * 16));
  const unsigned g_dense =
      (unsigned)std::max(1ll, std::min<long long>((n_dense + 255) / 256, (long long)ctx->num_sms * 16));
  const size_t sort_smem = (size_t)kSortMax * 16;
  if (cudaFuncSetAttribute(pq_pop_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem) !=
      cudaSuccess)
    return LABS_ERR_CUDA;

  // The survivor path, shared by the seeds and every round: dedup, best, cut, eviction, admission.
  auto survivor_path = [&](bool seed, cudaStream_t s) {
    if (seed) {
      pq_dedup_insert_kernel<true><<<g_dense, 256, 0, s>>>(b, n_seeds);
      pq_dedup_rep_kernel<true><<<g_dense, 256, 0, s>>>(b, n_seeds);
    } else {
      pq_dedup_insert_kernel<false><<<g_dense, 256, 0, s>>>(b, n_seeds);
      pq_dedup_rep_kernel<false><<<g_dense, 256, 0, s>>>(b, n_seeds);
    }
    pq_u_min_kernel<<<g_dense, 256, 0, s>>>(b);
    if (seed) pq_set_window_kernel<<<1, 1, 0, s>>>(b);
    pq_u_hist_kernel<<<g_dense, 256, 0, s>>>(b);
    pq_u_best_kernel<<<g_dense, 256, 0, s>>>(b);
    if (seed)
      pq_best_kernel<true><<<1, 1, 0, s>>>(b);
    else
      pq_best_kernel<false><<<1, 1, 0, s>>>(b);
    pq_select_kernel<false><<<1, kSelThreads, 0, s>>>(b);
    pq_gather_kernel<false, false><<<g_pool, 256, 0, s>>>(b);
    pq_gather_kernel<false, true><<<g_dense, 256, 0, s>>>(b);
    pq_boundary_kernel<false><<<1, kSelThreads, 0, s>>>(b);
    pq_evict_kernel<<<g_pool, 256, 0, s>>>(b);
    if (seed) {
      pq_admit_kernel<true><<<g_dense, 256, 0, s>>>(b);
      pq_round_end_kernel<true><<<1, 1, 0, s>>>(b);
    } else {
      pq_admit_kernel<false><<<g_dense, 256, 0, s>>>(b);
      pq_round_end_kernel<false><<<1, 1, 0, s>>>(b);
    }
    cudaMemsetAsync(b.hU, 0, 4 * kNB, s);
    cudaMemsetAsync(b.hU2, 0, 4 * kNC, s);
  };

  // ---- set-up: visited set, pool, histograms, dedup table, Zobrist keys; the seeds go through the
  // survivor path into the empty pool (equal seeds kept once, the cap smallest admitted)
  if (cudaMemsetAsync(b.H, 0xff, 8ull << cfg->H_log2, st) != cudaSuccess) return LABS_ERR_CUDA;
  if (cudaMemsetAsync(b.hP, 0, 4 * kNB, st) != cudaSuccess || cudaMemsetAsync(b.hP2, 0, 4 * kNC, st) != cudaSuccess ||
      cudaMemsetAsync(b.hU, 0, 4 * kNB, st) != cudaSuccess || cudaMemsetAsync(b.hU2, 0, 4 * kNC, st) != cudaSuccess ||
      cudaMemsetAsync(b.hkey, 0, 8ull << hs_log2, st) != cudaSuccess)
    return LABS_ERR_CUDA;
  pq_ztab_kernel<<<(L + 255) / 256, 256, 0, st>>>(b.ztab, L);
  pq_init_kernel<<<g_pool, 256, 0, st>>>(b);
  pq_seed_kernel<<<(unsigned)std::min<long long>((n_seeds + kPqWarps - 1) / kPqWarps, ctx->num_sms * 16), 32 * kPqWarps,
                   0, st>>>(b, n_seeds);
  survivor_path(true, st);
  if (cudaGetLastError() != cudaSuccess) return LABS_ERR_CUDA;

  // ---- rounds
  const long long max_rounds = (cfg->max_expansions + cfg->B - 1) / cfg->B + 1;
  const unsigned exp_blocks = (unsigned)std::max(1ll, std::min<long long>((cfg->B + kPqWarps - 1) / kPqWarps,
                                                                        (long long)ctx->num_sms * 8));
  // Every round issues the same launches with the same arguments (a round's sizes and stop state live
  // in device memory), so one round is captured as a CUDA graph and replayed.
  if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return LABS_ERR_CUDA;
  if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LABS_ERR_CUDA;
  {
    cudaStream_t cs = ctx->capture_stream;
    pq_round_begin_kernel<<<1, 1, 0, cs>>>(b);
    pq_select_kernel<true><<<1, kSelThreads, 0, cs>>>(b);
    pq_gather_kernel<true, false><<<g_pool, 256, 0, cs>>>(b);
    pq_boundary_kernel<true><<<1, kSelThreads, 0, cs>>>(b);
    pq_pop_sort_kernel<<<1, kSelThreads, sort_smem, cs>>>(b);
    pq_expand_kernel<<<exp_blocks, 32 * kPqWarps, 0, cs>>>(b, ly);
    survivor_path(false, cs);
  }
  cudaGraph_t round_graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &round_graph);
  cudaGraphExec_t round_exec = nullptr;
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&round_exec, round_graph, 0);
  if (round_graph) cudaGraphDestroy(round_graph);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return LABS_ERR_CUDA;
  }
  int* hstop = nullptr;
  if (cudaMallocHost(&hstop, sizeof(int)) != cudaSuccess) {
    cudaGraphExecDestroy(round_exec);
    return LABS_ERR_NOMEM;
  }
  int status = LABS_OK;
  for (long long r = 0; r < max_rounds; r++) {
    if (cudaGraphLaunch(round_exec, st) != cudaSuccess) {
      status = LABS_ERR_CUDA;
      break;
    }
    if ((r & 31) == 31 || r + 1 == max_rounds) {  // poll the stop flag
      if (cudaMemcpyAsync(hstop, &b.st->stop, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        status = LABS_ERR_CUDA;
        break;
      }
      if (*hstop) break;
    }
  }
  // the last round may end on the budget without a following begin: settle the stop reason
  pq_round_begin_kernel<<<1, 1, 0, st>>>(b);
  pq_write_stats_kernel<<<1, 1, 0, st>>>(b, best_E, stats);
  if (cudaMemcpyAsync(best_seq, b.best_seq, 8 * W, cudaMemcpyDeviceToDevice, st) != cudaSuccess) status = LABS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) status = LABS_ERR_CUDA;
  cudaFreeHost(hstop);
  cudaGraphExecDestroy(round_exec);
  return status;
}

}  // namespace labsg
