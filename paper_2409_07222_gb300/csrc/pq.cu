// pq.cu -- step 2 of the dual-step search: Algorithm 2's priority-queue refinement over the unrestricted
// space, in batch-synchronous form (labs_pq_refine).
//
// GB300 mapping.  The paper runs one priority queue per candidate in Rust on CPU cores; here one open
// set of the cap smallest (E, fp) keys lives in HBM as an UNORDERED pool of entries (energy,
// fingerprint, sequence) with a free-slot stack, and beside it a histogram of the entries' energies
// (one bin per energy, clamped at both ends of a 2^17-bin window, and a coarse level whose bins each
// cover 256 fine bins).  The B smallest keys, or the cap smallest, are then found without ordering the pool: the
// histogram's prefix sums give the bin where the count is reached, every entry below it is taken, and
// only the entries of that one boundary bin are ranked (a radix select on their full (E, fp) key, so a
// clamped bin holding several energies is still exact).  A round
//   pop      -- the b = min(B, open, budget left) smallest keys leave the pool (one pass over it), are
//               ranked among themselves (a 2-D grid counts, for each, the smaller keys) and become the
//               round's pivots in key order;
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
  long long n_dense;    // dense survivor entries of the round: b x width, or the seeds
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
  int pmax_bin;        // highest occupied bin of the pool after the pops (-1: empty pool)
  int hist_mode;       // survivor histogram: 0 none (everything fits), 1 bins <= pmax_bin only, 2 all
  long long nU_low;    // survivors in bins <= pmax_bin
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
  int32_t* popId;     // pool ids gathered for popping [B], with their keys
  int32_t* popE;
  uint64_t* popF;
  int32_t* pivE;      // pivots in key order [B]
  uint64_t* pivFp;
  uint64_t* pivSeq;   // [B][W]
  int32_t* candId;    // boundary candidates: pool id >= 0, or -(u + 1) for survivor u
  int32_t* cE;        // their keys, gathered contiguously
  uint64_t* cF;
  int32_t* popRank;   // rank of each popped entry among the pops (its pivot index)
  int32_t* dE;        // dense survivors [pivot][column]: energy, or INT32_MAX (visited)
  uint64_t* dFp;
  uint64_t* hkey;     // dedup hash table: mixed (E, fp) key, 0 = empty
  int32_t* hval;      // the unique survivor of a slot
  unsigned* uRep;     // per dense entry: ~0 unless it is the unique survivor of its key, whose
                      // representative (pivot << kColBits | column) is the smallest of the equal keys
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

// Block-wide sum added to *ctr with one atomic per block (every thread of the block calls it).
__device__ __forceinline__ void block_add(long long* ctr, long long v) {
  __shared__ long long part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane_id() == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    if (t) atomicAdd(reinterpret_cast<unsigned long long*>(ctr), (unsigned long long)t);
  }
  __syncthreads();
}

// Block-wide minimum folded into *dst with one atomic per block (every thread calls it).
__device__ __forceinline__ void block_min(int* dst, int v) {
  __shared__ int part[32];
  v = __reduce_min_sync(kFull, v);
  if (lane_id() == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = INT32_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = min(t, part[w]);
    if (t != INT32_MAX) atomicMin(dst, t);
  }
  __syncthreads();
}

// Adds delta to the fine and coarse histogram bins of every lane with bin >= 0, one atomic per distinct
// bin of the warp (every lane calls it): the energies of a round crowd into few bins, and same-address
// atomics from every thread would serialise there.
__device__ __forceinline__ void hist_add(unsigned* fine, unsigned* coarse, int bin, int delta) {
  if (!__any_sync(kFull, bin >= 0)) return;  // most warps of a pass change nothing
  const unsigned lt = (1u << lane_id()) - 1u;
  const unsigned pf = __match_any_sync(kFull, bin);
  if (bin >= 0 && (pf & lt) == 0) atomicAdd(&fine[bin], (unsigned)(delta * __popc(pf)));
  const int cb = bin >= 0 ? bin / kCoarse : -1;
  const unsigned pc = __match_any_sync(kFull, cb);
  if (cb >= 0 && (pc & lt) == 0) atomicAdd(&coarse[cb], (unsigned)(delta * __popc(pc)));
}

// Mixed key of (E, fp) for the dedup table; 0 marks an empty slot, so a mixed key of 0 becomes 1.
__device__ __forceinline__ uint64_t dedup_key(int E, uint64_t fp) {
  const uint64_t k = fp ^ ((uint64_t)(uint32_t)E * 0xD6E8FEB86659FD93ull);
  return k ? k : 1ull;
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
    z.pmax_bin = -1;
    z.n_dense = b.n_seeds;
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
  st->n_dense = 0;
  st->ev_round = 0;
  st->adm_round = 0;
  st->minE_round = INT32_MAX;
  st->minfp_round = ~0ull;
  st->best_rep_round = ~0u;
  st->nU_low = 0;
  st->hist_mode = 0;
  if (st->stop) {
    st->b = 0;
    return;
  }
  long long bb = min((long long)b.B, st->nP);
  bb = min(bb, b.max_exp - st->expansions);
  st->b = (int)bb;
  st->n_dense = bb * b.width;
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
      target = st->hist_mode ? b.cap : -1;
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
// boundary bin (popped) and those in it (candidates); the cut gathers the boundary bin's entries.  Each
// thread takes four consecutive entries with one 16-byte load of their energies (the pool and the dense
// arrays are 256-byte aligned, their sizes rounded to whole quads by the workspace layout).
template <bool POP, bool U>
__global__ void __launch_bounds__(256) pq_gather_kernel(PqBufs b) {
  PqState* st = b.st;
  if (POP ? st->b == 0 : st->sel_need <= 0) return;
  const int sel = st->sel_bin, Eb = st->E_base;
  const long long n = U ? st->n_dense : b.cap;
  const long long nq = (n + 3) >> 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nq; base += stride) {
    const long long qd = base + threadIdx.x;
    int4 e4 = make_int4(INT32_MAX, INT32_MAX, INT32_MAX, INT32_MAX);
    uint4 r4 = make_uint4(0u, 0u, 0u, 0u);
    if (qd < nq) {
      e4 = reinterpret_cast<const int4*>(U ? b.dE : b.pE)[qd];
      if (U) r4 = reinterpret_cast<const uint4*>(b.uRep)[qd];
    }
    const int ev[4] = {e4.x, e4.y, e4.z, e4.w};
    const unsigned rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const long long i = 4 * qd + e;
      int bin = kNB;
      int E = INT32_MAX;
      if (i < n) {
        E = U ? (rv[e] != ~0u ? ev[e] : INT32_MAX) : ev[e];
        if (E != INT32_MAX) bin = e_bin(E, Eb);
      }
      // the histogram bounds both counts (b entries below the boundary bin at most); a count beyond a
      // buffer can only come from an inconsistent state, which is reported instead of written
      if (POP) {
        const long long o = warp_append(&st->pop_cnt, bin < sel);
        if (o >= b.B) {
          st->error = 1;
        } else if (o >= 0) {
          b.popId[o] = (int32_t)i;
          b.popE[o] = E;
          b.popF[o] = b.pFp[i];
        }
      }
      const long long o2 = warp_append(&st->cand_cnt, bin == sel);
      if (o2 >= b.cand_cap) {
        st->error = 1;
      } else if (o2 >= 0) {
        b.candId[o2] = U ? -(int32_t)i - 1 : (int32_t)i;
        b.cE[o2] = E;
        b.cF[o2] = U ? b.dFp[i] : b.pFp[i];
      }
    }
  }
}

// One block: the sel_need smallest (E, fp) keys among the boundary candidates, by a most-significant-
// digit-first radix select over the 96-bit key (four energy bytes, then eight fingerprint bytes; the
// energy bytes are skipped when the boundary bin holds one energy, i.e. it is not clamped); keys are
// distinct, so exactly sel_need candidates are <= the selected key.  The candidates are streamed from the
// gather arrays until those that match the digits fixed so far fit in shared memory; they are staged
// there and the remaining digits rank only them.  POP appends the selected candidates to the pops.
constexpr int kCandSmem = 8192;  // candidates staged in shared memory (12 B each)
template <bool POP>
__global__ void __launch_bounds__(kSelThreads) pq_boundary_kernel(PqBufs b) {
  PqState* st = b.st;
  if (POP ? st->b == 0 : st->sel_need <= 0) return;
  const long long n = min(st->cand_cnt, b.cand_cap);
  extern __shared__ unsigned long long sm_cand[];
  uint64_t* sF = reinterpret_cast<uint64_t*>(sm_cand);
  int* sE = reinterpret_cast<int*>(sm_cand + kCandSmem);
  __shared__ unsigned hist[256];
  __shared__ unsigned wsum[8];                     // bin-count totals of the eight warps' 32 bins
  __shared__ unsigned long long s_pre_e, s_pre_f;  // the digits fixed so far
  __shared__ long long s_k, s_match;               // rank still to find; candidates matching the digits
  __shared__ int s_ns;                             // candidates staged
  const int t = threadIdx.x;
  const bool one_energy = st->sel_bin > 0 && st->sel_bin < kNB - 1;
  if (t == 0) {
    s_pre_e = one_energy ? (unsigned long long)(uint32_t)(st->E_base + st->sel_bin) : 0ull;
    s_pre_f = 0;
    s_k = st->sel_need;
    s_match = n;
    s_ns = 0;
  }
  __syncthreads();
  bool staged = false;
  const int d0 = one_energy ? 4 : 0;
  for (int d = d0; d < 12; d++) {
    // the shared selection state is read here, behind the previous iteration's last barrier: the thread
    // of the crossing bin rewrites it below while the others still test their bins
    const unsigned long long pe = s_pre_e, pf = s_pre_f;
    const long long k = s_k;
    // does key (ue, fp) match the digits fixed before digit d?
    auto match = [&](uint64_t ue, uint64_t fp) {
      if (d < 4) return d == 0 || (ue >> (32 - 8 * d)) == (pe >> (32 - 8 * d));
      return ue == pe && (d == 4 || (fp >> (64 - 8 * (d - 4))) == (pf >> (64 - 8 * (d - 4))));
    };
    if (!staged && s_match <= kCandSmem) {  // stage the matching candidates
      for (long long i = t; i < n; i += kSelThreads) {
        const uint64_t ue = (uint32_t)b.cE[i], fp = b.cF[i];
        if (d == d0 || match(ue, fp)) {
          const int w = atomicAdd(&s_ns, 1);
          if (w < kCandSmem) {
            sF[w] = fp;
            sE[w] = (int)(uint32_t)ue;
          }
        }
      }
      staged = true;
      __syncthreads();
    }
    if (t < 256) hist[t] = 0;
    __syncthreads();
    const long long nsel = staged ? min((long long)s_ns, (long long)kCandSmem) : n;
    for (long long i = t; i < nsel; i += kSelThreads) {
      const uint64_t ue = (uint32_t)(staged ? sE[i] : b.cE[i]);
      const uint64_t fp = staged ? sF[i] : b.cF[i];
      if (d == d0 || match(ue, fp)) {
        const unsigned digit = d < 4 ? (unsigned)(ue >> (24 - 8 * d)) & 255u : (unsigned)(fp >> (56 - 8 * (d - 4))) & 255u;
        atomicAdd(&hist[digit], 1u);
      }
    }
    __syncthreads();
    // the digit where the count reaches k: an inclusive scan of the 256 bins (a shuffle scan per warp of
    // 32 bins, then the eight warp totals), then the one bin that crosses k
    const unsigned own = t < 256 ? hist[t] : 0u;
    unsigned c = own;
    if (t < 256) {
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, c, off);
        if (lane_id() >= off) c += v;
      }
      if (lane_id() == 31) wsum[t >> 5] = c;
    }
    __syncthreads();
    if (t < 256) {
      unsigned add = 0;
      for (int w = 0; w < (t >> 5); w++) add += wsum[w];
      c += add;
      const long long before = (long long)(c - own);
      if (before < k && (long long)c >= k) {
        s_k = k - before;
        s_match = own;
        if (d < 4)
          s_pre_e = pe | ((unsigned long long)t << (24 - 8 * d));
        else
          s_pre_f = pf | ((unsigned long long)t << (56 - 8 * (d - 4)));
      }
    }
    __syncthreads();
    // one candidate left with the digits fixed so far: it is the selected key, whatever its remaining
    // digits (candidate keys are distinct)
    if (s_match == 1 && d < 11) {
      const unsigned long long pe2 = s_pre_e, pf2 = s_pre_f;
      const int dn = d + 1;  // digits fixed now
      const long long m2 = staged ? min((long long)s_ns, (long long)kCandSmem) : n;
      for (long long i = t; i < m2; i += kSelThreads) {
        const uint64_t ue = (uint32_t)(staged ? sE[i] : b.cE[i]);
        const uint64_t fp = staged ? sF[i] : b.cF[i];
        const bool hit = dn <= 4 ? (ue >> (32 - 8 * dn)) == (pe2 >> (32 - 8 * dn))
                                 : ue == pe2 && (fp >> (64 - 8 * (dn - 4))) == (pf2 >> (64 - 8 * (dn - 4)));
        if (hit) {
          s_pre_e = ue;
          s_pre_f = fp;
        }
      }
      __syncthreads();
      break;
    }
  }
  const int selE = (int)(uint32_t)s_pre_e;
  const uint64_t selF = s_pre_f;
  if (t == 0) {
    st->sel_E = selE;
    st->sel_fp = selF;
    if (s_ns > kCandSmem) st->error = 1;  // cannot happen: at most s_match <= kCandSmem are staged
  }
  if (POP) {
    for (long long i = t; i < n; i += kSelThreads) {
      if (key_le(b.cE[i], b.cF[i], selE, selF)) {
        const long long o = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&st->pop_cnt), 1ull);
        if (o < b.B) {
          b.popId[o] = b.candId[i];
          b.popE[o] = b.cE[i];
          b.popF[o] = b.cF[i];
        } else {
          st->error = 1;
        }
      }
    }
  }
}

// Grid (x: 256 popped entries per block, y: kRankChunks slices of the others): the popped entries in key
// order.  Keys are distinct, so the number of popped keys smaller than a key is its rank; every block
// adds its slice's count to the entry's rank.
constexpr int kRankChunks = 16;
__global__ void __launch_bounds__(256) pq_pop_rank_kernel(PqBufs b) {
  PqState* st = b.st;
  const int nb = st->b;
  if (nb == 0) return;
  if (st->pop_cnt != nb || st->error) {  // an inconsistent pop: stop the search (capacity status)
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      st->error = 1;
      st->b = 0;
      st->n_dense = 0;
    }
    return;
  }
  __shared__ uint64_t sF[kSortMax / kRankChunks];
  __shared__ int sE[kSortMax / kRankChunks];
  const int per = (nb + kRankChunks - 1) / kRankChunks;
  const int j0 = blockIdx.y * per, j1 = min(nb, j0 + per);
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    sF[j - j0] = b.popF[j];
    sE[j - j0] = b.popE[j];
  }
  __syncthreads();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += gridDim.x * blockDim.x) {
    const int E = b.popE[q];
    const uint64_t fp = b.popF[q];
    int r = 0;
    for (int j = 0; j < j1 - j0; j++) r += key_lt(sE[j], sF[j], E, fp) ? 1 : 0;
    if (r) atomicAdd(&b.popRank[q], r);
  }
}

// Grid: the pivots' sequences leave their pool slots, which are freed (pushed on the stack) and leave
// the histogram.
__global__ void __launch_bounds__(256) pq_pivot_kernel(PqBufs b) {
  PqState* st = b.st;
  const int nb = st->b;
  const int Eb = st->E_base;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nb; base += stride) {
    const long long q = base + threadIdx.x;
    const bool on = q < nb;
    int id = 0, bin = -1;
    if (on) {
      int r = b.popRank[q];  // pivot index = rank (keys are distinct, so 0 <= r < nb)
      if (r < 0 || r >= nb) {
        st->error = 1;
        r = (int)q;
      }
      id = b.popId[q];
      const int E = b.popE[q];
      b.pivE[r] = E;
      b.pivFp[r] = b.popF[q];
      for (int w = 0; w < b.W; w++) b.pivSeq[(size_t)r * b.W + w] = b.pSeq[(size_t)id * b.W + w];
      b.pE[id] = INT32_MAX;
      b.popRank[q] = 0;  // cleared for the next round
      bin = e_bin(E, Eb);
    }
    const long long o = warp_append(&st->free_top, on);
    if (on) b.freeIds[o] = id;
    hist_add(b.hP, b.hP2, bin, -1);
  }
}

// One block: the highest occupied bin of the pool (after the pops), -1 when it is empty.
__global__ void __launch_bounds__(kSelThreads) pq_pmax_kernel(PqBufs b) {
  __shared__ int s_cb, s_fb;
  const int t = threadIdx.x;
  if (t == 0) {
    s_cb = -1;
    s_fb = -1;
  }
  __syncthreads();
  if (t < kNC && b.hP2[t]) atomicMax(&s_cb, t);
  __syncthreads();
  const int cb = s_cb;
  if (cb >= 0 && t < kCoarse && b.hP[cb * kCoarse + t]) atomicMax(&s_fb, cb * kCoarse + t);
  __syncthreads();
  if (t == 0) b.st->pmax_bin = cb >= 0 ? s_fb : -1;
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

// Dedup, first pass: every survivor inserts its (E, fp) key; the first inserter of a key becomes the
// key's unique survivor (marked in uRep, its representative settled by the second pass) and the table
// slot points to its dense index.  Unique survivors stay at their dense index: nothing is compacted.
// Each thread takes four consecutive survivors and keeps their four probes in flight together (the
// pass is bound by the latency of the table's compare-and-swaps).
template <bool SEED>
__global__ void __launch_bounds__(256) pq_dedup_insert_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->n_dense;
  const long long nq = (n + 3) >> 2;
  const uint64_t mask = (1ull << b.hs_log2) - 1;
  const int Eb = st->E_base, pmax = st->pmax_bin;
  long long fresh_n = 0, low = 0;
  int mE = INT32_MAX;
  for (long long qd = (long long)blockIdx.x * blockDim.x + threadIdx.x; qd < nq; qd += (long long)gridDim.x * blockDim.x) {
    const int4 e4 = reinterpret_cast<const int4*>(b.dE)[qd];
    const int E[4] = {e4.x, e4.y, e4.z, e4.w};
    uint64_t k[4], s[4];
    bool act[4], fresh[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long i = 4 * qd + j;
      act[j] = i < n && E[j] != INT32_MAX;
      fresh[j] = false;
      k[j] = act[j] ? dedup_key(E[j], b.dFp[i]) : 0ull;
      s[j] = (k[j] * kGamma) >> (64 - b.hs_log2);
    }
    for (uint64_t it = 0; it <= mask && (act[0] || act[1] || act[2] || act[3]); it++) {  // at most half full
      unsigned long long old[4];
#pragma unroll
      for (int j = 0; j < 4; j++)
        old[j] = act[j] ? atomicCAS(reinterpret_cast<unsigned long long*>(&b.hkey[s[j]]), 0ull, k[j]) : 0ull;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if (!act[j]) continue;
        if (old[j] == 0ull) {
          fresh[j] = true;
          b.hval[s[j]] = (int32_t)(4 * qd + j);
          act[j] = false;
        } else if (old[j] == k[j]) {
          act[j] = false;
        } else {
          s[j] = (s[j] + 1) & mask;
        }
      }
    }
    reinterpret_cast<uint4*>(b.uRep)[qd] = make_uint4(fresh[0] ? 0xFFFFFFFEu : ~0u, fresh[1] ? 0xFFFFFFFEu : ~0u,
                                                       fresh[2] ? 0xFFFFFFFEu : ~0u, fresh[3] ? 0xFFFFFFFEu : ~0u);
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (fresh[j]) {
        fresh_n++;
        mE = min(mE, E[j]);
        low += e_bin(E[j], Eb) <= pmax ? 1 : 0;
      }
  }
  block_add(&st->nU, fresh_n);
  block_min(&st->minE_round, mE);
  block_add(&st->nU_low, low);
}

// Which survivors the cut needs counted.  Everything fits: none.  The pool's rest and the survivors
// inside its occupied bins reach the cap: the cut lies in those bins, so only they are counted.
// Otherwise all of them.
__device__ __forceinline__ int hist_mode_of(const PqState* st, long long cap) {
  const long long rest = st->nP - st->b;
  if (rest + st->nU <= cap) return 0;
  if (st->pmax_bin >= 0 && rest + st->nU_low >= cap) return 1;
  return 2;
}

// Dedup, second pass: each survivor finds its key's slot and lowers the representative of the key's
// unique survivor to the smallest (pivot, column) -- the pivots are in key order, so this is the
// sequential definition's first occurrence.  The unique survivors also enter the survivor histogram (the
// bins the cut needs) and give the smallest fingerprint among the smallest-energy survivors.  Four
// consecutive survivors per thread, their lookups in flight together; survivors the cut cannot reach
// are skipped.
template <bool SEED>
__global__ void __launch_bounds__(256) pq_dedup_rep_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->n_dense;
  const long long nq = (n + 3) >> 2;
  const uint64_t mask = (1ull << b.hs_log2) - 1;
  const int mode = hist_mode_of(st, b.cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->hist_mode = mode;
  const int Eb = st->E_base, pmax = st->pmax_bin, mE = st->minE_round;
  uint64_t mf = ~0ull;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nq; base += stride) {  // warp-uniform
    const long long qd = base + threadIdx.x;
    int E[4] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MAX};
    if (qd < nq) {
      const int4 e4 = reinterpret_cast<const int4*>(b.dE)[qd];
      E[0] = e4.x;
      E[1] = e4.y;
      E[2] = e4.z;
      E[3] = e4.w;
    }
    uint64_t fp[4], k[4], s[4];
    bool act[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long i = 4 * qd + j;
      // with the cut inside the pool's occupied bins (mode 1), a survivor above them is never admitted
      // nor the round's smallest (survivors inside them exist then), so its representative is not needed
      act[j] = qd < nq && i < n && E[j] != INT32_MAX && !(mode == 1 && e_bin(E[j], Eb) > pmax);
      fp[j] = act[j] ? b.dFp[i] : 0ull;
      k[j] = dedup_key(E[j], fp[j]);
      s[j] = (k[j] * kGamma) >> (64 - b.hs_log2);
    }
    bool look[4] = {act[0], act[1], act[2], act[3]};
    for (uint64_t it = 0; it <= mask && (look[0] || look[1] || look[2] || look[3]); it++) {
      uint64_t hk[4];
#pragma unroll
      for (int j = 0; j < 4; j++) hk[j] = look[j] ? b.hkey[s[j]] : 0ull;
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (look[j]) {
          if (hk[j] == k[j])
            look[j] = false;
          else
            s[j] = (s[j] + 1) & mask;
        }
    }
    int hv[4];
#pragma unroll
    for (int j = 0; j < 4; j++) hv[j] = act[j] ? b.hval[s[j]] : -1;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int bin = -1;
      if (act[j]) {
        const long long i = 4 * qd + j;
        const unsigned rep = SEED ? (unsigned)i << kColBits
                                  : ((unsigned)(i / b.width) << kColBits) | (unsigned)(i % b.width);
        atomicMin(&b.uRep[hv[j]], rep);
        if (hv[j] == (int32_t)i) {  // the key's unique survivor
          const int eb = e_bin(E[j], Eb);
          if (mode == 2 || (mode == 1 && eb <= pmax)) bin = eb;
          if (E[j] == mE) mf = min(mf, fp[j]);
        }
      }
      if (mode) hist_add(b.hU, b.hU2, bin, 1);
    }
  }
  if (mf != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(&st->minfp_round), (unsigned long long)mf);
}

// The histogram's energy window, from the smallest seed energy (improvements stay far inside it).
__global__ void pq_set_window_kernel(PqBufs b) {
  PqState* st = b.st;
  st->E_base = st->minE_round == INT32_MAX ? 0 : max(0, st->minE_round - kNB / 2);
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

// Pool pass: the entries beyond the cut are evicted (slot freed, histogram updated); four slots per
// thread, their energies in one 16-byte load.
__global__ void __launch_bounds__(256) pq_evict_kernel(PqBufs b) {
  PqState* st = b.st;
  if (st->sel_need < 0) return;
  const int Eb = st->E_base;
  const long long nq = (b.cap + 3) >> 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nq; base += stride) {
    const long long qd = base + threadIdx.x;
    int4 e4 = make_int4(INT32_MAX, INT32_MAX, INT32_MAX, INT32_MAX);
    if (qd < nq) e4 = reinterpret_cast<const int4*>(b.pE)[qd];
    const int ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const long long i = 4 * qd + e;
      bool out = false;
      int bin = 0;
      const int E = ev[e];
      if (i < b.cap && E != INT32_MAX) {
        bin = e_bin(E, Eb);
        out = bin > st->sel_bin || (bin == st->sel_bin && !key_le(E, b.pFp[i], st->sel_E, st->sel_fp));
      }
      const long long o = warp_append(&st->free_top, out);
      if (out) {
        b.freeIds[o] = (int32_t)i;
        b.pE[i] = INT32_MAX;
      }
      hist_add(b.hP, b.hP2, out ? bin : -1, -1);
      warp_add(&st->ev_round, out ? 1 : 0);
    }
  }
}

// Survivor pass: the survivors inside the cut take a free slot (the sequence built from the pivot, or
// copied from the seed) and enter the visited set; the smallest survivor key's representative is noted
// for the best.
template <bool SEED>
__global__ void __launch_bounds__(256) pq_admit_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = st->n_dense;
  const long long nq = (n + 3) >> 2;
  const int Eb = st->E_base;
  const bool cut = st->sel_need >= 0;
  const int sel_bin = st->sel_bin, minE = st->minE_round;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // four consecutive survivors per thread: their representatives and energies in one 16-byte load each;
  // a fingerprint is read only where the cut or the best test needs it
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nq; base += stride) {  // warp-uniform
    const long long qd = base + threadIdx.x;
    uint4 r4 = make_uint4(~0u, ~0u, ~0u, ~0u);
    int4 e4 = make_int4(INT32_MAX, INT32_MAX, INT32_MAX, INT32_MAX);
    if (qd < nq) {
      r4 = reinterpret_cast<const uint4*>(b.uRep)[qd];
      e4 = reinterpret_cast<const int4*>(b.dE)[qd];
    }
    const unsigned R[4] = {r4.x, r4.y, r4.z, r4.w};
    const int Ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long u = 4 * qd + j;
      bool in = false;
      const int E = Ev[j];
      int bin = 0;
      uint64_t fp = 0;
      if (u < n && R[j] != ~0u) {
        bin = e_bin(E, Eb);
        if (!cut || bin <= sel_bin || E == minE) {
          fp = b.dFp[u];
          in = below_cut(st, bin, E, fp);
          if (E == minE && fp == st->minfp_round) st->best_rep_round = R[j];  // the smallest key
        }
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
      const unsigned rep = in ? R[j] : 0u;
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
        ins = h_insert(b, fp);
      }
      hist_add(b.hP, b.hP2, in ? bin : -1, 1);
      h_count(b, ins);
      warp_add(&st->adm_round, in ? 1 : 0);
    }
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
  const size_t opE = take(4 * ((cap + 3) & ~3ll)), opF = take(8 * cap), opS = take(8 * cap * W), ofree = take(4 * cap);
  const size_t ohP = take(4 * kNB), ohP2 = take(4 * kNC), ohU = take(4 * kNB), ohU2 = take(4 * kNC);
  const size_t opop = take(4 * (size_t)cfg->B), opivE = take(4 * (size_t)cfg->B), opivF = take(8 * (size_t)cfg->B);
  const size_t opopE = take(4 * (size_t)cfg->B), opopF = take(8 * (size_t)cfg->B);
  const size_t opivS = take(8 * (size_t)cfg->B * W);
  const size_t ocand = take(4 * (size_t)(cap + n_dense)), ocE = take(4 * (size_t)(cap + n_dense));
  const size_t ocF = take(8 * (size_t)(cap + n_dense)), orank = take(4 * (size_t)cfg->B);
  const size_t odE = take(4 * ((n_dense + 3) & ~3ll)), odF = take(8 * n_dense);
  const size_t ohk = take(8ull << hs_log2), ohv = take(4ull << hs_log2);
  const size_t ouR = take(4 * ((n_dense + 3) & ~3ll));
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
  b.popE = reinterpret_cast<int32_t*>(base + opopE);
  b.popF = reinterpret_cast<uint64_t*>(base + opopF);
  b.pivE = reinterpret_cast<int32_t*>(base + opivE);
  b.pivFp = reinterpret_cast<uint64_t*>(base + opivF);
  b.pivSeq = reinterpret_cast<uint64_t*>(base + opivS);
  b.candId = reinterpret_cast<int32_t*>(base + ocand);
  b.cE = reinterpret_cast<int32_t*>(base + ocE);
  b.cF = reinterpret_cast<uint64_t*>(base + ocF);
  b.popRank = reinterpret_cast<int32_t*>(base + orank);
  b.dE = reinterpret_cast<int32_t*>(base + odE);
  b.dFp = reinterpret_cast<uint64_t*>(base + odF);
  b.hkey = reinterpret_cast<uint64_t*>(base + ohk);
  b.hval = reinterpret_cast<int32_t*>(base + ohv);
  b.uRep = reinterpret_cast<unsigned*>(base + ouR);
  b.ztab = reinterpret_cast<uint64_t*>(base + ozt);
  b.st = reinterpret_cast<PqState*>(base + ost);
  b.best_seq = reinterpret_cast<uint64_t*>(base + obest);
  b.H = reinterpret_cast<uint64_t*>(base + oH);
  b.seeds = seeds;

  const unsigned g_pool = (unsigned)std::max(1ll, std::min<long long>((cap + 255) / 256, (long long)ctx->num_sms * 16));
  const unsigned g_dense =
      (unsigned)std::max(1ll, std::min<long long>((n_dense + 255) / 256, (long long)ctx->num_sms * 16));
  const size_t cand_smem = (size_t)kCandSmem * 12;
  if (cudaFuncSetAttribute(pq_boundary_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cand_smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(pq_boundary_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cand_smem) !=
          cudaSuccess)
    return LABS_ERR_CUDA;
  const unsigned g_piv = (unsigned)std::max(1, std::min((cfg->B + 255) / 256, ctx->num_sms * 4));

  // The survivor path, shared by the seeds and every round: dedup, best, cut, eviction, admission.
  auto survivor_path = [&](bool seed, cudaStream_t s) {
    if (seed) {
      pq_dedup_insert_kernel<true><<<g_dense, 256, 0, s>>>(b);
      pq_set_window_kernel<<<1, 1, 0, s>>>(b);
      pq_dedup_rep_kernel<true><<<g_dense, 256, 0, s>>>(b);
    } else {
      pq_dedup_insert_kernel<false><<<g_dense, 256, 0, s>>>(b);
      pq_dedup_rep_kernel<false><<<g_dense, 256, 0, s>>>(b);
    }
    pq_select_kernel<false><<<1, kSelThreads, 0, s>>>(b);
    pq_gather_kernel<false, false><<<g_pool, 256, 0, s>>>(b);
    pq_gather_kernel<false, true><<<g_dense, 256, 0, s>>>(b);
    pq_boundary_kernel<false><<<1, kSelThreads, cand_smem, s>>>(b);
    pq_evict_kernel<<<g_pool, 256, 0, s>>>(b);
    if (seed) {
      pq_admit_kernel<true><<<g_dense, 256, 0, s>>>(b);
      pq_best_kernel<true><<<1, 1, 0, s>>>(b);
      pq_round_end_kernel<true><<<1, 1, 0, s>>>(b);
    } else {
      pq_admit_kernel<false><<<g_dense, 256, 0, s>>>(b);
      pq_best_kernel<false><<<1, 1, 0, s>>>(b);
      pq_round_end_kernel<false><<<1, 1, 0, s>>>(b);
    }
    cudaMemsetAsync(b.hU, 0, 4 * kNB, s);
    cudaMemsetAsync(b.hU2, 0, 4 * kNC, s);
    cudaMemsetAsync(b.hkey, 0, 8ull << hs_log2, s);  // the dedup table, for the next round
  };

  // ---- set-up: visited set, pool, histograms, dedup table, Zobrist keys; the seeds go through the
  // survivor path into the empty pool (equal seeds kept once, the cap smallest admitted)
  if (cudaMemsetAsync(b.H, 0xff, 8ull << cfg->H_log2, st) != cudaSuccess) return LABS_ERR_CUDA;
  if (cudaMemsetAsync(b.hP, 0, 4 * kNB, st) != cudaSuccess || cudaMemsetAsync(b.hP2, 0, 4 * kNC, st) != cudaSuccess ||
      cudaMemsetAsync(b.hU, 0, 4 * kNB, st) != cudaSuccess || cudaMemsetAsync(b.hU2, 0, 4 * kNC, st) != cudaSuccess ||
      cudaMemsetAsync(b.hkey, 0, 8ull << hs_log2, st) != cudaSuccess ||
      cudaMemsetAsync(b.popRank, 0, 4 * (size_t)cfg->B, st) != cudaSuccess)
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
    pq_boundary_kernel<true><<<1, kSelThreads, cand_smem, cs>>>(b);
    pq_pop_rank_kernel<<<dim3((unsigned)((cfg->B + 255) / 256), kRankChunks), 256, 0, cs>>>(b);
    pq_pivot_kernel<<<g_piv, 256, 0, cs>>>(b);
    pq_pmax_kernel<<<1, kSelThreads, 0, cs>>>(b);
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
