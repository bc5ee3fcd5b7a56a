// pq.cu -- step 2 of the dual-step search: Algorithm 2's priority-queue refinement over the unrestricted
// space, in batch-synchronous form (labs_pq_refine).
//
// GB300 mapping.  The paper runs one priority queue per candidate in Rust on CPU cores; here one open
// set of the cap smallest (E, fp) keys lives in HBM as a sorted array (double-buffered), and a round
//   expand   -- one warp per popped node: its correlation table, the all-position dp4a scan and a
//               visited-set lookup per neighbour, written to a dense [pop][position] survivor array;
//   compact  -- stable compaction of the survivors (pop order, position);
//   sort     -- stable LSD radix sort by the fingerprint's top 16 bits then the energy bytes (passes
//               whose byte is the same in every key are skipped), then runs of equal (E', fp' >> 48)
//               ordered by (fp', pop, pos) in place: order (E', fp', pop, pos);
//   dedup    -- stable compaction keeping the first of equal (E', fp');
//   best     -- strict improvement test on the smallest survivor;
//   merge    -- merge path of (open set minus the pops) with the survivors into the other buffer, cut at
//               cap; admitted survivors enter the visited set (open addressing, atomicCAS);
// keeps every result identical to the sequential definition whatever order threads run in.
// With T_r > 0 every popped pivot also offers its 2 T_r rotations (MAKE_ROTATIONS) as survivor columns
// L .. L + 2 T_r - 1, after its L flips.
#include <algorithm>
#include <new>

#include "labs_core.cuh"
#include "labs_internal.h"

namespace labsg {
namespace {

constexpr uint64_t kEmptyKey = ~0ull;  // free slot of the visited set (fp == ~0 is tracked by a flag)
constexpr int kPqWarps = 4;
constexpr int kPqM = 8;
constexpr int kTile = 1024;  // elements per block in the compaction and sort kernels (256 threads x 4)
constexpr int kMaxProbe = 1 << 20;

struct PqState {
  long long nP, nS, nU, n_dense;
  long long expansions, rounds, survivors, admitted, evicted, h_size, improvements, u;
  unsigned long long best_fp;
  int b, cur, stop, best_E, error, h_has_empty, pad0, pad1;
  // OR and AND of the sort keys' 32-bit halves (fingerprint high half, energy) over this sort's input:
  // a radix byte that is equal in every key orders nothing and its pass is skipped
  unsigned fph_or, fph_and, e_or, e_and;
};

struct PqBufs {
  int L, W, B, H_log2;
  int Tr, width;  // rotations per side (MAKE_ROTATIONS) and survivor columns per pop: L flips + 2 Tr rotations
  long long cap, max_exp, T_u;
  int32_t* PE[2];
  uint64_t* Pfp[2];
  uint64_t* Pseq[2];
  int32_t* dE;  // dense survivors [B * L] (or seeds)
  uint64_t* dfp;
  int32_t* sE[2];  // sort ping-pong
  uint64_t* sfp[2];
  int32_t* sidx[2];
  int32_t* uE;  // unique survivors
  uint64_t* ufp;
  int32_t* uidx;
  unsigned* counts;  // 256 * blocks
  unsigned* bsum;    // per-block counts (+ total)
  uint64_t* H;
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

// ---------------------------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------------------------
__global__ void pq_ztab_kernel(uint64_t* ztab, int L) {
  const uint64_t zk = stream_key(0, kPurposeZobrist, (uint64_t)L, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) ztab[i] = zobrist(zk, i + 1);
}

__global__ void pq_state_init_kernel(PqState* st, long long n_seeds) {
  PqState z{};
  z.n_dense = n_seeds;
  z.best_E = INT32_MAX;
  z.best_fp = ~0ull;
  *st = z;
}

// One warp per seed: energy over all lags and the fingerprint, into the dense arrays.
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
      b.dfp[q] = h;
    }
    __syncwarp();
  }
}

// Adds a block's insertion counts to h_size with one atomic per warp (every thread of the block calls it).
__device__ __forceinline__ void h_count(const PqBufs& b, int inserted) {
  const int w = __reduce_add_sync(kFull, inserted);
  if (lane_id() == 0 && w) atomicAdd(reinterpret_cast<unsigned long long*>(&b.st->h_size), (unsigned long long)w);
}

// Admits the sorted, de-duplicated seeds: the cap smallest become the open set and enter H.
__global__ void pq_seed_admit_kernel(PqBufs b) {
  PqState* st = b.st;
  const long long n = min((long long)st->nU, b.cap);
  int ins = 0;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const int q = b.uidx[o];
    b.PE[0][o] = b.uE[o];
    b.Pfp[0][o] = b.ufp[o];
    for (int t = 0; t < b.W; t++) b.Pseq[0][o * b.W + t] = b.seeds[(size_t)q * b.W + t];
    ins += h_insert(b, b.ufp[o]);
  }
  h_count(b, ins);
}

__global__ void pq_seed_finish_kernel(PqBufs b) {
  PqState* st = b.st;
  st->nP = min((long long)st->nU, b.cap);
  st->cur = 0;
  if (st->nU > 0) {
    st->best_E = b.uE[0];
    st->best_fp = b.ufp[0];
    const int q = b.uidx[0];
    for (int t = 0; t < b.W; t++) b.best_seq[t] = b.seeds[(size_t)q * b.W + t];
  }
}

// ---------------------------------------------------------------------------------------------
// Round kernels
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
  if (st->stop) {
    st->b = 0;
    st->n_dense = 0;
    return;
  }
  long long bb = min((long long)b.B, st->nP);
  bb = min(bb, b.max_exp - st->expansions);
  st->b = (int)bb;
  st->n_dense = bb * b.width;
}

// One warp per popped node: Delta E of all L single flips, visited-set test, dense survivor output.
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
  const int cur = st->cur;
  const int32_t* PE = b.PE[cur];
  const uint64_t* Pfp = b.Pfp[cur];
  const uint64_t* Pseq = b.Pseq[cur];
  for (int q = blockIdx.x * kPqWarps + (threadIdx.x >> 5); q < nb; q += gridDim.x * kPqWarps) {
    load_bits(sm, Pseq + (size_t)q * b.W, b.L);
    build_table(sm, ly);
    const bool fast = pack_c8(sm);
    const int SC = table_sum(sm);
    build_bytes(sm, ly);
    p_all(sm, ly, xbits, rbits, Pm);
    const int E = PE[q];
    const uint64_t fp = Pfp[q];
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
          b.dfp[di] = fv[j];
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
        b.dfp[di] = h;
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Stable compaction (MODE 0: dense survivors -> sort input; MODE 1: sorted -> first of equal keys)
// and stable LSD radix sort.  Element e of block k is k*1024 + w*128 + r*32 + lane (warp w, round r):
// increasing e is increasing (w, r, lane), so block-local ranks built warp by warp, round by round,
// are stable.
// ---------------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ long long compact_n(const PqBufs& b) {
  return MODE == 0 ? b.st->n_dense : b.st->nS;
}

// Radix passes of the sort: 0..1 the bytes of fp >> 48, 2..5 the bytes of E (least significant first).
// Bit p of the mask is set when pass p runs; pass p reads buffer popc(mask below p) & 1.
__device__ __forceinline__ unsigned sort_mask(const PqState* st) {
  const unsigned vf = st->fph_or ^ st->fph_and, ve = st->e_or ^ st->e_and;  // fph: fp >> 32
  unsigned m = 0;
#pragma unroll
  for (int p = 0; p < 2; p++)
    if ((vf >> (16 + 8 * p)) & 255u) m |= 1u << p;
#pragma unroll
  for (int p = 0; p < 4; p++)
    if ((ve >> (8 * p)) & 255u) m |= 1u << (p + 2);
  return m;
}
__device__ __forceinline__ int sort_src(unsigned mask, int pass) { return __popc(mask & ((1u << pass) - 1u)) & 1; }
__device__ __forceinline__ int sort_final(const PqState* st) { return __popc(sort_mask(st)) & 1; }

template <int MODE>
__device__ __forceinline__ bool compact_flag(const PqBufs& b, long long e, int fin) {
  if (MODE == 0) return b.dE[e] != INT32_MAX;
  return e == 0 || b.sE[fin][e] != b.sE[fin][e - 1] || b.sfp[fin][e] != b.sfp[fin][e - 1];
}

template <int MODE>
__global__ void __launch_bounds__(256) compact_count_kernel(PqBufs b) {
  const long long n = compact_n<MODE>(b);
  const long long base = (long long)blockIdx.x * kTile;
  if (MODE == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // the sort that follows starts its key summary
    b.st->fph_or = 0u;
    b.st->fph_and = ~0u;
    b.st->e_or = 0u;
    b.st->e_and = ~0u;
  }
  if (base >= n) {  // blocks past this round's count still publish a zero for the scan
    if (threadIdx.x == 0) b.bsum[blockIdx.x] = 0;
    return;
  }
  const int fin = MODE == 1 ? sort_final(b.st) : 0;
  int c = 0;
  for (int r = 0; r < 4; r++) {
    const long long e = base + (threadIdx.x >> 5) * 128 + r * 32 + lane_id();
    if (e < n && compact_flag<MODE>(b, e, fin)) c++;
  }
  c = __reduce_add_sync(kFull, c);
  __shared__ int ws[8];
  if (lane_id() == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; w++) t += ws[w];
    b.bsum[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of a[0..n) in place; *total receives the sum.
__global__ void __launch_bounds__(1024) scan_kernel(unsigned* a, long long n, long long* total) {
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;
  const long long chunk = (n + 1023) / 1024;
  const long long lo = t * chunk, hi = min(n, lo + chunk);
  unsigned long long s = 0;
  for (long long i = lo; i < hi; i++) s += a[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan of the partial sums
    unsigned long long v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned long long run = t ? part[t - 1] : 0;
  for (long long i = lo; i < hi; i++) {
    const unsigned v = a[i];
    a[i] = (unsigned)run;
    run += v;
  }
  if (t == 1023 && total) *total = (long long)part[1023];
}

// Number of blocks a compaction or sort over n elements uses.
__device__ __forceinline__ long long tiles_of(long long n) { return (n + kTile - 1) / kTile; }

template <int MODE>
__global__ void __launch_bounds__(256) compact_scatter_kernel(PqBufs b) {
  const long long n = compact_n<MODE>(b);
  const long long base = (long long)blockIdx.x * kTile;
  if (base >= n) return;
  __shared__ int wcount[8][4];
  __shared__ unsigned wkey[8][4];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const int fin = MODE == 1 ? sort_final(b.st) : 0;
  bool fl[4];
  for (int r = 0; r < 4; r++) {
    const long long e = base + w * 128 + r * 32 + lane;
    fl[r] = e < n && compact_flag<MODE>(b, e, fin);
    const unsigned m = __ballot_sync(kFull, fl[r]);
    if (lane == 0) wcount[w][r] = __popc(m);
  }
  __syncthreads();
  int off = b.bsum[blockIdx.x];
  for (int ww = 0; ww < w; ww++)
    for (int r = 0; r < 4; r++) off += wcount[ww][r];
  for (int r = 0; r < 4; r++) {
    const long long e = base + w * 128 + r * 32 + lane;
    const unsigned m = __ballot_sync(kFull, fl[r]);
    if (fl[r]) {
      const long long o = off + __popc(m & ((1u << lane) - 1u));
      if (MODE == 0) {
        b.sE[0][o] = b.dE[e];
        b.sfp[0][o] = b.dfp[e];
        b.sidx[0][o] = (int32_t)e;
      } else {
        b.uE[o] = b.sE[fin][e];
        b.ufp[o] = b.sfp[fin][e];
        b.uidx[o] = b.sidx[fin][e];
      }
    }
    off += __popc(m);
  }
  if (MODE == 0) {  // the block's share of the key summary
    unsigned fo = 0u, fa = ~0u, eo = 0u, ea = ~0u;
    for (int r = 0; r < 4; r++) {
      const long long e = base + w * 128 + r * 32 + lane;
      if (fl[r]) {
        const unsigned fh = (unsigned)(b.dfp[e] >> 32), ev = (unsigned)b.dE[e];
        fo |= fh;
        fa &= fh;
        eo |= ev;
        ea &= ev;
      }
    }
    fo = __reduce_or_sync(kFull, fo);
    fa = __reduce_and_sync(kFull, fa);
    eo = __reduce_or_sync(kFull, eo);
    ea = __reduce_and_sync(kFull, ea);
    if (lane == 0) {
      wkey[w][0] = fo;
      wkey[w][1] = fa;
      wkey[w][2] = eo;
      wkey[w][3] = ea;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int ww = 1; ww < 8; ww++) {
        fo |= wkey[ww][0];
        fa &= wkey[ww][1];
        eo |= wkey[ww][2];
        ea &= wkey[ww][3];
      }
      atomicOr(&b.st->fph_or, fo);
      atomicAnd(&b.st->fph_and, fa);
      atomicOr(&b.st->e_or, eo);
      atomicAnd(&b.st->e_and, ea);
    }
  }
}

// Radix digit of element e of buffer `src` at pass `pass` (0..1: bytes of fp >> 48, 2..5: energy bytes).
__device__ __forceinline__ unsigned radix_digit(const PqBufs& b, int src, long long e, int pass) {
  if (pass < 2) return (unsigned)(b.sfp[src][e] >> (48 + 8 * pass)) & 255u;
  return ((unsigned)b.sE[src][e] >> (8 * (pass - 2))) & 255u;
}

__global__ void __launch_bounds__(256) radix_hist_kernel(PqBufs b, int pass) {
  const long long n = b.st->nS;
  const long long nblk = tiles_of(n);
  const long long base = (long long)blockIdx.x * kTile;
  const unsigned mask = sort_mask(b.st);
  if (base >= n || !((mask >> pass) & 1u)) return;
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int src = sort_src(mask, pass);
  for (int r = 0; r < 4; r++) {
    const long long e = base + (threadIdx.x >> 5) * 128 + r * 32 + lane_id();
    if (e < n) atomicAdd(&h[radix_digit(b, src, e, pass)], 1u);
  }
  __syncthreads();
  b.counts[(long long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the digit-major radix counts (256 x blocks of this round), in three phases over
// segments of kSeg entries: segment sums, a scan of the sums, then each segment with its offset.
constexpr int kSeg = 4096;

__device__ __forceinline__ long long radix_count_len(const PqBufs& b) { return 256 * tiles_of(b.st->nS); }

__global__ void __launch_bounds__(256) seg_reduce_kernel(PqBufs b, int pass) {
  if (!((sort_mask(b.st) >> pass) & 1u)) return;
  const long long n = radix_count_len(b);
  const long long lo = (long long)blockIdx.x * kSeg;
  unsigned s = 0;
  if (lo < n)
    for (long long i = lo + threadIdx.x; i < min(n, lo + kSeg); i += 256) s += b.counts[i];
  s = __reduce_add_sync(kFull, s);
  __shared__ unsigned w[8];
  if (lane_id() == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int i = 0; i < 8; i++) t += w[i];
    b.bsum[blockIdx.x] = t;  // zero for segments past this round's length
  }
}

__global__ void __launch_bounds__(1024) seg_scan_sums_kernel(unsigned* a, int n, const PqState* st, int pass) {
  if (!((sort_mask(st) >> pass) & 1u)) return;
  __shared__ unsigned part[1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int lo = t * chunk, hi = min(n, lo + chunk);
  unsigned s = 0;
  for (int i = lo; i < hi; i++) s += a[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned run = t ? part[t - 1] : 0;
  for (int i = lo; i < hi; i++) {
    const unsigned v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(256) seg_down_kernel(PqBufs b, int pass) {
  const long long n = radix_count_len(b);
  const long long lo = (long long)blockIdx.x * kSeg;
  if (lo >= n || !((sort_mask(b.st) >> pass) & 1u)) return;
  // thread t owns entries lo + 16t .. lo + 16t + 15
  const long long first = lo + 16 * threadIdx.x;
  unsigned v[16], s = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    v[i] = first + i < n ? b.counts[first + i] : 0u;
    s += v[i];
  }
  // block exclusive scan of the thread sums
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned x = __shfl_up_sync(kFull, incl, o);
    if (lane_id() >= o) incl += x;
  }
  __shared__ unsigned wsum[8];
  if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
  __syncthreads();
  unsigned wofs = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); w++) wofs += wsum[w];
  unsigned run = b.bsum[blockIdx.x] + wofs + incl - s;
#pragma unroll
  for (int i = 0; i < 16; i++)
    if (first + i < n) {
      b.counts[first + i] = run;
      run += v[i];
    }
}

__global__ void __launch_bounds__(256) radix_scatter_kernel(PqBufs b, int pass) {
  const long long n = b.st->nS;
  const long long nblk = tiles_of(n);
  const long long base = (long long)blockIdx.x * kTile;
  const unsigned mask = sort_mask(b.st);
  if (base >= n || !((mask >> pass) & 1u)) return;
  __shared__ unsigned cnt[8][256];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const int src = sort_src(mask, pass), dst = src ^ 1;
  for (int d = threadIdx.x; d < 8 * 256; d += 256) (&cnt[0][0])[d] = 0;
  __syncthreads();
  unsigned dig[4];
  for (int r = 0; r < 4; r++) {
    const long long e = base + w * 128 + r * 32 + lane;
    dig[r] = e < n ? radix_digit(b, src, e, pass) : 256u;
    const unsigned peers = __match_any_sync(kFull, dig[r]);
    if (dig[r] < 256u && lane == __ffs(peers) - 1) cnt[w][dig[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: exclusive prefix over warps, plus the block's global offset
    const int d = threadIdx.x;
    unsigned run = b.counts[(long long)d * nblk + blockIdx.x];
    for (int ww = 0; ww < 8; ww++) {
      const unsigned v = cnt[ww][d];
      cnt[ww][d] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int r = 0; r < 4; r++) {
    const long long e = base + w * 128 + r * 32 + lane;
    const unsigned peers = __match_any_sync(kFull, dig[r]);
    if (dig[r] < 256u) {
      const unsigned o = cnt[w][dig[r]] + __popc(peers & ((1u << lane) - 1u));
      b.sE[dst][o] = b.sE[src][e];
      b.sfp[dst][o] = b.sfp[src][e];
      b.sidx[dst][o] = b.sidx[src][e];
    }
    __syncwarp();
    if (dig[r] < 256u && lane == __ffs(peers) - 1) cnt[w][dig[r]] += __popc(peers);
    __syncwarp();
  }
}

// After the radix passes the keys are ordered by (E, fp >> 48) and, within equal pairs, by input order
// (pop, pos).  Each run of equal (E, fp >> 48) is put in (fp, pop, pos) order in place by the thread at
// its start (runs are disjoint; they are short, fingerprints being uniform 64-bit keys).
__global__ void __launch_bounds__(256) sort_fixup_kernel(PqBufs b) {
  const long long n = b.st->nS;
  const int f = sort_final(b.st);
  int32_t* E = b.sE[f];
  uint64_t* fp = b.sfp[f];
  int32_t* ix = b.sidx[f];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (long long)gridDim.x * blockDim.x) {
    const int Ei = E[i];
    const unsigned hi = (unsigned)(fp[i] >> 48);
    if (E[i + 1] != Ei || (unsigned)(fp[i + 1] >> 48) != hi) continue;
    if (i > 0 && E[i - 1] == Ei && (unsigned)(fp[i - 1] >> 48) == hi) continue;
    long long j = i + 2;
    while (j < n && E[j] == Ei && (unsigned)(fp[j] >> 48) == hi) j++;
    for (long long a = i + 1; a < j; a++) {  // insertion sort of [i, j) by (fp, index)
      const uint64_t kf = fp[a];
      const int32_t ki = ix[a];
      long long c = a;
      while (c > i && (fp[c - 1] > kf || (fp[c - 1] == kf && ix[c - 1] > ki))) {
        fp[c] = fp[c - 1];
        ix[c] = ix[c - 1];
        c--;
      }
      fp[c] = kf;
      ix[c] = ki;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Best, merge, round end
// ---------------------------------------------------------------------------------------------
__global__ void pq_best_kernel(PqBufs b) {
  PqState* st = b.st;
  if (st->b == 0) return;
  st->survivors += st->nU;
  if (st->nU > 0 && b.uE[0] < st->best_E) {
    st->best_E = b.uE[0];
    st->best_fp = b.ufp[0];
    const int q = b.uidx[0] / b.width, col = b.uidx[0] % b.width;
    pq_child(b.Pseq[st->cur] + (size_t)q * b.W, b, col, b.best_seq);
    st->improvements++;
    st->u = 0;
  } else {
    st->u += st->b;
  }
}

// Number of open-set (rest) entries among the first o merged outputs.
// The search may start from any [lo, hi] that contains the answer (the predicate is monotone in mid).
__device__ __forceinline__ long long merge_split_in(const int32_t* RE, const uint64_t* Rfp, const int32_t* UE,
                                                    const uint64_t* Ufp, long long o, long long lo, long long hi) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    const long long ui = o - mid - 1;
    if (key_lt(RE[mid], Rfp[mid], UE[ui], Ufp[ui]))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ long long merge_split(const int32_t* RE, const uint64_t* Rfp, long long nR, const int32_t* UE,
                                                 const uint64_t* Ufp, long long nU, long long o) {
  return merge_split_in(RE, Rfp, UE, Ufp, o, max(0ll, o - nU), min(o, nR));
}

// The same split found by the whole block (every thread calls it, gets the answer): each step tests
// blockDim increasing points of the range at once, and the number that test true (a prefix, the
// predicate being monotone) narrows the range by a factor of blockDim + 1 -- three steps for 2^22.
__device__ long long block_merge_split(const int32_t* RE, const uint64_t* Rfp, long long nR, const int32_t* UE,
                                       const uint64_t* Ufp, long long nU, long long o) {
  long long lo = max(0ll, o - nU), hi = min(o, nR);
  const long long nt = blockDim.x, t = threadIdx.x;
  while (lo < hi) {  // the same on every thread
    const long long span = hi - lo;
    const bool dense = span <= nt;  // then the points are lo .. hi - 1 and one step ends the search
    auto point = [&](long long k) { return dense ? lo + k : lo + (span * (k + 1)) / (nt + 1); };
    const long long np = dense ? span : nt;
    bool pred = false;
    if (t < np) {
      const long long mid = point(t), ui = o - mid - 1;
      pred = key_lt(RE[mid], Rfp[mid], UE[ui], Ufp[ui]);
    }
    const long long c = __syncthreads_count(pred);
    const long long nlo = c > 0 ? point(c - 1) + 1 : lo;
    hi = c < np ? point(c) : hi;
    lo = nlo;
  }
  return lo;
}

// Merge path in tiles: a block takes kMergeTile consecutive outputs and finds the tile's two ends
// (block_merge_split); the tile's keys of both inputs (kMergeTile in all) are then staged in
// shared memory, and each thread finds its own output's source by a search there.  Warps write 32
// consecutive outputs at a time and copy their sequences together (lane l moves word l mod W of output
// l / W, and so on), so every store is coalesced.
constexpr int kMergeTile = 2048;

__global__ void __launch_bounds__(256) pq_merge_kernel(PqBufs b) {
  const PqState* st = b.st;
  if (st->b == 0) return;
  const int cur = st->cur, nxt = cur ^ 1;
  const long long nb = st->b, nR = st->nP - nb, nU = st->nU;
  const long long nOut = min(b.cap, nR + nU);
  const int32_t* RE = b.PE[cur] + nb;
  const uint64_t* Rfp = b.Pfp[cur] + nb;
  const uint64_t* Rseq = b.Pseq[cur] + nb * b.W;
  __shared__ int32_t sE[kMergeTile];   // the tile's open-set keys at [0, nr), survivor keys at [nr, nr + nu)
  __shared__ uint64_t sF[kMergeTile];
  int ins = 0;
  for (long long o0 = (long long)blockIdx.x * kMergeTile; o0 < nOut; o0 += (long long)gridDim.x * kMergeTile) {
    const long long o1 = min(o0 + kMergeTile, nOut);
    __syncthreads();  // the previous tile's keys are no longer read
    const long long ra = block_merge_split(RE, Rfp, nR, b.uE, b.ufp, nU, o0);
    const long long rb = block_merge_split(RE, Rfp, nR, b.uE, b.ufp, nU, o1);
    const long long ua = o0 - ra;
    const int nr = (int)(rb - ra), nu = (int)(o1 - rb - ua);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      sE[i] = RE[ra + i];
      sF[i] = Rfp[ra + i];
    }
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
      sE[nr + i] = b.uE[ua + i];
      sF[nr + i] = b.ufp[ua + i];
    }
    __syncthreads();
    for (long long ob = o0 + (threadIdx.x & ~31); ob < o1; ob += blockDim.x) {
      const long long o = ob + lane_id();
      int kind = 0, src = 0, col = 0;  // kind: 0 none, 1 open set entry src, 2 flip col of pivot src, 3 rotation
      if (o < o1) {
        const int ol = (int)(o - o0);
        int lo = max(0, ol - nu), hi = min(ol, nr);  // open-set entries among the tile's first ol outputs
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const int uj = nr + ol - mid - 1;
          if (key_lt(sE[mid], sF[mid], sE[uj], sF[uj]))
            lo = mid + 1;
          else
            hi = mid;
        }
        const int al = lo, ul = ol - lo;
        const bool from_rest = al < nr && (ul >= nu || key_lt(sE[al], sF[al], sE[nr + ul], sF[nr + ul]));
        if (from_rest) {
          b.PE[nxt][o] = sE[al];
          b.Pfp[nxt][o] = sF[al];
          kind = 1;
          src = (int)(ra + al);
        } else {
          const long long ui = ua + ul;
          const int q = b.uidx[ui] / b.width;
          col = b.uidx[ui] % b.width;
          b.PE[nxt][o] = sE[nr + ul];
          b.Pfp[nxt][o] = sF[nr + ul];
          kind = col < b.L ? 2 : 3;
          src = q;
          if (kind == 3) pq_child(b.Pseq[cur] + (size_t)q * b.W, b, col, b.Pseq[nxt] + o * b.W);
          ins += h_insert(b, sF[nr + ul]);
        }
      }
      for (int t = lane_id(); t < 32 * b.W; t += 32) {
        const int oo = t / b.W, word = t - oo * b.W;
        const int k2 = __shfl_sync(kFull, kind, oo), s2 = __shfl_sync(kFull, src, oo), c2 = __shfl_sync(kFull, col, oo);
        if (k2 == 1) {
          b.Pseq[nxt][(ob + oo) * b.W + word] = Rseq[(long long)s2 * b.W + word];
        } else if (k2 == 2) {
          const uint64_t wv = b.Pseq[cur][(size_t)s2 * b.W + word];
          b.Pseq[nxt][(ob + oo) * b.W + word] = wv ^ (word == (c2 >> 6) ? 1ull << (c2 & 63) : 0ull);
        }
      }
    }
  }
  h_count(b, ins);
}

// One block: the split of the merged output at the cap (how many open-set entries stayed) by the block
// search, then the round's bookkeeping by thread 0.
__global__ void __launch_bounds__(256) pq_round_end_kernel(PqBufs b) {
  PqState* st = b.st;
  if (st->b == 0) return;
  const int cur = st->cur;
  const long long nb = st->b, nR = st->nP - nb, nU = st->nU;
  const long long nOut = min(b.cap, nR + nU);
  const long long a = block_merge_split(b.PE[cur] + nb, b.Pfp[cur] + nb, nR, b.uE, b.ufp, nU, nOut);
  if (threadIdx.x != 0) return;
  st->admitted += nOut - a;
  st->evicted += nR - a;
  st->nP = nOut;
  st->expansions += nb;
  st->rounds++;
  st->cur = cur ^ 1;
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

// Issues compaction (MODE) over at most `max_n` elements.
template <int MODE>
void issue_compact(const PqBufs& b, long long max_n, long long* total, cudaStream_t st) {
  const long long nblk = std::max(1ll, (max_n + kTile - 1) / kTile);
  compact_count_kernel<MODE><<<(unsigned)nblk, 256, 0, st>>>(b);
  scan_kernel<<<1, 1024, 0, st>>>(b.bsum, nblk, total);
  compact_scatter_kernel<MODE><<<(unsigned)nblk, 256, 0, st>>>(b);
}

}  // namespace

int launch_pq_refine(labs_ctx* ctx, const labs_pq_cfg* cfg, const uint64_t* seeds, int n_seeds, uint64_t* best_seq,
                     int32_t* best_E, labs_pq_stats* stats, cudaStream_t st) {
  const int L = cfg->L, W = (L + 63) / 64;
  Layout ly;
  if (!make_layout(ly, L, 0, 0, kPqM)) return LABS_ERR_INVALID_ARG;
  const int width = L + 2 * cfg->T_r;
  const long long nmax = std::max<long long>((long long)cfg->B * width, n_seeds);
  const long long nblk = (nmax + kTile - 1) / kTile;
  // workspace layout (one region, 256-byte aligned pieces)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t oPE0 = take(4 * cfg->cap), oPE1 = take(4 * cfg->cap);
  const size_t oPf0 = take(8 * cfg->cap), oPf1 = take(8 * cfg->cap);
  const size_t oPs0 = take(8 * cfg->cap * W), oPs1 = take(8 * cfg->cap * W);
  const size_t odE = take(4 * nmax), odf = take(8 * nmax);
  const size_t osE0 = take(4 * nmax), osE1 = take(4 * nmax), osf0 = take(8 * nmax), osf1 = take(8 * nmax);
  const size_t osi0 = take(4 * nmax), osi1 = take(4 * nmax);
  const size_t ouE = take(4 * nmax), ouf = take(8 * nmax), oui = take(4 * nmax);
  const size_t ocnt = take(4 * 256 * nblk), obs = take(4 * (nblk + 1));
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
  b.cap = cfg->cap;
  b.max_exp = cfg->max_expansions;
  b.T_u = cfg->T_u;
  b.PE[0] = reinterpret_cast<int32_t*>(base + oPE0);
  b.PE[1] = reinterpret_cast<int32_t*>(base + oPE1);
  b.Pfp[0] = reinterpret_cast<uint64_t*>(base + oPf0);
  b.Pfp[1] = reinterpret_cast<uint64_t*>(base + oPf1);
  b.Pseq[0] = reinterpret_cast<uint64_t*>(base + oPs0);
  b.Pseq[1] = reinterpret_cast<uint64_t*>(base + oPs1);
  b.dE = reinterpret_cast<int32_t*>(base + odE);
  b.dfp = reinterpret_cast<uint64_t*>(base + odf);
  b.sE[0] = reinterpret_cast<int32_t*>(base + osE0);
  b.sE[1] = reinterpret_cast<int32_t*>(base + osE1);
  b.sfp[0] = reinterpret_cast<uint64_t*>(base + osf0);
  b.sfp[1] = reinterpret_cast<uint64_t*>(base + osf1);
  b.sidx[0] = reinterpret_cast<int32_t*>(base + osi0);
  b.sidx[1] = reinterpret_cast<int32_t*>(base + osi1);
  b.uE = reinterpret_cast<int32_t*>(base + ouE);
  b.ufp = reinterpret_cast<uint64_t*>(base + ouf);
  b.uidx = reinterpret_cast<int32_t*>(base + oui);
  b.counts = reinterpret_cast<unsigned*>(base + ocnt);
  b.bsum = reinterpret_cast<unsigned*>(base + obs);
  b.ztab = reinterpret_cast<uint64_t*>(base + ozt);
  b.st = reinterpret_cast<PqState*>(base + ost);
  b.best_seq = reinterpret_cast<uint64_t*>(base + obest);
  b.H = reinterpret_cast<uint64_t*>(base + oH);
  b.seeds = seeds;
  PqState* dst = b.st;

  // ---- set-up: visited set, Zobrist keys, seeds sorted by (E, fp, index), de-duplicated, admitted
  if (cudaMemsetAsync(b.H, 0xff, 8ull << cfg->H_log2, st) != cudaSuccess) return LABS_ERR_CUDA;
  pq_ztab_kernel<<<(L + 255) / 256, 256, 0, st>>>(b.ztab, L);
  pq_state_init_kernel<<<1, 1, 0, st>>>(dst, n_seeds);
  pq_seed_kernel<<<(unsigned)std::min<long long>((n_seeds + kPqWarps - 1) / kPqWarps, ctx->num_sms * 16), 32 * kPqWarps,
                   0, st>>>(b, n_seeds);
  auto sort_and_dedup = [&](long long max_n, cudaStream_t s) {
    const unsigned nb = (unsigned)std::max(1ll, (max_n + kTile - 1) / kTile);
    issue_compact<0>(b, max_n, &dst->nS, s);
    const int nseg = (int)((256ll * nb + kSeg - 1) / kSeg);
    for (int pass = 0; pass < 6; pass++) {
      radix_hist_kernel<<<nb, 256, 0, s>>>(b, pass);
      seg_reduce_kernel<<<nseg, 256, 0, s>>>(b, pass);
      seg_scan_sums_kernel<<<1, 1024, 0, s>>>(b.bsum, nseg, b.st, pass);
      seg_down_kernel<<<nseg, 256, 0, s>>>(b, pass);
      radix_scatter_kernel<<<nb, 256, 0, s>>>(b, pass);
    }
    sort_fixup_kernel<<<(unsigned)std::min<long long>((max_n + 255) / 256, (long long)ctx->num_sms * 8), 256, 0, s>>>(b);
    issue_compact<1>(b, max_n, &dst->nU, s);
  };
  sort_and_dedup(n_seeds, st);
  pq_seed_admit_kernel<<<(unsigned)std::min<long long>((std::min<long long>(n_seeds, cfg->cap) + 255) / 256, 4096), 256, 0,
                         st>>>(b);
  pq_seed_finish_kernel<<<1, 1, 0, st>>>(b);

  // ---- rounds
  const long long max_rounds = (cfg->max_expansions + cfg->B - 1) / cfg->B + 1;
  const unsigned exp_blocks = (unsigned)std::max(1ll, std::min<long long>((cfg->B + kPqWarps - 1) / kPqWarps,
                                                                        (long long)ctx->num_sms * 8));
  const unsigned merge_blocks =
      (unsigned)std::max(1ll, std::min<long long>((cfg->cap + kMergeTile - 1) / kMergeTile, (long long)ctx->num_sms * 16));
  // Every round issues the same launches with the same arguments (a round's sizes and stop state live
  // in device memory), so one round is captured as a CUDA graph and replayed: about 50 launches per
  // round become one.
  if (cudaGetLastError() != cudaSuccess) return LABS_ERR_CUDA;
  if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return LABS_ERR_CUDA;
  if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LABS_ERR_CUDA;
  {
    cudaStream_t cs = ctx->capture_stream;
    pq_round_begin_kernel<<<1, 1, 0, cs>>>(b);
    pq_expand_kernel<<<exp_blocks, 32 * kPqWarps, 0, cs>>>(b, ly);
    sort_and_dedup((long long)cfg->B * width, cs);
    pq_best_kernel<<<1, 1, 0, cs>>>(b);
    pq_merge_kernel<<<merge_blocks, 256, 0, cs>>>(b);
    pq_round_end_kernel<<<1, 256, 0, cs>>>(b);
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
      if (cudaMemcpyAsync(hstop, &dst->stop, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
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
