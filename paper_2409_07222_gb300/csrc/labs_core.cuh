// labs_core.cuh -- device building blocks shared by the LABS kernels (sm_103a).
//
// One walk (or one sequence) is owned by one warp.  Its state lives in the warp's shared-memory slab:
//   * the sequence, bit-packed (32-bit words, 1 = +1);
//   * the correlation table C_{lambda g}, g = 1..G, as int16 (master) and int8 (fast-path copy);
//   * "byte windows": for every neighbour m the kernel needs s_{m + lambda g} and s_{m - lambda g}
//     for g = 1..G.  They are stored as one byte per position, enc(s) = s + 1 in {0, 2} and 1 for a
//     position outside 1..L, in a forward array and a reversed array per position class, so that both
//     windows of every neighbour are contiguous and increasing in g.
//
// lambda is the lag stride: 2 for skew-symmetric walks (odd lags have C = 0 by Eq. 2 and stay 0 under
// skew-preserving flips, so only even lags are tracked and positions split by parity into two
// classes), 1 for unrestricted walks.
//
// Single-flip Delta E (Section 3, linear-time neighbour evaluation).  Flipping F in {{m}, {m, m'}}
// changes C_kappa by delta_kappa = -alpha s_m y_kappa with
//   y_kappa = s_{m+kappa}[valid] + s_{m-kappa}[valid]      (the pair (m, m') itself excluded),
//   alpha   = 2 (single flip, or the skew centre), 4 (skew pair m, m' = L+1-m: the mirror products
//             equal the direct ones for even kappa),
// so Delta E = sum_kappa delta(2C + delta) = -2 alpha s_m T_m + alpha^2 Q_m, where
//   T_m = sum_kappa C_kappa y_kappa                    -- O(#lags) per neighbour: the hot loop
//   Q_m = sum_kappa y_kappa^2 = n_f + n_b + 2 P_m      -- P_m = sum s_{m-kappa} s_{m+kappa}, kept
//                                                        incrementally (O(1) per neighbour per flip).
// The hot loop computes T_m four lags at a time: y' = fwd4 + bwd4 (bytes 0..4, no carries) and
// dp4a(y', C4) accumulates sum C (y + 2); 2 sum C is subtracted once.  With |C| <= 127 the table fits
// int8 (dp4a); otherwise the exact int16 path (dp2a) runs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "labs.h"

namespace labsg {

constexpr int kMaxL = LABS_MAX_L;
constexpr int kQOff = 3;             // class index of the first position of a class
constexpr int kDirBytes = 1216;      // byte-window array per direction (two 608-byte classes when skew)
constexpr int kClassBytes = 608;
constexpr int kCLen = 608;           // correlation table slots (>= 4 * padded group count, L <= 576)
constexpr int kBitWords = 20;        // 18 words for 576 bits + 2 zero words for funnel shifts
constexpr int kMaxR = 32;

// ------------------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter form: output i of the generator whose state
// starts at `key`.  Streams are keyed by chaining at(at(at(seed, purpose), a), b).
// ------------------------------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
enum : uint64_t { kPurposeWalk = 1, kPurposeThresh = 2, kPurposeZobrist = 0x5A0B };

__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1) * kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t purpose, uint64_t a, uint64_t b) {
  return sm64_at(sm64_at(sm64_at(seed, purpose), a), b);
}

// Zobrist key of position i (1-based) for length L, given zkey = stream_key(0, Zobrist, L, 0).
__device__ __forceinline__ uint64_t zobrist(uint64_t zkey, int i) { return sm64_at(zkey, (uint64_t)(i - 1)); }

// ------------------------------------------------------------------------------------------------
// Warp helpers
// ------------------------------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int warp_sum_i32(int v) { return __reduce_add_sync(kFull, v); }
__device__ __forceinline__ int warp_min_i32(int v) { return __reduce_min_sync(kFull, v); }
__device__ __forceinline__ int warp_max_i32(int v) { return __reduce_max_sync(kFull, v); }
__device__ __forceinline__ unsigned warp_min_u32(unsigned v) { return __reduce_min_sync(kFull, v); }

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ uint64_t warp_xor_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
  return v;
}

// ------------------------------------------------------------------------------------------------
// Lane groups: GL consecutive lanes (GL = 32: the whole warp; GL = 16: either half) own one walk or one
// sequence.  Every synchronising primitive names the group's own lanes only, so the two halves of a
// warp may hold different walks and diverge safely; shuffles use width GL, so source lanes are
// group-relative.
// ------------------------------------------------------------------------------------------------
template <int GL>
__device__ __forceinline__ int glane() {
  return (int)(threadIdx.x & (GL - 1));
}
template <int GL>
__device__ __forceinline__ int gbase() {  // first lane of the group inside the warp
  return (int)(threadIdx.x & 31 & ~(GL - 1));
}
template <int GL>
__device__ __forceinline__ unsigned gmask() {
  if (GL == 32) return kFull;
  return ((1u << (GL & 31)) - 1u) << gbase<GL>();
}
template <int GL>
__device__ __forceinline__ int gsum(int v) { return __reduce_add_sync(gmask<GL>(), v); }
template <int GL>
__device__ __forceinline__ int gmin(int v) { return __reduce_min_sync(gmask<GL>(), v); }
template <int GL>
__device__ __forceinline__ int gmax(int v) { return __reduce_max_sync(gmask<GL>(), v); }
template <int GL>
__device__ __forceinline__ unsigned gminu(unsigned v) { return __reduce_min_sync(gmask<GL>(), v); }
// group-relative ballot: bit j is group lane j
template <int GL>
__device__ __forceinline__ unsigned gballot(bool p) { return __ballot_sync(gmask<GL>(), p) >> gbase<GL>(); }
template <int GL>
__device__ __forceinline__ bool gall(bool p) { return __all_sync(gmask<GL>(), p); }
template <int GL>
__device__ __forceinline__ bool gany(bool p) { return __any_sync(gmask<GL>(), p); }
template <int GL>
__device__ __forceinline__ void gsync() { __syncwarp(gmask<GL>()); }
template <int GL, class T>
__device__ __forceinline__ T gshfl(T v, int src) { return __shfl_sync(gmask<GL>(), v, src, GL); }
template <int GL, class T>
__device__ __forceinline__ T gshfl_xor(T v, int o) { return __shfl_xor_sync(gmask<GL>(), v, o, GL); }
template <int GL>
__device__ __forceinline__ uint64_t gxor_u64(uint64_t v) {
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) v ^= gshfl_xor<GL>(v, o);
  return v;
}

// ------------------------------------------------------------------------------------------------
// Layout of one walk for (L, skew, p, M).  Identical on every lane (pure function of its inputs).
// ------------------------------------------------------------------------------------------------
struct Layout {
  int L, skew, p, lam, lsh, G, NG, c, mlast;  // lam = 1 << lsh
  int ncls;
  int tile_first[2], ntiles[2];
  int n_tiles;
  int Qr;
  int M, H;   // neighbours per tile, lag ranges per tile (lanes sharing a tile)
  int R;      // ring length M/4 + 1; group ranges are multiples of R
  int NGh;    // groups of lag range 0 (range 1, when H = 2, is [NGh, NGend))
  int NGend;  // padded end of the groups (C = 0 beyond NG)
  int n_tasks;
  // ceil(2^16 / tasks of the class): for 0 <= n <= 32, (n * fold_magic) >> 16 = n / tasks exactly (the
  // error n * (magic * tasks - 2^16) stays below 32 * tasks < 2^16), so a lane splits a class's tasks
  // without a divide
  int fold_magic[2];
  int cw;  // 32-bit words per class in the byte-window arrays (class `cls` starts at word cls * cw)
  int cl;  // correlation-table entries kept (C16 / C8 lengths): > G, a multiple of 8, zero beyond G
};

// word offset of class `cls` inside the fwd/bwd arrays (class 1 exists only for skew walks)
__host__ __device__ __forceinline__ int cls_words(const Layout& ly, int cls) { return cls * ly.cw; }

// class and class index of position i (1-based)
__host__ __device__ __forceinline__ int pos_cls(const Layout& ly, int i) { return ly.skew ? (i & 1) : 0; }
__host__ __device__ __forceinline__ int pos_q(const Layout& ly, int i) {
  return ly.skew ? ((i - ((i & 1) ? 1 : 2)) >> 1) + kQOff : i - 1 + kQOff;
}
__host__ __device__ __forceinline__ int q_pos(const Layout& ly, int cls, int q) {
  return ly.skew ? 2 * (q - kQOff) + (cls ? 1 : 2) : q - kQOff + 1;
}

__host__ __device__ inline bool make_layout(Layout& ly, int L, int skew, int p, int M, int H = 1) {
  ly.L = L;
  ly.skew = skew;
  ly.p = p;
  ly.M = M;
  ly.H = H;
  ly.R = M / 4 + 1;
  ly.lam = skew ? 2 : 1;
  ly.lsh = skew ? 1 : 0;
  ly.G = (L - 1) >> ly.lsh;
  ly.NG = (ly.G + 3) / 4;
  ly.c = (L + 1) / 2;
  ly.mlast = skew ? ly.c : L;
  ly.ncls = skew ? 2 : 1;
  ly.n_tiles = 0;
  int qmax_end = 0;
  for (int cls = 0; cls < 2; cls++) {
    ly.tile_first[cls] = 0;
    ly.ntiles[cls] = 0;
    if (cls >= ly.ncls) continue;
    int i_lo = p + 1, i_hi = ly.mlast;
    if (skew) {
      if ((i_lo & 1) != cls) i_lo++;
      if ((i_hi & 1) != cls) i_hi--;
    }
    if (i_lo > i_hi) continue;
    int q_lo = pos_q(ly, i_lo), q_hi = pos_q(ly, i_hi);
    int first = ((q_lo - 3) / 4) * 4 + 3;
    int nt = (q_hi - first + 1 + M - 1) / M;
    ly.tile_first[cls] = first;
    ly.ntiles[cls] = nt;
    ly.n_tiles += nt;
    int end = first + nt * M - 1;
    if (end > qmax_end) qmax_end = end;
  }
  ly.Qr = qmax_end + ((2 - (qmax_end & 3)) & 3);
  ly.n_tasks = ly.n_tiles * H;
  for (int cls = 0; cls < 2; cls++) {
    const int nt = ly.ntiles[cls] * H;
    ly.fold_magic[cls] = nt > 0 ? ((1 << 16) + nt - 1) / nt : 0;
  }
  if (H == 1) {
    ly.NGh = ((ly.NG + ly.R - 1) / ly.R) * ly.R;
    ly.NGend = ly.NGh;
  } else {
    int half = (ly.NG + 1) / 2;
    ly.NGh = ((half + ly.R - 1) / ly.R) * ly.R;
    int rest = ly.NG - ly.NGh;
    ly.NGend = ly.NGh + (rest > 0 ? ((rest + ly.R - 1) / ly.R) * ly.R : 0);
  }
  // byte windows must stay inside a class array (see the bound derivation in the design notes)
  int cap = skew ? kClassBytes : kDirBytes;
  int need_f = qmax_end + 4 * ly.NGend + 8;
  int need_b = ly.Qr + 4 * ly.NGend + 8;
  ly.cw = cap / 4;
  ly.cl = kCLen;
  // the walk's P bookkeeping reads class index 2q - q_f <= 2 * qmax_end
  return (H == 1 || H == 2) && M % 4 == 0 && need_f < cap && need_b < cap && 2 * qmax_end < cap &&
         4 * ly.NGend <= kCLen && L >= 2 && L <= kMaxL;
}

// Shrinks a valid layout's arrays to what its length needs (the walk kernels size their shared-memory
// slabs per launch with it): class arrays of the smallest multiple of 16 bytes above every window, the
// P bookkeeping's index 2 qmax_end and the class itself, and a table of the smallest multiple of 8
// entries above G and 4 NGend (its last entry, always zero, stands in for a missing pair term).
__host__ __device__ inline void compact_layout(Layout& ly) {
  int qmax_end = 0;
  for (int cls = 0; cls < ly.ncls; cls++)
    if (ly.ntiles[cls] > 0) {
      const int end = ly.tile_first[cls] + ly.ntiles[cls] * ly.M - 1;
      if (end > qmax_end) qmax_end = end;
    }
  int need = qmax_end + 4 * ly.NGend + 8;
  const int need_b = ly.Qr + 4 * ly.NGend + 8;
  if (need_b > need) need = need_b;
  if (2 * qmax_end + 1 > need) need = 2 * qmax_end + 1;
  const int n_cls = ly.skew ? (ly.L + 1) / 2 : ly.L;  // class indices kQOff .. kQOff + n_cls - 1 hold positions
  if (kQOff + n_cls + 1 > need) need = kQOff + n_cls + 1;
  ly.cw = (need + 15) / 16 * 4;
  int cl = 4 * ly.NGend;
  if (ly.G + 1 > cl) cl = ly.G + 1;
  ly.cl = (cl + 7) / 8 * 8;
}

// Tile tau -> (class, first class index).
__device__ __forceinline__ void tile_of(const Layout& ly, int tau, int& cls, int& q0) {
  if (tau < ly.ntiles[0]) {
    cls = 0;
    q0 = ly.tile_first[0] + tau * ly.M;
  } else {
    cls = 1;
    q0 = ly.tile_first[1] + (tau - ly.ntiles[0]) * ly.M;
  }
}

// ------------------------------------------------------------------------------------------------
// Shared-memory slab of one walk.  ScanSmem is the fixed-size form (every length up to 576); the walk
// kernels carve slabs sized for their launch's lengths out of dynamic shared memory and address them
// through a ScanView with the same members.  Class `cls` of fwd/bwd starts at word cls * ly.cw; the
// tables hold ly.cl entries.
// ------------------------------------------------------------------------------------------------
struct __align__(16) ScanSmem {
  uint32_t fwd[kDirBytes / 4];
  uint32_t bwd[kDirBytes / 4];
  int16_t C16[kCLen];  // C_{lambda (h+1)} at h, zero beyond G
  int8_t C8[kCLen];    // int8 copy, valid when every |C| <= 127
  uint32_t bits[kBitWords];
};

struct ScanView {
  uint32_t* fwd;
  uint32_t* bwd;
  int16_t* C16;
  int8_t* C8;
  uint32_t* bits;
};

template <class S>
__device__ __forceinline__ int seq_bit(const S& sm, int i) {
  return (sm.bits[(i - 1) >> 5] >> ((i - 1) & 31)) & 1;
}

template <class S>
__device__ __forceinline__ int fwd_byte(const S& sm, const Layout& ly, int cls, int q) {
  return reinterpret_cast<const uint8_t*>(sm.fwd + cls_words(ly, cls))[q];
}
template <class S>
__device__ __forceinline__ int bwd_byte(const S& sm, const Layout& ly, int cls, int t) {
  return reinterpret_cast<const uint8_t*>(sm.bwd + cls_words(ly, cls))[t];
}
// s_i in {-1, +1} read from the forward byte array
template <class S>
__device__ __forceinline__ int s_at(const S& sm, const Layout& ly, int i) {
  return fwd_byte(sm, ly, pos_cls(ly, i), pos_q(ly, i)) - 1;
}

// Byte windows from the packed bits (whole arrays, pads included).
// Bytes of positions p, p+d, p+2d, p+3d (d = 1 or 2): byte e = s + 1 (0 or 2) for a position inside
// 1..L, else the pad 1; rev: byte e holds position p + (3 - e) d.  Bits at and above L are zero in
// sm.bits.  Every other bit of the window is taken for d = 2 (the positions of one parity class).
template <class S>
__device__ __forceinline__ uint32_t window_bytes(const S& sm, int L, int p, int d, bool rev) {
  const int plast = p + 3 * d;
  if (p > L || plast < 1) return 0x01010101u;  // no position of the window inside 1..L
  const int b = p - 1;  // bit index of position p: -3d <= b <= L - 1
  uint32_t x;
  if (b >= 0) {
    const int wi = b >> 5;
    x = __funnelshift_r(sm.bits[wi], wi + 1 < kBitWords ? sm.bits[wi + 1] : 0u, b & 31);
  } else {
    x = sm.bits[0] << (-b);
  }
  if (d == 2) {  // bits 0, 2, 4, 6 -> bits 0..3
    x &= 0x55u;
    x = (x | (x >> 1)) & 0x33u;
    x = (x | (x >> 2)) & 0x0Fu;
  } else {
    x &= 0xFu;
  }
  const int lo = p < 1 ? (1 - p + d - 1) / d : 0;          // invalid positions at the low end
  const int hi = plast > L ? (plast - L + d - 1) / d : 0;  // and at the high end
  const uint32_t v = ((0xFu << lo) & (0xFu >> hi)) & 0xFu;
  uint32_t xv = x & v, pad = v ^ 0xFu;
  if (rev) {
    xv = __brev(xv) >> 28;
    pad = __brev(pad) >> 28;
  }
  // nibble -> one bit per byte: n * 0x204081 puts bit e at 7e + e = 8e, without carries
  return 2u * ((xv * 0x204081u) & 0x01010101u) + ((pad * 0x204081u) & 0x01010101u);
}

// The forward and reversed byte windows of every class: class index t is position q_pos(cls, t), i.e.
// lambda (t - kQOff) + first position of the class, so every word is four positions lambda apart.
template <int GL = 32, class S>
__device__ inline void build_bytes(S& sm, const Layout& ly) {
  const int words_per_cls = ly.cw;
  for (int cls = 0; cls < ly.ncls; cls++) {
    uint32_t* F = sm.fwd + cls_words(ly, cls);
    uint32_t* B = sm.bwd + cls_words(ly, cls);
    const int first = q_pos(ly, cls, kQOff);  // position of class index kQOff
    for (int w = glane<GL>(); w < words_per_cls; w += GL) {
      F[w] = window_bytes(sm, ly.L, first + ly.lam * (4 * w - kQOff), ly.lam, false);
      B[w] = window_bytes(sm, ly.L, first + ly.lam * (ly.Qr - 4 * w - 3 - kQOff), ly.lam, true);
    }
  }
  gsync<GL>();
}

// C_k = (L-k) - 2 popc((x XOR (x >> k)) restricted to the low L-k bits) from the packed bits.
__device__ __forceinline__ int corr_lag(const uint32_t* bits, int L, int k) {
  const int n = L - k;  // number of products s_i s_{i+k}
  const int ws = k >> 5, sh = k & 31;
  const int nw = (n + 31) >> 5;
  int dis = 0;
  for (int w = 0; w < nw; w++) {
    uint32_t x = bits[w] ^ __funnelshift_r(bits[w + ws], bits[w + ws + 1], sh);
    int rem = n - 32 * w;
    if (rem < 32) x &= (1u << rem) - 1u;
    dis += __popc(x);
  }
  return n - 2 * dis;
}

// sum_{i=0}^{n-1} a_i b_{i+d} for two sequences given by their bits (n = L - d products, d >= 0):
// n - 2 popc((a XOR (b >> d)) restricted to the low n bits).
__device__ __forceinline__ int corr_pair(const uint32_t* a, const uint32_t* b, int L, int d) {
  const int n = L - d;
  const int ws = d >> 5, sh = d & 31;
  const int nw = (n + 31) >> 5;
  int dis = 0;
  for (int w = 0; w < nw; w++) {
    uint32_t x = a[w] ^ __funnelshift_r(b[w + ws], b[w + ws + 1], sh);
    const int rem = n - 32 * w;
    if (rem < 32) x &= (1u << rem) - 1u;
    dis += __popc(x);
  }
  return n - 2 * dis;
}

// P_m = sum_{g} s_{m - lambda g} s_{m + lambda g} over the lags with both ends inside 1..L -- for a skew
// layout without the pair's own lag gd = c - m -- for every position m in [m_lo, m_hi] (by default all of
// them), into P_out[m - 1] (int16).
// Per position class (every position for lambda = 1, each parity for lambda = 2) the class sequence x
// (x_j = s at class index j) has the self-convolution (x * x)[k] = sum_j x_j x_{k-j}, which counts each
// product of P twice plus x_j^2: P = ((x * x)[2j] - 1) / 2.  (x * x)[k] is the correlation of x with its
// reversal at offset n-1-k, one popcount per 32 products.  xb, rb: per-warp scratch of kBitWords words.
__device__ inline void p_all(const ScanSmem& sm, const Layout& ly, uint32_t* xb, uint32_t* rb, int16_t* P_out,
                             int m_lo = 1, int m_hi = kMaxL) {
  const int lane = lane_id();
  for (int cls = 0; cls < ly.ncls; cls++) {
    const int b = ly.skew ? (cls ? 1 : 2) : 1;  // first position of the class
    const int n = ly.skew ? (b == 1 ? (ly.L + 1) / 2 : ly.L / 2) : ly.L;
    for (int w = 0; w < kBitWords; w++) {  // x and its reversal
      const int j = 32 * w + lane;
      int bx = 0, br = 0;
      if (j < n) {
        const int i = ly.lam * j + b, ir = ly.lam * (n - 1 - j) + b;
        bx = (int)((sm.bits[(i - 1) >> 5] >> ((i - 1) & 31)) & 1u);
        br = (int)((sm.bits[(ir - 1) >> 5] >> ((ir - 1) & 31)) & 1u);
      }
      const unsigned wx = __ballot_sync(kFull, bx), wr = __ballot_sync(kFull, br);
      if (lane == 0) {
        xb[w] = wx;
        rb[w] = wr;
      }
    }
    __syncwarp();
    // only the class indices whose positions lie in [m_lo, m_hi]
    const int j_lo = m_lo > b ? (m_lo - b + ly.lam - 1) / ly.lam : 0;
    const int j_end = m_hi >= b ? min(n, (m_hi - b) / ly.lam + 1) : 0;
    for (int j = j_lo + lane; j < j_end; j += 32) {
      const int d = n - 1 - 2 * j;
      const int conv = d >= 0 ? corr_pair(xb, rb, n, d) : corr_pair(rb, xb, n, -d);
      int P = (conv - 1) / 2;
      const int m = ly.lam * j + b;
      if (ly.skew && m < ly.c) {  // the pair (m, m') is not a product of P_m
        const int gd = ly.c - m;
        if (j - gd >= 0 && j + gd < n) {
          const int x0 = (int)((xb[(j - gd) >> 5] >> ((j - gd) & 31)) & 1u);
          const int x1 = (int)((xb[(j + gd) >> 5] >> ((j + gd) & 31)) & 1u);
          P -= (x0 == x1) ? 1 : -1;
        }
      }
      P_out[m - 1] = (int16_t)P;
    }
    __syncwarp();
  }
}

// C_{lambda g} for g = 1..G; lanes split the lags.  Writes C16 (zero-padded to ly.cl) and returns E on
// every lane of the group (sum over the tracked lags; for skew inputs the untracked odd lags are zero).
template <int GL = 32, class S>
__device__ inline int build_table(S& sm, const Layout& ly) {
  int e_part = 0;
  for (int h = glane<GL>(); h < ly.cl; h += GL) {
    int g = h + 1;
    int cval = (g <= ly.G) ? corr_lag(sm.bits, ly.L, ly.lam * g) : 0;
    sm.C16[h] = (int16_t)cval;
    e_part += cval * cval;
  }
  gsync<GL>();
  return gsum<GL>(e_part);
}

// int8 copy of the table; returns true on every lane if all |C| <= 127 (fast path allowed).
template <int GL = 32, class S>
__device__ inline bool pack_c8(S& sm, const Layout& ly) {
  bool ok = true;
  for (int h = glane<GL>(); h < ly.cl; h += GL) {
    int v = sm.C16[h];
    ok &= (v >= -127 && v <= 127);
    sm.C8[h] = (int8_t)max(-127, min(127, v));
  }
  gsync<GL>();
  return gall<GL>(ok);
}

template <int GL = 32, class S>
__device__ inline int table_sum(const S& sm, const Layout& ly) {
  int s = 0;
  for (int h = glane<GL>(); h < ly.cl; h += GL) s += sm.C16[h];
  return gsum<GL>(s);
}

// ------------------------------------------------------------------------------------------------
// Hot loop: acc[j] += sum_{u in [u_begin, u_end)} sum_{e<4} C8[4u+e] * y'_{4u+e+1}(m_j) for the M
// neighbours of one tile (class `cls`, class indices q0 .. q0+M-1; q0 = 3 mod 4 so every window has a
// static alignment).  Groups are read in turns of R = M/4 + 1 (the ring of realigned words); a range
// that is not a whole number of turns ends with a partial one.
// ------------------------------------------------------------------------------------------------
template <int M, bool WIDE, class S>
__device__ __forceinline__ void scan_range(const S& sm, const Layout& ly, int cls, int q0, int u_begin, int u_end,
                                           int (&acc)[M]) {
  // Word streams: plain words P[t] (ring of R) and, for byte offsets r = 1..3, the realigned words
  // S_r[t] = bytes 4t+r .. 4t+r+3 (rings of R).  Each new word costs one load and three funnel
  // shifts per direction, shared by every neighbour of the tile.
  constexpr int K4 = M / 4;
  constexpr int R = K4 + 1;
  const uint32_t* Fw = sm.fwd + cls_words(ly, cls);
  const uint32_t* Bw = sm.bwd + cls_words(ly, cls);
  const int tf0 = ((q0 + 1) >> 2) + u_begin;
  const int tb0 = ((ly.Qr - q0 + 1) >> 2) - K4 + u_begin;
  uint32_t pf[R], pb[R], sf[3][R], sb[3][R];
#pragma unroll
  for (int a = 0; a < R; a++) {
    pf[a] = Fw[tf0 + a];
    pb[a] = Bw[tb0 + a];
  }
#pragma unroll
  for (int a = 0; a < K4; a++)
#pragma unroll
    for (int r = 1; r < 4; r++) {
      sf[r - 1][a] = __funnelshift_r(pf[a], pf[a + 1], 8 * r);
      sb[r - 1][a] = __funnelshift_r(pb[a], pb[a + 1], 8 * r);
    }
  const uint32_t* C8w = reinterpret_cast<const uint32_t*>(sm.C8) + u_begin;
  const uint32_t* C16w = reinterpret_cast<const uint32_t*>(sm.C16) + 2 * u_begin;
  const int n = u_end > u_begin ? u_end - u_begin : 0;
  // group u of the range in ring slot du (du = u mod R, a constant after unrolling)
  auto step = [&](const int u, const int du) {
      uint32_t c4 = 0, clo = 0, chi = 0;
      if (WIDE) {
        clo = C16w[2 * u];
        chi = C16w[2 * u + 1];
      } else {
        c4 = C8w[u];
      }
#pragma unroll
      for (int j = 0; j < M; j++) {
        const int af = (du + (j >> 2)) % R;
        const int rf = j & 3;
        const uint32_t f = rf ? sf[rf - 1][af] : pf[af];
        const int ab = (du + K4 - ((j + 3) >> 2)) % R;
        const int rb = (4 - (j & 3)) & 3;
        const uint32_t b = rb ? sb[rb - 1][ab] : pb[ab];
        const int y4 = (int)(f + b);
        if (WIDE) {
          acc[j] = __dp2a_lo((int)clo, y4, acc[j]);
          acc[j] = __dp2a_hi((int)chi, y4, acc[j]);
        } else {
          acc[j] = __dp4a(y4, (int)c4, acc[j]);
        }
      }
      // advance: word u + R enters slot du; S_r[u + K4] goes to slot (du + K4) % R
      pf[du] = Fw[tf0 + u + R];
      pb[du] = Bw[tb0 + u + R];
      const int sl = (du + K4) % R;
#pragma unroll
      for (int r = 1; r < 4; r++) {
        sf[r - 1][sl] = __funnelshift_r(pf[sl], pf[du], 8 * r);
        sb[r - 1][sl] = __funnelshift_r(pb[sl], pb[du], 8 * r);
      }
  };
  // whole ring turns, then the last partial turn (groups beyond the range are not scanned: the table
  // is zero there, so the accumulators would not change)
  const int nfull = n - n % R;
  for (int u0 = 0; u0 < nfull; u0 += R) {
#pragma unroll
    for (int du = 0; du < R; du++) step(u0 + du, du);
  }
  if (nfull < n) {
#pragma unroll
    for (int du = 0; du < R - 1; du++) {
      if (nfull + du >= n) break;
      step(nfull + du, du);
    }
  }
}

// The whole lag range of one tile (single lane per tile).
template <int M, bool WIDE, class S>
__device__ __forceinline__ void scan_tile(const S& sm, const Layout& ly, int cls, int q0, int (&acc)[M]) {
#pragma unroll
  for (int j = 0; j < M; j++) acc[j] = 0;
  scan_range<M, WIDE>(sm, ly, cls, q0, 0, ly.NGh, acc);
}

// Per-neighbour constants of slot (cls, q): position, whether it is a neighbour, pair flag, counts.
struct SlotInfo {
  int m;       // position (1-based)
  int active;  // inside the free range
  int pair;    // skew pair flip (m != centre)
  int nf, nb;  // valid forward / backward lags
  int gd;      // lag index of the excluded pair (m, m') when pair, else 0
};

__device__ __forceinline__ SlotInfo slot_info(const Layout& ly, int cls, int q) {
  SlotInfo si;
  si.m = q_pos(ly, cls, q);
  si.active = (si.m >= ly.p + 1 && si.m <= ly.mlast) ? 1 : 0;
  si.pair = (ly.skew && si.m != ly.c) ? 1 : 0;
  si.nf = (ly.L - si.m) >> ly.lsh;
  si.nb = (si.m - 1) >> ly.lsh;
  si.gd = si.pair ? (ly.L + 1 - 2 * si.m) >> 1 : 0;
  return si;
}

// P_m from scratch: sum over g <= min(nf, nb), g != gd, of s_{m - lambda g} s_{m + lambda g}.
template <class S>
__device__ __forceinline__ int p_from_scratch(const S& sm, const Layout& ly, int cls, int q, const SlotInfo& si) {
  if (!si.active) return 0;
  int gmax = min(si.nf, si.nb);
  int P = 0;
  for (int g = 1; g <= gmax; g++) {
    if (g == si.gd) continue;
    P += (fwd_byte(sm, ly, cls, q + g) - 1) * (bwd_byte(sm, ly, cls, ly.Qr - q + g) - 1);
  }
  return P;
}

// Delta E of slot (cls, q) from its accumulator, the table sum SC and P.
template <class S>
__device__ __forceinline__ int finish_delta(const S& sm, const Layout& ly, int cls, int q, const SlotInfo& si, int acc,
                                            int SC, int P) {
  int s_m = fwd_byte(sm, ly, cls, q) - 1;
  int T = acc - 2 * SC;
  int alpha = si.pair ? 4 : 2;
  if (si.pair) {
    // s_{m'} = (-1)^{c-m} s_m by Eq. (2); remove the product with the mirror from the g = gd term
    int s_mp = ((ly.c - si.m) & 1) ? -s_m : s_m;
    T -= (int)sm.C16[si.gd - 1] * s_mp;
  }
  int Q = si.nf + si.nb - si.pair + 2 * P;
  return -2 * alpha * s_m * T + alpha * alpha * Q;
}

// Table update for flipping neighbour m* (pre-flip s): C_{lambda g} += -alpha s_m* y_g(m*) for g = 1..G,
// and the int8 copy alongside, four lags per lane and iteration: the windows s_{m* + lambda g} and
// s_{m* - lambda g} of lags 4u+1..4u+4 are one realigned word per direction and y + 2 = fwd4 + bwd4
// bytewise (as in the scan).  Lags beyond G have pads at both ends, so their y is 0 and C stays 0.
// Returns the change of the table sum; *fast receives whether every |C| <= 127 (the int8 copy is only
// read while that holds, and every step rewrites all of it).
template <int GL = 32, class S>
__device__ inline int table_update(S& sm, const Layout& ly, int mstar, bool* fast) {
  const int cls = pos_cls(ly, mstar), q = pos_q(ly, mstar);
  const int pair = (ly.skew && mstar != ly.c) ? 1 : 0;
  const int s_m = fwd_byte(sm, ly, cls, q) - 1;
  const int as = -(pair ? 4 : 2) * s_m;  // C_g += as * y_g
  const int gd = pair ? (ly.L + 1 - 2 * mstar) >> 1 : 0;
  const int s_mp = pair ? (((ly.c - mstar) & 1) ? -s_m : s_m) : 0;
  const uint32_t* Fw = sm.fwd + cls_words(ly, cls);
  const uint32_t* Bw = sm.bwd + cls_words(ly, cls);
  const int of = q + 1, ob = ly.Qr - q + 1;  // byte offsets of lag 1 in the two windows
  const int wf = of >> 2, sf = 8 * (of & 3), wb = ob >> 2, sb = 8 * (ob & 3);
  uint32_t* C16w = reinterpret_cast<uint32_t*>(sm.C16);
  uint32_t* C8w = reinterpret_cast<uint32_t*>(sm.C8);
  int dsum = 0;
  bool ok = true;
  for (int u = glane<GL>(); u < ly.NG; u += GL) {
    uint32_t y4 = __funnelshift_r(Fw[wf + u], Fw[wf + u + 1], sf) + __funnelshift_r(Bw[wb + u], Bw[wb + u + 1], sb);
    // the pair's own product is not part of C: lag gd drops s_m' from its byte, which holds
    // (s_m' + 1) + (the other end + 1 or a pad 1), so the byte stays in 0..4 and no borrow crosses bytes
    const int eg = gd - 1 - 4 * u;
    if ((unsigned)eg < 4u) y4 -= (uint32_t)s_mp << (8 * eg);
    const uint32_t lo = C16w[2 * u], hi = C16w[2 * u + 1];
    int c[4] = {(int)(int16_t)(lo & 0xffffu), (int)lo >> 16, (int)(int16_t)(hi & 0xffffu), (int)hi >> 16};
    dsum += as * ((int)__dp4a(y4, 0x01010101u, 0u) - 8);  // sum of the four y
    uint32_t c8 = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      c[e] += as * ((int)((y4 >> (8 * e)) & 0xffu) - 2);
      ok &= (unsigned)(c[e] + 127) <= 254u;
      c8 |= ((uint32_t)c[e] & 0xffu) << (8 * e);
    }
    C16w[2 * u] = ((uint32_t)c[0] & 0xffffu) | ((uint32_t)c[1] << 16);
    C16w[2 * u + 1] = ((uint32_t)c[2] & 0xffffu) | ((uint32_t)c[3] << 16);
    C8w[u] = c8;
  }
  gsync<GL>();
  *fast = gall<GL>(ok);
  return gsum<GL>(dsum);
}

// Negates s_i in the bits and both byte arrays (one lane per position, distinct positions may run
// on different lanes at once; then a group sync).
template <class S>
__device__ __forceinline__ void flip_position(S& sm, const Layout& ly, int i) {
  const int cls = pos_cls(ly, i), q = pos_q(ly, i);
  uint8_t* F = reinterpret_cast<uint8_t*>(sm.fwd + cls_words(ly, cls));
  uint8_t* B = reinterpret_cast<uint8_t*>(sm.bwd + cls_words(ly, cls));
  F[q] = (uint8_t)(2 - F[q]);
  B[ly.Qr - q] = (uint8_t)(2 - B[ly.Qr - q]);
  atomicXor(&sm.bits[(i - 1) >> 5], 1u << ((i - 1) & 31));
}

// Copies packed 64-bit words from global memory into the slab bits (zero-padded).
template <class S>
__device__ inline void load_bits(S& sm, const uint64_t* src, int L) {
  const int W32 = (L + 31) >> 5;
  for (int w = lane_id(); w < kBitWords; w += 32) {
    uint32_t v = 0;
    if (w < W32) {
      uint64_t x = src[w >> 1];
      v = (w & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
      int rem = L - 32 * w;
      if (rem < 32) v &= (1u << rem) - 1u;
    }
    sm.bits[w] = v;
  }
  __syncwarp();
}

// Builds a walk start into the bits: s_1..s_p from the prefix, free element j (position p+1+j) is +1
// iff bit j%64 of output j/64 of stream `key`; skew walks fill the last k by Eq. (2).  Each 32-bit word
// is assembled from 32 / GL group ballots.
template <int GL = 32, class S>
__device__ inline void build_start(S& sm, const Layout& ly, const uint64_t* prefix, uint64_t key) {
  const int lane = glane<GL>();
  const int W32 = (ly.L + 31) >> 5;
  for (int w = 0; w < kBitWords; w++) {
    unsigned word = 0;
#pragma unroll
    for (int part = 0; part < 32 / GL; part++) {
      int i = 32 * w + GL * part + lane + 1;
      int bit = 0;
      if (i <= ly.L) {
        int src = i;
        int neg = 0;
        if (ly.skew && i > ly.c) {
          src = 2 * ly.c - i;
          neg = (i - ly.c) & 1;
        }
        int b;
        if (src <= ly.p) {
          b = (int)((prefix[(src - 1) >> 6] >> ((src - 1) & 63)) & 1u);
        } else {
          int j = src - ly.p - 1;
          b = (int)((sm64_at(key, (uint64_t)(j >> 6)) >> (j & 63)) & 1u);
        }
        bit = b ^ neg;
      }
      const unsigned bal = gballot<GL>(bit != 0);
      word |= GL == 32 ? bal : (bal & ((1u << (GL & 31)) - 1u)) << (GL * part);
    }
    if (lane == 0) sm.bits[w] = (w < W32) ? word : 0u;
  }
  gsync<GL>();
}

// Zobrist fingerprint of the sequence in the bits.
template <int GL = 32, class S>
__device__ inline uint64_t fingerprint(const S& sm, int L, uint64_t zkey) {
  uint64_t h = 0;
  for (int i = glane<GL>() + 1; i <= L; i += GL)
    if (!seq_bit(sm, i)) h ^= zobrist(zkey, i);
  return gxor_u64<GL>(h);
}

}  // namespace labsg
