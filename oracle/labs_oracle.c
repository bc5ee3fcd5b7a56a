/*
 * labs_oracle.c -- plain, slow, obviously-correct CPU oracle for the LABS dual-step search
 * (Psenicnik, Mlinaric, Brest, Boskovic, "Dual-Step Optimization for Binary Sequences with High
 * Merit Factors", arXiv 2409.07222).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  It shares no code, header, table or helper with the CUDA
 * library; the only thing the two have in common is the packed sequence format of the interface and
 * the published definitions they are both written from.
 *
 * Representation inside the oracle: a sequence is an int8_t array s[0..L-1] holding s_1..s_L of the
 * paper (s[i-1] = s_i in {+1,-1}); every computation below works on these +-1 values with plain
 * loops -- no bit tricks.  The packed interface format is read and written only by unpack()/pack():
 * bit (i-1) mod 64 of word (i-1)/64 holds s_i, with bit value 1 meaning +1 (the paper's hex coding,
 * Section 4: a binary 0 stands for -1).
 *
 * Parity status of each function (what pins it is in tests/test_oracle_pins.py):
 *   energy / correlations       pinned: Barker sequences, closed forms, FFT identity, invariances
 *   flip deltas (definition)    pinned: brute recomputation, equals energy difference by construction
 *   linear-time flip deltas     pinned: against the definition on random and edge inputs
 *   skew fill                   pinned: odd-lag correlations vanish (Section 1, after Eq. 2)
 *   exhaustive skew search      pinned: brute force over all 2^L restricted to skew sequences
 *   walk search (Algorithm 1)   pinned: invariants + an independent set-based replay at tiny L
 *   threshold sampling          pinned: equals sorting the sampled energies (numpy)
 *   priority-queue refinement   pinned: B=1 equals a textbook best-first search (heapq) at tiny L
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#define ORACLE_MAX_L 576
#define ORACLE_MAX_W 9

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_CAPACITY = 2, ORC_ERR_NOMEM = 5 };

/* ------------------------------------------------------------------------------------------------
 * Packed format <-> +-1 arrays (interface layout only).
 * ---------------------------------------------------------------------------------------------- */
static void unpack(const uint64_t* w, int L, int8_t* s) {
  for (int i = 1; i <= L; i++) {
    uint64_t bit = (w[(i - 1) / 64] >> ((i - 1) % 64)) & 1u;
    s[i - 1] = bit ? 1 : -1;
  }
}

static void pack(const int8_t* s, int L, uint64_t* w) {
  int W = (L + 63) / 64;
  for (int j = 0; j < W; j++) w[j] = 0;
  for (int i = 1; i <= L; i++)
    if (s[i - 1] == 1) w[(i - 1) / 64] |= (uint64_t)1 << ((i - 1) % 64);
}

/* ------------------------------------------------------------------------------------------------
 * Section 1: C_k(S) = sum_{i=1}^{L-k} s_i s_{i+k};  E(S) = sum_{k=1}^{L-1} C_k(S)^2.
 * ---------------------------------------------------------------------------------------------- */
static int64_t correlation(const int8_t* s, int L, int k) {
  int64_t c = 0;
  for (int i = 1; i <= L - k; i++) c += (int64_t)s[i - 1] * s[i + k - 1];
  return c;
}

/* Fills C[k] for k = 0..L-1 (C[0] = L) and returns E. */
static int64_t energy_table(const int8_t* s, int L, int64_t* C) {
  int64_t E = 0;
  C[0] = L;
  for (int k = 1; k <= L - 1; k++) {
    C[k] = correlation(s, L, k);
    E += C[k] * C[k];
  }
  return E;
}

static int64_t energy(const int8_t* s, int L) {
  int64_t E = 0;
  for (int k = 1; k <= L - 1; k++) {
    int64_t c = correlation(s, L, k);
    E += c * c;
  }
  return E;
}

/* Batch energies of packed sequences; C_out (nullable) receives C_1..C_{L-1} per sequence. */
int oracle_energy_batch(const uint64_t* words, int L, int64_t n, int32_t* E_out, int32_t* C_out) {
  if (L < 1 || L > ORACLE_MAX_L || n < 0) return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  int8_t s[ORACLE_MAX_L];
  for (int64_t q = 0; q < n; q++) {
    unpack(words + q * W, L, s);
    int64_t E = 0;
    for (int k = 1; k <= L - 1; k++) {
      int64_t c = correlation(s, L, k);
      if (C_out) C_out[q * (L - 1) + (k - 1)] = (int32_t)c;
      E += c * c;
    }
    E_out[q] = (int32_t)E; /* E < L^3/3 < 2^31 for L <= 576 */
  }
  return ORC_OK;
}

/* Eq. (1): F = L^2 / (2E). */
double oracle_merit_factor(int L, int64_t E) { return (double)L * (double)L / (2.0 * (double)E); }

/* ------------------------------------------------------------------------------------------------
 * Eq. (2): skew symmetry for odd L = 2k+1:  s_{(k+1)+i} = (-1)^i s_{(k+1)-i},  i = 1..k.
 * ---------------------------------------------------------------------------------------------- */
static void skew_fill(int8_t* s, int L) {
  int k = (L - 1) / 2;
  for (int i = 1; i <= k; i++) {
    int sign = (i % 2 == 0) ? 1 : -1;
    s[(k + 1 + i) - 1] = (int8_t)(sign * s[(k + 1 - i) - 1]);
  }
}

static int is_skew(const int8_t* s, int L) {
  if (L % 2 == 0) return 0;
  int k = (L - 1) / 2;
  for (int i = 1; i <= k; i++) {
    int sign = (i % 2 == 0) ? 1 : -1;
    if (s[(k + 1 + i) - 1] != sign * s[(k + 1 - i) - 1]) return 0;
  }
  return 1;
}

/* Packed wrapper: positions 1..k+1 are read from `head`, the last k are filled by Eq. (2). */
int oracle_skew_fill(const uint64_t* head, int L, uint64_t* out) {
  if (L < 1 || L > ORACLE_MAX_L || L % 2 == 0) return ORC_ERR_ARG;
  int8_t s[ORACLE_MAX_L];
  unpack(head, L, s);
  skew_fill(s, L);
  pack(s, L, out);
  return ORC_OK;
}

int oracle_is_skew(const uint64_t* words, int L) {
  if (L < 1 || L > ORACLE_MAX_L) return 0;
  int8_t s[ORACLE_MAX_L];
  unpack(words, L, s);
  return is_skew(s, L);
}

/* ------------------------------------------------------------------------------------------------
 * Neighbourhoods.  Unrestricted (Algorithm 2, SEQUENCE_FLIP): the neighbour of position i flips
 * s_i, for every free position i = p+1..L.  Skew-symmetric (Algorithm 1, SEQUENCE_FLIP_SKEW): the
 * free position m in [p+1, k+1] of Eq. (3) flips s_m together with its mirror s_{L+1-m}, the only
 * pairing that keeps Eq. (2); the centre m = k+1 is its own mirror and flips alone.
 * ---------------------------------------------------------------------------------------------- */
static int flip_set(int L, int skew, int m, int* F) {
  if (!skew) { F[0] = m; return 1; }
  int mirror = L + 1 - m;
  F[0] = m;
  if (mirror == m) return 1;
  F[1] = mirror;
  return 2;
}

static void negate(int8_t* s, const int* F, int nF) {
  for (int a = 0; a < nF; a++) s[F[a] - 1] = (int8_t)-s[F[a] - 1];
}

/* Delta-E of every neighbour by definition: flip, recompute E from scratch, subtract.  Entries that
 * are not neighbours (outside the free range) hold INT32_MAX.  dE has L entries per sequence,
 * indexed by position - 1. */
int oracle_flip_deltas(const uint64_t* words, int L, int64_t n, int skew, int p, int32_t* dE) {
  if (L < 1 || L > ORACLE_MAX_L || n < 0 || p < 0) return ORC_ERR_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return ORC_ERR_ARG;
  if (!skew && p > L) return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  int last = skew ? (L - 1) / 2 + 1 : L;
  int8_t s[ORACLE_MAX_L];
  for (int64_t q = 0; q < n; q++) {
    unpack(words + q * W, L, s);
    int64_t E0 = energy(s, L);
    for (int i = 1; i <= L; i++) dE[q * L + (i - 1)] = INT32_MAX;
    for (int m = p + 1; m <= last; m++) {
      int F[2];
      int nF = flip_set(L, skew, m, F);
      negate(s, F, nF);
      dE[q * L + (m - 1)] = (int32_t)(energy(s, L) - E0);
      negate(s, F, nF);
    }
  }
  return ORC_OK;
}

/* Linear-time evaluation of one neighbour from the kept table C (Section 3: a neighbour is
 * evaluated in linear time and space, after Dimitrov 2021).  Flipping the set F changes only the
 * products s_i s_{i+k} that have exactly one factor in F; each changes sign, so
 *   delta_k = -2 * sum over those products,   Delta E = sum_k (C_k + delta_k)^2 - C_k^2.
 * Each lag sees at most 2|F| such products, so the cost is O(|F| L). */
static void flip_corr_change(const int8_t* s, int L, const int* F, int nF, int k, int64_t* delta) {
  int64_t d = 0;
  for (int a = 0; a < nF; a++) {
    int f = F[a];
    int partners[2] = {f - k, f + k};
    for (int b = 0; b < 2; b++) {
      int j = partners[b];
      if (j < 1 || j > L) continue;
      int in_F = 0;
      for (int c = 0; c < nF; c++) in_F |= (F[c] == j);
      if (in_F) continue; /* both factors flip: the product is unchanged */
      d += (int64_t)s[f - 1] * s[j - 1];
    }
  }
  *delta = -2 * d;
}

static int64_t delta_linear(const int8_t* s, const int64_t* C, int L, const int* F, int nF) {
  int64_t dE = 0;
  for (int k = 1; k <= L - 1; k++) {
    int64_t delta;
    flip_corr_change(s, L, F, nF, k, &delta);
    dE += (C[k] + delta) * (C[k] + delta) - C[k] * C[k];
  }
  return dE;
}

/* Applies the flip of F to s and updates the kept table C in O(|F| L). */
static void apply_flip(int8_t* s, int64_t* C, int L, const int* F, int nF) {
  for (int k = 1; k <= L - 1; k++) {
    int64_t delta;
    flip_corr_change(s, L, F, nF, k, &delta);
    C[k] += delta;
  }
  negate(s, F, nF);
}

/* Same output as oracle_flip_deltas, through the linear-time formula (pinned against it). */
int oracle_flip_deltas_linear(const uint64_t* words, int L, int64_t n, int skew, int p, int32_t* dE) {
  if (L < 1 || L > ORACLE_MAX_L || n < 0 || p < 0) return ORC_ERR_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return ORC_ERR_ARG;
  if (!skew && p > L) return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  int last = skew ? (L - 1) / 2 + 1 : L;
  int8_t s[ORACLE_MAX_L];
  int64_t C[ORACLE_MAX_L];
  for (int64_t q = 0; q < n; q++) {
    unpack(words + q * W, L, s);
    energy_table(s, L, C);
    for (int i = 1; i <= L; i++) dE[q * L + (i - 1)] = INT32_MAX;
    for (int m = p + 1; m <= last; m++) {
      int F[2];
      int nF = flip_set(L, skew, m, F);
      dE[q * L + (m - 1)] = (int32_t)delta_linear(s, C, L, F, nF);
    }
  }
  return ORC_OK;
}

/* Applies a list of flips (positions, one per move) to one packed sequence with the O(L) table
 * update and reports the energy after every move; used to pin the table update. */
int oracle_flip_trajectory(const uint64_t* words, int L, int skew, const int32_t* moves, int n_moves,
                           int32_t* E_after, uint64_t* final_words) {
  if (L < 1 || L > ORACLE_MAX_L || n_moves < 0) return ORC_ERR_ARG;
  int8_t s[ORACLE_MAX_L];
  int64_t C[ORACLE_MAX_L];
  unpack(words, L, s);
  int64_t E = energy_table(s, L, C);
  for (int t = 0; t < n_moves; t++) {
    int F[2];
    if (moves[t] < 1 || moves[t] > L) return ORC_ERR_ARG;
    int nF = flip_set(L, skew, moves[t], F);
    E += delta_linear(s, C, L, F, nF);
    apply_flip(s, C, L, F, nF);
    E_after[t] = (int32_t)E;
  }
  pack(s, L, final_words);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  The paper names no
 * generator; both implementations write this published one from its definition so that walk starts
 * and fingerprints agree.  Output i (0-based) of a generator whose state starts at `key`:
 *   z = key + (i+1) * 0x9E3779B97F4A7C15
 *   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;  z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  z ^ (z >> 31)
 * Streams are keyed by chaining: key(seed, purpose, a, b) = at(at(at(seed, purpose), a), b).
 * ---------------------------------------------------------------------------------------------- */
#define SM_GAMMA 0x9E3779B97F4A7C15ull
enum { PURPOSE_WALK = 1, PURPOSE_THRESH = 2, PURPOSE_ZOBRIST = 0x5A0B };

uint64_t oracle_sm64_at(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1) * SM_GAMMA;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t oracle_stream_key(uint64_t seed, uint64_t purpose, uint64_t a, uint64_t b) {
  return oracle_sm64_at(oracle_sm64_at(oracle_sm64_at(seed, purpose), a), b);
}

/* 64-bit Zobrist keys Z_L[i], i = 1..L (Algorithm 2's HASH_FLIP needs an O(1) neighbour hash). */
uint64_t oracle_zobrist(int L, int i) {
  return oracle_sm64_at(oracle_stream_key(0, PURPOSE_ZOBRIST, (uint64_t)L, 0), (uint64_t)(i - 1));
}

static void zobrist_table(int L, uint64_t* Z /* [L+1], Z[0] unused */) {
  for (int i = 1; i <= L; i++) Z[i] = oracle_zobrist(L, i);
}

/* fp(S) = XOR of Z_L[i] over the positions with s_i = -1. */
static uint64_t fingerprint(const int8_t* s, int L, const uint64_t* Z) {
  uint64_t h = 0;
  for (int i = 1; i <= L; i++)
    if (s[i - 1] == -1) h ^= Z[i];
  return h;
}

int oracle_fingerprint_batch(const uint64_t* words, int L, int64_t n, uint64_t* fp_out) {
  if (L < 1 || L > ORACLE_MAX_L || n < 0) return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  uint64_t Z[ORACLE_MAX_L + 1];
  int8_t s[ORACLE_MAX_L];
  zobrist_table(L, Z);
  for (int64_t q = 0; q < n; q++) {
    unpack(words + q * W, L, s);
    fp_out[q] = fingerprint(s, L, Z);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------
 * INIT_PARTITIONED_SEQUENCE (Algorithm 1, Eq. 3): s_1..s_p from the walk's prefix (restriction
 * class), free element number j (0-based) at position p+1+j is +1 iff bit j%64 of output j/64 of the
 * stream `key` is 1.  Skew walks draw positions p+1..k+1 and fill the last k by Eq. (2); unrestricted
 * walks draw positions p+1..L.
 * ---------------------------------------------------------------------------------------------- */
static void init_start(int8_t* s, int L, int skew, int p, const uint64_t* prefix, uint64_t key) {
  for (int i = 1; i <= p; i++) s[i - 1] = ((prefix[(i - 1) / 64] >> ((i - 1) % 64)) & 1u) ? 1 : -1;
  int last = skew ? (L - 1) / 2 + 1 : L;
  for (int i = p + 1; i <= last; i++) {
    int j = i - (p + 1);
    uint64_t r = oracle_sm64_at(key, (uint64_t)(j / 64));
    s[i - 1] = ((r >> (j % 64)) & 1u) ? 1 : -1;
  }
  if (skew) skew_fill(s, L);
}

int oracle_make_starts(int L, int skew, int p, const uint64_t* prefixes, int n_prefix, int prefix_words,
                       uint64_t seed, uint64_t purpose, int64_t first, int64_t n, uint64_t segment,
                       uint64_t* out_words) {
  if (L < 2 || L > ORACLE_MAX_L || n_prefix < 1 || p < 0 || p > 64 * prefix_words) return ORC_ERR_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  int8_t s[ORACLE_MAX_L];
  for (int64_t q = 0; q < n; q++) {
    int64_t id = first + q;
    const uint64_t* pre = prefixes + (id % n_prefix) * prefix_words;
    init_start(s, L, skew, p, pre, oracle_stream_key(seed, purpose, (uint64_t)id, segment));
    pack(s, L, out_words + q * W);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Bloom filter of visited states (Algorithm 1; Bloom 1970).  m = 2^log2 bits, K probes; probe j
 * sets bit (lo32(fp) + j * (hi32(fp) | 1)) mod m, in 32-bit unsigned arithmetic (Kirsch-Mitzenmacher
 * double hashing).
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  uint8_t* bits; /* one byte per bit: plain and obviously correct */
  uint32_t mask;
  int K;
} bloom_t;

static uint32_t bloom_probe(uint64_t fp, int j, uint32_t mask) {
  uint32_t lo = (uint32_t)fp, hi = (uint32_t)(fp >> 32);
  return (lo + (uint32_t)j * (hi | 1u)) & mask;
}

static void bloom_insert(bloom_t* b, uint64_t fp) {
  for (int j = 0; j < b->K; j++) b->bits[bloom_probe(fp, j, b->mask)] = 1;
}

static int bloom_contains(const bloom_t* b, uint64_t fp) {
  for (int j = 0; j < b->K; j++)
    if (!b->bits[bloom_probe(fp, j, b->mask)]) return 0;
  return 1;
}

/* ------------------------------------------------------------------------------------------------
 * Algorithm 1, one walk, under the readings stated in the design notes:
 *  - the walk restarts (fresh free elements from stream (seed, WALK, walk, segment), same prefix,
 *    Bloom filter cleared) after T_i accepted flips or when BEST_NEIGHBOUR finds no unexplored
 *    neighbour, until flip_budget accepted flips have been made in total;
 *  - BEST_NEIGHBOUR returns the free position m minimising (Delta E_m, m) among neighbours whose
 *    fingerprint is not in the Bloom filter (it may be uphill);
 *  - the sieve keeps, per walk, the R smallest distinct (E, fp) states with E <= E_thr reached by a
 *    flip (Algorithm 1 tests the energy only after a move).
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t E;
  uint32_t walk;
  uint32_t step;
  uint32_t pad;
  uint64_t fp;
  uint64_t seq[ORACLE_MAX_W];
} oracle_candidate; /* 96 bytes, the interface layout of a candidate record */

static int key_less(int32_t Ea, uint64_t fa, int32_t Eb, uint64_t fb) {
  return Ea < Eb || (Ea == Eb && fa < fb);
}

typedef struct {
  int L, skew, p, prefix_words, n_prefix, T_i, R, bloom_log2, bloom_k;
  const uint64_t* prefixes;
  int64_t walk_begin, n_walks, flip_budget;
  uint64_t seed;
  int32_t E_thr;
  const float* logits; /* nullable: [n_walks][n_chunks][L] proposal logits */
  int n_chunks, chunk;
  float lambda;
  oracle_candidate* out;
  int64_t* walk_stats;
  int n_threads, thread_id;
  int status;
} walk_job_t;

static void candidate_offer(oracle_candidate* slots, int R, int32_t E, uint64_t fp, const int8_t* s, int L,
                            uint32_t walk, uint32_t step) {
  /* distinct by fingerprint */
  for (int r = 0; r < R; r++)
    if (slots[r].E != INT32_MAX && slots[r].fp == fp) return;
  /* worst slot = largest (E, fp); empty slots (E = INT32_MAX, fp = ~0) are the largest */
  int worst = 0;
  for (int r = 1; r < R; r++)
    if (key_less(slots[worst].E, slots[worst].fp, slots[r].E, slots[r].fp)) worst = r;
  if (!key_less(E, fp, slots[worst].E, slots[worst].fp)) return;
  slots[worst].E = E;
  slots[worst].fp = fp;
  slots[worst].walk = walk;
  slots[worst].step = step;
  slots[worst].pad = 0;
  pack(s, L, slots[worst].seq);
  for (int j = (L + 63) / 64; j < ORACLE_MAX_W; j++) slots[worst].seq[j] = 0;
}

static int cmp_candidate(const void* a, const void* b) {
  const oracle_candidate* x = (const oracle_candidate*)a;
  const oracle_candidate* y = (const oracle_candidate*)b;
  if (key_less(x->E, x->fp, y->E, y->fp)) return -1;
  if (key_less(y->E, y->fp, x->E, x->fp)) return 1;
  return 0;
}

static void run_one_walk(walk_job_t* job, int64_t w, bloom_t* bloom, const uint64_t* Z) {
  int L = job->L, skew = job->skew, p = job->p, R = job->R;
  int last = skew ? (L - 1) / 2 + 1 : L;
  int8_t s[ORACLE_MAX_L];
  int64_t C[ORACLE_MAX_L];
  int64_t dE[ORACLE_MAX_L + 1];
  int8_t in_bloom[ORACLE_MAX_L + 1];
  double key[ORACLE_MAX_L + 1];
  oracle_candidate* slots = job->out + (w - job->walk_begin) * R;
  for (int r = 0; r < R; r++) {
    memset(&slots[r], 0, sizeof(oracle_candidate));
    slots[r].E = INT32_MAX;
    slots[r].fp = ~(uint64_t)0;
  }
  int64_t flips = 0, segments = 0, bloom_skips = 0, dead_ends = 0, best_E = INT32_MAX;
  const uint64_t* prefix = job->prefixes + (w % job->n_prefix) * job->prefix_words;
  uint32_t nbits = bloom->mask + 1u;
  while (flips < job->flip_budget) {
    memset(bloom->bits, 0, nbits);
    init_start(s, L, skew, p, prefix, oracle_stream_key(job->seed, PURPOSE_WALK, (uint64_t)w, (uint64_t)segments));
    segments++;
    uint64_t fp = fingerprint(s, L, Z);
    bloom_insert(bloom, fp);
    int64_t E = energy_table(s, L, C);
    int it = 0;
    while (it < job->T_i && flips < job->flip_budget) {
      it++;
      /* BEST_NEIGHBOUR */
      for (int m = p + 1; m <= last; m++) {
        int F[2];
        int nF = flip_set(L, skew, m, F);
        dE[m] = delta_linear(s, C, L, F, nF);
      }
      /* choice key: Delta E, or with a proposal the FP32 score fmaf(-lambda, logit, Delta E) (a
         non-finite logit counts as 0); ties go to the lower position */
      const float* lg = NULL;
      if (job->logits) {
        int64_t ch = flips / job->chunk;
        if (ch >= job->n_chunks) ch = job->n_chunks - 1;
        lg = job->logits + ((w - job->walk_begin) * job->n_chunks + ch) * (int64_t)L;
      }
      for (int m = p + 1; m <= last; m++) {
        if (lg) {
          float l = lg[m - 1];
          if (!isfinite(l)) l = 0.0f;
          key[m] = (double)(fmaf(-job->lambda, l, (float)dE[m]) + 0.0f);
        } else {
          key[m] = (double)dE[m];
        }
      }
      int best = -1;
      int64_t best_d = 0;
      double best_k = 0.0;
      for (int m = p + 1; m <= last; m++) {
        int F[2];
        int nF = flip_set(L, skew, m, F);
        uint64_t nfp = fp;
        for (int a = 0; a < nF; a++) nfp ^= Z[F[a]];
        in_bloom[m] = (int8_t)bloom_contains(bloom, nfp);
        if (in_bloom[m]) continue;
        if (best == -1 || key[m] < best_k) { best = m; best_d = dE[m]; best_k = key[m]; } /* ties keep the lower m */
      }
      /* statistics: explored neighbours that ranked ahead of the chosen one */
      for (int m = p + 1; m <= last; m++)
        if (in_bloom[m] && (best == -1 || key[m] < best_k || (key[m] == best_k && m < best))) bloom_skips++;
      if (best == -1) { dead_ends++; break; }
      int F[2];
      int nF = flip_set(L, skew, best, F);
      apply_flip(s, C, L, F, nF);
      for (int a = 0; a < nF; a++) fp ^= Z[F[a]];
      bloom_insert(bloom, fp);
      E += best_d;
      flips++;
      if (E < best_E) best_E = E;
      if (E <= job->E_thr) candidate_offer(slots, R, (int32_t)E, fp, s, L, (uint32_t)w, (uint32_t)flips);
    }
  }
  qsort(slots, (size_t)R, sizeof(oracle_candidate), cmp_candidate);
  if (job->walk_stats) {
    int64_t* st = job->walk_stats + (w - job->walk_begin) * 5;
    st[0] = flips; st[1] = segments; st[2] = bloom_skips; st[3] = dead_ends; st[4] = best_E;
  }
}

static void* walk_thread(void* arg) {
  walk_job_t* job = (walk_job_t*)arg;
  uint64_t Z[ORACLE_MAX_L + 1];
  zobrist_table(job->L, Z);
  bloom_t bloom;
  bloom.mask = (1u << job->bloom_log2) - 1u;
  bloom.K = job->bloom_k;
  bloom.bits = (uint8_t*)malloc((size_t)bloom.mask + 1u);
  if (!bloom.bits) { job->status = ORC_ERR_NOMEM; return NULL; }
  for (int64_t w = job->walk_begin + job->thread_id; w < job->walk_begin + job->n_walks; w += job->n_threads)
    run_one_walk(job, w, &bloom, Z);
  free(bloom.bits);
  job->status = ORC_OK;
  return NULL;
}

/* Algorithm 1 walks with an optional proposal bias (see oracle_walk_search below). */
int oracle_walk_search_biased(int L, int skew, int p, const uint64_t* prefixes, int n_prefix, int prefix_words,
                              int64_t walk_begin, int64_t n_walks, int64_t flip_budget, int T_i, uint64_t seed, int R,
                              int bloom_log2, int bloom_k, int32_t E_thr, const float* logits, int n_chunks, int chunk,
                              float lambda, oracle_candidate* out, int64_t* walk_stats, int n_threads) {
  if (L < 2 || L > ORACLE_MAX_L || n_prefix < 1 || p < 0 || p > 64 * prefix_words || R < 1 || T_i < 1)
    return ORC_ERR_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return ORC_ERR_ARG;
  if (!skew && p >= L) return ORC_ERR_ARG;
  if (bloom_log2 < 5 || bloom_log2 > 31 || bloom_k < 1 || n_threads < 1) return ORC_ERR_ARG;
  if (logits && (n_chunks < 1 || chunk < 1)) return ORC_ERR_ARG;
  walk_job_t* jobs = (walk_job_t*)calloc((size_t)n_threads, sizeof(walk_job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return ORC_ERR_NOMEM; }
  for (int t = 0; t < n_threads; t++) {
    walk_job_t* j = &jobs[t];
    j->L = L; j->skew = skew; j->p = p; j->prefix_words = prefix_words; j->n_prefix = n_prefix;
    j->T_i = T_i; j->R = R; j->bloom_log2 = bloom_log2; j->bloom_k = bloom_k; j->prefixes = prefixes;
    j->walk_begin = walk_begin; j->n_walks = n_walks; j->flip_budget = flip_budget; j->seed = seed;
    j->E_thr = E_thr; j->out = out; j->logits = logits; j->n_chunks = n_chunks; j->chunk = chunk;
    j->lambda = lambda; j->walk_stats = walk_stats;
    j->n_threads = n_threads; j->thread_id = t; j->status = ORC_OK;
  }
  int status = ORC_OK;
  if (n_threads == 1) {
    walk_thread(&jobs[0]);
  } else {
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, walk_thread, &jobs[t]);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
  }
  for (int t = 0; t < n_threads; t++)
    if (jobs[t].status != ORC_OK) status = jobs[t].status;
  free(jobs);
  free(th);
  return status;
}

/* Runs walks walk_begin .. walk_begin+n_walks-1 (global walk ids; walk w uses prefix w mod n_prefix).
 * out: [n_walks][R] candidates sorted by (E, fp), empty slots E = INT32_MAX, fp = ~0.
 * walk_stats (nullable): [n_walks][5] = flips, segments, bloom_skips, dead_ends, best_E, where
 * bloom_skips counts Bloom-positive neighbours whose key ranked ahead of the chosen move and best_E is
 * the lowest energy reached by a flip (INT32_MAX if none).  The _biased form takes the proposal logits
 * of each walk's chunks (a chunk is `chunk` accepted flips). */
int oracle_walk_search(int L, int skew, int p, const uint64_t* prefixes, int n_prefix, int prefix_words,
                       int64_t walk_begin, int64_t n_walks, int64_t flip_budget, int T_i, uint64_t seed, int R,
                       int bloom_log2, int bloom_k, int32_t E_thr, oracle_candidate* out, int64_t* walk_stats,
                       int n_threads) {
  return oracle_walk_search_biased(L, skew, p, prefixes, n_prefix, prefix_words, walk_begin, n_walks, flip_budget, T_i,
                                   seed, R, bloom_log2, bloom_k, E_thr, NULL, 0, 0, 0.0f, out, walk_stats, n_threads);
}

/* ------------------------------------------------------------------------------------------------
 * Sieve threshold E_l (Algorithm 1): n_samples starts drawn exactly like walk starts (sample i uses
 * prefix i mod n_prefix and stream (seed, THRESH, i, 0)); E_thr is the sampled energy of 0-based
 * rank `rank` in ascending order (nearest rank).
 * ---------------------------------------------------------------------------------------------- */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

int oracle_threshold(int L, int skew, int p, const uint64_t* prefixes, int n_prefix, int prefix_words,
                     uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr, int32_t* E_samples) {
  if (n_samples < 1 || rank < 0 || rank >= n_samples) return ORC_ERR_ARG;
  if (L < 2 || L > ORACLE_MAX_L || n_prefix < 1 || p < 0 || p > 64 * prefix_words) return ORC_ERR_ARG;
  if (skew && (L % 2 == 0 || p > (L - 1) / 2)) return ORC_ERR_ARG;
  int32_t* Es = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_samples);
  if (!Es) return ORC_ERR_NOMEM;
  int8_t s[ORACLE_MAX_L];
  for (int64_t i = 0; i < n_samples; i++) {
    const uint64_t* pre = prefixes + (i % n_prefix) * prefix_words;
    init_start(s, L, skew, p, pre, oracle_stream_key(seed, PURPOSE_THRESH, (uint64_t)i, 0));
    Es[i] = (int32_t)energy(s, L);
  }
  if (E_samples) memcpy(E_samples, Es, sizeof(int32_t) * (size_t)n_samples);
  qsort(Es, (size_t)n_samples, sizeof(int32_t), cmp_i32);
  *E_thr = Es[rank];
  free(Es);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Exhaustive skew-symmetric search (Eq. 2 and 3): every assignment of the k-p+1 free elements behind
 * a fixed prefix.  Free bit j of the assignment integer is 1 iff s_{p+1+j} = -1.  Reports the minimum
 * E, how many assignments reach it, and the smallest assignment integer among them.
 * ---------------------------------------------------------------------------------------------- */
int oracle_skew_exhaustive(int L, int p, const uint64_t* prefix, int32_t* min_E, uint64_t* count,
                           uint64_t* argmin_free, uint64_t* argmin_words) {
  if (L < 3 || L % 2 == 0 || L > 127 || p < 0 || p > (L - 1) / 2) return ORC_ERR_ARG;
  int k = (L - 1) / 2;
  int nfree = k - p + 1;
  if (nfree > 40) return ORC_ERR_ARG;
  int8_t s[ORACLE_MAX_L];
  for (int i = 1; i <= p; i++) s[i - 1] = ((prefix[(i - 1) / 64] >> ((i - 1) % 64)) & 1u) ? 1 : -1;
  int64_t best = INT64_MAX;
  uint64_t cnt = 0, arg = 0;
  for (uint64_t a = 0; a < ((uint64_t)1 << nfree); a++) {
    for (int j = 0; j < nfree; j++) s[p + j] = ((a >> j) & 1u) ? -1 : 1;
    skew_fill(s, L);
    int64_t E = energy(s, L);
    if (E < best) { best = E; cnt = 1; arg = a; }
    else if (E == best) cnt++;
  }
  *min_E = (int32_t)best;
  *count = cnt;
  *argmin_free = arg;
  for (int j = 0; j < nfree; j++) s[p + j] = ((arg >> j) & 1u) ? -1 : 1;
  skew_fill(s, L);
  pack(s, L, argmin_words);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Algorithm 2 in batch-synchronous form (readings in the design notes):
 *  - keys are (E, fp), compared lexicographically; the open set P holds at most `cap` entries;
 *  - a round pops the b = min(B, |P|, budget left) smallest keys; for every popped node (in key order)
 *    and every position i = 1..L, the neighbour's fingerprint fp ^ Z[i] is skipped when it is in H,
 *    otherwise the neighbour survives with E' = E + Delta E_i (linear-time evaluation);
 *  - survivors are sorted by (E', fp', pop order, i) and equal (E', fp') are kept once;
 *  - P becomes the cap smallest keys of P ∪ survivors; H receives exactly the admitted survivors;
 *  - the best improves on strict E' < E_best, to the smallest survivor key; u counts pops since the
 *    last improvement (reset to 0 by an improving round);
 *  - stop when max_expansions pops are done, P is empty, or T_u > 0 and u >= T_u.
 * With B = 1 and a cap that is never reached this is Algorithm 2 line by line, with H membership
 * as the skip test and rotations off (T_r = 0).
 * stats[8] = expansions, rounds, survivors, admitted, evicted, h_size, improvements, stop_reason
 * (1 budget, 2 empty, 3 T_u).
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t E;
  uint64_t fp;
  int64_t parent; /* survivors: pop order of the parent node; entries of P: -1 */
  int32_t pos;    /* survivors: flipped position */
  int8_t* s;      /* entries of P: owned +-1 array */
} pq_entry;

static int cmp_pq(const void* a, const void* b) {
  const pq_entry* x = (const pq_entry*)a;
  const pq_entry* y = (const pq_entry*)b;
  if (x->E != y->E) return x->E < y->E ? -1 : 1;
  if (x->fp != y->fp) return x->fp < y->fp ? -1 : 1;
  if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
  if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
  return 0;
}

typedef struct {
  uint64_t* keys;
  uint8_t* used;
  uint64_t mask;
  int64_t size;
} fpset_t;

static uint64_t fpset_slot(uint64_t fp, uint64_t mask) {
  uint64_t z = fp * 0x9E3779B97F4A7C15ull;
  return (z ^ (z >> 29)) & mask;
}

static int fpset_init(fpset_t* h, int log2) {
  h->mask = ((uint64_t)1 << log2) - 1;
  h->size = 0;
  h->keys = (uint64_t*)calloc((size_t)h->mask + 1, sizeof(uint64_t));
  h->used = (uint8_t*)calloc((size_t)h->mask + 1, 1);
  return (h->keys && h->used) ? ORC_OK : ORC_ERR_NOMEM;
}

static void fpset_free(fpset_t* h) { free(h->keys); free(h->used); }

static int fpset_contains(const fpset_t* h, uint64_t fp) {
  for (uint64_t i = fpset_slot(fp, h->mask);; i = (i + 1) & h->mask) {
    if (!h->used[i]) return 0;
    if (h->keys[i] == fp) return 1;
  }
}

static int fpset_insert(fpset_t* h, uint64_t fp);

static int fpset_grow(fpset_t* h) {
  fpset_t g;
  int log2 = 0;
  while (((uint64_t)1 << log2) <= h->mask) log2++;
  if (fpset_init(&g, log2 + 1) != ORC_OK) { fpset_free(&g); return ORC_ERR_NOMEM; }
  for (uint64_t i = 0; i <= h->mask; i++)
    if (h->used[i]) fpset_insert(&g, h->keys[i]);
  fpset_free(h);
  *h = g;
  return ORC_OK;
}

static int fpset_insert(fpset_t* h, uint64_t fp) {
  if ((uint64_t)(h->size + 1) * 2 > h->mask + 1) {
    int st = fpset_grow(h);
    if (st != ORC_OK) return st;
  }
  for (uint64_t i = fpset_slot(fp, h->mask);; i = (i + 1) & h->mask) {
    if (!h->used[i]) { h->used[i] = 1; h->keys[i] = fp; h->size++; return ORC_OK; }
    if (h->keys[i] == fp) return ORC_OK;
  }
}

/* MAKE_ROTATIONS (Section 3, Algorithm 2): rotation code c = 0 .. 2 T_r - 1 of a sequence; c < T_r moves
   the first c + 1 elements to the end (left rotation), c >= T_r moves the last c - T_r + 1 elements to the
   start (right rotation).  out[i] = s[(i + r) mod L] for the left shift r. */
static void rotate_seq(const int8_t* s, int L, int T_r, int c, int8_t* out) {
  int r = c < T_r ? c + 1 : L - ((c - T_r + 1) % L);
  r %= L;
  for (int i = 0; i < L; i++) out[i] = s[(i + r) % L];
}

/* child of pivot s: position pos (1..L) flipped, or rotation pos - L - 1 */
static void child_seq(const int8_t* s, int L, int T_r, int pos, int8_t* out) {
  if (pos <= L) {
    memcpy(out, s, (size_t)L);
    out[pos - 1] = (int8_t)-out[pos - 1];
  } else {
    rotate_seq(s, L, T_r, pos - L - 1, out);
  }
}

int oracle_pq_refine(int L, const uint64_t* seeds, int n_seeds, int64_t cap, int B, int64_t max_expansions,
                     int64_t T_u, int T_r, uint64_t* best_words, int32_t* best_E_out, uint64_t* best_fp_out,
                     int64_t* stats) {
  if (L < 2 || L > ORACLE_MAX_L || n_seeds < 1 || cap < 1 || B < 1 || max_expansions < 0 || T_r < 0 || 2 * T_r >= L)
    return ORC_ERR_ARG;
  int W = (L + 63) / 64;
  uint64_t Z[ORACLE_MAX_L + 1];
  zobrist_table(L, Z);
  int status = ORC_OK;
  fpset_t H;
  if (fpset_init(&H, 12) != ORC_OK) { fpset_free(&H); return ORC_ERR_NOMEM; }
  for (int t = 0; t < 8; t++) stats[t] = 0;

  /* seeds: dedup by (E, fp), keep the cap smallest */
  pq_entry* P = (pq_entry*)calloc((size_t)n_seeds, sizeof(pq_entry));
  if (!P) { fpset_free(&H); return ORC_ERR_NOMEM; }
  for (int q = 0; q < n_seeds; q++) {
    P[q].s = (int8_t*)malloc((size_t)L);
    unpack(seeds + (int64_t)q * W, L, P[q].s);
    P[q].E = (int32_t)energy(P[q].s, L);
    P[q].fp = fingerprint(P[q].s, L, Z);
    P[q].parent = q;
    P[q].pos = 0;
  }
  qsort(P, (size_t)n_seeds, sizeof(pq_entry), cmp_pq);
  int64_t nP = 0;
  for (int q = 0; q < n_seeds; q++) {
    if (nP > 0 && P[nP - 1].E == P[q].E && P[nP - 1].fp == P[q].fp) { free(P[q].s); continue; }
    P[nP++] = P[q];
  }
  while (nP > cap) free(P[--nP].s);
  for (int64_t q = 0; q < nP; q++) { P[q].parent = -1; fpset_insert(&H, P[q].fp); }

  int32_t best_E = P[0].E;
  uint64_t best_fp = P[0].fp;
  int8_t best_s[ORACLE_MAX_L];
  memcpy(best_s, P[0].s, (size_t)L);

  int64_t expansions = 0, u = 0;
  int64_t C[ORACLE_MAX_L];
  int stop = 0;
  while (!stop) {
    if (expansions >= max_expansions) { stop = 1; break; }
    if (nP == 0) { stop = 2; break; }
    if (T_u > 0 && u >= T_u) { stop = 3; break; }
    int64_t b = B;
    if (b > nP) b = nP;
    if (b > max_expansions - expansions) b = max_expansions - expansions;
    /* expand the b popped nodes */
    int64_t nS = 0, capS = b * (L + 2 * T_r);
    pq_entry* S = (pq_entry*)malloc(sizeof(pq_entry) * (size_t)(capS > 0 ? capS : 1));
    if (!S) { status = ORC_ERR_NOMEM; break; }
    for (int64_t q = 0; q < b; q++) {
      energy_table(P[q].s, L, C);
      for (int i = 1; i <= L; i++) {
        uint64_t nfp = P[q].fp ^ Z[i];
        if (fpset_contains(&H, nfp)) continue;
        int F[1] = {i};
        S[nS].E = (int32_t)(P[q].E + delta_linear(P[q].s, C, L, F, 1));
        S[nS].fp = nfp;
        S[nS].parent = q;
        S[nS].pos = i;
        S[nS].s = NULL;
        nS++;
      }
      /* MAKE_ROTATIONS of the pivot: energy and fingerprint from scratch, skipped when visited */
      for (int c = 0; c < 2 * T_r; c++) {
        int8_t rs[ORACLE_MAX_L];
        rotate_seq(P[q].s, L, T_r, c, rs);
        uint64_t rfp = fingerprint(rs, L, Z);
        if (fpset_contains(&H, rfp)) continue;
        S[nS].E = (int32_t)energy(rs, L);
        S[nS].fp = rfp;
        S[nS].parent = q;
        S[nS].pos = L + 1 + c;
        S[nS].s = NULL;
        nS++;
      }
    }
    qsort(S, (size_t)nS, sizeof(pq_entry), cmp_pq);
    int64_t nU = 0;
    for (int64_t t = 0; t < nS; t++) {
      if (nU > 0 && S[nU - 1].E == S[t].E && S[nU - 1].fp == S[t].fp) continue;
      S[nU++] = S[t];
    }
    stats[2] += nU;
    /* best */
    if (nU > 0 && S[0].E < best_E) {
      best_E = S[0].E;
      best_fp = S[0].fp;
      child_seq(P[S[0].parent].s, L, T_r, S[0].pos, best_s);
      stats[6]++;
      u = 0;
    } else {
      u += b;
    }
    /* merge the rest of P (sorted) with the survivors (sorted); keep the cap smallest */
    int64_t rest = nP - b;
    int64_t total = rest + nU;
    int64_t keep = total < cap ? total : cap;
    pq_entry* NP = (pq_entry*)malloc(sizeof(pq_entry) * (size_t)(keep > 0 ? keep : 1));
    if (!NP) { free(S); status = ORC_ERR_NOMEM; break; }
    int64_t ia = b, ib = 0, n_new = 0;
    while (n_new < keep) {
      int take_a;
      if (ia >= nP) take_a = 0;
      else if (ib >= nU) take_a = 1;
      else take_a = key_less(P[ia].E, P[ia].fp, S[ib].E, S[ib].fp);
      if (take_a) {
        NP[n_new++] = P[ia++];
      } else {
        pq_entry e = S[ib++];
        int8_t* ns = (int8_t*)malloc((size_t)L);
        child_seq(P[e.parent].s, L, T_r, e.pos, ns);
        e.s = ns;
        e.parent = -1;
        e.pos = 0;
        if (fpset_insert(&H, e.fp) != ORC_OK) status = ORC_ERR_NOMEM;
        stats[3]++;
        NP[n_new++] = e;
      }
    }
    stats[4] += (nP - ia); /* old entries that did not fit */
    for (int64_t q = 0; q < b; q++) free(P[q].s);
    for (int64_t q = ia; q < nP; q++) free(P[q].s);
    free(P);
    free(S);
    P = NP;
    nP = n_new;
    expansions += b;
    stats[1]++;
    if (status != ORC_OK) break;
  }
  stats[0] = expansions;
  stats[5] = H.size;
  stats[7] = stop;
  for (int64_t q = 0; q < nP; q++) free(P[q].s);
  free(P);
  fpset_free(&H);
  pack(best_s, L, best_words);
  *best_E_out = best_E;
  *best_fp_out = best_fp;
  return status;
}

/* ---------------------------------------------------------------------------------------------
 * End-element sequence operators (Section 3, the loop of Fig. 4 back into step 2): for every input
 * sequence S of length L the four sequences of length L+1 (S then +1, S then -1, +1 then S, -1 then S)
 * and the two of length L-1 (S without its last element, S without its first), with their energies by
 * the Section 1 definition.  Parity pinned by restating the operators with list slicing in the tests.
 * --------------------------------------------------------------------------------------------- */
int oracle_sequence_operators(const uint64_t* words, int L, int64_t n, uint64_t* grow, int32_t* E_grow,
                              uint64_t* shrink, int32_t* E_shrink) {
  if (L < 3 || L + 1 > ORACLE_MAX_L || n < 0) return ORC_ERR_ARG;
  const int W = (L + 63) / 64, Wg = (L + 64) / 64, Ws = (L + 62) / 64;
  int8_t s[ORACLE_MAX_L], t[ORACLE_MAX_L + 1];
  for (int64_t q = 0; q < n; q++) {
    unpack(words + q * W, L, s);
    for (int v = 0; v < 4; v++) {
      const int8_t x = (v & 1) ? -1 : 1;
      if (v < 2) {
        memcpy(t, s, (size_t)L);
        t[L] = x;
      } else {
        t[0] = x;
        memcpy(t + 1, s, (size_t)L);
      }
      pack(t, L + 1, grow + (q * 4 + v) * Wg);
      E_grow[q * 4 + v] = (int32_t)energy(t, L + 1);
    }
    for (int v = 0; v < 2; v++) {
      const int8_t* src = v == 0 ? s : s + 1;
      pack(src, L - 1, shrink + (q * 2 + v) * Ws);
      E_shrink[q * 2 + v] = (int32_t)energy(src, L - 1);
    }
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Legendre-sequence seeds (Section 4, Table 2): s_i = chi((i + off) mod p) for i = 0..L-1, the rotation of
 * the Legendre sequence of prime length p by off with its first L - p elements appended; chi(j) = +1 for a
 * non-zero square mod p, -1 otherwise (chi(0) = -1).  Squares found by listing k^2 mod p.  Pinned by the
 * construction column of Table 2 and by the two-valued periodic autocorrelation of Legendre sequences.
 * --------------------------------------------------------------------------------------------- */
int oracle_legendre_construct(int L, const int32_t* params, int64_t n, uint64_t* words, int32_t* E_out) {
  if (L < 3 || L > ORACLE_MAX_L || n < 0) return ORC_ERR_ARG;
  const int W = (L + 63) / 64;
  int8_t s[ORACLE_MAX_L];
  uint8_t square[ORACLE_MAX_L];
  for (int64_t q = 0; q < n; q++) {
    const int p = params[2 * q], off = params[2 * q + 1];
    if (p < 2 || p > L || off < 0 || off >= p) return ORC_ERR_ARG;
    memset(square, 0, (size_t)p);
    for (int k = 1; k < p; k++) square[(k * k) % p] = 1;
    for (int i = 0; i < L; i++) {
      const int j = (i + off) % p;
      s[i] = (j != 0 && square[j]) ? 1 : -1;
    }
    pack(s, L, words + q * W);
    E_out[q] = (int32_t)energy(s, L);
  }
  return ORC_OK;
}
