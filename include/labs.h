/*
 * labs.h -- C ABI of liblabs.so, a GB300 (sm_103a) implementation of the hot path of the dual-step
 * search for low-autocorrelation binary sequences of Psenicnik, Mlinaric, Brest and Boskovic,
 * "Dual-Step Optimization for Binary Sequences with High Merit Factors" (arXiv 2409.07222).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sequences S = (s_1..s_L), s_i in {+1,-1}, 2 <= L <= 576, are bit-packed into W = ceil(L/64)
 *    uint64 words: bit (i-1) % 64 of word (i-1) / 64 holds s_i, bit value 1 meaning +1 (the paper's
 *    hexadecimal coding, Section 4, where a binary 0 stands for -1).  Bits above L-1 must be zero.
 *  - Unless stated otherwise, pointers are DEVICE pointers owned by the caller; the library never
 *    frees caller memory.  Internal workspace lives in the opaque context.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *    stream-ordered and asynchronous: argument errors are returned immediately, device-side errors
 *    (capacity, timeouts) are reported through the stats/status outputs once the stream has reached
 *    them.  A context must not be used by two host threads at once.
 *  - Every call returns LABS_OK or one of the LABS_ERR_* codes below.
 *  - Energies are exact integers: E < L^3/3 < 2^31 for L <= 576.
 */
#ifndef LABS_H_
#define LABS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LABS_OK 0
#define LABS_ERR_INVALID_ARG 1 /* bad size, length, mode, alignment or layout */
#define LABS_ERR_CAPACITY 2    /* a bounded device structure (heap, hash table, buffer) overflowed */
#define LABS_ERR_TIMEOUT 3     /* a capped device-side wait gave up */
#define LABS_ERR_CUDA 4        /* a CUDA runtime call or launch failed */
#define LABS_ERR_NOMEM 5       /* workspace allocation failed */

#define LABS_MAX_L 576
#define LABS_MAX_W 9
#define LABS_AUTO_THRESHOLD ((int32_t)0x80000000) /* E_thr: sample it (Algorithm 1's E_l) */

typedef struct labs_ctx labs_ctx;

/* Creates a context bound to CUDA device `device`.  *out receives the handle. */
int labs_ctx_create(labs_ctx** out, int device);
/* Releases the context's workspace.  Synchronises the device first. */
void labs_ctx_destroy(labs_ctx* ctx);
/* Static string naming a status code. */
const char* labs_status_string(int status);
/* Version of this ABI (bumped on any incompatible change). */
int labs_abi_version(void);

/*
 * labs_energy_batch -- Section 1 definitions: C_k(S) = sum_{i=1}^{L-k} s_i s_{i+k} and
 * E(S) = sum_{k=1}^{L-1} C_k(S)^2, for n sequences at once (Algorithm 1's and 2's ENERGY).
 *   seqs   [n][W] uint64, device, 8-byte aligned.
 *   E_out  [n] int32, device.
 *   C_out  nullable; [n][L-1] int32, device: C_out[q*(L-1) + k-1] = C_k of sequence q.
 * Errors: LABS_ERR_INVALID_ARG if L outside [2, 576], n < 0 or a pointer is NULL/misaligned.
 */
int labs_energy_batch(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, int32_t* E_out, int32_t* C_out,
                      void* stream);

/*
 * labs_flip_deltas -- the single-flip neighbourhood scan of BEST_NEIGHBOUR (Algorithm 1, Section 3)
 * and of Algorithm 2's loop: Delta E of every neighbour, exactly.
 *   skew = 0: unrestricted neighbourhood (SEQUENCE_FLIP): dE[q][i-1] = E(S with s_i negated) - E(S)
 *             for i = p+1..L.
 *   skew = 1: skew-symmetric neighbourhood (SEQUENCE_FLIP_SKEW, Eq. 2-3; L odd, L = 2k+1, inputs
 *             must be skew-symmetric): for every free position m in [p+1, k+1] the neighbour negates
 *             s_m and its mirror s_{L+1-m} (the centre k+1 alone); dE[q][m-1] holds its Delta E.
 *   Entries outside the free range are INT32_MAX.  dE is [n][L] int32, device.
 *   C      nullable; [n][L-1] int32 correlation tables as written by labs_energy_batch.  When given,
 *          the kernel uses them instead of rebuilding them (results are identical when they match).
 * Errors: LABS_ERR_INVALID_ARG for L outside [2, 576], odd/even mismatch with `skew`, p out of range.
 */
int labs_flip_deltas(labs_ctx* ctx, const uint64_t* seqs, const int32_t* C, int L, int64_t n, int skew, int p,
                     int32_t* dE_out, void* stream);

/* One candidate record of the sieve (Algorithm 1's E < E_l test).  96 bytes. */
typedef struct {
  int32_t E;     /* energy of seq */
  uint32_t walk; /* global walk id that reached it */
  uint32_t step; /* that walk's accepted-flip count when it was reached (1-based) */
  uint32_t pad;
  uint64_t fp; /* 64-bit Zobrist fingerprint of seq */
  uint64_t seq[LABS_MAX_W];
} labs_candidate;

/*
 * Walk configuration (Algorithm 1).  Readings where the paper gives no value:
 *  - a walk restarts (fresh free elements, same prefix, Bloom filter cleared) after T_i accepted
 *    flips or when no unexplored neighbour is left; flip_budget counts accepted flips over all of a
 *    walk's segments;
 *  - BEST_NEIGHBOUR picks the smallest (Delta E, m) whose neighbour fingerprint is not in the Bloom
 *    filter (2^bloom_log2 bits, bloom_k probes, double hashing of the fingerprint);
 *  - the sieve keeps per walk the R smallest distinct (E, fp) states with E <= E_thr reached by a flip.
 * Walk w uses prefix w mod n_prefix and draws its free elements from the counter-based SplitMix64
 * stream (seed, walk=1, w, segment).
 */
typedef struct {
  int32_t L;            /* 2..576 */
  int32_t skew;         /* 1: skew-symmetric walk, L odd (Algorithm 1); 0: unrestricted walk */
  int32_t p;            /* prefix length (restriction class, Eq. 3); <= k (skew) or < L */
  int32_t T_i;          /* segment length; <= 0 means 8(L+1)/2 = 4(L+1) */
  int64_t n_walks;      /* walks; walk ids are walk_begin .. walk_begin+n_walks-1 */
  int64_t walk_begin;   /* first global walk id (lets a caller shard walks) */
  int64_t flip_budget;  /* accepted flips per walk */
  uint64_t seed;        /* stream seed */
  int32_t R;            /* candidates kept per walk, 1..32 */
  int32_t bloom_log2;   /* Bloom filter bits = 2^bloom_log2, 5..15 */
  int32_t bloom_k;      /* Bloom probes, 1..8 */
  int32_t E_thr;        /* sieve bound (E <= E_thr passes) or LABS_AUTO_THRESHOLD */
  int64_t n_thresh_samples; /* auto threshold: starts sampled (stream (seed, 2, i, 0)), e.g. 10^6 */
  int64_t thresh_rank;      /* auto threshold: 0-based rank of E_thr among the samples, e.g. 999 */
  int32_t E_target;     /* record each walk's first flip reaching E <= E_target; INT32_MIN = off */
  int32_t tile_m;       /* neighbours per tile (8, 12 or 16); 0 = chosen by the library */
  int32_t warps_per_cta;/* warps per CTA: 1..8 with 32 lanes per walk, 1..12 with 16; 0 = chosen by the library */
  int32_t lanes_per_walk; /* 32: one walk per warp; 16: two walks per warp (R <= 16); 0 = chosen by the library */
  const int32_t* E_thr_dev; /* nullable device int32: when set, the sieve bound is read from it (for
                               instance written by labs_sample_threshold on the same stream) and
                               E_thr is ignored */
} labs_walk_cfg;

/* Aggregates over all walks of one call, written to device memory. */
typedef struct {
  int64_t flips;        /* accepted flips */
  int64_t segments;     /* walk segments started */
  int64_t bloom_skips;  /* Bloom-positive neighbours that ranked ahead of the chosen move */
  int64_t dead_ends;    /* segments ended because every neighbour was explored */
  int32_t E_thr;        /* sieve bound actually used */
  int32_t best_E;       /* lowest energy reached by any flip */
  int32_t status;       /* LABS_OK or a device-side error */
  int32_t reserved;
} labs_walk_stats;

/*
 * labs_skew_search -- step 1 of the paper (Algorithm 1, Fig. 2-3): n_walks independent self-avoiding
 * walks, one per warp, each behind a fixed prefix, sieving candidates with E <= E_thr.
 *   prefixes   [n_prefix][ceil(p/64)] uint64, device: bit j of word 0 is 1 iff s_{j+1} = +1.
 *   out        [n_walks][R] labs_candidate, device, sorted by (E, fp) per walk; unused slots have
 *              E = INT32_MAX, fp = ~0 and zero elsewhere.
 *   walk_stats nullable; [n_walks][6] int64, device: flips, segments, bloom_skips, dead_ends, best_E,
 *              first flip count with E <= E_target (-1 if never or off).
 *   stats      labs_walk_stats, device.
 * Errors: LABS_ERR_INVALID_ARG on a bad configuration.
 */
int labs_skew_search(labs_ctx* ctx, const labs_walk_cfg* cfg, const uint64_t* prefixes, int n_prefix,
                     labs_candidate* out, int64_t* walk_stats, labs_walk_stats* stats, void* stream);

/*
 * Mixed-length batch (step 1 over many lengths at once; the paper runs lengths as separate jobs, so this
 * batching is the library's).  Odd lengths walk skew-symmetrically behind the prefix (Algorithm 1),
 * even lengths walk the unrestricted neighbourhood with no prefix.
 */
typedef struct {
  int32_t n_len;            /* lengths in the batch, 1..96 */
  int32_t p;                /* prefix length for odd lengths (<= k of the shortest odd length) */
  int64_t flip_budget;      /* accepted flips per walk, < 2^32 */
  uint64_t seed;            /* stream seed (walks: (seed, 1, walk, segment); samples: (seed, 2, i, 0)) */
  int32_t R;                /* candidates kept per walk, 1..32 */
  int32_t bloom_log2;       /* 5..15 */
  int32_t bloom_k;          /* 1..8 */
  int32_t T_i;              /* segment length; <= 0 means 4(L+1) for each length */
  int64_t n_thresh_samples; /* per-length sieve bound: samples (<= 2^31) */
  int64_t thresh_rank;      /* per-length sieve bound: 0-based rank */
  int32_t E_target;         /* per-walk first flip reaching E <= E_target (walk_stats[5]); INT32_MIN = off */
  int32_t tile_m;           /* 0: autotuned (timed trial, cached per length set and SM count); 8, 12, 16 */
  int32_t warps_per_cta;    /* 0: autotuned; 1..8 */
  int32_t use_graph;        /* 1: capture the step into a CUDA graph on first use and replay it */
} labs_batch_cfg;

/*
 * labs_batched_search -- every length's sieve bound (as labs_sample_threshold), then ONE persistent
 * launch over all (length, walk) work items, pulled from a device counter.
 *   lengths [n_len] int32 HOST, 3..576; walks [n_len] int64 HOST, walks per length (walk ids 0..walks-1
 *   within each length).
 *   prefixes as in labs_skew_search.  out [sum walks][R] candidates, DEVICE, grouped by length in the
 *   given order; walk_stats nullable [sum walks][6] int64 DEVICE; E_thr_out nullable [n_len] int32 DEVICE
 *   (the sieve bounds used); stats DEVICE (E_thr reports the first length's bound).
 *   With use_graph the first call with a given configuration and buffers captures the step into a CUDA
 *   graph (on a private stream) and later calls replay it on `stream`.
 * Errors: LABS_ERR_INVALID_ARG on a bad configuration or a length that fits no tile variant.
 */
int labs_batched_search(labs_ctx* ctx, const labs_batch_cfg* cfg, const int32_t* lengths, const int64_t* walks,
                        const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                        int32_t* E_thr_out, labs_walk_stats* stats, void* stream);

/*
 * labs_sample_threshold -- the sieve bound E_l of Algorithm 1 under the nearest-rank reading: draws
 * n_samples starts exactly like walk starts (sample i: prefix i mod n_prefix, stream (seed, 2, i, 0))
 * and writes the 0-based `rank`-th smallest sampled energy to *E_thr_out (device int32).
 *   E_samples nullable; [n_samples] int32, device: the sampled energies in sample order.
 */
int labs_sample_threshold(labs_ctx* ctx, int L, int skew, int p, const uint64_t* prefixes, int n_prefix,
                          uint64_t seed, int64_t n_samples, int64_t rank, int32_t* E_thr_out, int32_t* E_samples,
                          void* stream);

/*
 * labs_sample_threshold_noalloc -- the same sieve bound as labs_sample_threshold for callers that may
 * not allocate device memory: an application whose allocator owns every device byte (a framework memory
 * pool, a fixed arena sized at start-up) forbids direct cudaMalloc, and a latency-sensitive caller avoids
 * it because it can synchronise the device.  The paper has no counterpart; this is a property of the
 * library, not of the method.
 *   No context is needed and nothing is allocated: no cudaMalloc, cudaFree or allocating library routine
 *   is called.  The scratch (sampled energies and histograms) is one fixed device array of 4.26 MB that
 *   every GPU loading the library holds until the process exits.
 *   Runs on the current device and `stream`; arguments as in labs_sample_threshold (prefixes device,
 *   E_thr_out device int32); the sampled energies are not returned.
 *   n_samples may be at most 1,048,576 (2^20); larger values return LABS_ERR_CAPACITY.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress); make that
 *   first call before any stream capture.
 *   Every call shares the one array and clears the parts that must start at zero; calls that overlap on
 *   the GPU (other streams, other host threads) race on it and must be serialised by the caller.
 */
int labs_sample_threshold_noalloc(int L, int skew, int p, const uint64_t* prefixes, int n_prefix, uint64_t seed,
                                  int64_t n_samples, int64_t rank, int32_t* E_thr_out, void* stream);

/*
 * Step 2: Algorithm 2 (priority-queue refinement over the unrestricted space) in batch-synchronous form.
 * Readings where the paper gives no value or is ambiguous:
 *  - keys are (E, fp) compared lexicographically; the open set holds at most `cap` entries;
 *  - a round pops the b = min(B, open, budget left) smallest keys and scans every single-flip neighbour of
 *    each (all L positions), skipping neighbours whose fingerprint is in the visited set H;
 *  - the round's survivors are ordered by (E', fp', pop order, position), equal (E', fp') kept once;
 *  - the open set becomes the cap smallest keys of (rest of open set) u survivors; H receives exactly the
 *    admitted survivors;
 *  - the best improves on a strict E' < E_best (to the smallest survivor key); u counts pops since the
 *    last improvement;
 *  - MAKE_ROTATIONS: with T_r > 0 each popped pivot also offers its rotations by 1..T_r elements to the
 *    left (first elements moved to the end) and to the right (last elements moved to the start), energy
 *    and fingerprint computed from scratch, ordered after the pivot's L flips; they are survivors like
 *    the flips (visited-set test, admission, best).
 * With B = 1 and a cap never reached this is Algorithm 2 step by step.
 */
typedef struct {
  int32_t L;              /* 2..576 */
  int32_t B;              /* pops per round, 1..8192 */
  int64_t cap;            /* open-set capacity, 1..2^24 */
  int32_t H_log2;         /* visited set: 2^H_log2 slots of 8 bytes, 10..31; it must stay <= 3/4 full */
  int32_t T_r;            /* rotations per side: 0..64, 2 T_r < L */
  int64_t max_expansions; /* pops in total */
  int64_t T_u;            /* stop after T_u pops without improvement; <= 0: no limit */
} labs_pq_cfg;

typedef struct {
  int64_t expansions;   /* nodes popped and scanned */
  int64_t rounds;
  int64_t survivors;    /* distinct neighbours not in H, summed over rounds */
  int64_t admitted;     /* survivors that entered the open set (and H) */
  int64_t evicted;      /* open-set entries pushed out by the capacity */
  int64_t h_size;       /* fingerprints in H at the end */
  int64_t improvements; /* rounds that improved the best */
  uint64_t best_fp;
  int32_t stop_reason;  /* 1 expansion budget, 2 open set empty, 3 T_u */
  int32_t status;       /* LABS_OK, or LABS_ERR_CAPACITY if H filled past 3/4 (the search stops there) */
} labs_pq_stats;

/*
 * labs_pq_refine -- runs Algorithm 2 from n_seeds candidates (for instance the step-1 sieve output) on
 * the device until a stop condition holds.  The host drives the rounds and polls a device flag, so the
 * call returns after `stream` has finished the refinement.
 *   seeds [n_seeds][W] uint64 DEVICE; best_seq [W] uint64 DEVICE; best_E int32 DEVICE; stats DEVICE.
 *   Workspace: two open-set buffers (cap * (12 + 8W) bytes each), the visited set (8 * 2^H_log2 bytes),
 *   survivor and sort buffers (about 60 * B * L bytes).
 * Errors: LABS_ERR_INVALID_ARG on a bad configuration, LABS_ERR_NOMEM if the
 * workspace cannot be allocated.
 */
int labs_pq_refine(labs_ctx* ctx, const labs_pq_cfg* cfg, const uint64_t* seeds, int n_seeds, uint64_t* best_seq,
                   int32_t* best_E, labs_pq_stats* stats, void* stream);

/*
 * labs_pq_independent -- Algorithm 2 run separately for every candidate (the paper's parallelisation of
 * step 2): candidate q starts its own queue and visited set from seeds[q] and is refined with one pop per
 * step, the queue unbounded (nothing is evicted), until max_expansions pops, an empty queue, or T_u pops
 * without improvement.  Equivalent to labs_pq_refine with one seed, B = 1 and a cap never reached
 * (rotations included when T_r > 0).
 *   seeds [n][W] uint64, best_seqs [n][W] uint64, best_E [n] int32, stats [n] labs_pq_stats -- device.
 *   Memory: each resident warp holds max_expansions x (L + 2 T_r) x 16 B of queue records, 24 B per pop
 *   of run heads, 8 W B per pop of pivots, about 4 L B per pop of pivot tables (C_k and P_m) and
 *   2^H_log2 x 8 B of visited set; as many warps run as fit in max_workspace_bytes (0: 64 GiB) and the
 *   occupancy limit, the rest of the candidates wait for a warp.
 * Errors: LABS_ERR_INVALID_ARG on a bad configuration; per candidate, stats.status = LABS_ERR_CAPACITY if
 * its visited set passed 3/4 load (raise H_log2).
 */
typedef struct {
  int32_t L;                   /* 2..576 */
  int32_t T_r;                 /* rotations per side: 0..64, 2 T_r < L */
  int32_t H_log2;              /* visited set per candidate: 2^H_log2 slots, 10..30 */
  int32_t reserved;            /* 0 */
  int64_t max_expansions;      /* pops per candidate, 1..2^21 - 1 */
  int64_t T_u;                 /* stop after T_u pops without improvement; <= 0: no limit */
  int64_t max_workspace_bytes; /* device memory for the resident warps; 0: 64 GiB */
} labs_pq_indep_cfg;

int labs_pq_independent(labs_ctx* ctx, const labs_pq_indep_cfg* cfg, const uint64_t* seeds, int n, uint64_t* best_seqs,
                        int32_t* best_E, labs_pq_stats* stats, void* stream);

/*
 * Learned flip proposal (library extension; the paper has no learned component).  A small network --
 * features (s_i, C_k / sqrt(L-k)), three Conv1d(64, kernel 9) layers, Linear(64L -> 256), Linear(256 -> L)
 * -- scores the L positions of a sequence; walks may bias their neighbour choice with it while the exact
 * energy scan stays the judge.  Weights are BF16 with an FP32 master copy; sums accumulate in FP32.
 * Parameters are one flat FP32 array in the order w1 [64][2][9], b1 [64], w2 [64][64][9], b2, w3, b3,
 * W4 [256][64 L], b4 [256], W5 [L][256], b5 [L].
 */
typedef struct labs_policy labs_policy;

/* Number of parameters for length L. */
int labs_policy_param_count(int L, int64_t* n_out);
/* Creates a network for length L with He-uniform weights drawn from SplitMix64 stream (seed, 4, layer). */
int labs_policy_create(labs_ctx* ctx, int L, uint64_t seed, labs_policy** out);
void labs_policy_destroy(labs_policy* policy);
/* Replaces the parameters (device FP32 [n]) and resets the optimizer state. */
int labs_policy_set_params(labs_policy* policy, const float* params, void* stream);
/* Copies the FP32 master parameters to device memory [n]. */
int labs_policy_get_params(labs_policy* policy, float* params, void* stream);
/*
 * logits [n][L] FP32 (device) of n packed sequences (device).  Runs on the tensor cores (tcgen05): the
 * convolution outputs are stored as BF16 between layers (training keeps them in FP32), every sum
 * accumulates in FP32.  Workspace: about 0.2 KB x L per sample for up to 8,192 samples at a time.
 * A sample's logits do not depend on the batch it is evaluated in (fixed summation order).
 * A tensor-core wait that expires is reported by labs_policy_sync_status.
 */
int labs_policy_forward(labs_policy* policy, const uint64_t* seqs, int64_t n, float* logits, void* stream);
/*
 * Synchronises `stream` and returns LABS_ERR_TIMEOUT if a tensor-core wait of an earlier
 * labs_policy_forward expired (its logits are then invalid), else LABS_OK; clears the flag.
 */
int labs_policy_sync_status(labs_policy* policy, void* stream);
/*
 * One training step on n samples: forward, weighted cross-entropy over the free positions
 * [free_lo, free_hi] (0-based, the same for every sample) toward target[q] (0-based position), backward,
 * and Adam (lr 0: no update).  loss_out (nullable, device FP32 [1]) receives the mean weighted loss,
 * grads_out (nullable, device FP32 [n_params]) the gradient.  Device pointers throughout.
 */
int labs_policy_train_step(labs_policy* policy, const uint64_t* seqs, const int32_t* target, const float* weight,
                           int64_t n, int free_lo, int free_hi, float lr, float* loss_out, float* grads_out,
                           void* stream);

/*
 * labs_chunked_search -- labs_skew_search's walks run in chunks of `chunk` accepted flips per walk, with
 * each walk's state saved between launches.  With a policy, every walk's current sequence is scored before
 * each chunk (and before the first) and the neighbour choice becomes the smallest
 *     (fmaf(-lambda, logit[m-1], (float) Delta E_m), m)        (FP32; a non-finite logit counts as 0)
 * among the unexplored neighbours -- the energies stay exact, only the order of the choice changes.
 * Without a policy (or lambda = 0) the results are identical to labs_skew_search.  The paper has no
 * counterpart: this is the library's learned proposal.
 *   Arguments as in labs_skew_search, plus (all nullable, DEVICE, n_chunks = ceil(flip_budget / chunk)):
 *   logits_log [n_chunks][n_walks][L] FP32: the logits each chunk used;
 *   state_log  [n_chunks][n_walks][W] uint64: every walk's sequence when its chunk began;
 *   move_log   [n_chunks][n_walks][2] int32: the chunk's first move (position, Delta E), (-1, 0) if none.
 *   Workspace: about 5.5 KB per walk.  With a policy the call synchronises `stream` at its end and returns
 *   LABS_ERR_TIMEOUT if a tensor-core wait of the network expired.
 */
int labs_chunked_search(labs_ctx* ctx, const labs_walk_cfg* cfg, labs_policy* policy, float lambda, int chunk,
                        const uint64_t* prefixes, int n_prefix, labs_candidate* out, int64_t* walk_stats,
                        labs_walk_stats* stats, float* logits_log, uint64_t* state_log, int32_t* move_log,
                        void* stream);

/*
 * labs_sequence_operators -- the end-element operators of Section 3 (Fig. 4): appending or removing one
 * element at either end moves a candidate of length L to L+1 or L-1 with a comparable merit factor, and
 * the results re-enter step 2 (labs_pq_refine at the new length).  For each input sequence S (length L):
 *   grow[q][v], length L+1:   v = 0: S then +1,  1: S then -1,  2: +1 then S,  3: -1 then S;
 *   shrink[q][v], length L-1: v = 0: S without its last element,  1: S without its first element;
 * with the exact energies of the six results.
 *   seqs [n][W(L)] uint64; grow [n][4][W(L+1)] uint64; E_grow [n][4] int32; shrink [n][2][W(L-1)]
 *   uint64; E_shrink [n][2] int32 -- all device; any output may be NULL (not computed / not written).
 * Errors: LABS_ERR_INVALID_ARG for L outside [3, 575], n < 0, a NULL or misaligned pointer.
 */
int labs_sequence_operators(labs_ctx* ctx, const uint64_t* seqs, int L, int64_t n, uint64_t* grow, int32_t* E_grow,
                            uint64_t* shrink, int32_t* E_shrink, void* stream);

/*
 * Legendre-sequence seeds for step 2 (Section 4, Table 2).  A seed is the periodic extension of a
 * rotated Legendre sequence of prime length p <= L:
 *     s_i = chi((i + off) mod p),  i = 0 .. L-1   (the rotation by `off`, then its first L - p elements
 *                                                  appended),
 * chi(j) = +1 for a non-zero quadratic residue j mod p, -1 otherwise (j = 0 included).
 *
 * labs_legendre_family (host only, no device work) -- the parameter family of length L: every prime
 *   p <= L with L - p <= t_max * p and every rotation off < p with r_lo <= off / L <= r_hi, written as
 *   (p, off) int32 pairs to params [max_n][2] (host; NULL to count only), in increasing (p, off);
 *   *n_out receives the family size.  LABS_ERR_CAPACITY if it exceeds max_n (the first max_n are written).
 *   The family (0.20, 0.24, 0.1) reproduces the construction column of Table 2.
 * labs_legendre_construct -- the n seeds of params [n][2] (DEVICE int32 pairs, p prime, 0 <= off < p,
 *   p <= L) as packed sequences seqs [n][W] and exact energies E_out [n] (device; either may be NULL).
 *   A pair that is not a seed of length L (p not a prime in [2, L], off outside [0, p)) gets a zero
 *   sequence and E = INT32_MAX.
 * Errors: LABS_ERR_INVALID_ARG for L outside [3, 576], bad ranges or pointers.
 */
int labs_legendre_family(int L, double r_lo, double r_hi, double t_max, int32_t* params, int64_t max_n,
                         int64_t* n_out);
int labs_legendre_construct(labs_ctx* ctx, int L, const int32_t* params, int64_t n, uint64_t* seqs, int32_t* E_out,
                            void* stream);

/*
 * labs_skew_exhaustive -- every skew-symmetric sequence (Eq. 2) of odd length L <= 127 behind the
 * prefix (Eq. 3, p <= k), 2^(k-p+1) of them, with k-p+1 <= 40.  Free bit j of an assignment is 1 iff
 * s_{p+1+j} = -1.
 *   out_min_E [1] int32, out_count [1] uint64 (assignments reaching the minimum),
 *   out_argmin_free [1] uint64 (smallest such assignment), out_argmin_seq [W] uint64; all device.
 */
int labs_skew_exhaustive(labs_ctx* ctx, int L, int p, uint64_t prefix, int32_t* out_min_E, uint64_t* out_count,
                         uint64_t* out_argmin_free, uint64_t* out_argmin_seq, void* stream);

/*
 * Hexadecimal coding of sequences, as the paper prints its record sequences (Section 4, the paragraph
 * on the results' table): each hex digit stands for four bits, most significant first; the first
 * 4 * ceil(L/4) - L bits are zero pads and are dropped; of the remaining L bits the first is s_1 and a 0
 * stands for -1.  Host-only (no context, no device work, nothing allocated); all pointers are HOST.
 * labs_seq_to_hex -- writes the ceil(L/4) upper-case digits and a terminating NUL of the packed sequence
 *   seq [W] uint64 (the library's layout) to hex.  LABS_ERR_CAPACITY if hex_size < ceil(L/4) + 1,
 *   LABS_ERR_INVALID_ARG for L outside [1, 576] or a NULL pointer.
 * labs_hex_to_seq -- parses exactly ceil(L/4) digits (either case) into seq [W] uint64 (bits above L-1
 *   zero).  LABS_ERR_INVALID_ARG for another length, a character that is not a hex digit, a pad bit that
 *   is not zero, L outside [1, 576] or a NULL pointer; seq is left unchanged on error.
 */
int labs_seq_to_hex(const uint64_t* seq, int L, char* hex, size_t hex_size);
int labs_hex_to_seq(const char* hex, int L, uint64_t* seq);

/*
 * labs_measure_issue_rates -- measurement support for the rooflines (the paper has no counterpart): the
 * sustained issue rate of nine instruction classes on `device`, in lane-instructions per SM clock,
 * written to rates[0..8] (HOST doubles) in the order IADD (add.s32), LOP3, SHF (funnel shift), IMAD
 * (mad.lo.s32), DP4A, POPC, PRMT, FFMA (fma.rn.f32), DP2A.  Each class runs alone: one 1024-thread block
 * per SM, 16 independent chains per thread, timed in SM clocks with clock64(); the median over the SMs.
 * Synchronises the device; allocates and frees a few hundred bytes of device memory.
 * Errors: LABS_ERR_INVALID_ARG for a bad device or n_rates < 9, LABS_ERR_CUDA / LABS_ERR_NOMEM.
 */
int labs_measure_issue_rates(int device, double* rates, int n_rates);

#ifdef __cplusplus
}
#endif

#endif /* LABS_H_ */
