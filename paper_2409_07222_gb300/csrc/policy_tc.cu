// policy_tc.cu -- the proposal network's inference path on the 5th-generation tensor cores (tcgen05).
//
// Activations are BF16, channels-last ([sample][position][64 channels], 128 B per position); every sum
// accumulates in FP32 in tensor memory (TMEM).  Operands sit in shared memory in the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, rows 16 B apart, core matrices 128 B
// apart along M/N (the descriptor's stride byte offset) and LBO bytes apart along K (its leading byte
// offset).  LBO is padded by 16 B so that the row-major fills below hit all 32 banks.
//
//   conv64_tc_kernel -- Conv1d(64 -> 64, kernel 9, padding 4) + bias + ReLU as an implicit GEMM: a tile
//       is 128 positions x 64 output channels, K = 9 taps x 64 input channels.  The input rows
//       i0-4 .. i0+131 are staged once; the A operand of tap t is the same tile started t rows
//       (16 t bytes) later, so the 36 MMAs (M 128, N 64, K 16) of a tile read one 17.5 KB tile.  The
//       whole weight image (9 x 64 x 64 BF16, 72 KB) stays in shared memory; CTAs are persistent.
//   dense_tc_kernel -- Linear(64 L -> 256) + bias + ReLU: 128 samples x 256 outputs per CTA, K in
//       stages of 64 with two shared-memory stages, so the loads of stage k+1 overlap the MMAs of k.
//
// One thread issues the MMAs; tcgen05.commit arrives on an mbarrier that the CTA waits on with an
// iteration limit (on expiry the kernel records an error, stops issuing work and still frees its
// TMEM).  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w .. 32w+31).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "labs_internal.h"
#include "policy_tc.h"

namespace labsg {
namespace tc {
namespace {

constexpr int kWaitLimit = 1 << 26;  // try_wait polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}
// Waits for phase `parity` of the barrier; false if the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; it++)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
  return done != 0;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// 64 consecutive FP32 columns of this thread's TMEM lane, one load and one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,"
      "%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,"
      "%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 64; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 16-byte asynchronous global -> shared copy; valid = false writes zeros (nothing is read).
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// ------------------------------------------------------------------------------------------------
// Conv1d(64 -> 64, 9, pad 4) + bias + ReLU
// ------------------------------------------------------------------------------------------------
constexpr int kRows = 128 + 8;               // staged input rows of a tile
constexpr int kALbo = kRows * 16 + 16;       // K-chunk stride of the input tile (2192 B)
constexpr int kATile = 8 * kALbo;            // 17,536 B
constexpr int kWLbo = 64 * 16;               // K-chunk stride of one tap's weights (1024 B)
constexpr int kWTap = 8 * kWLbo;             // 8,192 B
constexpr int kWImg = 9 * kWTap;             // 73,728 B
constexpr int kConvSmem = kWImg + 2 * kATile + 1024;

// Warp-specialised: warps 0-3 fetch input tiles (cp.async) and drain accumulators, warp 4 issues the
// MMAs.  Two input buffers and two TMEM accumulators; per buffer b four mbarriers:
//   full[b]  -- the tile in buffer b has landed (128 arrivals)      -> the MMA warp may start,
//   mma[b]   -- the MMAs reading buffer b are done (commit)         -> buffer b may be refilled and
//                                                                      accumulator b read out,
//   drain[b] -- accumulator b has been read out (128 arrivals)      -> the MMA warp may overwrite it.
// Tile j of the CTA uses buffer and accumulator j & 1; every barrier completes once per use of b, so
// the parity of use u = j >> 1 is u & 1.
constexpr int kConvThreads = 160;

__device__ __forceinline__ void mbar_init_n(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)));
}
// cp.async completion of this thread's copies counted as one arrival on bar (non-blocking).
__device__ __forceinline__ void cp_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)));
}

__global__ void __launch_bounds__(kConvThreads, 2) conv64_tc_kernel(const __nv_bfloat16* __restrict__ in,
                                                                    const __nv_bfloat16* __restrict__ wimg,
                                                                    const float* __restrict__ bias,
                                                                    __nv_bfloat16* __restrict__ out, int L, long long n,
                                                                    int tiles_per_sample, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
  unsigned char* Ws = base;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[2], mmad[2], drain[2], wbar;
  __shared__ float bias_s[64];
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long n_tiles = n * tiles_per_sample;
  const long long my_tiles = (long long)blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_id = [&](long long j) { return (long long)blockIdx.x + j * gridDim.x; };
  if (tid < 64) bias_s[tid] = bias[tid];
  if (warp == 0) tmem_alloc(&tmem_base, 128);
  if (tid == 0) {
    for (int b = 0; b < 2; b++) {
      mbar_init_n(&full[b], 128);
      mbar_init_n(&mmad[b], 1);
      mbar_init_n(&drain[b], 128);
    }
    mbar_init_n(&wbar, 128);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp < 4) {
    // ---- loader / drain warps
    for (int e = tid; e < kWImg / 16; e += 128) cp16(Ws + 16 * e, reinterpret_cast<const uint4*>(wimg) + e, true);
    cp_arrive(&wbar);
    for (long long j = 0; j <= my_tiles; j++) {
      // fetch tile j into buffer j & 1 once the MMAs of tile j - 2 have released it
      if (j < my_tiles) {
        const int b = (int)(j & 1);
        if (j >= 2 && !mbar_wait(&mmad[b], (uint32_t)(((j >> 1) - 1) & 1))) atomicExch(&fail, 1);
        unsigned char* As = base + kWImg + b * kATile;
        const long long tile = tile_id(j);
        const long long s = tile / tiles_per_sample;
        const int i0 = (int)(tile % tiles_per_sample) * 128;
        const __nv_bfloat16* src = in + s * (long long)L * 64;
        for (int e = tid; e < kRows * 8; e += 128) {
          const int r = e >> 3, c8 = e & 7, pos = i0 - 4 + r;
          const bool ok = pos >= 0 && pos < L;
          cp16(As + c8 * kALbo + r * 16, ok ? src + (long long)pos * 64 + c8 * 8 : src, ok);
        }
        cp_arrive(&full[b]);
      }
      // drain tile j - 1
      if (j >= 1) {
        const long long jj = j - 1;
        const int b = (int)(jj & 1);
        if (!mbar_wait(&mmad[b], (uint32_t)((jj >> 1) & 1))) atomicExch(&fail, 1);
        fence_after();
        const long long tile = tile_id(jj);
        const long long s = tile / tiles_per_sample;
        const int i = (int)(tile % tiles_per_sample) * 128 + warp * 32 + lane;
        float v[64];
        tmem_ld64(tmem_base + (uint32_t)(b * 64) + ((uint32_t)(warp * 32) << 16), v);
        fence_before();
        mbar_arrive(&drain[b]);
        uint32_t w[32];
#pragma unroll
        for (int k = 0; k < 32; k++)
          w[k] = pack_bf16(fmaxf(v[2 * k] + bias_s[2 * k], 0.f), fmaxf(v[2 * k + 1] + bias_s[2 * k + 1], 0.f));
        if (i < L) {
          uint4* dst = reinterpret_cast<uint4*>(out + (s * (long long)L + i) * 64);
#pragma unroll
          for (int k = 0; k < 8; k++) dst[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        }
      }
      if (*reinterpret_cast<volatile int*>(&fail)) break;
    }
  } else if (lane == 0) {
    // ---- MMA warp (one lane)
    const uint32_t idesc = idesc_bf16(128, 64);
    const uint64_t adesc0 = sdesc(smem_u32(base + kWImg), kALbo, 128);
    const uint64_t wdesc0 = sdesc(smem_u32(Ws), kWLbo, 128);
    bool ok = mbar_wait(&wbar, 0);
    for (long long j = 0; j < my_tiles && ok; j++) {
      const int b = (int)(j & 1);
      const uint32_t u = (uint32_t)((j >> 1) & 1);
      ok = mbar_wait(&full[b], u);                                 // the input tile has landed
      if (ok && j >= 2) ok = mbar_wait(&drain[b], u ^ 1u);          // accumulator b was read out
      if (!ok) break;
      asm volatile("fence.proxy.async.shared::cta;");
      fence_after();
      const uint64_t ab = adesc0 + (uint64_t)((b * kATile) >> 4);
      const uint32_t d = tmem_base + (uint32_t)(b * 64);
#pragma unroll
      for (int t = 0; t < 9; t++)
#pragma unroll
        for (int c = 0; c < 4; c++)
          mma_bf16(d, ab + (uint64_t)((16 * t + 2 * c * kALbo) >> 4), wdesc0 + (uint64_t)((t * kWTap + 2 * c * kWLbo) >> 4),
                   idesc, (t | c) ? 1u : 0u);
      mma_commit(&mmad[b]);
    }
    if (!ok) atomicExch(&fail, 1);
  }
  cp_wait<0>();
  fence_before();
  __syncthreads();
  fence_after();
  if (fail && tid == 0) atomicExch(err, 1);
  if (warp == 0) tmem_dealloc(tmem_base, 128);
}

// ------------------------------------------------------------------------------------------------
// Linear(K -> 256): partial sums part[split][q][j] = sum over the split's K range of A[q][k] B[j][k].
// K in stages of 64 (4 MMAs of M 128, N 256, K 16), three shared-memory stages filled by cp.async two
// stages ahead.  The splits of K spread the 64 L-long rows over the SMs; dense_reduce_kernel adds the
// partial sums in split order (deterministic), the bias and the ReLU.
// ------------------------------------------------------------------------------------------------
constexpr int kDLboA = 128 * 16 + 16;  // 2,064 B
constexpr int kDLboB = 256 * 16 + 16;  // 4,112 B
constexpr int kDStageA = 8 * kDLboA;   // 16,512 B
constexpr int kDStageB = 8 * kDLboB;   // 32,896 B
constexpr int kDStage = kDStageA + kDStageB;
constexpr int kDStages = 3;
constexpr int kDenseSmem = kDStages * kDStage + 1024;

__global__ void __launch_bounds__(128, 1) dense_tc_kernel(const __nv_bfloat16* __restrict__ A,
                                                          const __nv_bfloat16* __restrict__ B, float* __restrict__ part,
                                                          long long n, int K, int kb_per_split, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar[kDStages];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * 128;
  const int nk = K / 64;
  const int kb0 = blockIdx.y * kb_per_split;
  const int nkb = max(0, min(nk, kb0 + kb_per_split) - kb0);
  auto load = [&](int i) {
    unsigned char* As = base + (i % kDStages) * kDStage;
    unsigned char* Bs = As + kDStageA;
    const long long k0 = (long long)(kb0 + i) * 64;
    for (int e = tid; e < 128 * 8; e += 128) {
      const int r = e >> 3, c8 = e & 7;
      const bool ok = m0 + r < n;
      cp16(As + c8 * kDLboA + r * 16, ok ? A + (m0 + r) * (long long)K + k0 + c8 * 8 : A, ok);
    }
    for (int e = tid; e < 256 * 8; e += 128) {
      const int r = e >> 3, c8 = e & 7;
      cp16(Bs + c8 * kDLboB + r * 16, B + (long long)r * K + k0 + c8 * 8, true);
    }
  };
  if (nkb > 0) load(0);
  cp_commit();
  if (nkb > 1) load(1);
  cp_commit();
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  if (tid == 0)
    for (int b = 0; b < kDStages; b++) mbar_init(&bar[b]);
  const uint32_t idesc = idesc_bf16(128, 256);
  uint32_t phase[kDStages] = {0u, 0u, 0u};
  bool failed = false;
  for (int i = 0; i < nkb; i++) {
    const int st = i % kDStages;
    cp_wait<1>();  // stage i has landed (only the most recent group may still be in flight)
    fence_smem_to_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t a0 = smem_u32(base + st * kDStage), b0 = a0 + kDStageA;
#pragma unroll
      for (int c = 0; c < 4; c++)
        mma_bf16(tmem_base, sdesc(a0 + 2 * c * kDLboA, kDLboA, 128), sdesc(b0 + 2 * c * kDLboB, kDLboB, 128), idesc,
                 (i | c) ? 1u : 0u);
      mma_commit(&bar[st]);
    }
    if (i >= 1) {  // the MMAs of stage i-1 are done: its buffer takes stage i+2
      const int sp = (i - 1) % kDStages;
      const bool ok = mbar_wait(&bar[sp], phase[sp]);
      phase[sp] ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    if (i + 2 < nkb) load(i + 2);
    cp_commit();
  }
  if (!failed && nkb > 0) {
    const int sl = (nkb - 1) % kDStages;
    const bool ok = mbar_wait(&bar[sl], phase[sl]);
    if (__syncthreads_or(!ok)) failed = true;
  }
  cp_wait<0>();
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    fence_after();
    const long long q = m0 + warp * 32 + lane;
    float* dst = part + ((long long)blockIdx.y * n + q) * 256;
#pragma unroll 1
    for (int c0 = 0; c0 < 256; c0 += 64) {
      float v[64];
      if (nkb > 0) {
        tmem_ld64(tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 64; j++) v[j] = 0.f;
      }
      if (q < n) {
#pragma unroll
        for (int j = 0; j < 16; j++)
          reinterpret_cast<float4*>(dst + c0)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, 256);
}

// out[q][j] = relu(bias[j] + sum over splits of part[s][q][j]), splits added in order.
__global__ void dense_reduce_kernel(const float* __restrict__ part, const float* __restrict__ bias,
                                    float* __restrict__ out, long long n, int splits) {
  const long long total = n * 256;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    float v = part[e];
    for (int s = 1; s < splits; s++) v += part[(long long)s * total + e];
    out[e] = fmaxf(v + bias[e & 255], 0.f);
  }
}

// ------------------------------------------------------------------------------------------------
// CUDA-core pieces of the inference path: the first convolution (2 input channels) into BF16
// channels-last, and the weight images.
// ------------------------------------------------------------------------------------------------
// One block per (sample, 128 positions), 256 threads: thread (cp, g) keeps the 36 weights of output
// channels 2cp, 2cp+1 in registers and slides over positions i0 + 16g .. i0 + 16g + 15 of the two input
// channels staged in shared memory; a warp's 32 channel pairs write one 128-byte position row.
__global__ void __launch_bounds__(256) conv1_cl_kernel(const float* __restrict__ x, const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                       int L, long long n) {
  __shared__ float xs[2][136];
  const int cp = threadIdx.x & 31, g = threadIdx.x >> 5;
  float wr[2][2][9];
#pragma unroll
  for (int o = 0; o < 2; o++)
#pragma unroll
    for (int ci = 0; ci < 2; ci++)
#pragma unroll
      for (int t = 0; t < 9; t++) wr[o][ci][t] = __bfloat162float(w[((2 * cp + o) * 2 + ci) * 9 + t]);
  const float b0 = bias[2 * cp], b1 = bias[2 * cp + 1];
  const int tps = (L + 127) / 128;
  for (long long tile = blockIdx.x; tile < n * tps; tile += gridDim.x) {
    const long long s = tile / tps;
    const int i0 = (int)(tile % tps) * 128;
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * 136; e += blockDim.x) {
      const int ci = e / 136, r = e % 136, pos = i0 - 4 + r;
      xs[ci][r] = (pos >= 0 && pos < L) ? x[(s * 2 + ci) * L + pos] : 0.f;
    }
    __syncthreads();
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + (s * L + i0 + 16 * g) * 64) + cp;
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
      float a0 = b0, a1 = b1;
#pragma unroll
      for (int ci = 0; ci < 2; ci++)
#pragma unroll
        for (int t = 0; t < 9; t++) {
          const float xv = xs[ci][16 * g + k + t];
          a0 = fmaf(wr[0][ci][t], xv, a0);
          a1 = fmaf(wr[1][ci][t], xv, a1);
        }
      if (i0 + 16 * g + k < L) dst[k * 32] = pack_bf16(fmaxf(a0, 0.f), fmaxf(a1, 0.f));
    }
  }
}

// Shared-memory image of a 64 -> 64 kernel-9 convolution: element (co, ci) of tap t at byte
// t * 8192 + (ci / 8) * 1024 + co * 16 + (ci % 8) * 2, from the FP32 weights w[co][ci][t].
__global__ void conv_image_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ img) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 9 * 64 * 64; e += gridDim.x * blockDim.x) {
    const int t = e / 4096, r = e % 4096, cc = r / 512, co = (r / 8) % 64, c8 = r % 8;
    const int ci = cc * 8 + c8;
    img[e] = __float2bfloat16_rn(w[(co * 64 + ci) * 9 + t]);
  }
}

// The dense layer's weights in channels-last input order: Bp[j][i * 64 + c] = W4[j][c * L + i].
__global__ void dense_perm_kernel(const float* __restrict__ W4, __nv_bfloat16* __restrict__ Bp, int L) {
  const long long K = 64ll * L;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 256 * K; e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / K, k = e % K;
    const long long i = k / 64, c = k % 64;
    Bp[e] = __float2bfloat16_rn(W4[j * K + c * L + i]);
  }
}

}  // namespace

int tc_conv_smem_bytes() { return kConvSmem; }
int tc_dense_smem_bytes() { return kDenseSmem; }

int tc_prepare_weights(const float* w2, const float* w3, const float* W4, int L, __nv_bfloat16* img2,
                       __nv_bfloat16* img3, __nv_bfloat16* W4p, cudaStream_t st) {
  conv_image_kernel<<<36, 1024, 0, st>>>(w2, img2);
  conv_image_kernel<<<36, 1024, 0, st>>>(w3, img3);
  dense_perm_kernel<<<1024, 256, 0, st>>>(W4, W4p, L);
  return cuda_status(cudaGetLastError());
}

int tc_conv1(const float* x, const __nv_bfloat16* w1, const float* b1, __nv_bfloat16* h1, int L, long long n,
             int num_sms, cudaStream_t st) {
  const long long tiles = n * ((L + 127) / 128);
  const long long blocks = std::min<long long>(tiles, (long long)num_sms * 8);
  if (blocks > 0) conv1_cl_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, w1, b1, h1, L, n);
  return cuda_status(cudaGetLastError());
}

int tc_conv64(const __nv_bfloat16* in, const __nv_bfloat16* img, const float* bias, __nv_bfloat16* out, int L,
              long long n, int num_sms, int* err, cudaStream_t st) {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {
    if (cudaFuncSetAttribute(conv64_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem) != cudaSuccess)
      return LABS_ERR_CUDA;
    configured[dev] = true;
  }
  const int tps = (L + 127) / 128;
  const long long tiles = n * tps;
  const long long blocks = std::min<long long>(tiles, 2ll * num_sms);
  if (blocks > 0) conv64_tc_kernel<<<(unsigned)blocks, kConvThreads, kConvSmem, st>>>(in, img, bias, out, L, n, tps, err);
  return cuda_status(cudaGetLastError());
}

// Splits of K: a function of K alone (about 64 stages each, at most 8), so a sample's logits do not
// depend on the batch it is evaluated in.
int tc_dense_splits(int K) { return std::max(1, std::min(8, (K / 64) / 64)); }

int tc_dense(const __nv_bfloat16* A, const __nv_bfloat16* Bp, const float* bias, float* part, float* out, long long n,
             int K, int num_sms, int* err, cudaStream_t st) {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {
    if (cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem) != cudaSuccess)
      return LABS_ERR_CUDA;
    configured[dev] = true;
  }
  if (K % 64 || n <= 0) return n == 0 ? LABS_OK : LABS_ERR_INVALID_ARG;
  const int splits = tc_dense_splits(K);
  const int nk = K / 64, per = (nk + splits - 1) / splits;
  dense_tc_kernel<<<dim3((unsigned)((n + 127) / 128), (unsigned)splits), 128, kDenseSmem, st>>>(A, Bp, part, n, K, per, err);
  dense_reduce_kernel<<<(unsigned)std::min<long long>((n * 256 + 255) / 256, (long long)num_sms * 16), 256, 0, st>>>(
      part, bias, out, n, splits);
  return cuda_status(cudaGetLastError());
}

}  // namespace tc
}  // namespace labsg
