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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
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
constexpr int kConvSmem = kWImg + kATile + 1024;

__global__ void __launch_bounds__(128, 2) conv64_tc_kernel(const __nv_bfloat16* __restrict__ in,
                                                           const __nv_bfloat16* __restrict__ wimg,
                                                           const float* __restrict__ bias,
                                                           __nv_bfloat16* __restrict__ out, int L, long long n,
                                                           int tiles_per_sample, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
  unsigned char* Ws = base;
  unsigned char* As = base + kWImg;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar;
  __shared__ float bias_s[64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < kWImg / 16; e += 128)
    reinterpret_cast<uint4*>(Ws)[e] = reinterpret_cast<const uint4*>(wimg)[e];
  if (tid < 64) bias_s[tid] = bias[tid];
  if (warp == 0) tmem_alloc(&tmem_base, 64);
  if (tid == 0) mbar_init(&bar);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(128, 64);
  const uint32_t a0 = smem_u32(As), w0 = smem_u32(Ws);
  uint32_t phase = 0;
  const long long n_tiles = n * tiles_per_sample;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long s = tile / tiles_per_sample;
    const int i0 = (int)(tile % tiles_per_sample) * 128;
    const __nv_bfloat16* src = in + s * (long long)L * 64;
    for (int e = tid; e < kRows * 8; e += 128) {
      const int r = e >> 3, c8 = e & 7, pos = i0 - 4 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (pos >= 0 && pos < L) v = *reinterpret_cast<const uint4*>(src + (long long)pos * 64 + c8 * 8);
      *reinterpret_cast<uint4*>(As + c8 * kALbo + r * 16) = v;
    }
    fence_smem_to_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
#pragma unroll 1
      for (int t = 0; t < 9; t++)
#pragma unroll
        for (int c = 0; c < 4; c++)
          mma_bf16(tmem, sdesc(a0 + 16 * t + 2 * c * kALbo, kALbo, 128), sdesc(w0 + t * kWTap + 2 * c * kWLbo, kWLbo, 128),
                   idesc, (t | c) ? 1u : 0u);
      mma_commit(&bar);
    }
    const bool ok = mbar_wait(&bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    fence_after();
    const int i = i0 + warp * 32 + lane;
    __nv_bfloat16* dst = out + (s * (long long)L + i) * 64;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 8; j++)
        w[j] = pack_bf16(fmaxf(v[2 * j] + bias_s[c0 + 2 * j], 0.f), fmaxf(v[2 * j + 1] + bias_s[c0 + 2 * j + 1], 0.f));
      if (i < L) {
        reinterpret_cast<uint4*>(dst + c0)[0] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4*>(dst + c0)[1] = make_uint4(w[4], w[5], w[6], w[7]);
      }
    }
    fence_before();
    __syncthreads();  // the next tile overwrites the input tile and the accumulator
    fence_after();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

// ------------------------------------------------------------------------------------------------
// Linear(K -> 256) + bias + ReLU, FP32 output: out[q][j] = relu(bias[j] + sum_k A[q][k] B[j][k])
// ------------------------------------------------------------------------------------------------
constexpr int kDLboA = 128 * 16 + 16;  // 2,064 B
constexpr int kDLboB = 256 * 16 + 16;  // 4,112 B
constexpr int kDStageA = 8 * kDLboA;   // 16,512 B
constexpr int kDStageB = 8 * kDLboB;   // 32,896 B
constexpr int kDStage = kDStageA + kDStageB;
constexpr int kDenseSmem = 2 * kDStage + 1024;

__global__ void __launch_bounds__(128, 1) dense_tc_kernel(const __nv_bfloat16* __restrict__ A,
                                                          const __nv_bfloat16* __restrict__ B,
                                                          const float* __restrict__ bias, float* __restrict__ out,
                                                          long long n, int K, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * 128;
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(128, 256);
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool failed = false;
  const int nk = K / 64;
  for (int kb = 0; kb < nk && !failed; kb++) {
    const int st = kb & 1;
    unsigned char* As = base + st * kDStage;
    unsigned char* Bs = As + kDStageA;
    if (pending[st]) {  // the MMAs of stage kb - 2 still read this buffer
      const bool ok = mbar_wait(&bar[st], phase[st]);
      phase[st] ^= 1u;
      pending[st] = false;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    const long long k0 = (long long)kb * 64;
    for (int e = tid; e < 128 * 8; e += 128) {
      const int r = e >> 3, c8 = e & 7;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (m0 + r < n) v = *reinterpret_cast<const uint4*>(A + (m0 + r) * (long long)K + k0 + c8 * 8);
      *reinterpret_cast<uint4*>(As + c8 * kDLboA + r * 16) = v;
    }
    for (int e = tid; e < 256 * 8; e += 128) {
      const int r = e >> 3, c8 = e & 7;
      *reinterpret_cast<uint4*>(Bs + c8 * kDLboB + r * 16) =
          *reinterpret_cast<const uint4*>(B + (long long)r * K + k0 + c8 * 8);
    }
    fence_smem_to_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int c = 0; c < 4; c++)
        mma_bf16(tmem, sdesc(a0 + 2 * c * kDLboA, kDLboA, 128), sdesc(b0 + 2 * c * kDLboB, kDLboB, 128), idesc,
                 (kb | c) ? 1u : 0u);
      mma_commit(&bar[st]);
    }
    pending[st] = true;
  }
  for (int st = 0; st < 2; st++)
    if (pending[st]) {
      const bool ok = mbar_wait(&bar[st], phase[st]);
      phase[st] ^= 1u;
      if (!ok) failed = true;
    }
  if (__syncthreads_or(failed)) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    fence_after();
    const long long q = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < 256; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (q < n) {
        float4* dst = reinterpret_cast<float4*>(out + q * 256 + c0);
#pragma unroll
        for (int j = 0; j < 4; j++)
          dst[j] = make_float4(fmaxf(v[4 * j] + bias[c0 + 4 * j], 0.f), fmaxf(v[4 * j + 1] + bias[c0 + 4 * j + 1], 0.f),
                               fmaxf(v[4 * j + 2] + bias[c0 + 4 * j + 2], 0.f),
                               fmaxf(v[4 * j + 3] + bias[c0 + 4 * j + 3], 0.f));
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------------------------------------
// CUDA-core pieces of the inference path: the first convolution (2 input channels) into BF16
// channels-last, and the weight images.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) conv1_cl_kernel(const float* __restrict__ x, const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                       int L, long long n) {
  __shared__ float ws[64 * 18];
  __shared__ float bs[64];
  for (int e = threadIdx.x; e < 64 * 18; e += blockDim.x) ws[e] = __bfloat162float(w[e]);
  if (threadIdx.x < 64) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const long long total = n * L;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const long long s = g / L;
    const int i = (int)(g % L);
    float xin[2][9];
#pragma unroll
    for (int ci = 0; ci < 2; ci++)
#pragma unroll
      for (int t = 0; t < 9; t++) {
        const int pos = i + t - 4;
        xin[ci][t] = (pos >= 0 && pos < L) ? x[(s * 2 + ci) * L + pos] : 0.f;
      }
    uint32_t pk[32];
#pragma unroll
    for (int co = 0; co < 64; co += 2) {
      float acc0 = bs[co], acc1 = bs[co + 1];
#pragma unroll
      for (int ci = 0; ci < 2; ci++)
#pragma unroll
        for (int t = 0; t < 9; t++) {
          acc0 = fmaf(ws[(co * 2 + ci) * 9 + t], xin[ci][t], acc0);
          acc1 = fmaf(ws[((co + 1) * 2 + ci) * 9 + t], xin[ci][t], acc1);
        }
      pk[co >> 1] = pack_bf16(fmaxf(acc0, 0.f), fmaxf(acc1, 0.f));
    }
    uint4* dst = reinterpret_cast<uint4*>(out + g * 64);
#pragma unroll
    for (int j = 0; j < 8; j++) dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
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
  const long long total = n * L;
  const long long blocks = std::min<long long>((total + 127) / 128, (long long)num_sms * 16);
  conv1_cl_kernel<<<(unsigned)blocks, 128, 0, st>>>(x, w1, b1, h1, L, n);
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
  conv64_tc_kernel<<<(unsigned)blocks, 128, kConvSmem, st>>>(in, img, bias, out, L, n, tps, err);
  return cuda_status(cudaGetLastError());
}

int tc_dense(const __nv_bfloat16* A, const __nv_bfloat16* Bp, const float* bias, float* out, long long n, int K,
             int* err, cudaStream_t st) {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {
    if (cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem) != cudaSuccess)
      return LABS_ERR_CUDA;
    configured[dev] = true;
  }
  if (K % 64) return LABS_ERR_INVALID_ARG;
  dense_tc_kernel<<<(unsigned)((n + 127) / 128), 128, kDenseSmem, st>>>(A, Bp, bias, out, n, K, err);
  return cuda_status(cudaGetLastError());
}

}  // namespace tc
}  // namespace labsg
