// policy.cu -- the learned flip-proposal network (labs_policy_*): an optional bias for Algorithm 1's
// neighbour choice.  The paper has no learned component; the exact energy scan stays the judge and a
// zero bias is the plain walk.
//
// Network: features x[0][i] = s_{i+1}, x[1][k] = C_k / sqrt(L-k) (x[1][0] = 0); three Conv1d layers
// (2 -> 64 -> 64 -> 64 channels, kernel 9, padding 4, ReLU); Linear(64 L -> 256, ReLU); Linear(256 -> L).
// Weights are stored in BF16 (an FP32 master copy is kept for the optimizer), all sums accumulate in
// FP32.  Training minimises the weighted cross-entropy over each sample's free positions toward the
// flip it took, with Adam.
//
// Inference (labs_policy_forward, the learned walks) runs on the tensor cores (policy_tc.cu): BF16
// channels-last activations, tcgen05 implicit-GEMM convolutions and a tcgen05 GEMM for the 64 L -> 256
// layer; the first convolution and the 256 -> L layer stay on CUDA cores.
// Training (labs_policy_train_step) runs on CUDA cores with FP32 activations: direct convolution tiles
// (64 output channels x 128 positions per block, 8x4 outputs per thread, input and weight chunks staged
// in shared memory) for the forward pass and the data gradient (the same kernel on flipped, transposed
// weights); an outer-product kernel for the weight gradient; a 64x64-tile GEMM with strided operands for
// the two dense layers and their gradients.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "labs_core.cuh"
#include "labs_internal.h"
#include "policy_tc.h"

struct labs_policy {
  labs_ctx* ctx;
  int L;
  long long n_params;
  long long off[11];  // offsets of w1 b1 w2 b2 w3 b3 W4 b4 W5 b5 (and the end)
  float* master;      // FP32 parameters
  __nv_bfloat16* wbf; // BF16 copy used by every forward pass
  __nv_bfloat16* wT2; // conv2 / conv3 weights flipped and transposed (data gradients)
  __nv_bfloat16* wT3;
  float* grad;
  float* m1;
  float* m2;
  long long step;
  // training activations for up to cap_n samples
  long long cap_n;
  float *x, *h1, *h2, *h3, *a, *logits, *d_logits, *da, *dh_a, *dh_b, *wsum, *loss, *lossv, *wpart;
  // tensor-core inference: weight images (rebuilt when tc_stale) and activations for up to cap_i samples
  __nv_bfloat16 *img2, *img3, *W4p;
  bool tc_stale;
  int* tc_err;
  long long cap_i;
  float *xi, *ai, *part;
  __nv_bfloat16 *h1b, *h2b, *h3b;
};

namespace labsg {
namespace {

constexpr int kC = 64, kKW = 9, kPad = 4, kHid = 256;

// ---------------------------------------------------------------------------------------------
// Features
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) features_kernel(const uint64_t* __restrict__ seqs, int L, long long n,
                                                       float* __restrict__ x) {
  __shared__ uint32_t bits_all[4][kBitWords];
  uint32_t* bits = bits_all[threadIdx.x >> 5];
  const int lane = lane_id();
  const int W = (L + 63) >> 6;
  for (long long q = (long long)blockIdx.x * 4 + (threadIdx.x >> 5); q < n; q += (long long)gridDim.x * 4) {
    if (lane < kBitWords) {
      const int W32 = (L + 31) >> 5;
      uint32_t v = 0;
      if (lane < W32) {
        const uint64_t w = seqs[q * W + (lane >> 1)];
        v = (lane & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
        const int rem = L - 32 * lane;
        if (rem < 32) v &= (1u << rem) - 1u;
      }
      bits[lane] = v;
    }
    __syncwarp();
    float* xs = x + q * 2 * L;
    for (int i = lane; i < L; i += 32) xs[i] = ((bits[i >> 5] >> (i & 31)) & 1u) ? 1.f : -1.f;
    if (lane == 0) xs[L] = 0.f;
    for (int k = lane + 1; k < L; k += 32) xs[L + k] = (float)corr_lag(bits, L, k) / sqrtf((float)(L - k));
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Direct convolution: out[n][co][i] = bias[co] + sum_{ci,t} w[co][ci][t] in[n][ci][i+t-4] (ReLU), or
// for a data gradient (no bias) times (mask[n][co][i] > 0).  64 output channels, 128 positions per block.
// ---------------------------------------------------------------------------------------------
constexpr int kCT = 16;  // input channels per chunk

template <int CIN>
__global__ void __launch_bounds__(256) conv_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                   const float* __restrict__ bias, const float* __restrict__ mask,
                                                   float* __restrict__ out, int L, int relu) {
  constexpr int CH = CIN < kCT ? CIN : kCT;
  __shared__ float in_s[CH][128 + 8];
  __shared__ float w_s[kC][CH * kKW + 1];
  const int n = blockIdx.y;
  const int i0 = blockIdx.x * 128;
  const int ty = threadIdx.x >> 5;  // output channels 8ty .. 8ty+7
  const int tx = threadIdx.x & 31;  // positions i0 + 4tx .. +3
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
  const float* inn = in + (long long)n * CIN * L;
  for (int c0 = 0; c0 < CIN; c0 += CH) {
    for (int e = threadIdx.x; e < CH * 136; e += 256) {
      const int ci = e / 136, j = e % 136;
      const int pos = i0 + j - kPad;
      in_s[ci][j] = (pos >= 0 && pos < L) ? inn[(long long)(c0 + ci) * L + pos] : 0.f;
    }
    for (int e = threadIdx.x; e < kC * CH * kKW; e += 256) {
      const int co = e / (CH * kKW), r = e % (CH * kKW);
      w_s[co][r] = __bfloat162float(w[((long long)co * CIN + c0) * kKW + r]);
    }
    __syncthreads();
#pragma unroll 2
    for (int ci = 0; ci < CH; ci++)
#pragma unroll
      for (int t = 0; t < kKW; t++) {
        float wv[8], iv[4];
#pragma unroll
        for (int a = 0; a < 8; a++) wv[a] = w_s[8 * ty + a][ci * kKW + t];
#pragma unroll
        for (int b = 0; b < 4; b++) iv[b] = in_s[ci][4 * tx + b + t];
#pragma unroll
        for (int a = 0; a < 8; a++)
#pragma unroll
          for (int b = 0; b < 4; b++) acc[a][b] = fmaf(wv[a], iv[b], acc[a][b]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; a++) {
    const int co = 8 * ty + a;
    const float bb = bias ? bias[co] : 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int i = i0 + 4 * tx + b;
      if (i >= L) continue;
      const long long o = ((long long)n * kC + co) * L + i;
      float v = acc[a][b] + bb;
      if (relu) v = fmaxf(v, 0.f);
      if (mask) v = mask[o] > 0.f ? v : 0.f;
      out[o] = v;
    }
  }
}

// Weight gradient of a convolution for a chunk of samples per block: part[block][(co * CIN + ci) * 9 + t] =
// sum_{n in chunk, i} dout[n][co][i] in[n][ci][i+t-4] and part[block][64 * CIN * 9 + co] = sum dout[n][co][i];
// wgrad_reduce_kernel adds the blocks in order (deterministic).
template <int CIN>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const float* __restrict__ in, const float* __restrict__ dout,
                                                         float* __restrict__ part, int L, long long n, int per_block) {
  constexpr int CH = CIN < kCT ? CIN : kCT;
  __shared__ float do_s[kC][129];
  __shared__ float in_s[CH][128 + 8];
  const int c0 = blockIdx.y * CH;
  const int cg = threadIdx.x >> 4;  // output channels 4cg .. 4cg+3
  const int cig = threadIdx.x & 15; // input channel c0 + cig (only if cig < CH)
  float acc[4][kKW];
  float dbs[4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    dbs[a] = 0.f;
#pragma unroll
    for (int t = 0; t < kKW; t++) acc[a][t] = 0.f;
  }
  const long long nb = (long long)blockIdx.x * per_block, ne = min(n, nb + per_block);
  for (long long s = nb; s < ne; s++) {
    for (int i0 = 0; i0 < L; i0 += 128) {
      for (int e = threadIdx.x; e < kC * 128; e += 256) {
        const int co = e >> 7, j = e & 127;
        do_s[co][j] = (i0 + j < L) ? dout[((s * kC) + co) * L + i0 + j] : 0.f;
      }
      for (int e = threadIdx.x; e < CH * 136; e += 256) {
        const int ci = e / 136, j = e % 136;
        const int pos = i0 + j - kPad;
        in_s[ci][j] = (pos >= 0 && pos < L) ? in[((s * CIN) + c0 + ci) * L + pos] : 0.f;
      }
      __syncthreads();
      if (cig < CH) {
        for (int j = 0; j < 128; j++) {
          float dv[4];
#pragma unroll
          for (int a = 0; a < 4; a++) dv[a] = do_s[4 * cg + a][j];
#pragma unroll
          for (int t = 0; t < kKW; t++) {
            const float iv = in_s[cig][j + t];
#pragma unroll
            for (int a = 0; a < 4; a++) acc[a][t] = fmaf(dv[a], iv, acc[a][t]);
          }
          if (cig == 0 && blockIdx.y == 0)
#pragma unroll
            for (int a = 0; a < 4; a++) dbs[a] += dv[a];
        }
      }
      __syncthreads();
    }
  }
  float* pb = part + (long long)blockIdx.x * (kC * CIN * kKW + kC);
  if (cig < CH) {
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const int co = 4 * cg + a;
#pragma unroll
      for (int t = 0; t < kKW; t++) pb[(co * CIN + c0 + cig) * kKW + t] = acc[a][t];
      if (cig == 0 && blockIdx.y == 0) pb[kC * CIN * kKW + co] = dbs[a];
    }
  }
}

// dw[e] += sum over blocks of part[b][e] (e < 64 CIN 9), db likewise, blocks in order.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int blocks, int nw, float* __restrict__ dw,
                                    float* __restrict__ db) {
  const int stride = nw + kC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < stride; e += gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int b = 0; b < blocks; b++) v += part[(long long)b * stride + e];
    if (e < nw)
      dw[e] += v;
    else
      db[e - nw] += v;
  }
}

// wT[ci][co][t] = w[co][ci][8 - t]: a convolution with wT maps output gradients to input gradients.
__global__ void flip_transpose_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wT, int cout, int cin) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cout * cin * kKW) return;
  const int co = e / (cin * kKW), r = e % (cin * kKW), ci = r / kKW, t = r % kKW;
  wT[((long long)ci * cout + co) * kKW + (kKW - 1 - t)] = __float2bfloat16_rn(w[e]);
}

// ---------------------------------------------------------------------------------------------
// GEMM with strided operands: C[m][n] (+)= sum_k A(m,k) B(k,n), A(m,k) = A[m*am + k*ak],
// B(k,n) = B[k*bk + n*bn]; epilogue: + bias[n], ReLU, times (mask[m][n] > 0).  64x64 tiles, 16-deep.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float ld_as_float(const T* p, long long i);
template <>
__device__ __forceinline__ float ld_as_float<float>(const float* p, long long i) {
  return p[i];
}
template <>
__device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, long long K, const TA* __restrict__ A, long long am,
                                                   long long ak, const TB* __restrict__ B, long long bk, long long bn,
                                                   float* __restrict__ C, long long ldc, const float* __restrict__ bias,
                                                   int relu, const float* __restrict__ mask, int accumulate) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
  for (long long k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e >> 6, mm = e & 63;
      const long long k = k0 + kk;
      const int m = m0 + mm, nn = n0 + mm;
      As[kk][mm] = (m < M && k < K) ? ld_as_float(A, m * am + k * ak) : 0.f;
      Bs[kk][mm] = (nn < N && k < K) ? ld_as_float(B, k * bk + nn * bn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) av[a] = As[kk][4 * ty + a];
#pragma unroll
      for (int b = 0; b < 4; b++) bv[b] = Bs[kk][4 * tx + b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int m = m0 + 4 * ty + a;
    if (m >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int nn = n0 + 4 * tx + b;
      if (nn >= N) continue;
      const long long o = m * ldc + nn;
      float v = acc[a][b] + (bias ? bias[nn] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      if (mask) v = mask[o] > 0.f ? v : 0.f;
      C[o] = accumulate ? C[o] + v : v;
    }
  }
}

template <typename TA, typename TB>
void gemm(cudaStream_t st, int M, int N, long long K, const TA* A, long long am, long long ak, const TB* B, long long bk,
          long long bn, float* C, long long ldc, const float* bias, int relu, const float* mask, int accumulate) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, am, ak, B, bk, bn, C, ldc, bias, relu, mask, accumulate);
}

// column sums: out[j] += sum_i d[i][j]
__global__ void colsum_kernel(const float* __restrict__ d, long long rows, int cols, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (long long i = 0; i < rows; i++) s += d[i * cols + j];
  out[j] += s;
}

// ---------------------------------------------------------------------------------------------
// Loss: weighted cross-entropy over the free positions [lo, hi] (0-based) toward target[n].
// ---------------------------------------------------------------------------------------------
__global__ void wsum_kernel(const float* __restrict__ wgt, long long n, float* __restrict__ out) {
  float s = 0.f;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += wgt[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  __shared__ float ws[32];
  if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += ws[i];
    *out = t;
  }
}

__global__ void __launch_bounds__(128) loss_kernel(const float* __restrict__ logits, int L, long long n, int lo, int hi,
                                                   const int32_t* __restrict__ target, const float* __restrict__ wgt,
                                                   const float* __restrict__ wsum, float* __restrict__ dlogits,
                                                   float* __restrict__ loss) {
  const int lane = lane_id();
  const float inv = 1.f / *wsum;
  for (long long q = (long long)blockIdx.x * 4 + (threadIdx.x >> 5); q < n; q += (long long)gridDim.x * 4) {
    const float* lg = logits + q * L;
    float mx = -INFINITY;
    for (int i = lo + lane; i <= hi; i += 32) mx = fmaxf(mx, lg[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    float z = 0.f;
    for (int i = lo + lane; i <= hi; i += 32) z += expf(lg[i] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(kFull, z, o);
    const int t = target[q];
    const float w = wgt[q] * inv;
    for (int i = lane; i < L; i += 32) {
      float d = 0.f;
      if (i >= lo && i <= hi) d = expf(lg[i] - mx) / z;
      if (i == t) d -= 1.f;
      dlogits[q * L + i] = d * w;
    }
    if (lane == 0) loss[q] = w * (mx + logf(z) - lg[t]);  // summed in order by wsum_kernel
  }
}

// ---------------------------------------------------------------------------------------------
// Adam (FP32 master weights), BF16 copy refreshed
// ---------------------------------------------------------------------------------------------
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, __nv_bfloat16* __restrict__ wbf, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float x = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = x;
    wbf[i] = __float2bfloat16_rn(x);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ wbf, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wbf[i] = __float2bfloat16_rn(p[i]);
}

// SplitMix64 uniform in [-lim, lim] for He-uniform initialisation (purpose 4, parameter index i).
__global__ void init_params_kernel(float* __restrict__ p, long long lo, long long hi, float lim, uint64_t key) {
  for (long long i = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
       i += (long long)gridDim.x * blockDim.x) {
    const uint64_t r = sm64_at(key, (uint64_t)i);
    const float u = (float)(r >> 40) * (1.f / 16777216.f);  // 24 random bits in [0, 1)
    p[i] = (2.f * u - 1.f) * lim;
  }
}

constexpr int kWgradSamples = 4;  // samples per block of the weight-gradient kernels

int ensure_acts(labs_policy* P, long long n) {
  if (n <= P->cap_n) return LABS_OK;
  float* bufs[] = {P->x, P->h1, P->h2, P->h3, P->a, P->logits, P->d_logits, P->da, P->dh_a, P->dh_b, P->lossv, P->wpart};
  for (float* b : bufs)
    if (b) cudaFree(b);
  const long long L = P->L;
  const size_t sz[] = {(size_t)n * 2 * L, (size_t)n * kC * L, (size_t)n * kC * L, (size_t)n * kC * L,
                       (size_t)n * kHid, (size_t)n * L, (size_t)n * L, (size_t)n * kHid, (size_t)n * kC * L,
                       (size_t)n * kC * L, (size_t)n, (size_t)((n + kWgradSamples - 1) / kWgradSamples) * (kC * kC * kKW + kC)};
  float** dst[] = {&P->x, &P->h1, &P->h2, &P->h3, &P->a, &P->logits, &P->d_logits, &P->da, &P->dh_a, &P->dh_b,
                   &P->lossv, &P->wpart};
  for (int i = 0; i < 12; i++) {
    *dst[i] = nullptr;
    if (cudaMalloc(dst[i], sizeof(float) * sz[i]) != cudaSuccess) {
      P->cap_n = 0;
      return LABS_ERR_NOMEM;
    }
  }
  P->cap_n = n;
  return LABS_OK;
}

// Forward pass for n samples already featurised in P->x; logits into `logits` (stride L).
void forward(labs_policy* P, long long n, float* logits, cudaStream_t st) {
  const int L = P->L;
  const dim3 g((L + 127) / 128, (unsigned)n);
  const __nv_bfloat16* w = P->wbf;
  const float* m = P->master;
  conv_kernel<2><<<g, 256, 0, st>>>(P->x, w + P->off[0], m + P->off[1], nullptr, P->h1, L, 1);
  conv_kernel<64><<<g, 256, 0, st>>>(P->h1, w + P->off[2], m + P->off[3], nullptr, P->h2, L, 1);
  conv_kernel<64><<<g, 256, 0, st>>>(P->h2, w + P->off[4], m + P->off[5], nullptr, P->h3, L, 1);
  const long long K4 = (long long)kC * L;
  // a[n][j] = relu(b4[j] + sum_k h3[n][k] W4[j][k])
  gemm(st, (int)n, kHid, K4, P->h3, K4, 1ll, w + P->off[6], 1ll, K4, P->a, kHid, m + P->off[7], 1, (const float*)nullptr,
       0);
  // logits[n][i] = b5[i] + sum_j a[n][j] W5[i][j]
  gemm(st, (int)n, L, (long long)kHid, P->a, (long long)kHid, 1ll, w + P->off[8], 1ll, (long long)kHid, logits, L,
       m + P->off[9], 0, (const float*)nullptr, 0);
}

int ensure_inference(labs_policy* P, long long n) {
  if (n <= P->cap_i) return LABS_OK;
  void* bufs[] = {P->xi, P->ai, P->part, P->h1b, P->h2b, P->h3b};
  for (void* b : bufs)
    if (b) cudaFree(b);
  P->xi = P->ai = P->part = nullptr;
  P->h1b = P->h2b = P->h3b = nullptr;
  P->cap_i = 0;
  const size_t L = (size_t)P->L, act = (size_t)n * L * kC * 2;
  const size_t part_rows = (size_t)tc::tc_dense_splits(kC * P->L) * (size_t)n;  // split-K partial sums
  if (cudaMalloc(&P->xi, 4 * (size_t)n * 2 * L) != cudaSuccess || cudaMalloc(&P->ai, 4 * (size_t)n * kHid) != cudaSuccess ||
      cudaMalloc(&P->part, 4 * part_rows * kHid) != cudaSuccess ||
      cudaMalloc(&P->h1b, act) != cudaSuccess || cudaMalloc(&P->h2b, act) != cudaSuccess ||
      cudaMalloc(&P->h3b, act) != cudaSuccess)
    return LABS_ERR_NOMEM;
  P->cap_i = n;
  return LABS_OK;
}

// Inference for n packed sequences: features, conv1 (CUDA cores, BF16 channels-last out), conv2 and
// conv3 (tcgen05), the 64 L -> 256 layer (tcgen05), the 256 -> L layer (CUDA cores).
int forward_tc(labs_policy* P, const uint64_t* seqs, long long n, float* logits, cudaStream_t st) {
  const int L = P->L;
  const float* m = P->master;
  const int sms = P->ctx->num_sms;
  int s = LABS_OK;
  if (P->tc_stale) {
    s = tc::tc_prepare_weights(m + P->off[2], m + P->off[4], m + P->off[6], L, P->img2, P->img3, P->W4p, st);
    if (s != LABS_OK) return s;
    P->tc_stale = false;
  }
  features_kernel<<<(unsigned)std::min<long long>((n + 3) / 4, 4096), 128, 0, st>>>(seqs, L, n, P->xi);
  s = tc::tc_conv1(P->xi, P->wbf + P->off[0], m + P->off[1], P->h1b, L, n, sms, st);
  if (s == LABS_OK) s = tc::tc_conv64(P->h1b, P->img2, m + P->off[3], P->h2b, L, n, sms, P->tc_err, st);
  if (s == LABS_OK) s = tc::tc_conv64(P->h2b, P->img3, m + P->off[5], P->h3b, L, n, sms, P->tc_err, st);
  if (s == LABS_OK) s = tc::tc_dense(P->h3b, P->W4p, m + P->off[7], P->part, P->ai, n, kC * L, sms, P->tc_err, st);
  if (s != LABS_OK) return s;
  gemm(st, (int)n, L, (long long)kHid, P->ai, (long long)kHid, 1ll, P->wbf + P->off[8], 1ll, (long long)kHid, logits, L,
       m + P->off[9], 0, (const float*)nullptr, 0);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int policy_length(const labs_policy* P) { return P->L; }

}  // namespace labsg

using namespace labsg;

extern "C" {

int labs_policy_param_count(int L, int64_t* n_out) {
  if (L < 2 || L > LABS_MAX_L || !n_out) return LABS_ERR_INVALID_ARG;
  *n_out = (int64_t)kC * 2 * kKW + kC + 2 * ((int64_t)kC * kC * kKW + kC) + (int64_t)kHid * kC * L + kHid +
           (int64_t)L * kHid + L;
  return LABS_OK;
}

int labs_policy_create(labs_ctx* ctx, int L, uint64_t seed, labs_policy** out) {
  if (!ctx || !out || L < 2 || L > LABS_MAX_L) return LABS_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LABS_ERR_CUDA;
  labs_policy* P = new (std::nothrow) labs_policy();
  if (!P) return LABS_ERR_NOMEM;
  P->ctx = ctx;
  P->L = L;
  const long long sizes[10] = {(long long)kC * 2 * kKW, kC, (long long)kC * kC * kKW, kC, (long long)kC * kC * kKW,
                               kC, (long long)kHid * kC * L, kHid, (long long)L * kHid, L};
  long long o = 0;
  for (int i = 0; i < 10; i++) {
    P->off[i] = o;
    o += sizes[i];
  }
  P->off[10] = o;
  P->n_params = o;
  const size_t n = (size_t)o;
  if (cudaMalloc(&P->master, 4 * n) != cudaSuccess || cudaMalloc(&P->wbf, 2 * n) != cudaSuccess ||
      cudaMalloc(&P->grad, 4 * n) != cudaSuccess || cudaMalloc(&P->m1, 4 * n) != cudaSuccess ||
      cudaMalloc(&P->m2, 4 * n) != cudaSuccess || cudaMalloc(&P->wT2, 2 * sizes[2]) != cudaSuccess ||
      cudaMalloc(&P->wT3, 2 * sizes[4]) != cudaSuccess || cudaMalloc(&P->wsum, 8) != cudaSuccess ||
      cudaMalloc(&P->loss, 8) != cudaSuccess || cudaMalloc(&P->img2, 2 * sizes[2]) != cudaSuccess ||
      cudaMalloc(&P->img3, 2 * sizes[4]) != cudaSuccess || cudaMalloc(&P->W4p, 2 * sizes[6]) != cudaSuccess ||
      cudaMalloc(&P->tc_err, sizeof(int)) != cudaSuccess) {
    labs_policy_destroy(P);
    return LABS_ERR_NOMEM;
  }
  cudaMemset(P->master, 0, 4 * n);
  cudaMemset(P->tc_err, 0, sizeof(int));
  P->tc_stale = true;
  cudaMemset(P->m1, 0, 4 * n);
  cudaMemset(P->m2, 0, 4 * n);
  // He-uniform weights, zero biases
  const int fan[10] = {2 * kKW, 0, kC * kKW, 0, kC * kKW, 0, kC * L, 0, kHid, 0};
  for (int i = 0; i < 10; i += 2) {
    const float lim = sqrtf(6.f / (float)fan[i]);
    init_params_kernel<<<256, 256>>>(P->master, P->off[i], P->off[i] + sizes[i], lim, stream_key(seed, 4, (uint64_t)i, 0));
  }
  to_bf16_kernel<<<1024, 256>>>(P->master, P->wbf, o);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    labs_policy_destroy(P);
    return LABS_ERR_CUDA;
  }
  *out = P;
  return LABS_OK;
}

void labs_policy_destroy(labs_policy* P) {
  if (!P) return;
  cudaSetDevice(P->ctx->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {P->master, P->wbf, P->grad, P->m1, P->m2, P->wT2, P->wT3, P->wsum, P->loss, P->x, P->h1,
                  P->h2, P->h3, P->a, P->logits, P->d_logits, P->da, P->dh_a, P->dh_b, P->lossv, P->wpart, P->img2, P->img3,
                  P->W4p, P->tc_err, P->xi, P->ai, P->part, P->h1b, P->h2b, P->h3b};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete P;
}

int labs_policy_set_params(labs_policy* P, const float* params, void* stream) {
  if (!P || !params) return LABS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(P->master, params, 4 * (size_t)P->n_params, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LABS_ERR_CUDA;
  to_bf16_kernel<<<1024, 256, 0, st>>>(P->master, P->wbf, P->n_params);
  cudaMemsetAsync(P->m1, 0, 4 * (size_t)P->n_params, st);
  cudaMemsetAsync(P->m2, 0, 4 * (size_t)P->n_params, st);
  P->step = 0;
  P->tc_stale = true;
  return cuda_status(cudaGetLastError());
}

int labs_policy_get_params(labs_policy* P, float* params, void* stream) {
  if (!P || !params) return LABS_ERR_INVALID_ARG;
  return cuda_status(cudaMemcpyAsync(params, P->master, 4 * (size_t)P->n_params, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

int labs_policy_forward(labs_policy* P, const uint64_t* seqs, int64_t n, float* logits, void* stream) {
  LABS_TRACE("labs_policy_forward");
  if (!P || n < 0 || (n > 0 && (!seqs || !logits))) return LABS_ERR_INVALID_ARG;
  if (n == 0) return LABS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long chunk = 8192;
  int s = ensure_inference(P, std::min<long long>(n, chunk));
  if (s != LABS_OK) return s;
  const int W = (P->L + 63) / 64;
  for (long long b = 0; b < n && s == LABS_OK; b += chunk)
    s = forward_tc(P, seqs + b * W, std::min<long long>(chunk, n - b), logits + b * P->L, st);
  return s;
}

int labs_policy_train_step(labs_policy* P, const uint64_t* seqs, const int32_t* target, const float* weight, int64_t n,
                           int free_lo, int free_hi, float lr, float* loss_out, float* grads_out, void* stream) {
  LABS_TRACE("labs_policy_train_step");
  if (!P || n < 1 || !seqs || !target || !weight || free_lo < 0 || free_hi >= P->L || free_lo > free_hi)
    return LABS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int s = ensure_acts(P, n);
  if (s != LABS_OK) return s;
  const int L = P->L;
  const long long K4 = (long long)kC * L;
  features_kernel<<<(unsigned)std::min<long long>((n + 3) / 4, 4096), 128, 0, st>>>(seqs, L, n, P->x);
  forward(P, n, P->logits, st);
  cudaMemsetAsync(P->grad, 0, 4 * (size_t)P->n_params, st);
  wsum_kernel<<<1, 1024, 0, st>>>(weight, n, P->wsum);
  loss_kernel<<<(unsigned)std::min<long long>((n + 3) / 4, 4096), 128, 0, st>>>(P->logits, L, n, free_lo, free_hi,
                                                                                  target, weight, P->wsum,
                                                                                  P->d_logits, P->lossv);
  wsum_kernel<<<1, 1024, 0, st>>>(P->lossv, n, P->loss);
  float* g = P->grad;
  const __nv_bfloat16* w = P->wbf;
  // fc2: dW5[i][j] = sum_n dl[n][i] a[n][j]; db5; da[n][j] = sum_i dl[n][i] W5[i][j], masked by a > 0
  gemm(st, L, kHid, n, P->d_logits, 1ll, (long long)L, P->a, (long long)kHid, 1ll, g + P->off[8], kHid,
       (const float*)nullptr, 0, (const float*)nullptr, 1);
  colsum_kernel<<<(L + 255) / 256, 256, 0, st>>>(P->d_logits, n, L, g + P->off[9]);
  gemm(st, (int)n, kHid, (long long)L, P->d_logits, (long long)L, 1ll, w + P->off[8], (long long)kHid, 1ll, P->da, kHid,
       (const float*)nullptr, 0, P->a, 0);
  // fc1: dW4[j][k] = sum_n da[n][j] h3[n][k]; db4; dh3[n][k] = sum_j da[n][j] W4[j][k], masked by h3 > 0
  gemm(st, kHid, (int)K4, n, P->da, 1ll, (long long)kHid, P->h3, K4, 1ll, g + P->off[6], K4, (const float*)nullptr, 0,
       (const float*)nullptr, 1);
  colsum_kernel<<<1, 256, 0, st>>>(P->da, n, kHid, g + P->off[7]);
  gemm(st, (int)n, (int)K4, (long long)kHid, P->da, (long long)kHid, 1ll, w + P->off[6], K4, 1ll, P->dh_a, K4,
       (const float*)nullptr, 0, P->h3, 0);
  // conv3: weight gradient from (h2, dc3); data gradient into h2's grid, masked by h2 > 0
  const int per_block = kWgradSamples;
  const unsigned nbk = (unsigned)((n + per_block - 1) / per_block);
  const int nw64 = kC * kC * kKW, nw2 = kC * 2 * kKW;
  conv_wgrad_kernel<64><<<dim3(nbk, kC / kCT), 256, 0, st>>>(P->h2, P->dh_a, P->wpart, L, n, per_block);
  wgrad_reduce_kernel<<<(nw64 + kC + 255) / 256, 256, 0, st>>>(P->wpart, (int)nbk, nw64, g + P->off[4], g + P->off[5]);
  flip_transpose_kernel<<<(kC * kC * kKW + 255) / 256, 256, 0, st>>>(P->master + P->off[4], P->wT3, kC, kC);
  const dim3 gc((L + 127) / 128, (unsigned)n);
  conv_kernel<64><<<gc, 256, 0, st>>>(P->dh_a, P->wT3, nullptr, P->h2, P->dh_b, L, 0);
  // conv2
  conv_wgrad_kernel<64><<<dim3(nbk, kC / kCT), 256, 0, st>>>(P->h1, P->dh_b, P->wpart, L, n, per_block);
  wgrad_reduce_kernel<<<(nw64 + kC + 255) / 256, 256, 0, st>>>(P->wpart, (int)nbk, nw64, g + P->off[2], g + P->off[3]);
  flip_transpose_kernel<<<(kC * kC * kKW + 255) / 256, 256, 0, st>>>(P->master + P->off[2], P->wT2, kC, kC);
  conv_kernel<64><<<gc, 256, 0, st>>>(P->dh_b, P->wT2, nullptr, P->h1, P->dh_a, L, 0);
  // conv1 (input features need no gradient)
  conv_wgrad_kernel<2><<<dim3(nbk, 1), 256, 0, st>>>(P->x, P->dh_a, P->wpart, L, n, per_block);
  wgrad_reduce_kernel<<<(nw2 + kC + 255) / 256, 256, 0, st>>>(P->wpart, (int)nbk, nw2, g + P->off[0], g + P->off[1]);
  if (grads_out && cudaMemcpyAsync(grads_out, g, 4 * (size_t)P->n_params, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LABS_ERR_CUDA;
  if (loss_out && cudaMemcpyAsync(loss_out, P->loss, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LABS_ERR_CUDA;
  if (lr != 0.f) {
    P->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)P->step), c2 = 1.f - powf(b2, (float)P->step);
    adam_kernel<<<1024, 256, 0, st>>>(P->master, g, P->m1, P->m2, P->wbf, P->n_params, lr, b1, b2, 1e-8f, c1, c2);
    P->tc_stale = true;
  }
  return cuda_status(cudaGetLastError());
}

int labs_policy_sync_status(labs_policy* P, void* stream) {
  if (!P) return LABS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LABS_ERR_CUDA;
  int e = 0;
  if (cudaMemcpy(&e, P->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LABS_ERR_CUDA;
  if (e && cudaMemset(P->tc_err, 0, sizeof(int)) != cudaSuccess) return LABS_ERR_CUDA;
  return e ? LABS_ERR_TIMEOUT : LABS_OK;
}

}  // extern "C"
