// policy_tc.h -- launchers of the proposal network's tensor-core inference path (policy_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace labsg {
namespace tc {

// BF16 weight images from the FP32 parameters: the two 64 -> 64 convolutions' shared-memory images
// (9 * 64 * 64 elements each) and the dense layer's weights permuted to channels-last input order
// ([256][64 L]).
int tc_prepare_weights(const float* w2, const float* w3, const float* W4, int L, __nv_bfloat16* img2,
                       __nv_bfloat16* img3, __nv_bfloat16* W4p, cudaStream_t st);
// Conv1d(2 -> 64) + bias + ReLU from the features x[n][2][L] into BF16 channels-last h1[n][L][64].
int tc_conv1(const float* x, const __nv_bfloat16* w1, const float* b1, __nv_bfloat16* h1, int L, long long n,
             int num_sms, cudaStream_t st);
// Conv1d(64 -> 64, 9, pad 4) + bias + ReLU, BF16 channels-last in and out; *err = 1 if a wait expired.
int tc_conv64(const __nv_bfloat16* in, const __nv_bfloat16* img, const float* bias, __nv_bfloat16* out, int L,
              long long n, int num_sms, int* err, cudaStream_t st);
// out[n][256] = relu(bias + A[n][K] . Bp[256][K]^T) in FP32; K a multiple of 64; *err = 1 if a wait expired.
// part: FP32 scratch of tc_dense_splits(K) * n * 256 floats (partial sums of the K splits).
int tc_dense(const __nv_bfloat16* A, const __nv_bfloat16* Bp, const float* bias, float* part, float* out, long long n,
             int K, int num_sms, int* err, cudaStream_t st);
int tc_dense_splits(int K);

int tc_conv_smem_bytes();
int tc_dense_smem_bytes();

}  // namespace tc
}  // namespace labsg
