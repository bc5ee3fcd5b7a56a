// issue_rates.cu -- measured integer and FP32 issue rates of the GPU (labs_measure_issue_rates).
//
// The walk kernels are bound by integer issue, and the ALU/POPC/DP4A rooflines they are judged against
// need the chip's sustained rate for each instruction class.  Each probe kernel runs one block per SM
// (its dynamic shared memory is sized so that no second block fits), 1024 threads, and every thread
// issues NITER x 16 instructions of one class in 16 independent dependency chains, written as inline
// PTX so that exactly that instruction is issued.  The block times itself with clock64() between two
// barriers; the rate is lane-instructions per SM clock = 1024 x NITER x 16 / cycles, the median over
// the SMs.  Clock-independent: multiply by SMs and SM clock to get a peak in ops/s.
#include <algorithm>
#include <vector>

#include "labs_internal.h"

namespace labsg {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 16;

template <int OP>
__device__ __forceinline__ void probe_op(uint32_t (&r)[kChains], uint32_t a, uint32_t b) {
#pragma unroll
  for (int j = 0; j < kChains; j++) {
    uint32_t x = r[j];
    // the add's second operand is the next chain's current value, which that chain's own add also
    // reads: no intermediate sum is single-use, so no two adds can be merged into one three-input add
    if (OP == 0) asm volatile("add.s32 %0, %0, %1;" : "+r"(x) : "r"(r[(j + 1) % kChains]));
    if (OP == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 2) asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 3) asm volatile("mad.lo.s32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 4) asm volatile("dp4a.s32.s32 %0, %1, %2, %0;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 5) asm volatile("popc.b32 %0, %0;" : "+r"(x));
    if (OP == 6) asm volatile("prmt.b32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 7) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
    if (OP == 8) asm volatile("dp2a.lo.s32.s32 %0, %1, %2, %0;" : "+r"(x) : "r"(a), "r"(b));
    r[j] = x;
  }
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1) probe_kernel(int niter, uint32_t a, uint32_t b,
                                                                  long long* cycles, uint32_t* sink) {
  uint32_t r[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) r[j] = threadIdx.x * 2654435761u + j;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < niter; i++) probe_op<OP>(r, a, b);
  __syncthreads();
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s ^= r[j];
  if (s == 0x9E3779B9u) sink[0] = s;  // keeps every chain live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
int run_probe(int sms, size_t smem, int niter, long long* d_cycles, uint32_t* d_sink, double* rate) {
  auto k = probe_kernel<OP>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return LABS_ERR_CUDA;
  for (int pass = 0; pass < 2; pass++) {  // the first pass warms the clocks and the instruction cache
    k<<<sms, kProbeThreads, smem>>>(niter, 0x01020304u, 0x05060708u, d_cycles, d_sink);
    if (cudaDeviceSynchronize() != cudaSuccess) return LABS_ERR_CUDA;
  }
  std::vector<long long> cyc(sms);
  if (cudaMemcpy(cyc.data(), d_cycles, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LABS_ERR_CUDA;
  std::sort(cyc.begin(), cyc.end());
  const double c = (double)cyc[sms / 2];
  *rate = c > 0 ? (double)kProbeThreads * niter * kChains / c : 0.0;
  return LABS_OK;
}

}  // namespace
}  // namespace labsg

extern "C" int labs_measure_issue_rates(int device, double* rates, int n_rates) {
  LABS_TRACE("labs_measure_issue_rates");
  using namespace labsg;
  if (!rates || n_rates < 9) return LABS_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LABS_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return LABS_ERR_CUDA;
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (sms < 1 || optin < 1) return LABS_ERR_CUDA;
  // more than half of the per-block limit: one resident block per SM
  const size_t smem = (size_t)optin / 2 + 1024;
  long long* d_cycles = nullptr;
  uint32_t* d_sink = nullptr;
  if (cudaMalloc(&d_cycles, sizeof(long long) * sms) != cudaSuccess) return LABS_ERR_NOMEM;
  if (cudaMalloc(&d_sink, 64) != cudaSuccess) {
    cudaFree(d_cycles);
    return LABS_ERR_NOMEM;
  }
  const int it = 4096;
  int s = LABS_OK;
  if (s == LABS_OK) s = run_probe<0>(sms, smem, it, d_cycles, d_sink, &rates[0]);
  if (s == LABS_OK) s = run_probe<1>(sms, smem, it, d_cycles, d_sink, &rates[1]);
  if (s == LABS_OK) s = run_probe<2>(sms, smem, it, d_cycles, d_sink, &rates[2]);
  if (s == LABS_OK) s = run_probe<3>(sms, smem, it, d_cycles, d_sink, &rates[3]);
  if (s == LABS_OK) s = run_probe<4>(sms, smem, it, d_cycles, d_sink, &rates[4]);
  if (s == LABS_OK) s = run_probe<5>(sms, smem, it / 4, d_cycles, d_sink, &rates[5]);  // a slow pipe
  if (s == LABS_OK) s = run_probe<6>(sms, smem, it, d_cycles, d_sink, &rates[6]);
  if (s == LABS_OK) s = run_probe<7>(sms, smem, it, d_cycles, d_sink, &rates[7]);
  if (s == LABS_OK) s = run_probe<8>(sms, smem, it, d_cycles, d_sink, &rates[8]);
  cudaFree(d_cycles);
  cudaFree(d_sink);
  return s;
}
