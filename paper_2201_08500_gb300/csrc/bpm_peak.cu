// Measured CUDA-core peaks: the denominators of the march kernels' rooflines.
//
// The march is bound by FP32 arithmetic on the CUDA cores, and the setup and
// time-sum kernels use FP64.  The unit-count peak (SMs x 128 FP32 lanes x 2 x
// the maximum clock) assumes the clock the part sustains under that load; this
// kernel measures the rate instead.  Every thread runs kChains independent
// fused multiply-add chains x <- x * a + b (a, b kernel arguments, so nothing
// folds), kUnroll rounds per loop trip, on a grid of kBlocksPerSm blocks per
// SM.  Work per launch: 2 x kChains x kUnroll x iters flop per thread.
#include <cuda_runtime.h>

#include "../../include/bpm.h"
#include "bpm_internal.h"
#include "bpm_tma.cuh"

namespace bpm {
namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 8;
constexpr int kPeakThreads = 256;
constexpr int kBlocksPerSm = 4;

// Written only when the chains reach a value they cannot reach, so that the
// compiler keeps every chain and the store never happens.
__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == T(-1.2345e-7)) g_peak_sink = double(s);
}

// The bounded wait of the bulk-copy kernels, made to run out: one block's
// mbarrier is told to expect 16 bytes that no copy will bring, and every
// thread waits on it with mbar_wait (the function the streamed column pass
// uses) at `limit` polls; a thread that gives up records the status the
// kernels record.  No copy is in flight, so the block exits cleanly.
__global__ void bounded_wait_probe_kernel(uint32_t limit, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
  __syncthreads();
  if (!mbar_wait(&bar, 0u, limit)) atomicExch(status, kStatusTmaTimeout);
}

// Status word of the probe.
__device__ int g_probe_status;

}  // namespace
}  // namespace bpm

using namespace bpm;

extern "C" {

BPM_API bpm_status bpm_measure_peak(int kind, int iters, double* flop_per_s, float* ms,
                                    void* cuda_stream) {
  BPM_NVTX();
  if (!flop_per_s || !ms || iters < 1 || (kind != BPM_PEAK_FP32 && kind != BPM_PEAK_FP64))
    return BPM_ERR_INVALID_ARG;
  int sms = 0;
  if (!device_ready(&sms)) return BPM_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return BPM_ERR_CUDA;
  }
  const dim3 grid(unsigned(sms * kBlocksPerSm));
  cudaEventRecord(e0, st);
  if (kind == BPM_PEAK_FP32)
    fma_chain_kernel<float><<<grid, kPeakThreads, 0, st>>>(iters, 0.99999994f, 1e-7f);
  else
    fma_chain_kernel<double><<<grid, kPeakThreads, 0, st>>>(iters, 0.9999999999999999, 1e-16);
  cudaError_t e = cudaGetLastError();
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(t > 0.f)) return BPM_ERR_CUDA;
  const double flop = 2.0 * kChains * kUnroll * double(iters) * double(grid.x) * kPeakThreads;
  *ms = t;
  *flop_per_s = flop / (double(t) * 1e-3);
  return BPM_OK;
}

BPM_API bpm_status bpm_check_bounded_wait(int poll_limit, int* gave_up, void* cuda_stream) {
  BPM_NVTX();
  if (!gave_up || poll_limit < 1) return BPM_ERR_INVALID_ARG;
  int sms = 0;
  if (!device_ready(&sms)) return BPM_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* status = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&status), g_probe_status) != cudaSuccess)
    return BPM_ERR_CUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return BPM_ERR_CUDA;
  bounded_wait_probe_kernel<<<1, 64, 0, st>>>(uint32_t(poll_limit), status);
  int h = 0;
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BPM_ERR_CUDA;
  *gave_up = h == kStatusTmaTimeout ? 1 : 0;
  return BPM_OK;
}

}  // extern "C"
