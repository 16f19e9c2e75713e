// Work-queue form of the resident march: one persistent launch marches many
// plans (instances of different Nx, z-step counts and channel counts).
//
// Items are (plan, first channel) pairs sorted longest-first on the host.
// Every block repeatedly takes the next item with an atomic counter and runs
// the resident march of that item's transform size on G = 256 / T channels
// (T = Nx/16 threads per channel): Nx = 256, 512, 1024, 2048, 4096 pack 16, 8,
// 4, 2, 1 channels into the 256-thread block, each with its own shared-memory
// slot (at most 196 KB).  Nx = 8192 needs 512 threads and runs in a sibling
// kernel of the same structure, with the parked-envelope body (bpm_parked.cuh).  The counter lives in global memory and is
// cleared before each launch; the queue never waits, so no block can hang.
#include <cuda_runtime.h>

#include "bpm_parked.cuh"
#include "bpm_resident.cuh"

namespace bpm {

namespace {

constexpr int kSmallThreads = 256;

template <int N>
constexpr size_t item_smem() {
  return Resident<N, kSmallThreads / (N / 16)>::smem_bytes();
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

constexpr size_t kSmallSmem =
    cmax(cmax(cmax(item_smem<256>(), item_smem<512>()), cmax(item_smem<1024>(), item_smem<2048>())),
         item_smem<4096>());

template <bool STRANG>
__global__ void __launch_bounds__(kSmallThreads, 1)
    batch_kernel(const MarchArgs* __restrict__ plans, const BatchItem* __restrict__ items,
                 int n_items, int* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const MarchArgs& A = plans[item.plan];
    switch (item.n) {
      case 256: Resident<256, 16, STRANG ? 2 : 1>::run_item(A, item.ch0, smem); break;
      case 512: Resident<512, 8, STRANG ? 2 : 1>::run_item(A, item.ch0, smem); break;
      case 1024: Resident<1024, 4, STRANG ? 2 : 1>::run_item(A, item.ch0, smem); break;
      case 2048: Resident<2048, 2, STRANG ? 2 : 1>::run_item(A, item.ch0, smem); break;
      case 4096: Resident<4096, 1, STRANG ? 2 : 1>::run_item(A, item.ch0, smem); break;
      default: break;
    }
  }
}

template <bool STRANG>
__global__ void __launch_bounds__(512, 1)
    batch_kernel_8192(const MarchArgs* __restrict__ plans, const BatchItem* __restrict__ items,
                      int n_items, int* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    if (item.n == 8192) Parked<8192, STRANG ? 2 : 1>::run_item(plans[item.plan], item.ch0, smem);
  }
}

}  // namespace

int batch_group(int n) { return n == 8192 ? 1 : kSmallThreads / (n / 16); }

cudaError_t launch_batch(const MarchArgs* plans, const BatchItem* items, int n_items, int* counter,
                         bool big, bool strang, int blocks, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const size_t big_smem = Parked<8192, 1>::smem_bytes();
  if (!big && !strang)
    batch_kernel<false><<<blocks, kSmallThreads, kSmallSmem, s>>>(plans, items, n_items, counter);
  else if (!big)
    batch_kernel<true><<<blocks, kSmallThreads, kSmallSmem, s>>>(plans, items, n_items, counter);
  else if (!strang)
    batch_kernel_8192<false><<<blocks, 512, big_smem, s>>>(plans, items, n_items, counter);
  else
    batch_kernel_8192<true><<<blocks, 512, big_smem, s>>>(plans, items, n_items, counter);
  return cudaGetLastError();
}

cudaError_t batch_set_attributes() {
  const int small = int(kSmallSmem), big = int(Parked<8192, 1>::smem_bytes());
  cudaError_t r[] = {
      cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, small),
      cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, small),
      cudaFuncSetAttribute(batch_kernel_8192<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big),
      cudaFuncSetAttribute(batch_kernel_8192<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace bpm
