// Work-queue form of the resident march: one persistent launch marches many
// plans (instances of different Nx, z-step counts and channel counts).
//
// Items are (plan, first channel) pairs sorted longest-first on the host.
// Every block repeatedly takes the next item with an atomic counter and runs
// the resident march of that item's transform size on G = 256 / T channels
// (T = Nx/16 threads per channel): Nx = 256, 512, 1024, 2048, 4096 pack 16, 8,
// 4, 2, 1 channels into the 256-thread block, each with its own shared-memory
// slot (at most 196 KB).  Nx = 8192 needs 512 threads and runs in a sibling
// kernel of the same structure, with the parked-envelope body (bpm_parked.cuh).
// First-order items at Nx >= 1024 run in the tensor-memory kernels below;
// second- and fourth-order items in their own instantiations of the two
// kernels above (one queue per order and size class).  The counter lives in global memory and is
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
static_assert(Resident<4096, 1, 4>::smem_bytes() <= kSmallSmem &&
                  Resident<256, 16, 4>::smem_bytes() <= kSmallSmem &&
                  Resident<256, 16, 2>::smem_bytes() <= kSmallSmem,
              "every order's resident slot fits the first-order bound");

// SPLIT: Eq. split-op order of the queue's plans (1, 2 or 4).  The resident
// body keeps its tables in shared memory only at first and second order, so
// kSmallSmem (first order) bounds every order.
template <int SPLIT>
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
      case 256: Resident<256, 16, SPLIT>::run_item(A, item.ch0, smem); break;
      case 512: Resident<512, 8, SPLIT>::run_item(A, item.ch0, smem); break;
      case 1024: Resident<1024, 4, SPLIT>::run_item(A, item.ch0, smem); break;
      case 2048: Resident<2048, 2, SPLIT>::run_item(A, item.ch0, smem); break;
      case 4096: Resident<4096, 1, SPLIT>::run_item(A, item.ch0, smem); break;
      default: break;
    }
  }
}

template <int SPLIT>
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
    if (item.n == 8192) Parked<8192, SPLIT>::run_item(plans[item.plan], item.ch0, smem);
  }
}

// Body of the TMEM queues: first order in the narrow layout (fewer spills in
// the work-queue kernel, measured faster), Strang in the layout of its
// single-plan kernel (wide at N <= 4096).
template <int N, int SPLIT>
using TmBody = Parked<N, SPLIT, true, SPLIT == 2 && N <= 4096>;

// First-order and Strang items at Nx = 2048, 4096, 8192 in the parked form
// with the tables in tensor memory (Parked<N, SPLIT, true>, the fastest
// single-plan form there): one channel per item, N/16 threads per block,
// 512/(N/16) blocks per SM; every block allocates its TMEM columns once and
// frees them on exit.
template <int N, int SPLIT>
__global__ void __launch_bounds__(N / 16, 512 / (N / 16))
    batch_kernel_tm(const MarchArgs* __restrict__ plans, const BatchItem* __restrict__ items,
                    int n_items, int* counter) {
  using P = TmBody<N, SPLIT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ uint32_t s_tbase;
  if (threadIdx.x / 32 == 0) tmem_alloc<P::kCols>(&s_tbase);
  tmem_sync();
  const uint32_t tcol = P::tmem_thread(s_tbase, threadIdx.x);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const MarchArgs& A = plans[item.plan];
    if (item.ch0 < A.n_ch) P::march_channel(A, item.ch0, smem, threadIdx.x, tcol);
  }
  tmem_sync();
  if (threadIdx.x / 32 == 0) tmem_dealloc<P::kCols>(s_tbase);
}

// First-order items at Nx = 1024 in the tensor-memory parked form with two
// channels per 128-thread block (Parked<1024, 1, true, true, 2>, the fastest
// single-plan form there): each channel group of 64 threads takes its own
// items (its own slot for the counter's answer, its own named barrier), so
// the two groups march at independent phases; four blocks per SM fill the
// SM's 512 TMEM columns.
template <int N>
__global__ void __launch_bounds__(2 * (N / 16), 512 / (2 * (N / 16)))
    batch_kernel_tm2(const MarchArgs* __restrict__ plans, const BatchItem* __restrict__ items,
                     int n_items, int* counter) {
  using P = Parked<N, 1, true, true, 2>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item[2];
  __shared__ uint32_t s_tbase;
  if (threadIdx.x / 32 == 0) tmem_alloc<P::kCols>(&s_tbase);
  tmem_sync();
  const int grp = threadIdx.x / P::T;
  const int t = threadIdx.x % P::T;
  const uint32_t tcol = P::tmem_thread(s_tbase, threadIdx.x);
  unsigned char* gsmem = smem + size_t(grp) * P::group_bytes();
  for (;;) {
    P::gsync();
    if (t == 0) s_item[grp] = atomicAdd(counter, 1);
    P::gsync();
    const int it = s_item[grp];
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const MarchArgs& A = plans[item.plan];
    if (item.ch0 < A.n_ch) P::march_channel(A, item.ch0, gsmem, t, tcol);
  }
  tmem_sync();  // both groups are done (their TMEM loads waited)
  if (threadIdx.x / 32 == 0) tmem_dealloc<P::kCols>(s_tbase);
}

// Fourth-order items at Nx = 1024, 2048, 4096 in the parked form with both
// table sets read from L2 (Parked<N, 4>, the fastest single-plan form there):
// one channel per item, N/16 threads per block, 512/(N/16) blocks per SM.
template <int N, int SPLIT>
__global__ void __launch_bounds__(N / 16, 512 / (N / 16))
    batch_kernel_pk(const MarchArgs* __restrict__ plans, const BatchItem* __restrict__ items,
                    int n_items, int* counter) {
  using P = Parked<N, SPLIT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    P::run_item(plans[item.plan], item.ch0, smem);
  }
}

}  // namespace

int batch_group(int n) { return n == 8192 ? 1 : kSmallThreads / (n / 16); }

int batch_item_channels(int n, int split_order) {
  const bool parked = (split_order <= 2 && n >= 2048) || (split_order == 1 && n == 1024) ||
                      (split_order == 4 && n >= 1024 && n <= 4096);
  return parked ? 1 : batch_group(n);
}

int batch_queue(int n, int split_order) {
  if (split_order == 1) {
    if (n == 8192) return kQueueTm8192;
    if (n == 4096) return kQueueTm4096;
    if (n == 2048) return kQueueTm2048;
    if (n == 1024) return kQueueTm1024;
    return kQueueSmall;
  }
  if (split_order == 4) {
    if (n == 8192) return kQueueBig4;
    if (n == 4096) return kQueuePk4096s4;
    if (n == 2048) return kQueuePk2048s4;
    if (n == 1024) return kQueuePk1024s4;
    return kQueueSmall4;
  }
  if (n == 8192) return kQueueTm8192s2;
  if (n == 4096) return kQueueTm4096s2;
  if (n == 2048) return kQueueTm2048s2;
  return kQueueSmall2;
}

int batch_blocks_per_sm(int queue) {
  switch (queue) {
    case kQueueTm4096:
    case kQueueTm4096s2:
    case kQueuePk4096s4: return 2;
    case kQueueTm2048:
    case kQueueTm2048s2:
    case kQueuePk2048s4:
    case kQueueTm1024: return 4;
    case kQueuePk1024s4: return 8;
    default: return 1;
  }
}

namespace {

template <int N, int SPLIT>
void tm_launch(const MarchArgs* plans, const BatchItem* items, int n_items, int* counter,
               int blocks, cudaStream_t s) {
  batch_kernel_tm<N, SPLIT><<<blocks, N / 16, TmBody<N, SPLIT>::smem_bytes(), s>>>(
      plans, items, n_items, counter);
}

template <int N, int SPLIT>
void pk_launch(const MarchArgs* plans, const BatchItem* items, int n_items, int* counter,
               int blocks, cudaStream_t s) {
  batch_kernel_pk<N, SPLIT><<<blocks, N / 16, Parked<N, SPLIT>::smem_bytes(), s>>>(
      plans, items, n_items, counter);
}

template <int N, int SPLIT>
cudaError_t tm_attr() {
  return cudaFuncSetAttribute(batch_kernel_tm<N, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(TmBody<N, SPLIT>::smem_bytes()));
}

template <int N, int SPLIT>
cudaError_t pk_attr() {
  return cudaFuncSetAttribute(batch_kernel_pk<N, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(Parked<N, SPLIT>::smem_bytes()));
}

}  // namespace

cudaError_t launch_batch(const MarchArgs* plans, const BatchItem* items, int n_items, int* counter,
                         int queue, int blocks, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const size_t big_smem = Parked<8192, 4>::smem_bytes();
  switch (queue) {
    case kQueueTm8192: tm_launch<8192, 1>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm4096: tm_launch<4096, 1>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm2048: tm_launch<2048, 1>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm8192s2: tm_launch<8192, 2>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm4096s2: tm_launch<4096, 2>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm2048s2: tm_launch<2048, 2>(plans, items, n_items, counter, blocks, s); break;
    case kQueuePk4096s4: pk_launch<4096, 4>(plans, items, n_items, counter, blocks, s); break;
    case kQueuePk2048s4: pk_launch<2048, 4>(plans, items, n_items, counter, blocks, s); break;
    case kQueuePk1024s4: pk_launch<1024, 4>(plans, items, n_items, counter, blocks, s); break;
    case kQueueTm1024:
      batch_kernel_tm2<1024><<<blocks, 128, Parked<1024, 1, true, true, 2>::smem_bytes(), s>>>(
          plans, items, n_items, counter);
      break;
    case kQueueSmall:
      batch_kernel<1><<<blocks, kSmallThreads, kSmallSmem, s>>>(plans, items, n_items, counter);
      break;
    case kQueueSmall2:
      batch_kernel<2><<<blocks, kSmallThreads, kSmallSmem, s>>>(plans, items, n_items, counter);
      break;
    case kQueueSmall4:
      batch_kernel<4><<<blocks, kSmallThreads, kSmallSmem, s>>>(plans, items, n_items, counter);
      break;
    case kQueueBig4:
      batch_kernel_8192<4><<<blocks, 512, big_smem, s>>>(plans, items, n_items, counter);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t batch_set_attributes() {
  const int small = int(kSmallSmem), big = int(Parked<8192, 4>::smem_bytes());
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t r[] = {cudaFuncSetAttribute(batch_kernel<1>, attr, small),
                     cudaFuncSetAttribute(batch_kernel<2>, attr, small),
                     cudaFuncSetAttribute(batch_kernel<4>, attr, small),
                     cudaFuncSetAttribute(batch_kernel_8192<4>, attr, big),
                     tm_attr<8192, 1>(), tm_attr<4096, 1>(), tm_attr<2048, 1>(),
                     tm_attr<8192, 2>(), tm_attr<4096, 2>(), tm_attr<2048, 2>(),
                     pk_attr<4096, 4>(), pk_attr<2048, 4>(), pk_attr<1024, 4>(),
                     cudaFuncSetAttribute(batch_kernel_tm2<1024>, attr,
                                          int(Parked<1024, 1, true, true, 2>::smem_bytes()))};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace bpm
