// Single-plan launch wrappers of the resident march kernel, shared by the
// translation units of each splitting order (bpm_march.cu: first order,
// bpm_march_strang.cu: second, bpm_march_split4.cu: fourth) and form.
#pragma once

#include <cuda_runtime.h>

#include "bpm_parked.cuh"
#include "bpm_resident.cuh"

namespace bpm {

// Per-channel march body of a launch form: the register-resident form for
// N <= 4096, the parked-envelope form for N = 8192.
template <int N, int G, int SPLIT, bool L2TAB>
struct MarchBody {
  using type = Resident<N, G, SPLIT, L2TAB>;
};
template <int SPLIT>
struct MarchBody<8192, 1, SPLIT, false> {
  using type = Parked<8192, SPLIT>;
};

namespace {

template <int N, int G, int SPLIT, bool L2TAB = false>
__global__ void __launch_bounds__((N / 16) * G, L2TAB ? 2 : 1) march_kernel(MarchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  MarchBody<N, G, SPLIT, L2TAB>::type::run(A, smem);
}

template <int N, int G, int SPLIT, bool L2TAB = false>
cudaError_t launch_one(int blocks, const MarchArgs& a, cudaStream_t s) {
  march_kernel<N, G, SPLIT, L2TAB>
      <<<blocks, (N / 16) * G, MarchBody<N, G, SPLIT, L2TAB>::type::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

template <int N, int G, int SPLIT, bool L2TAB = false>
cudaError_t attr_one() {
  return cudaFuncSetAttribute(march_kernel<N, G, SPLIT, L2TAB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(MarchBody<N, G, SPLIT, L2TAB>::type::smem_bytes()));
}

}  // namespace
}  // namespace bpm
