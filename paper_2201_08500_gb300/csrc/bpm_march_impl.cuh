// Single-plan launch wrappers of the resident march kernel, shared by the
// translation units of each splitting order (bpm_march.cu: first order,
// bpm_march_strang.cu: second, bpm_march_split4.cu: fourth) and form.
#pragma once

#include <cuda_runtime.h>

#include "bpm_parked.cuh"
#include "bpm_resident.cuh"

namespace bpm {

// Per-channel march body of a launch form: FORM 0 the register-resident form
// for N <= 4096 and the parked-envelope form for N = 8192; FORM 1 the L2-table
// resident form; FORM 2 the parked form at N <= 4096; FORM 3 the parked form
// with the tables in tensor memory (at N = 1024 two channels a block).
template <int N, int G, int SPLIT, int FORM>
struct MarchBody {
  using type = Resident<N, G, SPLIT, FORM == 1>;
};
template <int SPLIT>
struct MarchBody<8192, 1, SPLIT, 0> {
  using type = Parked<8192, SPLIT>;
};
template <int N, int SPLIT>
struct MarchBody<N, 1, SPLIT, 2> {
  using type = Parked<N, SPLIT>;
};
template <int N, int SPLIT>
struct MarchBody<N, 1, SPLIT, 3> {
  using type = Parked<N, SPLIT, true>;
};
// N = 1024: two channels of 64 threads per block, so that a block's 128
// tensor-memory lanes all hold tables (four blocks of 128 columns per SM).
template <>
struct MarchBody<1024, 2, 1, 3> {
  using type = Parked<1024, 1, true, true, 2>;
};

// Resident blocks per SM the form is compiled for (128 registers unless 1).
__host__ __device__ constexpr int march_min_blocks(int n, int g, int form) {
  return form == 1 ? 2 : (form == 2 || form == 3) ? 512 / (n / 16 * g) : 1;
}

namespace {

template <int N, int G, int SPLIT, int FORM = 0>
__global__ void __launch_bounds__((N / 16) * G, march_min_blocks(N, G, FORM))
    march_kernel(MarchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  MarchBody<N, G, SPLIT, FORM>::type::run(A, smem);
}

template <int N, int G, int SPLIT, int FORM = 0>
cudaError_t launch_one(int blocks, const MarchArgs& a, cudaStream_t s) {
  march_kernel<N, G, SPLIT, FORM>
      <<<blocks, (N / 16) * G, MarchBody<N, G, SPLIT, FORM>::type::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

template <int N, int G, int SPLIT, int FORM = 0>
cudaError_t attr_one() {
  return cudaFuncSetAttribute(march_kernel<N, G, SPLIT, FORM>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(MarchBody<N, G, SPLIT, FORM>::type::smem_bytes()));
}

}  // namespace
}  // namespace bpm
