// Diagnostic entry point: the FP64 division the kernels use (nr_div, stencil2d.cuh) applied
// elementwise, so that tests can bound its error against correctly rounded IEEE division.
#include <cuda_runtime.h>

#include "../../include/mpdata.h"
#include "stencil2d.cuh"

namespace {

__global__ void k_div(const double* __restrict__ n, const double* __restrict__ d, double* __restrict__ q,
                      long long count) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    q[i] = mpd::dev::nr_div(n[i], d[i]);
}

}  // namespace

extern "C" int mpdata_selftest_division(const double* n, const double* d, double* q, int64_t count,
                                        void* cuda_stream) {
  if (count < 0 || (count > 0 && (!n || !d || !q))) return MPDATA_EINVAL;
  if (count == 0) return MPDATA_OK;
  const int bs = 256;
  const long long blocks = (count + bs - 1) / bs < 4096 ? (count + bs - 1) / bs : 4096;
  k_div<<<static_cast<unsigned>(blocks), bs, 0, static_cast<cudaStream_t>(cuda_stream)>>>(n, d, q, count);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}
