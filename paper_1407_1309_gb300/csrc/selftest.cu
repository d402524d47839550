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

namespace {

// Fused multiply-add issue rate: every thread runs kChains independent FMA chains for `iters`
// rounds (independent chains hide the pipe latency); the result is stored only when it equals
// a value no chain reaches, so nothing is optimised away and nothing is written.
constexpr int kChains = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(long long iters, T b, T c, T never, T* __restrict__ sink) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = static_cast<T>(threadIdx.x + j) * T(1e-3);
  for (long long r = 0; r < iters; ++r) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == never) sink[0] = s;
}

}  // namespace

extern "C" int mpdata_selftest_fma_rate(int dtype, int64_t iters, void* sink, int64_t* fma_count,
                                        void* cuda_stream) {
  if (iters < 1 || !sink || !fma_count || (dtype != MPDATA_F32 && dtype != MPDATA_F64)) return MPDATA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPDATA_ECUDA;
  const unsigned blocks = static_cast<unsigned>(sms) * 8u;  // 8 x 256 threads: every SM full
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (dtype == MPDATA_F32)
    k_fma_rate<float><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-6f, -1.0f, static_cast<float*>(sink));
  else
    k_fma_rate<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-6, -1.0, static_cast<double*>(sink));
  *fma_count = static_cast<int64_t>(blocks) * 256 * kChains * iters;
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}
