// FP64 reductions: total mass sum(G psi) per field, difference norms, and the
// donor-cell Courant check.  Deterministic: each block reduces a fixed strided
// subset in FP64, a second kernel reduces the block partials in a fixed order.
#include <cuda_runtime.h>

#include "internal.h"

namespace mpd {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// block-wide reduction; result valid in thread 0
template <bool kMax>
__device__ double block_reduce(double v) {
  __shared__ double sh[kThreads / 32];
  v = kMax ? warp_max(v) : warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kThreads / 32) ? sh[l] : (kMax ? 0.0 : 0.0);
    v = kMax ? warp_max(v) : warp_sum(v);
  }
  __syncthreads();
  return v;
}

template <typename T>
__global__ void k_mass_partial(const T* __restrict__ psi, const T* __restrict__ g,
                               const FieldSpan* __restrict__ spans, double* __restrict__ partial) {
  const FieldSpan sp = spans[blockIdx.y];
  double acc = 0.0;
  for (long long j = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; j < sp.n;
       j += static_cast<long long>(gridDim.x) * kThreads) {
    const long long i = sp.offset + j;
    const double p = static_cast<double>(psi[i]);
    acc += g ? static_cast<double>(g[i]) * p : p;
  }
  acc = block_reduce<false>(acc);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

template <typename T>
__global__ void k_diff_partial(const T* __restrict__ a, const T* __restrict__ b,
                               const FieldSpan* __restrict__ spans, double* __restrict__ psum,
                               double* __restrict__ pmax) {
  const FieldSpan sp = spans[blockIdx.y];
  double s = 0.0, m = 0.0;
  for (long long j = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; j < sp.n;
       j += static_cast<long long>(gridDim.x) * kThreads) {
    const long long i = sp.offset + j;
    const double d = static_cast<double>(a[i]) - static_cast<double>(b[i]);
    s += d * d;
    m = fmax(m, fabs(d));
  }
  s = block_reduce<false>(s);
  m = block_reduce<true>(m);
  if (threadIdx.x == 0) {
    psum[blockIdx.y * gridDim.x + blockIdx.x] = s;
    pmax[blockIdx.y * gridDim.x + blockIdx.x] = m;
  }
}

template <bool kMax>
__global__ void k_final(const double* __restrict__ partial, int nper, double* __restrict__ out) {
  double v = 0.0;
  for (int j = threadIdx.x; j < nper; j += kThreads) {
    const double x = partial[blockIdx.x * nper + j];
    v = kMax ? fmax(v, x) : v + x;
  }
  v = block_reduce<kMax>(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// max over cells of sum_d ([gc_d(i)]+ - [gc_d(i - e_d)]-) / G_i
template <typename T>
__global__ void k_courant(Grid gr, const T* __restrict__ g0, const T* __restrict__ g1,
                          const T* __restrict__ g2, const T* __restrict__ G, double* __restrict__ partial) {
  const T* gc[3] = {g0, g1, g2};
  double m = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < gr.N;
       i += static_cast<long long>(gridDim.x) * kThreads) {
    long long c[3];
    c[2] = i % gr.n[2];
    const long long r = i / gr.n[2];
    c[1] = r % gr.n[1];
    c[0] = r / gr.n[1];
    double out = 0.0;
    for (int d = 0; d < gr.nd; ++d) {
      const int a = 3 - gr.nd + d;
      long long cm[3] = {c[0], c[1], c[2]};
      cm[a] = (c[a] + gr.n[a] - 1) % gr.n[a];
      const long long im = (cm[0] * gr.n[1] + cm[1]) * gr.n[2] + cm[2];
      const double vp = static_cast<double>(gc[d][i]), vm = static_cast<double>(gc[d][im]);
      out += (vp > 0 ? vp : 0.0) - (vm < 0 ? vm : 0.0);
    }
    if (G) out /= static_cast<double>(G[i]);
    m = fmax(m, out);
  }
  m = block_reduce<true>(m);
  if (threadIdx.x == 0) partial[blockIdx.x] = m;
}

}  // namespace

template <typename T>
cudaError_t reduce_mass(const T* psi, const T* g, const FieldSpan* d_spans, int n_fields,
                        double* d_partial, double* d_out, cudaStream_t st) {
  k_mass_partial<T><<<dim3(kRedBlocks, n_fields), kThreads, 0, st>>>(psi, g, d_spans, d_partial);
  k_final<false><<<n_fields, kThreads, 0, st>>>(d_partial, kRedBlocks, d_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t reduce_diff(const T* a, const T* b, const FieldSpan* d_spans, int n_fields,
                        double* d_partial, double* d_out, cudaStream_t st) {
  double* psum = d_partial;
  double* pmax = d_partial + static_cast<long long>(kRedBlocks) * n_fields;
  k_diff_partial<T><<<dim3(kRedBlocks, n_fields), kThreads, 0, st>>>(a, b, d_spans, psum, pmax);
  k_final<false><<<n_fields, kThreads, 0, st>>>(psum, kRedBlocks, d_out);
  k_final<true><<<n_fields, kThreads, 0, st>>>(pmax, kRedBlocks, d_out + n_fields);
  return cudaGetLastError();
}

template <typename T>
cudaError_t reduce_courant(const Grid* grids, const long long* offsets, int n_fields, const T* const* gc,
                           const T* g, double* d_partial, double* d_out, cudaStream_t st) {
  for (int f = 0; f < n_fields; ++f) {
    const long long o = offsets[f];
    const Grid& gr = grids[f];
    k_courant<T><<<kRedBlocks, kThreads, 0, st>>>(gr, gc[0] + o, gr.nd > 1 ? gc[1] + o : nullptr,
                                                  gr.nd > 2 ? gc[2] + o : nullptr, g ? g + o : nullptr,
                                                  d_partial + static_cast<long long>(f) * kRedBlocks);
  }
  k_final<true><<<n_fields, kThreads, 0, st>>>(d_partial, kRedBlocks, d_out);
  return cudaGetLastError();
}

template cudaError_t reduce_mass<float>(const float*, const float*, const FieldSpan*, int, double*, double*, cudaStream_t);
template cudaError_t reduce_mass<double>(const double*, const double*, const FieldSpan*, int, double*, double*, cudaStream_t);
template cudaError_t reduce_diff<float>(const float*, const float*, const FieldSpan*, int, double*, double*, cudaStream_t);
template cudaError_t reduce_diff<double>(const double*, const double*, const FieldSpan*, int, double*, double*, cudaStream_t);
template cudaError_t reduce_courant<float>(const Grid*, const long long*, int, const float* const*, const float*, double*, double*, cudaStream_t);
template cudaError_t reduce_courant<double>(const Grid*, const long long*, int, const double* const*, const double*, double*, double*, cudaStream_t);

}  // namespace mpd
