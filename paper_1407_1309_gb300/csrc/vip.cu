// Prognosed velocity (Sect. 5.1-5.2) and the shallow-water momentum sources of Sect. 5.3-5.4.
//
// k_vip_cells: velocities u_d = q_d / h where h > eps (else 0) at the cell centres, extrapolated
//   linearly in time to n + 1/2 (1.5 u^n - 0.5 u^{n-1}; at the first step of a run u^{n-1} = u^n),
//   and u^n kept for the next step.
// k_vip_faces: the extrapolated velocities interpolated linearly to the cell walls, times dt/dx:
//   the advector of the step (face i+1/2 at index i; along an open dimension the last, unread,
//   entry takes the edge cell's value on both sides).
// k_sw_force: q_d += (dt/2) R_d with R_d = -h (h_{i+e_d} - h_{i-e_d}) / (2 dx) (beyond an open edge
//   h is the edge value): the two halves of the trapezoidal scheme (Sect. 4.1), each with the
//   depth of its own time level.
#include <cuda_runtime.h>

#include "internal.h"

namespace mpd {
namespace {

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }
__device__ __forceinline__ int wrapv(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// coordinates of cell i on the internal axes
__device__ __forceinline__ void coords(const Grid& g, long long i, int (&c)[3]) {
  c[2] = static_cast<int>(i % g.n[2]);
  const long long r = i / g.n[2];
  c[1] = static_cast<int>(r % g.n[1]);
  c[0] = static_cast<int>(r / g.n[1]);
}
// index of the neighbour s = +-1 cells along internal axis a (clamped along an open axis)
__device__ __forceinline__ long long nb(const Grid& g, const int (&c)[3], long long i, int a, int s) {
  const int v = g.open[a] ? clampi(c[a] + s, g.n[a]) : wrapv(c[a] + s, g.n[a]);
  long long stride = 1;
  for (int b = 2; b > a; --b) stride *= g.n[b];
  return i + static_cast<long long>(v - c[a]) * stride;
}

template <typename T>
__global__ void k_vip_cells(long long n, int nd, const T* __restrict__ state, T* __restrict__ uprev,
                            T* __restrict__ ext, bool first, T eps) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const T h = state[i];
    for (int d = 0; d < nd; ++d) {
      const T u = h > eps ? state[(1 + d) * n + i] / h : T(0);
      const T up = first ? u : uprev[d * n + i];
      ext[d * n + i] = T(1.5) * u - T(0.5) * up;
      uprev[d * n + i] = u;
    }
  }
}

template <typename T>
__global__ void k_vip_faces(Grid g, const T* __restrict__ ext, T* __restrict__ adv, T courant) {
  const long long n = g.N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    int c[3];
    coords(g, i, c);
    for (int d = 0; d < g.nd; ++d) {
      const int a = 3 - g.nd + d;
      const T* e = ext + d * n;
      adv[d * n + i] = T(0.5) * (e[i] + e[nb(g, c, i, a, +1)]) * courant;
    }
  }
}

template <typename T>
__global__ void k_sw_force(Grid g, T* __restrict__ state, T half_dt, T inv2dx) {
  const long long n = g.N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    int c[3];
    coords(g, i, c);
    const T h = state[i];
    for (int d = 0; d < g.nd; ++d) {
      const int a = 3 - g.nd + d;
      const T R = -h * (state[nb(g, c, i, a, +1)] - state[nb(g, c, i, a, -1)]) * inv2dx;
      state[(1 + d) * n + i] = state[(1 + d) * n + i] + half_dt * R;
    }
  }
}

unsigned blocks_of(long long n) {
  const long long b = (n + 255) / 256;
  return static_cast<unsigned>(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

}  // namespace

template <typename T>
cudaError_t vip_advector(const Grid& g, const T* state, T* uprev, T* ext, T* adv, bool first, T eps, T courant,
                         cudaStream_t st) {
  k_vip_cells<T><<<blocks_of(g.N), 256, 0, st>>>(g.N, g.nd, state, uprev, ext, first, eps);
  k_vip_faces<T><<<blocks_of(g.N), 256, 0, st>>>(g, ext, adv, courant);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sw_force(const Grid& g, T* state, T half_dt, T dx, cudaStream_t st) {
  k_sw_force<T><<<blocks_of(g.N), 256, 0, st>>>(g, state, half_dt, T(1) / (T(2) * dx));
  return cudaGetLastError();
}

template cudaError_t vip_advector<float>(const Grid&, const float*, float*, float*, float*, bool, float, float,
                                         cudaStream_t);
template cudaError_t vip_advector<double>(const Grid&, const double*, double*, double*, double*, bool, double,
                                          double, cudaStream_t);
template cudaError_t sw_force<float>(const Grid&, float*, float, float, cudaStream_t);
template cudaError_t sw_force<double>(const Grid&, double*, double, double, cudaStream_t);

}  // namespace mpd
