// Trapezoidal (Crank-Nicolson) source scheme of Sect. 4.1,
//   psi^{n+1} = ADV(psi^n + dt/2 R^n) + dt/2 R^{n+1},
// for a system of equations whose sources are affine in the state, R = A psi + b per cell
// (A: E x E constant, b: a field per equation).  R^{n+1} makes the scheme implicit: per cell
// (I - dt/2 A) psi^{n+1} = psi* + dt/2 b with psi* = ADV(psi^n + dt/2 R^n) (for the translating
// oscillator of Sect. 4.2 this is the closed form given there).  The advection itself runs on
// the usual kernels between the two element-wise kernels below.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace mpd {
namespace {

template <typename T>
__global__ void k_trapez_pre(const TrapezMat m, long long n, T half_dt, const T* __restrict__ psi,
                             const T* __restrict__ b, T* __restrict__ out) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    T x[kTrapezMax];
#pragma unroll
    for (int f = 0; f < kTrapezMax; ++f) x[f] = f < m.E ? psi[f * n + i] : T(0);
#pragma unroll
    for (int e = 0; e < kTrapezMax; ++e) {
      if (e >= m.E) break;
      T R = T(0);
#pragma unroll
      for (int f = 0; f < kTrapezMax; ++f)
        if (f < m.E) R = R + static_cast<T>(m.A[e * kTrapezMax + f]) * x[f];
      if (b) R = R + b[e * n + i];
      out[e * n + i] = x[e] + half_dt * R;
    }
  }
}

template <typename T>
__global__ void k_trapez_post(const TrapezMat m, long long n, T half_dt, const T* __restrict__ b,
                              T* __restrict__ psi) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    T y[kTrapezMax];
#pragma unroll
    for (int f = 0; f < kTrapezMax; ++f) {
      y[f] = f < m.E ? psi[f * n + i] : T(0);
      if (b && f < m.E) y[f] = y[f] + half_dt * b[f * n + i];
    }
#pragma unroll
    for (int e = 0; e < kTrapezMax; ++e) {
      if (e >= m.E) break;
      T s = T(0);
#pragma unroll
      for (int f = 0; f < kTrapezMax; ++f)
        if (f < m.E) s = s + static_cast<T>(m.Minv[e * kTrapezMax + f]) * y[f];
      psi[e * n + i] = s;
    }
  }
}

unsigned blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return static_cast<unsigned>(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

bool trapez_matrix(TrapezMat& m, const double* A, int E, double dt) {
  if (E < 1 || E > kTrapezMax) return false;
  m.E = E;
  double M[kTrapezMax][2 * kTrapezMax];
  for (int e = 0; e < kTrapezMax; ++e)
    for (int f = 0; f < kTrapezMax; ++f) {
      const double a = (e < E && f < E) ? A[e * E + f] : 0.0;
      m.A[e * kTrapezMax + f] = a;
      m.Minv[e * kTrapezMax + f] = 0.0;
    }
  // [I - dt/2 A | I] -> [I | (I - dt/2 A)^{-1}]
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 2 * E; ++f)
      M[e][f] = f < E ? (e == f ? 1.0 : 0.0) - 0.5 * dt * A[e * E + f] : (f - E == e ? 1.0 : 0.0);
  for (int c = 0; c < E; ++c) {
    int piv = c;
    for (int r = c + 1; r < E; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (!(std::fabs(M[piv][c]) > 0.0)) return false;
    if (piv != c)
      for (int f = 0; f < 2 * E; ++f) { const double t = M[c][f]; M[c][f] = M[piv][f]; M[piv][f] = t; }
    const double inv = 1.0 / M[c][c];
    for (int f = 0; f < 2 * E; ++f) M[c][f] *= inv;
    for (int r = 0; r < E; ++r) {
      if (r == c || M[r][c] == 0.0) continue;
      const double q = M[r][c];
      for (int f = 0; f < 2 * E; ++f) M[r][f] -= q * M[c][f];
    }
  }
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < E; ++f) m.Minv[e * kTrapezMax + f] = M[e][E + f];
  return true;
}

template <typename T>
cudaError_t trapez_pre(const TrapezMat& m, long long n, T dt, const T* psi, const T* b, T* out, cudaStream_t st) {
  k_trapez_pre<T><<<blocks_for(n), 256, 0, st>>>(m, n, T(0.5) * dt, psi, b, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t trapez_post(const TrapezMat& m, long long n, T dt, const T* b, T* psi, cudaStream_t st) {
  k_trapez_post<T><<<blocks_for(n), 256, 0, st>>>(m, n, T(0.5) * dt, b, psi);
  return cudaGetLastError();
}

template cudaError_t trapez_pre<float>(const TrapezMat&, long long, float, const float*, const float*, float*,
                                       cudaStream_t);
template cudaError_t trapez_pre<double>(const TrapezMat&, long long, double, const double*, const double*, double*,
                                        cudaStream_t);
template cudaError_t trapez_post<float>(const TrapezMat&, long long, float, const float*, float*, cudaStream_t);
template cudaError_t trapez_post<double>(const TrapezMat&, long long, double, const double*, double*, cudaStream_t);

}  // namespace mpd
