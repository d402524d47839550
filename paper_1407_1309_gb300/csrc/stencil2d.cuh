// Device helpers shared by the fused 2D kernels (fused2d.cu, band2d.cu): the
// donor-cell flux of Eq. 5, the guarded psi-fraction of Eq. 6, the donor update
// of Eq. 4, cp.async wrappers and the lane-neighbour shuffles of a row held as
// NC adjacent columns per lane.
#pragma once

#include <cuda_runtime.h>

namespace mpd {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int wrapi(int c, int n) {
  int r = c % n;
  return r < 0 ? r + n : r;
}

template <typename T> __device__ __forceinline__ T fdiv(T a, T b);
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
// FP64 n / d for the arithmetic-bound FP64 kernels: Newton-Raphson reciprocal iteration
// r <- r + r (1 - d r) (quadratic convergence) from the PTX approximate FP64 reciprocal
// (rcp.approx.ftz.f64, full exponent range), two iterations, and Markstein's remainder
// correction q <- q + r (n - d q) of the quotient: within one unit in the last place of the
// exact quotient for normal operands.  A zero, infinite or NaN divisor gives NaN (the
// kernels never rely on it: the psi-ratio guards zero sums, and the FCT factors' min(1, x)
// maps the inf or NaN of a zero flux sum to 1 alike).
__device__ __forceinline__ double nr_div(double n, double d) {
  double r0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(d));
  double e = fma(-d, r0, 1.0);
  double r = fma(r0, e, r0);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  const double q = n * r;
  return fma(r, fma(-d, q, n), q);
}
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return nr_div(a, b); }

template <typename T> __device__ __forceinline__ T posp(T x) { return x > T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T negp(T x) { return x < T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T absv(T x) { return x < T(0) ? -x : x; }
template <typename T> __device__ __forceinline__ T maxv(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T minv(T a, T b) { return a < b ? a : b; }
// min(1, x); a NaN x gives 1 (fmin returns the non-NaN operand)
__device__ __forceinline__ float min1(float x) { return fminf(1.0f, x); }
__device__ __forceinline__ double min1(double x) { return fmin(1.0, x); }
// donor-cell flux (Eq. 5) in advector units: [V]+ L + [V]- R, one term of which is zero
template <typename T> __device__ __forceinline__ T flux(T L, T R, T V) { return V * (V > T(0) ? L : R); }
// A divisor the fast divisions can take: not zero and not below the smallest normal number (their
// approximate reciprocals flush such a divisor to zero).  A psi-sum that small counts as zero in
// the guard of the psi-fraction: the fraction it would give changes no flux by more than that.
__device__ __forceinline__ bool divisible(float d) { return fabsf(d) >= 1.17549435e-38f; }
__device__ __forceinline__ bool divisible(double d) { return ((__double_as_longlong(d) >> 52) & 0x7FF) != 0; }

// psi-fraction of Eq. 6 with the zero-denominator guard
template <typename T> __device__ __forceinline__ T ratio(T n, T d) { return divisible(d) ? fdiv(n, d) : T(0); }

// x > 0 (the upwind choice of a flux, the limiter's direction)
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }

// FP64: sign tests, extrema and magnitudes on the integer pipe.  GB300's FP64 pipe runs at a
// small fraction of the FP32 rate and bounds the FP64 step, so the operations that need no
// FP64 arithmetic (comparisons with zero, ordering of two values, |x|) are taken off it.  For
// finite arguments they give the floating-point forms' results, up to the sign of a zero
// result (an ordering key makes -0 < +0).
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool lt0(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool nonzero(double x) { return (__double_as_longlong(x) << 1) != 0; }
// a signed integer in the order of the doubles (finite arguments)
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
template <> __device__ __forceinline__ double posp<double>(double x) { return gt0(x) ? x : 0.0; }
template <> __device__ __forceinline__ double negp<double>(double x) { return lt0(x) ? x : 0.0; }
template <> __device__ __forceinline__ double absv<double>(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL);
}
template <> __device__ __forceinline__ double maxv<double>(double a, double b) { return order_key(a) > order_key(b) ? a : b; }
template <> __device__ __forceinline__ double minv<double>(double a, double b) { return order_key(a) < order_key(b) ? a : b; }
template <> __device__ __forceinline__ double flux<double>(double L, double R, double V) { return V * (gt0(V) ? L : R); }


template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& comp, T t) {
  const T y = t - comp;
  const T u = s + y;
  comp = (u - s) - y;
  s = u;
}

// Donor-cell update of Eq. 4 from the four face fluxes, rG = 1/G.  The flux
// differences are added first and psi last, so only one rounding happens at the
// scale of psi; with the Kahan option the terms psi - Fp0 + Fm0 - Fp1 + Fm1 are
// summed in that order with compensation instead.
template <typename T, bool NUG, bool KAHAN>
__device__ __forceinline__ T donor(T p, T Fp0, T Fm0, T Fp1, T Fm1, T rG) {
  if (KAHAN) {
    if (NUG) {
      Fp0 *= rG;
      Fm0 *= rG;
      Fp1 *= rG;
      Fm1 *= rG;
    }
    T s = p, comp = T(0);
    kahan_add(s, comp, -Fp0);
    kahan_add(s, comp, Fm0);
    kahan_add(s, comp, -Fp1);
    kahan_add(s, comp, Fm1);
    return s;
  }
  const T div = (Fm0 - Fp0) + (Fm1 - Fp1);
  return NUG ? p + div * rG : p + div;
}

// s + t = u + err exactly (Knuth's two-sum, no magnitude condition); s <- u, e += err.
template <typename T>
__device__ __forceinline__ void two_sum_acc(T& s, T& e, T t) {
  const T u = s + t;
  const T bp = u - s;
  const T err = (s - (u - bp)) + (t - bp);
  s = u;
  e = e + err;
}

// Donor-cell update of Eq. 4 on a compensated state psi = hi + lo: the flux divergence of
// the high parts is formed in FP32 as in the plain update (fluxes differenced first), added to
// hi with a two-sum whose rounding error joins lo together with the low parts' own flux
// divergence (lo_div), and the pair is renormalised so that the returned hi is the value of
// the representable sum nearest hi + lo.  The rounding of psi + divergence, at the scale of
// psi, is the one that biases the plain FP32 state over long runs; it is kept exactly.
// lo_div: the divergence of the low parts' own face fluxes (added to lo, scaled by 1/G).
template <typename T, bool NUG>
__device__ __forceinline__ T donor_comp(T p, T lo, T Fp0, T Fm0, T Fp1, T Fm1, T rG, T lo_div, T& lo_out) {
  T div = (Fm0 - Fp0) + (Fm1 - Fp1);
  if (NUG) {
    div *= rG;
    lo_div *= rG;
  }
  const T s = p + div;
  const T bp = s - p;
  const T err = (p - (s - bp)) + (div - bp);
  const T e = (lo + lo_div) + err;
  // renormalise with a full two-sum: after cancellation |e| may exceed |s|
  const T h = s + e;
  const T bq = h - s;
  lo_out = (s - (h - bq)) + (e - bq);
  return h;
}

// A row of NC columns held by one lane; the columns just outside come from the
// neighbouring lanes.
template <typename T, int NC> __device__ __forceinline__ T from_left(const T (&a)[NC]) {
  return __shfl_up_sync(kFull, a[NC - 1], 1);
}
template <typename T, int NC> __device__ __forceinline__ T from_right(const T (&a)[NC]) {
  return __shfl_down_sync(kFull, a[0], 1);
}
template <typename T, int NC> __device__ __forceinline__ T left_of(const T (&a)[NC], int c, T aL) {
  return c == 0 ? aL : a[c > 0 ? c - 1 : 0];
}
template <typename T, int NC> __device__ __forceinline__ T right_of(const T (&a)[NC], int c, T aR) {
  return c == NC - 1 ? aR : a[c < NC - 1 ? c + 1 : NC - 1];
}
template <typename T, int N> __device__ __forceinline__ void copy_row(T (&d)[N], const T (&s)[N]) {
#pragma unroll
  for (int c = 0; c < N; ++c) d[c] = s[c];
}

}  // namespace dev
}  // namespace mpd
