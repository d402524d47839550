// Adjoint (reverse mode) of one MPDATA step: given dL/dpsi^{n+1}, produce
// dL/dpsi^n and add dL/dGC to the advector adjoints.  The forward step is first
// recomputed on the staged kernels with every pass's intermediates kept
// (staged_forward_tape, or a tape the caller recorded); then the passes are
// reversed, last first:
//
//   ka_fct_a        (FCT) donor-cell pass k (Eqs. 4-5), the limiter V^ = V min(1, a, b)
//                   and the factors G[psi_max - psi]+/in, ...: gather over the cell's
//                   faces; scatters the flux adjoints (atomics)
//   ka_fct_b        (FCT) the unlimited fluxes of pass k, the antidiffusive advector
//                   (Eq. 6 + cross terms) and, after pass 2, the bounds over psi^n and
//                   psi^(1): scatter (atomics)
//   ka_donor_flux   (no FCT) donor-cell pass k: gather
//   ka_antidiff     (no FCT) antidiffusive advector: scatter (atomics)
// (the pseudo-advector's reverse has a second form, for the third-order terms, |psi| and the
// divergent-flow term)
//   ka_donor_flux   the first pass, which writes the step's outputs
//
// Adjoint arrays that receive scatters start at zero; the others are set by their
// first writer, so the order of the kernels is the reverse of the forward sub-steps.
// Conventions at the kinks: d[x]+/dx = d[x]-/dx = 1/2 at x = 0 (so d|x|/dx = 0
// there), a max/min passes the derivative of the first extremal candidate in the
// forward candidate order, the limiter's min(1, a, b) that of the first minimum.
// The Euler source terms (a given R added after or before the advection) enter only the one-call
// reverse step: the reverse passes psi_bar through the addition, euler_b reverses the step about
// psi^n + dt R, and dL/dR = dt psi_bar is accumulated where asked.
#include <cuda_runtime.h>

#include "kernels.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

template <typename T> __device__ __forceinline__ T posp(T x) { return x > T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T negp(T x) { return x < T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T dpos(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(0) : T(0.5)); }
template <typename T> __device__ __forceinline__ T dneg(T x) { return x < T(0) ? T(1) : (x > T(0) ? T(0) : T(0.5)); }
template <typename T> __device__ __forceinline__ T sgn(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0)); }
template <typename T> __device__ __forceinline__ T absv(T x) { return x < T(0) ? -x : x; }
// x > 0, x < 0, x != 0 and a < b: native for FP32 (x < 0 only in the generic templates above);
// FP64 on the integer pipe (the FP64 kernels are bound by the FP64 pipe; stencil2d.cuh), the
// same results for finite arguments up to the sign of a zero
__device__ __forceinline__ bool gtz(float x) { return x > 0.0f; }
__device__ __forceinline__ bool nez(float x) { return x != 0.0f; }
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool gtz(double x) { return dev::gt0(x); }
__device__ __forceinline__ bool ltz(double x) { return dev::lt0(x); }
__device__ __forceinline__ bool nez(double x) { return dev::nonzero(x); }
__device__ __forceinline__ bool lt(double a, double b) { return dev::order_key(a) < dev::order_key(b); }
template <> __device__ __forceinline__ double posp<double>(double x) { return gtz(x) ? x : 0.0; }
template <> __device__ __forceinline__ double negp<double>(double x) { return ltz(x) ? x : 0.0; }
template <> __device__ __forceinline__ double dpos<double>(double x) { return gtz(x) ? 1.0 : (ltz(x) ? 0.0 : 0.5); }
template <> __device__ __forceinline__ double dneg<double>(double x) { return ltz(x) ? 1.0 : (gtz(x) ? 0.0 : 0.5); }
template <> __device__ __forceinline__ double sgn<double>(double x) { return gtz(x) ? 1.0 : (ltz(x) ? -1.0 : 0.0); }
template <> __device__ __forceinline__ double absv<double>(double x) { return dev::absv(x); }
// n / d as in the forward kernels: fast division in FP32, Newton-Raphson division (within one
// ulp) in FP64; every divisor here is a G, a nonzero psi sum or a nonzero flux sum
template <typename T> __device__ __forceinline__ T adiv(T n, T d);
template <> __device__ __forceinline__ float adiv<float>(float n, float d) { return __fdividef(n, d); }
template <> __device__ __forceinline__ double adiv<double>(double n, double d) { return dev::nr_div(n, d); }

template <typename T> struct P3 { const T* p[3]; };
template <typename T> struct W3 { T* p[3]; };

struct Coord { int c[3]; };
__device__ __forceinline__ long long lin(const Grid& g, const Coord& x) {
  return (static_cast<long long>(x.c[0]) * g.n[1] + x.c[1]) * g.n[2] + x.c[2];
}
template <int ND>
__device__ __forceinline__ Coord sh(const Grid& g, Coord x, int d, int s) {
  const int a = 3 - ND + d;
  const int n = g.n[a];
  // |s| <= 2: two corrections each way wrap any extent n >= 1 (no loop)
  int v = x.c[a] + s;
  if (v < 0) v += n;
  if (v < 0) v += n;
  if (v >= n) v -= n;
  if (v >= n) v -= n;
  x.c[a] = v;
  return x;
}
inline dim3 cell_grid(const Grid& g, int bs) {
  return dim3(static_cast<unsigned>((g.n[2] + bs - 1) / bs), static_cast<unsigned>(g.n[1] < 65535 ? g.n[1] : 65535),
              static_cast<unsigned>(g.n[0] < 65535 ? g.n[0] : 65535));
}

// Linear index of a cell and the index offsets of its periodic neighbours (s = -2..2 along d);
// a diagonal neighbour is the sum of two offsets.
template <int ND>
struct Nbr {
  long long i;
  long long off[ND][5];
  __device__ __forceinline__ Nbr(const Grid& g, const Coord& x) {
    i = lin(g, x);
    long long stride = 1;
#pragma unroll
    for (int a = 2; a >= 0; --a) {
      const int d = a - (3 - ND);
      if (d >= 0) {
#pragma unroll
        for (int s = -2; s <= 2; ++s) off[d][s + 2] = (sh<ND>(g, x, d, s).c[a] - x.c[a]) * stride;
      }
      stride *= g.n[a];
    }
  }
  __device__ __forceinline__ long long at(int d, int s) const { return i + off[d][s + 2]; }
  __device__ __forceinline__ long long at2(int d, int s, int q, int t) const { return i + off[d][s + 2] + off[q][t + 2]; }
  __device__ __forceinline__ long long at3(int d, int s, int q, int t, int e, int u) const {
    return i + off[d][s + 2] + off[q][t + 2] + off[e][u + 2];
  }
};

// 2D: 32-bit cell indices (the reverse step refuses 2D fields of 2^31 cells or more) and the
// wrap of each neighbour formed from the cell's own row and column
template <>
struct Nbr<2> {
  int i;
  int off[2][5];
  __device__ __forceinline__ Nbr(const Grid& g, const Coord& x) {
    const int n1 = g.n[1], n2 = g.n[2], r = x.c[1], c = x.c[2];
    i = r * n2 + c;
#pragma unroll
    for (int s = -2; s <= 2; ++s) {
      int v = r + s;
      if (v < 0) v += n1;
      if (v < 0) v += n1;
      if (v >= n1) v -= n1;
      if (v >= n1) v -= n1;
      off[0][s + 2] = (v - r) * n2;
      int u = c + s;
      if (u < 0) u += n2;
      if (u < 0) u += n2;
      if (u >= n2) u -= n2;
      if (u >= n2) u -= n2;
      off[1][s + 2] = u - c;
    }
  }
  __device__ __forceinline__ int at(int d, int s) const { return i + off[d][s + 2]; }
  __device__ __forceinline__ int at2(int d, int s, int q, int t) const { return i + off[d][s + 2] + off[q][t + 2]; }
};

template <typename T> __device__ __forceinline__ T flux(T L, T R, T V, bool unit) {
  return unit ? V : posp(V) * L + negp(V) * R;
}

// Programmatic dependent launch: a kernel launched with launch_after() may start while its
// predecessor on the stream finishes; it calls grid_wait() before it reads anything the
// predecessor wrote (no-ops for kernels launched the ordinary way).  grid_release() lets the
// successor's launch begin as soon as every block of this grid has started.
__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... KArgs, typename... Args>
cudaError_t launch_after(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// loop over the cells on a (fast, middle, slow) launch grid; closed by CELL_END
#define CELL_INDEX                                                                    \
  for (int c0_ = blockIdx.z; c0_ < g.n[0]; c0_ += gridDim.z)                            \
    for (int c1_ = blockIdx.y; c1_ < g.n[1]; c1_ += gridDim.y)                          \
      for (int c2_ = blockIdx.x * blockDim.x + threadIdx.x; c2_ < g.n[2];               \
           c2_ += gridDim.x * blockDim.x) {                                           \
        const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});                                   \
        const auto i = nb.i;
#define CELL_END }

// Reverse of the donor-cell pass k, psi_k = psi_{k-1} + sum_d (F_{i-e_d} - F_i)/G_i with
// F = flux(psi_{k-1}, V^k): pb_prev += dL/dpsi_{k-1}, vhb[d] += dL/dV^k.  FINAL (the first
// pass, reversed last): the step's outputs are written here instead, psi_out = pb_prev +
// this pass's part, and gc_out[d] += vhb[d] + this pass's part (gc_out[d] may be null);
// then the cell's element of each of the nz arrays at zb (stride zn; they include pb_prev
// and vhb) is cleared for the next reverse step.
template <typename T, int ND, bool FINAL>
__global__ void ka_donor_flux(Grid g, const T* __restrict__ pb, const T* __restrict__ psi, P3<T> V,
                              const T* __restrict__ G, bool unit, T* pb_prev, W3<T> vhb, T* __restrict__ psi_out,
                              W3<T> gc_out, T* zb, int nz, long long zn) {
  grid_wait();
  CELL_INDEX
  const T gi = G ? adiv(pb[i], G[i]) : pb[i];
  T acc = pb[i];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const auto ip = nb.at(d, +1), im = nb.at(d, -1);
    const T gp = G ? adiv(pb[ip], G[ip]) : pb[ip];
    const T gm = G ? adiv(pb[im], G[im]) : pb[im];
    const T fp = gp - gi;  // dL/dF on the face (d, i)
    const T fm = gi - gm;  // dL/dF on the face (d, i - e_d)
    const T v = V.p[d][i], vm = V.p[d][im];
    T dv = T(1);
    if (!unit) {
      acc += fp * posp(v) + fm * negp(vm);
      dv = dpos(v) * psi[i] + dneg(v) * psi[ip];
    }
    if (!FINAL) {
      vhb.p[d][i] += fp * dv;
    } else if (gc_out.p[d]) {
      gc_out.p[d][i] += vhb.p[d][i] + fp * dv;
    }
  }
  if (FINAL) {
    psi_out[i] = pb_prev[i] + acc;
    for (int a = 0; a < nz; ++a) zb[a * zn + i] = T(0);
  } else {
    pb_prev[i] += acc;
  }
  CELL_END
}

// Reverse of the antidiffusive advector (Eq. 6 with the multi-D cross terms) on the face
// (d, i) for the adjoint gout of its output:
//   out = (|V| - V^2/Gb) A - sum_q 0.5 V Vq/Gb B_q,  A = (p1-p0)/(p0+p1),  B = (T-Bt)/(T+Bt)
// (A = (p1-p0)/2 and B = (T-Bt)/4 under infinite gauge); scatters to pb and vhb.
template <typename T, int ND>
__device__ __forceinline__ void antidiff_face_rev(const Nbr<ND>& nb, const decltype(Nbr<ND>::i) i, const int d, const T gout,
                                                  const T* __restrict__ psi, const P3<T>& Vin,
                                                  const T* __restrict__ G, const bool iga, T* pb, const W3<T>& vhb) {
  const auto ip = nb.at(d, +1);
  const T Gb = G ? T(0.5) * (G[i] + G[ip]) : T(1);
  const T V = Vin.p[d][i];
  const T p0 = psi[i], p1 = psi[ip];
  T A, dA0, dA1;
  if (iga) {
    A = (p1 - p0) * T(0.5); dA0 = T(-0.5); dA1 = T(0.5);
  } else {
    const T s = p0 + p1;
    if (dev::divisible(s)) {
      const T r = adiv(T(1), s);
      A = (p1 - p0) * r; dA0 = T(-2) * p1 * (r * r); dA1 = T(2) * p0 * (r * r);
    } else {
      A = dA0 = dA1 = T(0);
    }
  }
  const T rGb = G ? adiv(T(1), Gb) : T(1);
  const T c = absv(V) - V * V * rGb;
  T gV = gout * (sgn(V) - T(2) * V * rGb) * A;
  atomicAdd(&pb[i], gout * c * dA0);
  atomicAdd(&pb[ip], gout * c * dA1);
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    if (q == d) continue;
    const auto iqp = nb.at(q, +1), idqp = nb.at2(q, +1, d, +1);
    const auto iqm = nb.at(q, -1), idqm = nb.at2(q, -1, d, +1);
    const T* Q = Vin.p[q];
    const T Vq = T(0.25) * ((Q[i] + Q[ip]) + (Q[iqm] + Q[idqm]));
    const T Tp = psi[iqp] + psi[idqp], Bt = psi[iqm] + psi[idqm];
    T B, dBT, dBB;
    if (iga) {
      B = (Tp - Bt) * T(0.25); dBT = T(0.25); dBB = T(-0.25);
    } else {
      const T S = Tp + Bt;
      if (dev::divisible(S)) {
        const T r = adiv(T(1), S);
        B = (Tp - Bt) * r; dBT = T(2) * Bt * (r * r); dBB = T(-2) * Tp * (r * r);
      } else {
        B = dBT = dBB = T(0);
      }
    }
    gV += gout * (T(-0.5) * Vq * rGb * B);
    const T gq = gout * (T(-0.5) * V * rGb * B) * T(0.25);
    atomicAdd(&vhb.p[q][i], gq);
    atomicAdd(&vhb.p[q][ip], gq);
    atomicAdd(&vhb.p[q][iqm], gq);
    atomicAdd(&vhb.p[q][idqm], gq);
    const T gB = gout * (T(-0.5) * V * Vq * rGb);
    atomicAdd(&pb[iqp], gB * dBT);
    atomicAdd(&pb[idqp], gB * dBT);
    atomicAdd(&pb[iqm], gB * dBB);
    atomicAdd(&pb[idqm], gB * dBB);
  }
  atomicAdd(&vhb.p[d][i], gV);
}

// The same with the options the form above leaves out, selected at run time: |psi| in every
// psi-fraction (abs_psi, Sect. 3.1.5; d|psi|/dpsi = sgn psi, 0 at 0), the divergent-flow term
// (dfl, Sect. 3.1.3) -1/4 V (div_i + div_{i+e_d}) / Gb with div_j = sum_q (V_q at face j - at
// face j - e_q), and the third-order terms (tot, Sect. 3.1.2), with C = V/Gb and C_q = Vq/Gb:
//   + Gb (3 C|C| - 2 C^3 - C)/3 D_dd + sum_q Gb |C| C_q (1 - 2|C|) D_dq - (2/3) Gb C C_q1 C_q2 D_q1q2
// D_dd = (psi_{i+2} - psi_{i+1} - psi_i + psi_{i-1}) over their sum along d; D_dq = ((psi at
// i+e_d+e_q) - (i+e_q) - (i+e_d-e_q) + (i-e_q)) over their sum; D_q1q2 the same of the four
// pairs psi_j + psi_{j+e_d} at j = i +-e_q1 +-e_q2, signs (+,+) +, (+,-) -, (-,+) -, (-,-) +
// (over their count, 4, 4 and 8, under infinite gauge).  A fraction n/S of values with signs s_j
// in n has the derivatives (s_j - n/S)/S.  Scatters to pb and vhb.
template <typename T, int ND>
__device__ __forceinline__ void antidiff_face_rev_ext(const Nbr<ND>& nb, const decltype(Nbr<ND>::i) i, const int d,
                                                      const T gout, const T* __restrict__ psi, const P3<T>& Vin,
                                                      const T* __restrict__ G, const bool iga, const bool tot,
                                                      const bool abs_psi, const bool dfl, T* pb, const W3<T>& vhb) {
  using I = decltype(Nbr<ND>::i);
  auto ps = [&](I j) { return abs_psi ? absv(psi[j]) : psi[j]; };
  auto scat = [&](I j, T v) { atomicAdd(&pb[j], abs_psi ? v * sgn(psi[j]) : v); };
  // a fraction and its derivatives for the entries of sign +1 (kp) and -1 (km); cnt under infinite gauge
  auto fraction = [&](T n, T S, T cnt, T& D, T& kp, T& km) {
    if (iga) {
      D = n / cnt; kp = T(1) / cnt; km = T(-1) / cnt;
    } else if (dev::divisible(S)) {
      const T r = adiv(T(1), S);
      D = n * r; kp = (T(1) - D) * r; km = (T(-1) - D) * r;
    } else {
      D = kp = km = T(0);
    }
  };
  const auto ip = nb.at(d, +1);
  const T Gb = G ? T(0.5) * (G[i] + G[ip]) : T(1);
  const T V = Vin.p[d][i];
  const T p0 = ps(i), p1 = ps(ip);
  T A, dA0, dA1;
  if (iga) {
    A = (p1 - p0) * T(0.5); dA0 = T(-0.5); dA1 = T(0.5);
  } else {
    const T s = p0 + p1;
    if (dev::divisible(s)) {
      const T r = adiv(T(1), s);
      A = (p1 - p0) * r; dA0 = T(-2) * p1 * (r * r); dA1 = T(2) * p0 * (r * r);
    } else {
      A = dA0 = dA1 = T(0);
    }
  }
  const T rGb = G ? adiv(T(1), Gb) : T(1);
  const T c = absv(V) - V * V * rGb;
  T gV = gout * (sgn(V) - T(2) * V * rGb) * A;
  scat(i, gout * c * dA0);
  scat(ip, gout * c * dA1);
  const T aV = absv(V), sV = sgn(V);
  const T c2 = aV * rGb * (T(1) - T(2) * aV * rGb);     // the coefficient of Vq D_dq
  const T dc2 = sV * (rGb - T(4) * aV * (rGb * rGb));   // and its derivative in V
  T Vq[3] = {T(0), T(0), T(0)}, gVq[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    if (q == d) continue;
    const auto iqp = nb.at(q, +1), idqp = nb.at2(q, +1, d, +1);
    const auto iqm = nb.at(q, -1), idqm = nb.at2(q, -1, d, +1);
    const T* Q = Vin.p[q];
    Vq[q] = T(0.25) * ((Q[i] + Q[ip]) + (Q[iqm] + Q[idqm]));
    const T a = ps(iqp), b = ps(idqp), e = ps(iqm), f = ps(idqm);
    const T Tp = a + b, Bt = e + f;
    T B, dBT, dBB;
    if (iga) {
      B = (Tp - Bt) * T(0.25); dBT = T(0.25); dBB = T(-0.25);
    } else {
      const T S = Tp + Bt;
      if (dev::divisible(S)) {
        const T r = adiv(T(1), S);
        B = (Tp - Bt) * r; dBT = T(2) * Bt * (r * r); dBB = T(-2) * Tp * (r * r);
      } else {
        B = dBT = dBB = T(0);
      }
    }
    gV += gout * (T(-0.5) * Vq[q] * rGb * B);
    gVq[q] = gout * (T(-0.5) * V * rGb * B);
    const T gB = gout * (T(-0.5) * V * Vq[q] * rGb);
    T ga = gB * dBT, gb = gB * dBT, ge = gB * dBB, gf = gB * dBB;
    if (tot) {  // D_dq
      T D2, kp, km;
      fraction((b - a) - (f - e), (a + b) + (e + f), T(4), D2, kp, km);
      gV += gout * dc2 * Vq[q] * D2;
      gVq[q] += gout * c2 * D2;
      const T g2 = gout * c2 * Vq[q];
      gb += g2 * kp; ga += g2 * km; gf += g2 * km; ge += g2 * kp;
    }
    scat(iqp, ga);
    scat(idqp, gb);
    scat(iqm, ge);
    scat(idqm, gf);
  }
  if (tot) {
    {  // D_dd
      const auto im = nb.at(d, -1), ip2 = nb.at(d, +2);
      const T pm = ps(im), p2 = ps(ip2);
      T D, kp, km;
      fraction(((p2 - p1) - p0) + pm, ((p2 + p1) + p0) + pm, T(4), D, kp, km);
      const T cD = ((T(3) * V * aV) * rGb - (T(2) * V * V * V) * (rGb * rGb) - V) * (T(1) / T(3));
      gV += gout * ((T(6) * aV * rGb - T(6) * V * V * (rGb * rGb) - T(1)) * (T(1) / T(3))) * D;
      const T gd = gout * cD;
      scat(ip2, gd * kp);
      scat(ip, gd * km);
      scat(i, gd * km);
      scat(im, gd * kp);
    }
    if constexpr (ND == 3) {  // D_q1q2: q1 < q2 the two dimensions other than d
      const int q1 = d == 0 ? 1 : 0, q2 = d == 2 ? 1 : 2;
      const int s1[4] = {+1, +1, -1, -1}, s2[4] = {+1, -1, +1, -1};
      I j0[4], j1[4];
      T pr[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        j0[k] = nb.at2(q1, s1[k], q2, s2[k]);
        j1[k] = nb.at3(q1, s1[k], q2, s2[k], d, +1);
        pr[k] = ps(j0[k]) + ps(j1[k]);
      }
      T D3, kp, km;
      fraction((pr[0] - pr[1]) - (pr[2] - pr[3]), (pr[0] + pr[1]) + (pr[2] + pr[3]), T(8), D3, kp, km);
      const T w3 = T(-2) / T(3) * (rGb * rGb);
      gV += gout * (w3 * Vq[q1] * Vq[q2]) * D3;
      gVq[q1] += gout * (w3 * V * Vq[q2]) * D3;
      gVq[q2] += gout * (w3 * V * Vq[q1]) * D3;
      const T g3 = gout * (w3 * V * Vq[q1] * Vq[q2]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T gk = g3 * ((k == 0 || k == 3) ? kp : km);
        scat(j0[k], gk);
        scat(j1[k], gk);
      }
    }
  }
  if (dfl) {
    // the advector's differences across cells i and i+e_d (for q = d the face between them
    // enters both with opposite signs)
    T dsum = T(0);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const T* Q = Vin.p[q];
      const auto im_q = nb.at(q, -1);
      const auto ipm_q = q == d ? i : nb.at2(q, -1, d, +1);
      dsum = dsum + ((Q[i] - Q[im_q]) + (Q[ip] - Q[ipm_q]));
    }
    gV += gout * (T(-0.25) * dsum * rGb);
    const T gw = gout * (T(-0.25) * V * rGb);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      atomicAdd(&vhb.p[q][i], gw);
      atomicAdd(&vhb.p[q][nb.at(q, -1)], -gw);
      atomicAdd(&vhb.p[q][ip], gw);
      atomicAdd(&vhb.p[q][q == d ? i : nb.at2(q, -1, d, +1)], -gw);
    }
  }
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    if (q == d) continue;
    const T gq = gVq[q] * T(0.25);
    atomicAdd(&vhb.p[q][i], gq);
    atomicAdd(&vhb.p[q][ip], gq);
    atomicAdd(&vhb.p[q][nb.at(q, -1)], gq);
    atomicAdd(&vhb.p[q][nb.at2(q, -1, d, +1)], gq);
  }
  atomicAdd(&vhb.p[d][i], gV);
}

// Reverse of the antidiffusive advector of a pass without the limiter: vb holds the adjoint
// of its output on every face.
template <typename T, int ND, bool EXT>
__global__ void ka_antidiff(Grid g, P3<T> vb, const T* __restrict__ psi, P3<T> Vin, const T* __restrict__ G,
                            bool iga, bool tot, bool abs_psi, bool dfl, T* pb, W3<T> vhb) {
  CELL_INDEX
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const T gout = vb.p[d][i];
    if (nez(gout)) {
      if constexpr (EXT) antidiff_face_rev_ext<T, ND>(nb, i, d, gout, psi, Vin, G, iga, tot, abs_psi, dfl, pb, vhb);
      else antidiff_face_rev<T, ND>(nb, i, d, gout, psi, Vin, G, iga, pb, vhb);
    }
  }
  CELL_END
}

// The limiter's choice on the face between cells l and r = l + e_d:
// V^ = V min(1, a, b), a, b the factors of the upwind/downwind cells for the flux's direction;
// sel = 0 (the 1), 1 (a, a factor of l) or 2 (b, a factor of r), the first minimum.
template <typename T>
__device__ __forceinline__ T limit_choice(const T F, const T v, const T* __restrict__ bu, const T* __restrict__ bd,
                                          const long long l, const long long r, bool& right, int& sel) {
  right = gtz(F) || (!nez(F) && gtz(v));
  const T a = right ? bd[l] : bu[l];
  const T b = right ? bu[r] : bd[r];
  T m = T(1);
  sel = 0;
  if (lt(a, m)) { m = a; sel = 1; }
  if (lt(b, m)) { m = b; sel = 2; }
  return m;
}

// Reverse of corrective pass k under FCT, first half, per cell i: the donor-cell pass driven
// by the limited advector V^ (Eqs. 4-5), the limiter V^ = V min(1, a, b) and the factors
// beta_up = G[mx - psi]+/in, beta_dn = G[psi - mn]+/out (1 when the sum is 0; Sect. 3.1.4).
// V^ is re-derived from the unlimited advector and the limiter's choice (the product the
// forward formed).  The adjoint of V^ is formed on the cell's own faces (d, i) and on the
// faces (d, i - e_d) below it (donor part plus the scatter vhs of pass k + 1, nullable), so
// the factor adjoints of the cell are gathered from its 2 ND faces without atomics.  Writes
// pb_prev[i] = dL/dpsi^(k-1) of these sub-steps, vb[d][i] = dL/dV through the limiter, the
// bounds adjoints (set on the first pass reversed, accumulated on later ones), and scatters
// the adjoints of the unlimited fluxes into fb.  Branches follow the forward's choices.
template <typename T, int ND>
__global__ void ka_fct_a(Grid g, const T* __restrict__ pb, const T* __restrict__ psi, P3<T> Vu, P3<T> vhs,
                         const T* __restrict__ G, bool unit, const T* __restrict__ bu, const T* __restrict__ bd,
                         const T* __restrict__ mx, const T* __restrict__ mn, bool first, T* __restrict__ pb_prev,
                         W3<T> vb, T* __restrict__ mxb, T* __restrict__ mnb, W3<T> fb) {
  grid_wait();
  grid_release();
  CELL_INDEX
  const T p = psi[i];
  const T gi = G ? adiv(pb[i], G[i]) : pb[i];
  T acc = pb[i];
  T gu = T(0), gd = T(0);  // adjoints of beta_up and beta_dn of this cell
  T Fp[3], Fm[3];
  decltype(nb.i) im[3];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const auto ip = nb.at(d, +1);
    im[d] = nb.at(d, -1);
    const T pp = psi[ip], pm = psi[im[d]];
    const T v = Vu.p[d][i], vm = Vu.p[d][im[d]];
    Fp[d] = flux(p, pp, v, unit);
    Fm[d] = flux(pm, p, vm, unit);
    bool right, right_m;
    int sel, sel_m;
    const T m = limit_choice(Fp[d], v, bu, bd, i, ip, right, sel);               // this cell is l
    const T m_m = limit_choice(Fm[d], vm, bu, bd, im[d], i, right_m, sel_m);     // this cell is r
    const T vh = v * m, vhm = vm * m_m;
    const T gp = G ? adiv(pb[ip], G[ip]) : pb[ip];
    const T gm = G ? adiv(pb[im[d]], G[im[d]]) : pb[im[d]];
    const T fp = gp - gi;  // dL/dF on the face (d, i)
    const T fm = gi - gm;  // dL/dF on the face (d, i - e_d)
    T dv = T(1), dvm = T(1);
    if (!unit) {
      acc += fp * posp(vh) + fm * negp(vhm);
      dv = dpos(vh) * p + dneg(vh) * pp;
      dvm = dpos(vhm) * pm + dneg(vhm) * p;
    }
    T gq = fp * dv, gqm = fm * dvm;  // dL/dV^ on the two faces
    if (vhs.p[d]) { gq += vhs.p[d][i]; gqm += vhs.p[d][im[d]]; }
    vb.p[d][i] = gq * m;
    if (sel == 1) (right ? gd : gu) += gq * v;
    if (sel_m == 2) (right_m ? gu : gd) += gqm * vm;
  }
  T in = T(0), ou = T(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    in = in + (posp(Fm[d]) - negp(Fp[d]));
    ou = ou + (posp(Fp[d]) - negp(Fm[d]));
  }
  const T Gi = G ? G[i] : T(1);
  T gin = T(0), gout = T(0), pacc = T(0), dmx = T(0), dmn = T(0);
  if (gtz(in) && nez(gu)) {
    const T beta = adiv(Gi * posp(mx[i] - p), in);
    const T t = adiv(gu * Gi * dpos(mx[i] - p), in);
    dmx = t;
    pacc -= t;
    gin = adiv(-gu * beta, in);
  }
  if (gtz(ou) && nez(gd)) {
    const T beta = adiv(Gi * posp(p - mn[i]), ou);
    const T t = adiv(gd * Gi * dpos(p - mn[i]), ou);
    pacc += t;
    dmn = -t;
    gout = adiv(-gd * beta, ou);
  }
  if (nez(gin) || nez(gout)) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      atomicAdd(&fb.p[d][i], -gin * dneg(Fp[d]) + gout * dpos(Fp[d]));
      atomicAdd(&fb.p[d][im[d]], gin * dpos(Fm[d]) - gout * dneg(Fm[d]));
    }
  }
  pb_prev[i] = acc + pacc;
  mxb[i] = first ? dmx : mxb[i] + dmx;
  mnb[i] = first ? dmn : mnb[i] + dmn;
  CELL_END
}

// Reverse of the FCT bounds at cell i: the adjoint of each extremum goes to its first extremal
// candidate (order: the cell, then per dimension its -e_d and +e_d neighbours; psi^n before
// psi^(1)).
template <typename T, int ND>
__device__ __forceinline__ void bounds_rev(const Nbr<ND>& nb, const decltype(Nbr<ND>::i) i, const T gmx, const T gmn,
                                           const T* __restrict__ p0, const T* __restrict__ p1, T* pb0, T* pb1) {
  decltype(Nbr<ND>::i) loc[7];
  int nl = 0;
  loc[nl++] = i;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    loc[nl++] = nb.at(d, -1);
    loc[nl++] = nb.at(d, +1);
  }
  T hi = p0[i], lo = p0[i];
  int ha = 0, la = 0;
  auto hj = i, lj = i;
  for (int j = 0; j < nl; ++j) {
    const T a = p0[loc[j]], b = p1[loc[j]];
    if (lt(hi, a)) { hi = a; ha = 0; hj = loc[j]; }
    if (lt(hi, b)) { hi = b; ha = 1; hj = loc[j]; }
    if (lt(a, lo)) { lo = a; la = 0; lj = loc[j]; }
    if (lt(b, lo)) { lo = b; la = 1; lj = loc[j]; }
  }
  if (nez(gmx)) atomicAdd(ha == 0 ? &pb0[hj] : &pb1[hj], gmx);
  if (nez(gmn)) atomicAdd(la == 0 ? &pb0[lj] : &pb1[lj], gmn);
}

// Reverse of corrective pass k under FCT, second half, per cell i: the unlimited fluxes
// F = flux(psi^(k-1), V) that fed the factors (adjoints fb, complete after ka_fct_a), which
// complete dL/dV on the face (d, i) with the limiter's part vbl, then the antidiffusive
// advector that produced V (Eq. 6, scattered into pb and vhb).  On the last pass reversed
// (mxb not null) also the bounds over psi^n = p0 and psi^(1) = psi.
template <typename T, int ND, bool EXT>
__global__ void ka_fct_b(Grid g, P3<T> fb, P3<T> vbl, const T* __restrict__ psi, P3<T> Vu, P3<T> Vin,
                         const T* __restrict__ G, bool unit, bool tot, bool abs_psi, bool dfl, T* pb, W3<T> vhb,
                         const T* __restrict__ mxb, const T* __restrict__ mnb, const T* __restrict__ p0, T* pb0) {
  grid_wait();
  grid_release();
  CELL_INDEX
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const auto ip = nb.at(d, +1), im = nb.at(d, -1);
    const T fp = fb.p[d][i], fm = fb.p[d][im];
    const T v = Vu.p[d][i], vm = Vu.p[d][im];
    T dv = T(1);
    if (!unit) {
      acc += fp * posp(v) + fm * negp(vm);
      dv = dpos(v) * psi[i] + dneg(v) * psi[ip];
    }
    const T gout = vbl.p[d][i] + fp * dv;
    if (nez(gout)) {
      if constexpr (EXT) antidiff_face_rev_ext<T, ND>(nb, i, d, gout, psi, Vin, G, unit, tot, abs_psi, dfl, pb, vhb);
      else antidiff_face_rev<T, ND>(nb, i, d, gout, psi, Vin, G, unit, pb, vhb);
    }
  }
  if (nez(acc)) atomicAdd(&pb[i], acc);
  if (mxb) bounds_rev<T, ND>(nb, i, mxb[i], mnb[i], p0, psi, pb0, pb);
  CELL_END
}

template <typename T>
__global__ void ka_accumulate(long long n, const T* __restrict__ src, T* __restrict__ dst) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// dst += a x (the source adjoint dL/dR = dt psi_bar)
template <typename T>
__global__ void ka_axpy(long long n, T a, const T* __restrict__ x, T* __restrict__ dst) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] += a * x[i];
}

// psi^0 = psi^n + dt R of a step with the euler_b source (the forward's pre-add, same expression)
template <typename T>
__global__ void ka_pre(long long n, const T* __restrict__ psi, const T* __restrict__ r, T dt, T* __restrict__ out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = psi[i] + dt * r[i];
}

// Arrays of one step's tape: psi levels 1..K-1, the unlimited pseudo-advectors of passes
// 2..K and, under FCT, the limited ones, the bounds and the factors.
size_t tape_arrays(int K, int D, bool fct) {
  size_t n = static_cast<size_t>(K - 1) * (1 + D);
  if (fct) n += static_cast<size_t>(D) * (K - 1) + 2 + 2 * (K - 1);
  return n;
}

// Arrays of the reverse sweep: psi adjoints 0..K-1, advector adjoints of passes 1..K and,
// under FCT, the unlimited-advector (limiter part), flux and bounds adjoints.
size_t adj_arrays(int K, int D, bool fct) {
  size_t n = static_cast<size_t>(K) * (1 + D);
  if (fct) n += static_cast<size_t>(D) * (K - 1) + D + 2;
  return n;
}

// The tape of one step carved from `base` (tape_arrays(...) arrays of N elements).
template <typename T>
void carve_tape(T* base, long long N, int K, int D, bool fct, const T* psi_n, const T* const* gc, Tape<T>& tp,
                T** levels) {
  T* cur = base;
  auto take = [&]() { T* q = cur; cur += N; return q; };
  tp = Tape<T>{};
  for (int k = 0; k < kTapeMax; ++k) levels[k] = nullptr;
  tp.psi[0] = psi_n;
  for (int k = 1; k < K; ++k) { levels[k] = take(); tp.psi[k] = levels[k]; }
  for (int d = 0; d < 3; ++d) tp.vh[1][d] = d < D ? gc[d] : nullptr;
  for (int k = 2; k <= K; ++k)
    for (int d = 0; d < D; ++d) tp.v[k][d] = take();
  if (fct) {
    for (int k = 2; k <= K; ++k)
      for (int d = 0; d < D; ++d) tp.vh[k][d] = take();
    tp.mx = take();
    tp.mn = take();
    for (int k = 2; k <= K; ++k) { tp.bu[k] = take(); tp.bd[k] = take(); }
  } else {
    for (int k = 2; k <= K; ++k)
      for (int d = 0; d < D; ++d) tp.vh[k][d] = tp.v[k][d];
  }
}

// The handle's adjoint scratch: size, device pointer, and where its zero-initialised arrays
// started when the last call left them cleared (null when not known to be clear).
struct AdjScratch {
  size_t bytes;
  void* ptr;
  void* clean;
};

// What one call does: the whole reverse step (tape recomputed into the handle's scratch),
// only the tape (into the caller's buffer, plus the step's result), or only the reverse
// sweep from a tape the caller recorded.
enum class AdjMode { kStep, kRecord, kReplay };

// R, dt, r_bar: the Euler source of the step (one-call reverse step only; R null without one).
template <typename T, int ND>
int adjoint_nd(mpdata_s* h, const Grid& g, const Opts& o, const T* psi_n, const T* const* gc, const T* G,
               T* psi_bar, void* const* gc_bar, cudaStream_t st, AdjMode mode = AdjMode::kStep,
               T* tape = nullptr, T* psi_next = nullptr, const T* R = nullptr, T dt = T(0), T* r_bar = nullptr) {
  const int K = o.n_iters, D = ND;
  const long long N = g.N;
  Tape<T> tp{};
  T* levels[kTapeMax];
  if (mode == AdjMode::kRecord) {
    if constexpr (ND == 2) {
      // 2D: one launch of the fused step writes the tape and the step's result
      if (!o.staged && psi_next) {
        const StepArgs<T> a{psi_n, psi_next, {gc[0], gc[1], nullptr}, nullptr, nullptr, T(0), T(1)};
        const int rc = fused_tape<T>(g, o, a, tape, st);
        if (rc != MPDATA_EUNSUPPORTED) return rc;
      }
    }
    carve_tape<T>(tape, N, K, D, o.fct, psi_n, gc, tp, levels);
    if (staged_forward_tape<T>(g, o, gc, G, tp, levels, psi_next, st) != cudaSuccess) return MPDATA_ECUDA;
    return MPDATA_OK;
  }
  // the one-call reverse step keeps its tape (and the recorded step's unused result, and under
  // euler_b the advected state psi^n + dt R) in the scratch
  const size_t tape_n = mode == AdjMode::kStep ? tape_arrays(K, D, o.fct) + 1 + (o.rhs_b ? 1 : 0) : 0;
  const size_t need = (tape_n + adj_arrays(K, D, o.fct)) * static_cast<size_t>(N) * sizeof(T);
  void** slot = handle_adj(h);
  // the adjoint scratch is allocated on first use and kept with the handle
  AdjScratch* hdr = static_cast<AdjScratch*>(*slot);
  if (hdr == nullptr || hdr->bytes < need) {
    if (hdr) { cudaFree(hdr->ptr); delete hdr; *slot = nullptr; }
    hdr = new AdjScratch{need, nullptr, nullptr};
    if (cudaMalloc(&hdr->ptr, need) != cudaSuccess) { delete hdr; return MPDATA_ENOMEM; }
    *slot = hdr;
  }
  // the adjoint arrays first, so that they sit at the same place whether or not the tape is
  // kept in the scratch too (behind them)
  T* cur = static_cast<T*>(hdr->ptr);
  T* const tape_base = mode == AdjMode::kStep ? cur + adj_arrays(K, D, o.fct) * static_cast<size_t>(N) : tape;
  const int bs0 = 256;
  const unsigned nb0 = static_cast<unsigned>((N + bs0 - 1) / bs0);
  if (mode == AdjMode::kStep && o.rhs_b) {  // the step advects psi^n + dt R: its tape starts there
    T* const p0 = tape_base + (tape_arrays(K, D, o.fct) + 1) * static_cast<size_t>(N);
    ka_pre<T><<<nb0, bs0, 0, st>>>(N, psi_n, R, dt, p0);
    psi_n = p0;
  }
  // euler_a: dL/dR = dt dL/dpsi^{n+1}, taken before the sweep overwrites psi_bar
  if (mode == AdjMode::kStep && o.rhs_a && r_bar) ka_axpy<T><<<nb0, bs0, 0, st>>>(N, dt, psi_bar, r_bar);
  carve_tape<T>(tape_base, N, K, D, o.fct, psi_n, gc, tp, levels);
  auto take = [&]() { T* q = cur; cur += N; return q; };
  // adjoint arrays: first those that only receive atomic scatters (zeroed), then those
  // whose first writer sets them
  T* const adj_begin = cur;
  T* pbl[kTapeMax];
  pbl[0] = take();
  T* vhb[kTapeMax + 1][3] = {};
  for (int k = 1; k < K; ++k)
    for (int d = 0; d < D; ++d) vhb[k][d] = take();
  T* fb[3] = {nullptr, nullptr, nullptr};
  if (o.fct)
    for (int d = 0; d < D; ++d) fb[d] = take();
  T* const dirty_end = cur;  // under FCT the reverse sweep never writes vhb[K]: it stays zero
  for (int d = 0; d < D; ++d) vhb[K][d] = take();
  T* const zero_end = cur;
  for (int k = 1; k < K; ++k) pbl[k] = take();
  T* vbk[kTapeMax + 1][3] = {};
  T *mxb = nullptr, *mnb = nullptr;
  if (o.fct) {
    for (int k = 2; k <= K; ++k)
      for (int d = 0; d < D; ++d) vbk[k][d] = take();
    mxb = take();
    mnb = take();
  }
  // Without the limiter the donor-cell reverse accumulates into every psi adjoint, which are
  // cleared on every call.  With it only the arrays before zero_end must start at zero, and
  // the last kernel of every call clears them again, so only the first call on a scratch
  // buffer clears them (a CUDA graph captured after that first call holds no memset).
  const bool chain = o.fct && K >= 2;
  T* const zero_to = o.fct ? zero_end : cur;
  if (!chain || hdr->clean != adj_begin) {
    if (cudaMemsetAsync(adj_begin, 0, static_cast<size_t>(zero_to - adj_begin) * sizeof(T), st) != cudaSuccess)
      return MPDATA_ECUDA;
  }
  hdr->clean = nullptr;
  if (mode == AdjMode::kStep) {
    int rc = MPDATA_EUNSUPPORTED;
    if constexpr (ND == 2) {
      if (!o.staged) {
        T* const unused = tape_base + tape_arrays(K, D, o.fct) * static_cast<size_t>(N);
        const StepArgs<T> a{psi_n, unused, {gc[0], gc[1], nullptr}, nullptr, nullptr, T(0), T(1)};
        rc = fused_tape<T>(g, o, a, tape_base, st);
      }
    }
    if (rc == MPDATA_EUNSUPPORTED)
      rc = staged_forward_tape<T>(g, o, gc, G, tp, levels, nullptr, st) == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
    if (rc != MPDATA_OK) return rc;
  }

  const int bs = 256;
  const unsigned nb = static_cast<unsigned>((N + bs - 1) / bs);
  // the pseudo-advector's reverse with the third-order terms, |psi| or the divergent-flow term
  const bool ext = o.tot || o.abs || o.dfl;
  for (int k = K; k >= 2; --k) {
    const T* pbk = (k == K) ? psi_bar : pbl[k];
    P3<T> vh{{tp.vh[k][0], tp.vh[k][1], tp.vh[k][2]}};
    P3<T> vu{{tp.v[k][0], tp.v[k][1], tp.v[k][2]}};
    P3<T> vprev{{tp.vh[k - 1][0], tp.vh[k - 1][1], tp.vh[k - 1][2]}};
    W3<T> vhbp{{vhb[k - 1][0], vhb[k - 1][1], vhb[k - 1][2]}};
    if (o.fct) {
      // two kernels per pass: donor pass + limiter + factors (gather), then the unlimited
      // fluxes + antidiffusive advector (+ the bounds on the last pass reversed)
      if (k < K && cudaMemsetAsync(fb[0], 0, static_cast<size_t>(N) * D * sizeof(T), st) != cudaSuccess)
        return MPDATA_ECUDA;
      P3<T> vhs{{k < K ? vhb[k][0] : nullptr, k < K ? vhb[k][1] : nullptr, k < K ? vhb[k][2] : nullptr}};
      W3<T> vbw{{vbk[k][0], vbk[k][1], vbk[k][2]}};
      W3<T> fbw{{fb[0], fb[1], fb[2]}};
      if (launch_after(ka_fct_a<T, ND>, cell_grid(g, bs), dim3(bs), st, g, pbk, tp.psi[k - 1], vu, vhs, G,
                       static_cast<bool>(o.iga), tp.bu[k], tp.bd[k], tp.mx, tp.mn, k == K, pbl[k - 1], vbw, mxb,
                       mnb, fbw) != cudaSuccess)
        return MPDATA_ECUDA;
      P3<T> fbr{{fb[0], fb[1], fb[2]}};
      P3<T> vbr{{vbk[k][0], vbk[k][1], vbk[k][2]}};
      const bool last = k == 2;
      if (launch_after(ext ? ka_fct_b<T, ND, true> : ka_fct_b<T, ND, false>, cell_grid(g, bs), dim3(bs), st, g, fbr,
                       vbr, tp.psi[k - 1], vu, vprev, G, static_cast<bool>(o.iga), static_cast<bool>(o.tot),
                       static_cast<bool>(o.abs), static_cast<bool>(o.dfl), pbl[k - 1], vhbp, last ? mxb : nullptr,
                       last ? mnb : nullptr,
                       tp.psi[0], pbl[0]) != cudaSuccess)
        return MPDATA_ECUDA;
    } else {
      W3<T> vhbk{{vhb[k][0], vhb[k][1], vhb[k][2]}};
      ka_donor_flux<T, ND, false><<<cell_grid(g, bs), bs, 0, st>>>(g, pbk, tp.psi[k - 1], vh, G, o.iga, pbl[k - 1],
                                                                   vhbk, nullptr, W3<T>{}, nullptr, 0, 0);
      P3<T> gv{{vhb[k][0], vhb[k][1], vhb[k][2]}};  // dL/dV^k of the advector the antidiff produced
      if (ext)
        ka_antidiff<T, ND, true><<<cell_grid(g, bs), bs, 0, st>>>(g, gv, tp.psi[k - 1], vprev, G, o.iga, o.tot, o.abs,
                                                                  o.dfl, pbl[k - 1], vhbp);
      else
        ka_antidiff<T, ND, false><<<cell_grid(g, bs), bs, 0, st>>>(g, gv, tp.psi[k - 1], vprev, G, o.iga, false, false,
                                                                   false, pbl[k - 1], vhbp);
    }
  }
  P3<T> v1{{gc[0], D > 1 ? gc[1] : nullptr, D > 2 ? gc[2] : nullptr}};
  W3<T> vhb1{{vhb[1][0], vhb[1][1], vhb[1][2]}};
  if (K >= 2) {
    // the first pass, reversed last, writes the step's outputs: psi_bar (consumed by pass K
    // already) and gc_bar
    W3<T> out{{nullptr, nullptr, nullptr}};
    for (int d = 0; d < D; ++d) out.p[d] = gc_bar ? static_cast<T*>(gc_bar[d]) : nullptr;
    if (launch_after(ka_donor_flux<T, ND, true>, cell_grid(g, bs), dim3(bs), st, g, pbl[1], tp.psi[0], v1, G, false,
                     pbl[0], vhb1, psi_bar, out, adj_begin, static_cast<int>((dirty_end - adj_begin) / N), N) !=
        cudaSuccess)
      return MPDATA_ECUDA;
    if (chain) hdr->clean = adj_begin;
  } else {
    // one pass: psi_bar is this kernel's input, so the result goes through scratch
    ka_donor_flux<T, ND, false><<<cell_grid(g, bs), bs, 0, st>>>(g, psi_bar, tp.psi[0], v1, G, false, pbl[0], vhb1,
                                                                 nullptr, W3<T>{}, nullptr, 0, 0);
    if (cudaMemcpyAsync(psi_bar, pbl[0], static_cast<size_t>(N) * sizeof(T), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return MPDATA_ECUDA;
    if (gc_bar)
      for (int d = 0; d < D; ++d)
        if (gc_bar[d]) ka_accumulate<T><<<nb, bs, 0, st>>>(N, vhb[1][d], static_cast<T*>(gc_bar[d]));
  }
  // euler_b: dL/dR = dt dL/dpsi^0 = dt dL/dpsi^n
  if (mode == AdjMode::kStep && o.rhs_b && r_bar) ka_axpy<T><<<nb, bs, 0, st>>>(N, dt, psi_bar, r_bar);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template <typename T>
int adjoint_dispatch(mpdata_s* h, const T* psi_n, const void* const* gcv, const T* g, T* psi_bar,
                     void* const* gc_bar, AdjMode mode, T* tape, T* psi_next, const T* R = nullptr, T dt = T(0),
                     T* r_bar = nullptr) {
  Opts o = make_opts(handle_opts(h), handle_n_iters(h));
  handle_tuning(h, &o.kernel, &o.tile_rows);  // the fused recording follows the forward's kernel
  // the Euler sources only in the one-call reverse step, which is given R
  if (((o.rhs_a || o.rhs_b) && (mode != AdjMode::kStep || !R)) || o.n_iters > kTapeMax) return MPDATA_EUNSUPPORTED;
  const Grid& gr = handle_grids(h)[0];
  if (gr.nd == 2 && gr.N >= (1LL << 31)) return MPDATA_EUNSUPPORTED;  // 32-bit indices of Nbr<2>
  const T* gc[3] = {static_cast<const T*>(gcv[0]), gr.nd > 1 ? static_cast<const T*>(gcv[1]) : nullptr,
                    gr.nd > 2 ? static_cast<const T*>(gcv[2]) : nullptr};
  const T* G = o.nug ? g : nullptr;
  cudaStream_t st = handle_stream(h);
  switch (gr.nd) {
    case 1: return adjoint_nd<T, 1>(h, gr, o, psi_n, gc, G, psi_bar, gc_bar, st, mode, tape, psi_next, R, dt, r_bar);
    case 2: return adjoint_nd<T, 2>(h, gr, o, psi_n, gc, G, psi_bar, gc_bar, st, mode, tape, psi_next, R, dt, r_bar);
    case 3: return adjoint_nd<T, 3>(h, gr, o, psi_n, gc, G, psi_bar, gc_bar, st, mode, tape, psi_next, R, dt, r_bar);
  }
  return MPDATA_EINVAL;
}

}  // namespace

void adjoint_free(mpdata_s* h) {
  void** slot = handle_adj(h);
  AdjScratch* hdr = static_cast<AdjScratch*>(*slot);
  if (hdr) {
    cudaFree(hdr->ptr);
    delete hdr;
    *slot = nullptr;
  }
}

size_t adjoint_tape_bytes(mpdata_s* h, size_t esize) {
  const Opts o = make_opts(handle_opts(h), handle_n_iters(h));
  const Grid& gr = handle_grids(h)[0];
  return tape_arrays(o.n_iters, gr.nd, o.fct) * static_cast<size_t>(gr.N) * esize;
}

template <typename T>
int adjoint_step(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, T* psi_bar, void* const* gc_bar) {
  return adjoint_dispatch<T>(h, psi_n, gc, g, psi_bar, gc_bar, AdjMode::kStep, nullptr, nullptr);
}

template <typename T>
int adjoint_step_rhs(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, const T* r, T dt, T* psi_bar,
                     void* const* gc_bar, T* r_bar) {
  return adjoint_dispatch<T>(h, psi_n, gc, g, psi_bar, gc_bar, AdjMode::kStep, nullptr, nullptr, r, dt, r_bar);
}

template <typename T>
int adjoint_record(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, T* tape, T* psi_next) {
  return adjoint_dispatch<T>(h, psi_n, gc, g, nullptr, nullptr, AdjMode::kRecord, tape, psi_next);
}

template <typename T>
int adjoint_replay(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, const T* tape, T* psi_bar,
                   void* const* gc_bar) {
  return adjoint_dispatch<T>(h, psi_n, gc, g, psi_bar, gc_bar, AdjMode::kReplay, const_cast<T*>(tape), nullptr);
}

template int adjoint_step<float>(mpdata_s*, const float*, const void* const*, const float*, float*, void* const*);
template int adjoint_step<double>(mpdata_s*, const double*, const void* const*, const double*, double*, void* const*);
template int adjoint_step_rhs<float>(mpdata_s*, const float*, const void* const*, const float*, const float*, float,
                                     float*, void* const*, float*);
template int adjoint_step_rhs<double>(mpdata_s*, const double*, const void* const*, const double*, const double*,
                                      double, double*, void* const*, double*);
template int adjoint_record<float>(mpdata_s*, const float*, const void* const*, const float*, float*, float*);
template int adjoint_record<double>(mpdata_s*, const double*, const void* const*, const double*, double*, double*);
template int adjoint_replay<float>(mpdata_s*, const float*, const void* const*, const float*, const float*, float*,
                                   void* const*);
template int adjoint_replay<double>(mpdata_s*, const double*, const void* const*, const double*, const double*,
                                    double*, void* const*);

}  // namespace mpd
