// Staged MPDATA step: one kernel per sub-step over the whole field, with the
// intermediates of the step in library-owned device scratch.
//
// This path handles every dimension (1-3) and every option combination; the
// fused tile kernels (fused2d.cu) take over the cases they cover.  It is also
// the forward recomputation that the adjoint kernels reverse.
//
// Sub-steps (paper Sect. 3.1.1, 3.1.2, 3.1.4, 3.1.5, 4.1):
//   pre      psi0 = psi + dt R                           (euler_b)
//   donor    psi_k = psi_{k-1} - F_{i+1/2}/G + F_{i-1/2}/G per dimension (Eqs. 4-5)
//   bounds   FCT extrema of psi0 and psi1 over the cell and its face neighbours
//   antidiff pseudo-advector of Eq. 6 with multi-D cross and third-order terms
//   beta     FCT in/out flux sums and limiting factors
//   limit    limited advector
#include <cuda_runtime.h>

#include "internal.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

template <typename T> __device__ __forceinline__ T posp(T x) { return x > T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T negp(T x) { return x < T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T absv(T x) { return x < T(0) ? -x : x; }
// n / d: FP32 uses the fast division (rcp and multiply, 2 ulp), FP64 the Newton-Raphson
// division with remainder correction of stencil2d.cuh (within 1 ulp; NaN for a zero divisor,
// which the callers guard or map to a factor of 1)
template <typename T> __device__ __forceinline__ T qdiv(T n, T d);
template <> __device__ __forceinline__ float qdiv<float>(float n, float d) { return __fdividef(n, d); }
template <> __device__ __forceinline__ double qdiv<double>(double n, double d) { return dev::nr_div(n, d); }
// psi-fraction with the zero-denominator guard (the ratio of Eq. 6 is 0 when its sum is 0)
// (a divisor below the smallest normal number counts as zero: stencil2d.cuh)
template <typename T> __device__ __forceinline__ T fracg(T n, T d) { return dev::divisible(d) ? qdiv(n, d) : T(0); }
// FP64: the sign tests, extrema and |x| on the integer pipe (stencil2d.cuh)
template <> __device__ __forceinline__ double posp<double>(double x) { return dev::gt0(x) ? x : 0.0; }
template <> __device__ __forceinline__ double negp<double>(double x) { return dev::lt0(x) ? x : 0.0; }
template <> __device__ __forceinline__ double absv<double>(double x) { return dev::absv(x); }
// extrema (the first argument on ties) and the limiter's direction, through the same helpers
template <typename T> __device__ __forceinline__ T maxe(T a, T b) { return dev::maxv(a, b); }
template <typename T> __device__ __forceinline__ T mine(T a, T b) { return dev::minv(a, b); }
__device__ __forceinline__ bool goes_right(float F, float V) { return F > 0.0f || (F == 0.0f && V > 0.0f); }
__device__ __forceinline__ bool goes_right(double F, double V) {
  return dev::gt0(F) || (!dev::nonzero(F) && dev::gt0(V));
}
// a flux sum that takes a limiting factor (0 or a subnormal sum gives the factor 1: the FP64
// division has no reciprocal of a subnormal, and such a sum cannot move the cell's value)
__device__ __forceinline__ bool factor_sum(float x) { return x > 0.0f; }
__device__ __forceinline__ bool factor_sum(double x) { return dev::gt0(x) && dev::divisible(x); }

template <typename T> struct In3 { const T* p[3]; };
template <typename T> struct Out3 { T* p[3]; };

struct Coord { int c[3]; };

__device__ __forceinline__ long long lin(const Grid& g, const Coord& x) {
  return (static_cast<long long>(x.c[0]) * g.n[1] + x.c[1]) * g.n[2] + x.c[2];
}
// cell x moved by s cells along dimension d: periodic, or clamped to the edge cell along an
// open dimension (the halo beyond an open edge holds the edge value, Sect. 2.4)
template <int ND>
__device__ __forceinline__ Coord sh(const Grid& g, Coord x, int d, int s) {
  const int a = 3 - ND + d;
  const int n = g.n[a];
  int v = x.c[a] + s;
  if (g.open[a]) {
    v = v < 0 ? 0 : (v > n - 1 ? n - 1 : v);
  } else {
    // |s| <= 2: two corrections each way wrap any extent n >= 1 (no loop)
    if (v < 0) v += n;
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if (v >= n) v -= n;
  }
  x.c[a] = v;
  return x;
}

// storage position of face x_d + s + 1/2 of a vector component along its own dimension d:
// periodic, or, along an open dimension, clamped to the interior faces 0 .. n-2 (a boundary
// face carries the adjacent interior face's value: the zero-divergence condition, Sect. 2.4)
template <int ND>
__device__ __forceinline__ int face_pos(const Grid& g, const Coord& x, int d, int s) {
  const int a = 3 - ND + d;
  const int n = g.n[a];
  int v = x.c[a] + s;
  if (g.open[a]) return v < 0 ? 0 : (v > n - 2 ? n - 2 : v);
  if (v < 0) v += n;
  if (v >= n) v -= n;
  return v;
}

// Loop over the cells of a field launched on a (fast, middle, slow) grid: coordinates come
// from the block indices, so no division is needed.
#define FOR_CELLS(g)                                                                  \
  for (int c0_ = blockIdx.z; c0_ < (g).n[0]; c0_ += gridDim.z)                          \
    for (int c1_ = blockIdx.y; c1_ < (g).n[1]; c1_ += gridDim.y)                        \
      for (int c2_ = blockIdx.x * blockDim.x + threadIdx.x; c2_ < (g).n[2];             \
           c2_ += gridDim.x * blockDim.x)

inline dim3 cell_grid(const Grid& g, int bs) {
  const unsigned gx = static_cast<unsigned>((g.n[2] + bs - 1) / bs);
  const unsigned gy = static_cast<unsigned>(g.n[1] < 65535 ? g.n[1] : 65535);
  const unsigned gz = static_cast<unsigned>(g.n[0] < 65535 ? g.n[0] : 65535);
  return dim3(gx, gy, gz);
}

inline dim3 march3_grid(const Grid& g);

// Linear index of a cell and the index offsets of its neighbours: off[d][s+2] moves s = -2..2
// cells along dimension d (wrapped, or clamped along an open dimension); fo[d][s+1] moves to
// the storage of face x_d + s + 1/2 of the component along d, s = -1..1 (face_pos).  Shifts
// along different dimensions are independent, so a diagonal neighbour, or the q-face of a
// neighbour along d, is the sum of two offsets.
template <int ND>
struct Nbr {
  long long i;
  long long off[ND][5];
  long long fo[ND][3];
  __device__ __forceinline__ Nbr(const Grid& g, const Coord& x) {
    i = lin(g, x);
    long long stride = 1;
#pragma unroll
    for (int a = 2; a >= 0; --a) {
      const int d = a - (3 - ND);
      if (d >= 0) {
#pragma unroll
        for (int s = -2; s <= 2; ++s) off[d][s + 2] = (sh<ND>(g, x, d, s).c[a] - x.c[a]) * stride;
#pragma unroll
        for (int s = -1; s <= 1; ++s) fo[d][s + 1] = (face_pos<ND>(g, x, d, s) - x.c[a]) * stride;
      }
      stride *= g.n[a];
    }
  }
  __device__ __forceinline__ long long at(int d, int s) const { return i + off[d][s + 2]; }
  __device__ __forceinline__ long long at2(int d, int s, int q, int t) const { return i + off[d][s + 2] + off[q][t + 2]; }
  // face x_d + s + 1/2 of the component along d, of this cell or of the cell j on its row
  __device__ __forceinline__ long long face(int d, int s) const { return i + fo[d][s + 1]; }
  __device__ __forceinline__ long long face_of(long long j, int d, int s) const { return j + fo[d][s + 1]; }
};

// donor-cell flux of Eq. 5 in advector units; psi -> 1 under infinite gauge
template <typename T>
__device__ __forceinline__ T flux(T L, T R, T V, bool unit) {
  return unit ? V : posp(V) * L + negp(V) * R;
}

template <typename T>
__global__ void k_pre(long long N, const T* __restrict__ psi, const T* __restrict__ r, T dt,
                      T* __restrict__ out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < N) out[i] = psi[i] + dt * r[i];
}

// Donor-cell pass (Eqs. 4-5): psi_i - F_{i+1/2}/G_i + F_{i-1/2}/G_i, dimension 0 first,
// optionally with compensated (Kahan) summation; euler_a source added when post.
template <typename T, int ND>
__global__ void k_donor(Grid g, const T* __restrict__ psi, In3<T> V, T vscale, bool unit,
                        const T* __restrict__ G, bool kahan, const T* __restrict__ R, T dt,
                        bool post, T* __restrict__ out) {
  FOR_CELLS(g) {
  const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});
  const long long i = nb.i;
  const T p = psi[i];
  T s = p, comp = T(0);
  const T Gi = G ? G[i] : T(1);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const long long ip = nb.at(d, +1);
    const long long im = nb.at(d, -1);
    const T vp = V.p[d][nb.face(d, 0)] * vscale, vm = V.p[d][nb.face(d, -1)] * vscale;
    const T Fp = flux(p, psi[ip], vp, unit);
    const T Fm = flux(psi[im], p, vm, unit);
    const T t0 = G ? -qdiv(Fp, Gi) : -Fp;
    const T t1 = G ? qdiv(Fm, Gi) : Fm;
    if (kahan) {
      T y = t0 - comp;
      T u = s + y;
      comp = (u - s) - y;
      s = u;
      y = t1 - comp;
      u = s + y;
      comp = (u - s) - y;
      s = u;
    } else {
      s = s + t0;
      s = s + t1;
    }
  }
  if (post) s = s + dt * R[i];
  out[i] = s;
  }
}

// FCT bounds (Sect. 3.1.4): extrema of psi0 and psi1 over the cell and its face neighbours.
template <typename T, int ND>
__global__ void k_bounds(Grid g, const T* __restrict__ p0, const T* __restrict__ p1,
                         T* __restrict__ mx, T* __restrict__ mn) {
  FOR_CELLS(g) {
  const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});
  const long long i = nb.i;
  T hi = p0[i] > p1[i] ? p0[i] : p1[i];
  T lo = p0[i] < p1[i] ? p0[i] : p1[i];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
#pragma unroll
    for (int s = -1; s <= 1; s += 2) {
      const long long j = nb.at(d, s);
      const T a = p0[j], b = p1[j];
      hi = maxe(a, hi);
      hi = maxe(b, hi);
      lo = mine(a, lo);
      lo = mine(b, lo);
    }
  }
  mx[i] = hi;
  mn[i] = lo;
  }
}

// Antidiffusive pseudo-advector of pass k at every face i+1/2 of cell i (Eq. 6 with the
// multi-D cross terms, Sect. 3.1.1, and the third-order terms, Sect. 3.1.2):
//   (|V| - V^2/Gb) A - sum_q 0.5 V Vq/Gb B_q
//   + tot: Gb(3C|C| - 2C^3 - C)/3 D_dd + sum_q Gb|C|C_q(1 - 2|C|) D_dq - (2/3) Gb C C_q1 C_q2 D_q1q2
//   + dfl: -1/4 V (div_i + div_{i+e_d}) / Gb       (divergent flow, Sect. 3.1.3)
// with C = V/Gb, C_q = Vq/Gb; each psi ratio is a difference over the sum of the psi
// values it uses (over their count under infinite gauge; of their magnitudes with abs_psi,
// Sect. 3.1.5).
template <typename T, int ND>
__global__ void k_antidiff(Grid g, const T* __restrict__ psi, In3<T> Vin, T vscale,
                           const T* __restrict__ G, bool iga, bool tot, bool abs_psi, bool dfl, Out3<T> Vout) {
  // variable-sign option (Sect. 3.1.5): psi enters every psi-fraction as |psi|
  auto ps = [&](long long j) { const T v = psi[j]; return abs_psi ? absv(v) : v; };
  FOR_CELLS(g) {
  const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});
  const long long i = nb.i;
  const T p0 = ps(i);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const long long ip = nb.at(d, +1);
    // every 1/Gb of the face is one reciprocal, multiplied in
    const T rGb = G ? qdiv(T(1), T(0.5) * (G[i] + G[ip])) : T(1);
    const T V = Vin.p[d][nb.face(d, 0)] * vscale;
    const T p1 = ps(ip);
    const T A = iga ? (p1 - p0) * T(0.5) : fracg(p1 - p0, p0 + p1);
    T out = (absv(V) - V * V * rGb) * A;
    T Vq[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      if (q == d) continue;
      const long long iqp = nb.at(q, +1), idqp = nb.at2(q, +1, d, +1);
      const long long iqm = nb.at(q, -1), idqm = nb.at2(q, -1, d, +1);
      const T* Q = Vin.p[q];
      // the q-faces q+1/2 and q-1/2 of cells i and i+e_d
      Vq[q] = T(0.25) * ((Q[nb.face(q, 0)] * vscale + Q[nb.face_of(ip, q, 0)] * vscale) +
                         (Q[nb.face(q, -1)] * vscale + Q[nb.face_of(ip, q, -1)] * vscale));
      const T Tp = ps(iqp) + ps(idqp);
      const T Bt = ps(iqm) + ps(idqm);
      const T B = iga ? (Tp - Bt) * T(0.25) : fracg(Tp - Bt, Tp + Bt);
      out = out - T(0.5) * V * Vq[q] * rGb * B;
    }
    if (tot) {
      const T pm = ps(nb.at(d, -1));
      const T p2 = ps(nb.at(d, +2));
      const T num = ((p2 - p1) - p0) + pm;
      const T D = iga ? num * T(0.25) : fracg(num, ((p2 + p1) + p0) + pm);
      out = out + ((T(3) * V * absv(V)) * rGb - (T(2) * V * V * V) * (rGb * rGb) - V) * T(1.0 / 3.0) * D;
      int qs[2] = {0, 0}, nq = 0;
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        if (q == d) continue;
        qs[nq++] = q;
        const T a = ps(nb.at(q, +1)), b = ps(nb.at2(q, +1, d, +1));
        const T e = ps(nb.at(q, -1)), f = ps(nb.at2(q, -1, d, +1));
        const T n2 = (b - a) - (f - e);
        const T D2 = iga ? n2 * T(0.25) : fracg(n2, (a + b) + (e + f));
        out = out + absv(V) * Vq[q] * rGb * (T(1) - T(2) * absv(V) * rGb) * D2;
      }
      if (ND == 3) {
        T pr[4];
        int m = 0;
#pragma unroll
        for (int s1 = 1; s1 >= -1; s1 -= 2) {
#pragma unroll
          for (int s2 = 1; s2 >= -1; s2 -= 2) {
            const long long y = nb.i + nb.off[qs[0]][s1 + 2] + nb.off[qs[1]][s2 + 2];
            pr[m++] = ps(y) + ps(y + nb.off[d][3]);
          }
        }
        // pr = {(+,+), (+,-), (-,+), (-,-)}
        const T n3 = (pr[0] - pr[1]) - (pr[2] - pr[3]);
        const T D3 = iga ? n3 * T(0.125) : fracg(n3, (pr[0] + pr[1]) + (pr[2] + pr[3]));
        out = out - (T(2) / T(3)) * V * Vq[qs[0]] * Vq[qs[1]] * (rGb * rGb) * D3;
      }
    }
    if (dfl) {
      // divergent-flow term (Sect. 3.1.3): -1/4 V (div_i + div_{i+e_d}) / Gb, div_j the sum over
      // the dimensions of the advector's difference across cell j
      T div = T(0);
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        const T* Q = Vin.p[q];
        // faces q+1/2 and q-1/2 of cell i, then of cell i+e_d (along q == d: faces x+3/2, x+1/2)
        const long long a0 = nb.face(q, 0), a1 = nb.face(q, -1);
        const long long b0 = q == d ? nb.face(d, +1) : nb.face_of(ip, q, 0);
        const long long b1 = q == d ? nb.face(d, 0) : nb.face_of(ip, q, -1);
        div = div + ((Q[a0] * vscale - Q[a1] * vscale) + (Q[b0] * vscale - Q[b1] * vscale));
      }
      out = out - T(0.25) * V * div * rGb;
    }
    Vout.p[d][i] = out;
  }
  }
}

// The same pseudo-advector for 3D fields as a z-march: a block owns a 32 x 8 tile of
// (x, y) and walks down a chunk of z-planes, keeping rings of planes with their halos in
// shared memory: psi on planes z-1 .. z+2 with x, y in [-1, +2] around the tile (the
// third-order stencil reaches psi_{i-1} .. psi_{i+2} along the face's dimension and one
// cell across it), the advector components and G on two planes with a one-cell halo.
// Each cell's three faces are formed from the planes with the arithmetic of k_antidiff
// (same expressions, same order).
constexpr int kAx = 32, kAy = 8, kAz = 16;  // tile and z-chunk of the 3D march
constexpr int kPw = kAx + 3, kPh = kAy + 3;  // psi plane with halo [-1, +2]
constexpr int kVw = kAx + 2, kVh = kAy + 2;  // advector / G plane with halo [-1, +1]

inline dim3 march3_grid(const Grid& g) {
  return dim3(static_cast<unsigned>((g.n[2] + kAx - 1) / kAx), static_cast<unsigned>((g.n[1] + kAy - 1) / kAy),
              static_cast<unsigned>((g.n[0] + kAz - 1) / kAz));
}

__device__ __forceinline__ int wrapc(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// rings of the z-march, one slot more than the planes in use so that the next step's
// planes can be copied (cp.async) while this step computes
constexpr int kA3P = 5, kA3V = 3;
template <typename T>
constexpr size_t antidiff3_smem() {
  return sizeof(T) * (kA3P * kPw * kPh + (3 + 1) * kA3V * kVw * kVh);
}

// guarded psi-fractions n1/d and n2/d with one denominator (0 when d == 0): in FP32 one
// approximate reciprocal serves both quotients; FP64 divides each with the remainder-corrected
// Newton-Raphson division
template <typename T>
__device__ __forceinline__ void frac2(T n1, T n2, T d, T& r1, T& r2) {
  if constexpr (sizeof(T) == 4) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(d));
    r1 = dev::divisible(d) ? n1 * r : T(0);
    r2 = dev::divisible(d) ? n2 * r : T(0);
  } else {
    r1 = fracg(n1, d);
    r2 = fracg(n2, d);
  }
}

// s + j modulo n, for 0 <= s, j < n (ring slots)
__device__ __forceinline__ int rot(int s, int j, int n) {
  const int v = s + j;
  return v >= n ? v - n : v;
}

template <typename T, bool ABS>
__global__ void __launch_bounds__(kAx * kAy) k_antidiff3(Grid g, const T* __restrict__ psi, In3<T> Vin,
                                                         T vscale, const T* __restrict__ G, bool iga, bool tot,
                                                         Out3<T> Vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int nP = kPw * kPh, nV = kVw * kVh;
  T* const sP = reinterpret_cast<T*>(smem_raw);  // [kA3P][nP]
  T* const sV = sP + kA3P * nP;                   // [3 dimensions][kA3V][nV]
  T* const sG = sV + 3 * kA3V * nV;               // [kA3V][nV]
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kAx + tx;
  constexpr int kT = kAx * kAy;
  const int x0 = blockIdx.x * kAx, y0 = blockIdx.y * kAy;
  const int zb = blockIdx.z * kAz;
  const int ze = zb + kAz < nz ? zb + kAz : nz;
  const long long plane = static_cast<long long>(ny) * nx;

  // Every plane is copied with the same element assignment: this thread copies tile
  // elements tid and tid + kT (when they exist); their in-plane source offsets are fixed.
  static_assert(nP <= 2 * kT && nV <= 2 * kT, "two elements per thread cover a plane");
  int offP[2], offV[2];
  const bool hasP1 = tid + kT < nP, hasV1 = tid + kT < nV;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = tid + r * kT;
    int yy = k / kPw;
    offP[r] = wrapc(y0 - 1 + yy, ny) * nx + wrapc(x0 - 1 + (k - yy * kPw), nx);
    yy = k / kVw;
    offV[r] = wrapc(y0 - 1 + yy, ny) * nx + wrapc(x0 - 1 + (k - yy * kVw), nx);
  }
  auto zoff = [&](int z) { return static_cast<long long>(wrapc(z, nz)) * plane; };
  auto copyP = [&](T* dst, long long zo) {
    const T* src = psi + zo;
    dev::cp_async<sizeof(T)>(dst + tid, src + offP[0]);
    if (hasP1) dev::cp_async<sizeof(T)>(dst + tid + kT, src + offP[1]);
  };
  auto copyV = [&](T* dst, const T* base, long long zo) {
    const T* src = base + zo;
    dev::cp_async<sizeof(T)>(dst + tid, src + offV[0]);
    if (hasV1) dev::cp_async<sizeof(T)>(dst + tid + kT, src + offV[1]);
  };
  // after its copy has landed, this thread scales the advector elements it copied
  auto scaleV = [&](T* dst) {
    dst[tid] *= vscale;
    if (hasV1) dst[tid + kT] *= vscale;
  };
  // Ring slots, advanced by one at every step z: the psi planes z-1 .. z+2 are in slots
  // cp .. cp+3 (mod kA3P, the fifth takes plane z+3 in flight); the z component planes z-1, z in
  // cz, cz+1 (mod kA3V; z+1 in flight); the y, x components and G planes z, z+1 in cq, cq+1
  // (z+2 in flight).
  int cp = 0, cz = 0, cq = 0;
  auto Vzs = [&](int s) { return sV + s * nV; };
  auto Vys = [&](int s) { return sV + (kA3V + s) * nV; };
  auto Vxs = [&](int s) { return sV + (2 * kA3V + s) * nV; };
  auto Gs = [&](int s) { return sG + s * nV; };

  {  // prologue: psi planes zb-1 .. zb+2, z component zb-1, zb, the others and G zb, zb+1
    for (int j = 0; j < 4; ++j) copyP(sP + j * nP, zoff(zb - 1 + j));
    copyV(Vzs(0), Vin.p[0], zoff(zb - 1));
    copyV(Vzs(1), Vin.p[0], zoff(zb));
    for (int j = 0; j < 2; ++j) {
      const long long zo = zoff(zb + j);
      copyV(Vys(j), Vin.p[1], zo);
      copyV(Vxs(j), Vin.p[2], zo);
      if (G) copyV(Gs(j), G, zo);
    }
    dev::cp_commit();
    dev::cp_wait<0>();
    if (vscale != T(1)) {
      for (int j = 0; j < 2; ++j) {
        scaleV(Vzs(j));
        scaleV(Vys(j));
        scaleV(Vxs(j));
      }
    }
  }

  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < nx && y < ny;
  const int cP = (ty + 1) * kPw + (tx + 1), cV = (ty + 1) * kVw + (tx + 1);  // this cell in a plane
  const long long row = static_cast<long long>(y) * nx + x;
  for (int z = zb; z < ze; ++z) {
    __syncthreads();  // step z's planes are in (each thread waited for its own copies)
    const int fp = rot(cp, 4, kA3P), fz = rot(cz, 2, kA3V), fq = rot(cq, 2, kA3V);  // in-flight slots
    if (z + 1 < ze) {  // the next step's planes fly while this one computes
      copyP(sP + fp * nP, zoff(z + 3));
      copyV(Vzs(fz), Vin.p[0], zoff(z + 1));
      const long long zo = zoff(z + 2);
      copyV(Vys(fq), Vin.p[1], zo);
      copyV(Vxs(fq), Vin.p[2], zo);
      if (G) copyV(Gs(fq), G, zo);
    }
    dev::cp_commit();
    if (inside) {
      // this cell's position in each plane of the rings; every neighbour below is a fixed
      // offset from one of these
      const T* pz[4] = {sP + cp * nP + cP, sP + rot(cp, 1, kA3P) * nP + cP, sP + rot(cp, 2, kA3P) * nP + cP,
                        sP + rot(cp, 3, kA3P) * nP + cP};
      const int cq1 = rot(cq, 1, kA3V);
      const T* vz[2] = {Vzs(cz) + cV, Vzs(rot(cz, 1, kA3V)) + cV};  // z component, planes z-1, z
      const T* vy[2] = {Vys(cq) + cV, Vys(cq1) + cV};               // y component, planes z, z+1
      const T* vx[2] = {Vxs(cq) + cV, Vxs(cq1) + cV};               // x component, planes z, z+1
      const T* gz[2] = {Gs(cq) + cV, Gs(cq1) + cV};
      // ABS, the variable-sign option (Sect. 3.1.5): psi enters every psi-fraction as |psi|
      auto P = [&](int dz, int dy, int dx) {
        const T v = pz[dz + 1][dy * kPw + dx];
        if constexpr (ABS) return absv(v);
        else return v;
      };
      auto Q = [&](int q, int dz, int dy, int dx) {
        return q == 0 ? vz[dz + 1][dy * kVw + dx] : (q == 1 ? vy[dz][dy * kVw + dx] : vx[dz][dy * kVw + dx]);
      };
      auto Gv = [&](int dz, int dy, int dx) { return gz[dz][dy * kVw + dx]; };
      const T p0 = P(0, 0, 0);
      T res[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // unit offsets of dimension d (0 = z, 1 = y, 2 = x)
        const int dz = d == 0, dy = d == 1, dx = d == 2;
        const T rGb = G ? qdiv(T(1), T(0.5) * (Gv(0, 0, 0) + Gv(dz, dy, dx))) : T(1);
        const T V = Q(d, 0, 0, 0);
        const T p1 = P(dz, dy, dx);
        const T A = iga ? (p1 - p0) * T(0.5) : fracg(p1 - p0, p0 + p1);
        T out = (absv(V) - V * V * rGb) * A;
        T Vq[3] = {T(0), T(0), T(0)};
        T Dq[3] = {T(0), T(0), T(0)};  // the third-order pair terms D_dq, formed with B_q
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (q == d) continue;
          const int qz = q == 0, qy = q == 1, qx = q == 2;
          Vq[q] = T(0.25) * ((Q(q, 0, 0, 0) + Q(q, dz, dy, dx)) + (Q(q, -qz, -qy, -qx) + Q(q, dz - qz, dy - qy, dx - qx)));
          const T a = P(qz, qy, qx), b = P(qz + dz, qy + dy, qx + dx);
          const T e = P(-qz, -qy, -qx), f = P(dz - qz, dy - qy, dx - qx);
          const T Tp = a + b, Bt = e + f;
          T B;
          if (iga) {
            B = (Tp - Bt) * T(0.25);
            Dq[q] = ((b - a) - (f - e)) * T(0.25);
          } else {
            // B_q and D_dq share the denominator (a + b) + (e + f) = Tp + Bt
            frac2(Tp - Bt, (b - a) - (f - e), Tp + Bt, B, Dq[q]);
          }
          out = out - T(0.5) * V * Vq[q] * rGb * B;
        }
        if (tot) {
          const T pm = P(-dz, -dy, -dx);
          const T p2 = P(2 * dz, 2 * dy, 2 * dx);
          const T num = ((p2 - p1) - p0) + pm;
          const T D = iga ? num * T(0.25) : fracg(num, ((p2 + p1) + p0) + pm);
          out = out + ((T(3) * V * absv(V)) * rGb - (T(2) * V * V * V) * (rGb * rGb) - V) * T(1.0 / 3.0) * D;
          int qs[2] = {0, 0}, nq = 0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if (q == d) continue;
            qs[nq++] = q;
            out = out + absv(V) * Vq[q] * rGb * (T(1) - T(2) * absv(V) * rGb) * Dq[q];
          }
          T pr[4];
          int m = 0;
#pragma unroll
          for (int s1 = 1; s1 >= -1; s1 -= 2) {
#pragma unroll
            for (int s2 = 1; s2 >= -1; s2 -= 2) {
              const int oz = s1 * (qs[0] == 0) + s2 * (qs[1] == 0);
              const int oy = s1 * (qs[0] == 1) + s2 * (qs[1] == 1);
              const int ox = s1 * (qs[0] == 2) + s2 * (qs[1] == 2);
              pr[m++] = P(oz, oy, ox) + P(oz + dz, oy + dy, ox + dx);
            }
          }
          // pr = {(+,+), (+,-), (-,+), (-,-)}
          const T n3 = (pr[0] - pr[1]) - (pr[2] - pr[3]);
          const T D3 = iga ? n3 * T(0.125) : fracg(n3, (pr[0] + pr[1]) + (pr[2] + pr[3]));
          out = out - (T(2) / T(3)) * V * Vq[qs[0]] * Vq[qs[1]] * (rGb * rGb) * D3;
        }
        res[d] = out;
      }
      // stored after all three faces, so that no store separates the shared-memory reads
      const long long i = static_cast<long long>(z) * plane + row;
      Vout.p[0][i] = res[0];
      Vout.p[1][i] = res[1];
      Vout.p[2][i] = res[2];
    }
    dev::cp_wait<0>();
    if (z + 1 < ze && vscale != T(1)) {  // only planes copied in this step are scaled
      scaleV(Vzs(fz));
      scaleV(Vys(fq));
      scaleV(Vxs(fq));
    }
    cp = rot(cp, 1, kA3P);
    cz = rot(cz, 1, kA3V);
    cq = rot(cq, 1, kA3V);
  }
}

// Pass 1 and the FCT bounds of a 3D field as one z-march (the work of k_donor and k_bounds,
// same expressions, same order): at step z the donor-cell pass (Eqs. 4-5) forms psi^(1) of
// plane z on the tile and a one-cell halo into a ring of three planes; then the bounds of
// plane z-1 (Sect. 3.1.4: extrema of psi^n and psi^(1) over the cell and its face neighbours)
// are formed and plane z-1 of psi^(1), mx and mn is written.  Shared tiles: psi^n with a
// two-cell halo on planes z-2 .. z+1; the x and y advector components with halo [-2, +1] and
// G with halo 1 on plane z; the z component with halo 1 on planes z-1, z.  Each ring has one
// slot more, into which the next step's plane is copied (cp.async) while this step computes.
constexpr int kBw = kAx + 4, kBh = kAy + 4;  // psi^n
constexpr int kXw = kAx + 3, kXh = kAy + 3;  // x and y advector components
constexpr int kHw = kAx + 2, kHh = kAy + 2;  // z component, G, psi^(1)
constexpr int kP1N = 5, kP1X = 2, kP1Z = 3, kP1Q = 3;  // ring slots: psi^n, x/y/G, z, psi^(1)
template <typename T>
constexpr size_t p1b3_smem() {
  return sizeof(T) * (kP1N * kBw * kBh + 2 * kP1X * kXw * kXh + (kP1Z + kP1X + kP1Q) * kHw * kHh);
}

template <typename T>
__global__ void __launch_bounds__(kAx * kAy) k_p1b3(Grid g, const T* __restrict__ psi, In3<T> V, T vscale,
                                                    const T* __restrict__ G, bool kahan, T* __restrict__ p1,
                                                    T* __restrict__ mx, T* __restrict__ mn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int nB = kBw * kBh, nX = kXw * kXh, nH = kHw * kHh;
  T* const sN = reinterpret_cast<T*>(smem_raw);  // [kP1N][nB] psi^n
  T* const sX = sN + kP1N * nB;                   // [kP1X][nX] x component
  T* const sY = sX + kP1X * nX;                   // [kP1X][nX] y component
  T* const sZ = sY + kP1X * nX;                   // [kP1Z][nH] z component
  T* const sG = sZ + kP1Z * nH;                   // [kP1X][nH] G
  T* const s1 = sG + kP1X * nH;                   // [kP1Q][nH] psi^(1)
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kAx + tx;
  constexpr int kT = kAx * kAy;
  const int x0 = blockIdx.x * kAx, y0 = blockIdx.y * kAy;
  const int zb = blockIdx.z * kAz;
  const int ze = zb + kAz < nz ? zb + kAz : nz;
  const long long plane = static_cast<long long>(ny) * nx;
  // Every plane region is copied with the same element assignment: this thread copies region
  // elements tid and tid + kT (when they exist), whose in-plane source offsets are fixed.
  static_assert(nB <= 2 * kT && nX <= 2 * kT && nH <= 2 * kT, "two elements per thread cover a plane");
  int offB[2], offX[2], offH[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = tid + r * kT;
    int yy = k / kBw;
    offB[r] = wrapc(y0 - 2 + yy, ny) * nx + wrapc(x0 - 2 + (k - yy * kBw), nx);
    yy = k / kXw;
    offX[r] = wrapc(y0 - 2 + yy, ny) * nx + wrapc(x0 - 2 + (k - yy * kXw), nx);
    yy = k / kHw;
    offH[r] = wrapc(y0 - 1 + yy, ny) * nx + wrapc(x0 - 1 + (k - yy * kHw), nx);
  }
  const bool hasB1 = tid + kT < nB, hasX1 = tid + kT < nX, hasH1 = tid + kT < nH;
  auto zsrc = [&](const T* base, int z) { return base + static_cast<long long>(wrapc(z, nz)) * plane; };
  auto copy = [&](T* dst, const T* src, const int (&off)[2], bool has1) {
    dev::cp_async<sizeof(T)>(dst + tid, src + off[0]);
    if (has1) dev::cp_async<sizeof(T)>(dst + tid + kT, src + off[1]);
  };
  // Ring slots: kn, kx, kz are the slots of plane z at step z in the rings of kP1N, kP1X and
  // kP1Z = kP1Q planes (advanced by one per step); plane z + j sits in slot k + j (mod size).
  int kn = kP1N - 1, kx = kP1X - 1, kz = kP1Z - 1;  // plane zb - 1
  static_assert(kP1Z == kP1Q, "psi^(1) and the z component share their ring counter");
  auto rj = [](int k, int j, int n) { const int v = k + j; return v >= n ? v - n : (v < 0 ? v + n : v); };
  auto slotN = [&](int j) { return rj(kn, j, kP1N); };
  auto slotX = [&](int j) { return rj(kx, j, kP1X); };
  auto slotZ = [&](int j) { return rj(kz, j, kP1Z); };
  auto slot1 = [&](int j) { return rj(kz, j, kP1Q); };
  // the planes step zz = z + j reads that step zz-1 did not: psi^n zz+1; the x, y, z components
  // and G of zz (z the current step)
  auto copy_step = [&](int zz, int j) {
    copy(sN + slotN(j + 1) * nB, zsrc(psi, zz + 1), offB, hasB1);
    copy(sX + slotX(j) * nX, zsrc(V.p[2], zz), offX, hasX1);
    copy(sY + slotX(j) * nX, zsrc(V.p[1], zz), offX, hasX1);
    copy(sZ + slotZ(j) * nH, zsrc(V.p[0], zz), offH, hasH1);
    if (G) copy(sG + slotX(j) * nH, zsrc(G, zz), offH, hasH1);
  };

  // prologue (step zb-1): psi^n planes zb-2, zb-1, the z component of plane zb-2, then step zb-1's planes
  copy(sN + slotN(-1) * nB, zsrc(psi, zb - 2), offB, hasB1);
  copy(sN + slotN(0) * nB, zsrc(psi, zb - 1), offB, hasB1);
  copy(sZ + slotZ(-1) * nH, zsrc(V.p[0], zb - 2), offH, hasH1);
  copy_step(zb - 1, 0);
  dev::cp_commit();
  dev::cp_wait<0>();
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < nx && y < ny;
  for (int z = zb - 1; z <= ze; ++z) {
    __syncthreads();  // step z's planes are in (each thread waited for its own copies)
    if (z < ze) copy_step(z + 1, 1);  // the next step's planes fly while this one computes
    dev::cp_commit();
    {  // pass 1 on plane z, tile and one-cell halo
      const T* Nm = sN + slotN(-1) * nB;
      const T* Nc = sN + slotN(0) * nB;
      const T* Np = sN + slotN(1) * nB;
      const T* Zm = sZ + slotZ(-1) * nH;
      const T* Zc = sZ + slotZ(0) * nH;
      const T* Xc = sX + slotX(0) * nX;
      const T* Yc = sY + slotX(0) * nX;
      const T* Gc = sG + slotX(0) * nH;
      T* const P1 = s1 + slot1(0) * nH;
      for (int k = tid; k < nH; k += kT) {
        const int hy = k / kHw, hx = k - hy * kHw;
        const int b = (hy + 1) * kBw + (hx + 1);  // the cell in the psi^n planes
        const int q = (hy + 1) * kXw + (hx + 1);  // its x and y faces in the advector planes
        const T p = Nc[b];
        T sum = p, comp = T(0);
        const T Gi = G ? Gc[k] : T(1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T pp = d == 0 ? Np[b] : (d == 1 ? Nc[b + kBw] : Nc[b + 1]);
          const T pm = d == 0 ? Nm[b] : (d == 1 ? Nc[b - kBw] : Nc[b - 1]);
          const T vp = (d == 0 ? Zc[k] : (d == 1 ? Yc[q] : Xc[q])) * vscale;
          const T vm = (d == 0 ? Zm[k] : (d == 1 ? Yc[q - kXw] : Xc[q - 1])) * vscale;
          const T Fp = flux(p, pp, vp, false);
          const T Fm = flux(pm, p, vm, false);
          const T t0 = G ? -qdiv(Fp, Gi) : -Fp;
          const T t1 = G ? qdiv(Fm, Gi) : Fm;
          if (kahan) {
            T yk = t0 - comp;
            T u = sum + yk;
            comp = (u - sum) - yk;
            sum = u;
            yk = t1 - comp;
            u = sum + yk;
            comp = (u - sum) - yk;
            sum = u;
          } else {
            sum = sum + t0;
            sum = sum + t1;
          }
        }
        P1[k] = sum;
      }
    }
    __syncthreads();
    if (z - 1 >= zb && inside) {  // bounds of plane z-1
      const int zc = z - 1;
      const int b = (ty + 2) * kBw + (tx + 2), h = (ty + 1) * kHw + (tx + 1);
      const T* N0 = sN + slotN(-1) * nB;  // plane zc = z - 1
      const T* Q0 = s1 + slot1(-1) * nH;
      const T a0 = N0[b], b0 = Q0[h];
      T hi = a0 > b0 ? a0 : b0;
      T lo = a0 < b0 ? a0 : b0;
      // neighbours in k_bounds's order: z-1, z+1, y-1, y+1, x-1, x+1
      const T cand[6][2] = {{sN[slotN(-2) * nB + b], s1[slot1(-2) * nH + h]},
                            {sN[slotN(0) * nB + b], s1[slot1(0) * nH + h]},
                            {N0[b - kBw], Q0[h - kHw]},
                            {N0[b + kBw], Q0[h + kHw]},
                            {N0[b - 1], Q0[h - 1]},
                            {N0[b + 1], Q0[h + 1]}};
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const T a = cand[j][0], c = cand[j][1];
        hi = maxe(a, hi);
        hi = maxe(c, hi);
        lo = mine(a, lo);
        lo = mine(c, lo);
      }
      const long long i = static_cast<long long>(zc) * plane + static_cast<long long>(y) * nx + x;
      p1[i] = b0;
      mx[i] = hi;
      mn[i] = lo;
    }
    dev::cp_wait<0>();
    kn = rj(kn, 1, kP1N);
    kx = rj(kx, 1, kP1X);
    kz = rj(kz, 1, kP1Z);
  }
}

// One FCT corrective pass of a 3D field as a z-march (the work of k_beta, k_limit and
// k_donor, same expressions, same order): at plane z the limiting factors of plane z are
// formed on the tile and a one-cell halo into a ring of three planes; then plane z-1 is
// limited (its faces' factors are all there) and advanced by the donor-cell pass.  The
// limited advector is written out only when another pass follows (lim != null).
// Shared tiles: psi with halo [-2, +2] on planes z-2 .. z+1; the x and y pseudo-advector
// components with halo [-2, +1] on planes z-1, z; the z component, the factors, the bounds
// and G with halo [-1, +1] (z component on planes z-2 .. z, factors on z-2 .. z, G on z-1, z).
constexpr int kCPw = kAx + 4, kCPh = kAy + 4;  // psi
constexpr int kCVw = kAx + 3, kCVh = kAy + 3;  // x, y components
constexpr int kCBw = kAx + 2, kCBh = kAy + 2;  // z component, factors, bounds, G
// ring depths: planes in use plus one being copied (cp.async) for the next step
constexpr int kC3P = 5, kC3Vq = 3, kC3Vz = 4, kC3B = 3, kC3M = 2, kC3G = 3;
template <typename T>
constexpr size_t corr3_smem() {
  return sizeof(T) * (kC3P * kCPw * kCPh + 2 * kC3Vq * kCVw * kCVh +
                      (kC3Vz + 2 * kC3B + 2 * kC3M + kC3G) * kCBw * kCBh);
}

template <typename T>
__global__ void __launch_bounds__(kAx * kAy) k_corr3(Grid g, const T* __restrict__ psi, In3<T> Vu,
                                                     const T* __restrict__ G, bool unit, bool kahan,
                                                     const T* __restrict__ mxg, const T* __restrict__ mng,
                                                     const T* __restrict__ R, T dt, bool post, Out3<T> lim,
                                                     T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const sm = reinterpret_cast<T*>(smem_raw);
  constexpr int nP = kCPw * kCPh, nV = kCVw * kCVh, nB = kCBw * kCBh;
  // layout of sm: psi [kC3P][nP], x and y components [kC3Vq][nV] each, then the z component
  // [kC3Vz][nB], the factors [kC3B][nB] each, the bounds [kC3M][nB] each and G [kC3G][nB]
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kAx + tx;
  constexpr int kT = kAx * kAy;
  const int x0 = blockIdx.x * kAx, y0 = blockIdx.y * kAy;
  const int zb = blockIdx.z * kAz;
  const int ze = zb + kAz < nz ? zb + kAz : nz;
  const long long plane = static_cast<long long>(ny) * nx;
  static_assert(nP <= 2 * kT && nV <= 2 * kT && nB <= 2 * kT, "two elements per thread cover a plane");

  // fixed in-plane source offsets of the (at most two) tile elements this thread copies
  int offP[2], offV[2], offB[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = tid + r * kT;
    int yy = k / kCPw;
    offP[r] = wrapc(y0 - 2 + yy, ny) * nx + wrapc(x0 - 2 + (k - yy * kCPw), nx);
    yy = k / kCVw;
    offV[r] = wrapc(y0 - 2 + yy, ny) * nx + wrapc(x0 - 2 + (k - yy * kCVw), nx);
    yy = k / kCBw;
    offB[r] = wrapc(y0 - 1 + yy, ny) * nx + wrapc(x0 - 1 + (k - yy * kCBw), nx);
  }
  auto zoff = [&](int z) { return static_cast<long long>(wrapc(z, nz)) * plane; };
  auto copy = [&](T* dst, const T* src, const int (&off)[2], int count) {
    dev::cp_async<sizeof(T)>(dst + tid, src + off[0]);
    if (tid + kT < count) dev::cp_async<sizeof(T)>(dst + tid + kT, src + off[1]);
  };
  // Ring planes as pointers indexed by the plane's offset from the current step z, rotated by
  // one slot per step: P[i] plane z-2+i (i = 0..4), Vx/Vy[i] z-1+i, Vz[i] z-2+i, Bu/Bd[i]
  // z-2+i, Mx/Mn[i] z+i, G[i] z-1+i.  The last slot of each input ring takes the next step's
  // plane (cp.async) while this step computes.
  static_assert(kC3P == 5 && kC3Vz == 4 && kC3Vq == 3 && kC3B == 3 && kC3G == 3 && kC3M == 2, "ring sizes");
  int P[kC3P], VX[kC3Vq], VY[kC3Vq], VZ[kC3Vz], BU[kC3B], BD[kC3B], MX[kC3M], MN[kC3M], GG[kC3G];  // offsets in sm
#pragma unroll
  for (int i = 0; i < kC3P; ++i) P[i] = i * nP;
#pragma unroll
  for (int i = 0; i < kC3Vq; ++i) { VX[i] = kC3P * nP + i * nV; VY[i] = kC3P * nP + (kC3Vq + i) * nV; }
  constexpr int oB = kC3P * nP + 2 * kC3Vq * nV;  // start of the [nB] rings
#pragma unroll
  for (int i = 0; i < kC3Vz; ++i) VZ[i] = oB + i * nB;
#pragma unroll
  for (int i = 0; i < kC3B; ++i) {
    BU[i] = oB + (kC3Vz + i) * nB;
    BD[i] = oB + (kC3Vz + kC3B + i) * nB;
    GG[i] = oB + (kC3Vz + 2 * kC3B + 2 * kC3M + i) * nB;
  }
#pragma unroll
  for (int i = 0; i < kC3M; ++i) {
    MX[i] = oB + (kC3Vz + 2 * kC3B + i) * nB;
    MN[i] = oB + (kC3Vz + 2 * kC3B + kC3M + i) * nB;
  }
  // the planes that become needed at step zz (its psi plane zz+1 into psi slot jp; the
  // components, bounds and G of plane zz into slots jq, jz, jm, jg)
  auto copy_step = [&](long long zo_p, long long zo, int jp, int jq, int jz, int jm, int jg) {
    copy(sm + P[jp], psi + zo_p, offP, nP);
    copy(sm + VX[jq], Vu.p[2] + zo, offV, nV);
    copy(sm + VY[jq], Vu.p[1] + zo, offV, nV);
    copy(sm + VZ[jz], Vu.p[0] + zo, offB, nB);
    copy(sm + MX[jm], mxg + zo, offB, nB);
    copy(sm + MN[jm], mng + zo, offB, nB);
    if (G) copy(sm + GG[jg], G + zo, offB, nB);
  };
  // wrapped plane indices advanced by one per step
  auto next = [&](int v) { return v + 1 == nz ? 0 : v + 1; };
  int zq = wrapc(zb - 1, nz);  // plane z (step z = zb - 1 first)
  // prologue (step zb-1): psi planes zb-2, zb-1, the z component of plane zb-2, then step zb-1's planes
  copy(sm + P[1], psi + zoff(zb - 2), offP, nP);
  copy(sm + P[2], psi + static_cast<long long>(zq) * plane, offP, nP);
  copy(sm + VZ[1], Vu.p[0] + zoff(zb - 2), offB, nB);
  copy_step(static_cast<long long>(next(zq)) * plane, static_cast<long long>(zq) * plane, 3, 1, 2, 0, 1);
  dev::cp_commit();
  dev::cp_wait<0>();
  // the factor cells of this thread (the tile and a one-cell ring: nB cells, two passes of the
  // block at most), fixed for the whole march
  constexpr int kFac = (nB + kT - 1) / kT;
  int fr[kFac], fcp[kFac], fcv[kFac];
#pragma unroll
  for (int j = 0; j < kFac; ++j) {
    const int r = tid + j * kT;
    const int by = r / kCBw, bx = r - by * kCBw;  // cell (bx - 1, by - 1) of the tile
    fr[j] = r < nB ? r : -1;
    fcp[j] = (by + 1) * kCPw + (bx + 1);  // in the psi tile
    fcv[j] = (by + 1) * kCVw + (bx + 1);  // in the x, y component tiles
  }
  const int x = x0 + tx, y = y0 + ty;
  const int cpc = (ty + 2) * kCPw + (tx + 2), cvc = (ty + 2) * kCVw + (tx + 2), cbc = (ty + 1) * kCBw + (tx + 1);
  // this thread's cell of plane q = z - 1 (first step z = zb - 1)
  long long oq = static_cast<long long>(zb - 2) * plane + static_cast<long long>(y) * nx + x;

  for (int z = zb - 1; z <= ze; ++z) {
    __syncthreads();  // step z's planes are in (each thread waited for its own copies)
    const int zn = next(zq);           // plane z + 1
    if (z + 1 <= ze) copy_step(static_cast<long long>(next(zn)) * plane, static_cast<long long>(zn) * plane, 4, 2, 3, 1, 2);
    dev::cp_commit();
    {  // limiting factors of plane z on the tile and a one-cell halo (k_beta)
      const T* pm = sm + P[1];
      const T* p0 = sm + P[2];
      const T* pp = sm + P[3];
      const T* vx = sm + VX[1];
      const T* vy = sm + VY[1];
      const T* vzm = sm + VZ[1];
      const T* vz0 = sm + VZ[2];
      const T* gz = sm + GG[1];
      const T* sMxz = sm + MX[0];
      const T* sMnz = sm + MN[0];
      T* bu = sm + BU[2];
      T* bd = sm + BD[2];
#pragma unroll
      for (int j = 0; j < kFac; ++j) {
        const int r = fr[j];
        if (r < 0) continue;
        const int cp = fcp[j], cv = fcv[j];
        const T p = p0[cp];
        T in = T(0), ou = T(0);
        {  // dimension 0 (z)
          const T Fp = flux(p, pp[cp], vz0[r], unit);
          const T Fm = flux(pm[cp], p, vzm[r], unit);
          in = in + (posp(Fm) - negp(Fp));
          ou = ou + (posp(Fp) - negp(Fm));
        }
        {  // dimension 1 (y)
          const T Fp = flux(p, p0[cp + kCPw], vy[cv], unit);
          const T Fm = flux(p0[cp - kCPw], p, vy[cv - kCVw], unit);
          in = in + (posp(Fm) - negp(Fp));
          ou = ou + (posp(Fp) - negp(Fm));
        }
        {  // dimension 2 (x)
          const T Fp = flux(p, p0[cp + 1], vx[cv], unit);
          const T Fm = flux(p0[cp - 1], p, vx[cv - 1], unit);
          in = in + (posp(Fm) - negp(Fp));
          ou = ou + (posp(Fp) - negp(Fm));
        }
        const T Gi = G ? gz[r] : T(1);
        bu[r] = factor_sum(in) ? qdiv(Gi * posp(sMxz[r] - p), in) : T(1);
        bd[r] = factor_sum(ou) ? qdiv(Gi * posp(p - sMnz[r]), ou) : T(1);
      }
    }
    __syncthreads();
    const int q = z - 1;
    if (q >= zb && x < nx && y < ny) {  // limit and donor of plane q (k_limit, k_donor)
      // plane q = z - 1: ring offsets 0 .. 2 of psi and the factors
      const T* ps[3] = {sm + P[0], sm + P[1], sm + P[2]};
      const T* bus[3] = {sm + BU[0], sm + BU[1], sm + BU[2]};
      const T* bds[3] = {sm + BD[0], sm + BD[1], sm + BD[2]};
      const T* vx = sm + VX[0];
      const T* vy = sm + VY[0];
      const T* vzm = sm + VZ[0];
      const T* vz0 = sm + VZ[1];
      const int cp = cpc, cv = cvc, cb = cbc;
      const T p = ps[1][cp];
      // limited advector at a face: V m, m = min(1, factor of the upwind side, factor of the downwind side)
      auto limit = [&](T L, T Rr, T V, T buL, T bdL, T buR, T bdR) {
        const T F = flux(L, Rr, V, unit);
        const bool right = goes_right(F, V);
        const T a = right ? bdL : buL;
        const T b = right ? buR : bdR;
        T m = T(1);
        m = mine(a, m);
        m = mine(b, m);
        return V * m;
      };
      // faces (d, +) and (d, -) of this cell: psi, limited advector
      const T pz_p = ps[2][cp], pz_m = ps[0][cp];
      const T py_p = ps[1][cp + kCPw], py_m = ps[1][cp - kCPw];
      const T px_p = ps[1][cp + 1], px_m = ps[1][cp - 1];
      const T hz_p = limit(p, pz_p, vz0[cb], bus[1][cb], bds[1][cb], bus[2][cb], bds[2][cb]);
      const T hz_m = limit(pz_m, p, vzm[cb], bus[0][cb], bds[0][cb], bus[1][cb], bds[1][cb]);
      const T hy_p = limit(p, py_p, vy[cv], bus[1][cb], bds[1][cb], bus[1][cb + kCBw], bds[1][cb + kCBw]);
      const T hy_m = limit(py_m, p, vy[cv - kCVw], bus[1][cb - kCBw], bds[1][cb - kCBw], bus[1][cb], bds[1][cb]);
      const T hx_p = limit(p, px_p, vx[cv], bus[1][cb], bds[1][cb], bus[1][cb + 1], bds[1][cb + 1]);
      const T hx_m = limit(px_m, p, vx[cv - 1], bus[1][cb - 1], bds[1][cb - 1], bus[1][cb], bds[1][cb]);
      const long long i = oq;
      if (lim.p[0]) {
        lim.p[0][i] = hz_p;
        lim.p[1][i] = hy_p;
        lim.p[2][i] = hx_p;
      }
      const T Gi = G ? sm[GG[0] + cb] : T(1);
      T s = p, comp = T(0);
      const T hp[3] = {hz_p, hy_p, hx_p}, hm[3] = {hz_m, hy_m, hx_m};
      const T np_[3] = {pz_p, py_p, px_p}, nm_[3] = {pz_m, py_m, px_m};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T Fp = flux(p, np_[d], hp[d], unit);
        const T Fm = flux(nm_[d], p, hm[d], unit);
        const T t0 = G ? -qdiv(Fp, Gi) : -Fp;
        const T t1 = G ? qdiv(Fm, Gi) : Fm;
        if (kahan) {
          T yk = t0 - comp;
          T u = s + yk;
          comp = (u - s) - yk;
          s = u;
          yk = t1 - comp;
          u = s + yk;
          comp = (u - s) - yk;
          s = u;
        } else {
          s = s + t0;
          s = s + t1;
        }
      }
      if (post) s = s + dt * R[i];
      out[i] = s;
    }
    oq += plane;
    dev::cp_wait<0>();
    // rotate the rings by one plane
    {
      int t = P[0];
#pragma unroll
      for (int k = 0; k < kC3P - 1; ++k) P[k] = P[k + 1];
      P[kC3P - 1] = t;
      t = VZ[0];
#pragma unroll
      for (int k = 0; k < kC3Vz - 1; ++k) VZ[k] = VZ[k + 1];
      VZ[kC3Vz - 1] = t;
      const int tx_ = VX[0], ty_ = VY[0], tu = BU[0], td = BD[0], tg = GG[0];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        VX[k] = VX[k + 1]; VY[k] = VY[k + 1]; BU[k] = BU[k + 1]; BD[k] = BD[k + 1]; GG[k] = GG[k + 1];
      }
      VX[2] = tx_; VY[2] = ty_; BU[2] = tu; BD[2] = td; GG[2] = tg;
      t = MX[0]; MX[0] = MX[1]; MX[1] = t;
      t = MN[0]; MN[0] = MN[1]; MN[1] = t;
    }
    zq = zn;
  }
}

// FCT limiting factors (Sect. 3.1.4): in/out sums of the unlimited fluxes and
// beta_up = G [psi_max - psi]+ / in, beta_dn = G [psi - psi_min]+ / out (1 when the sum is 0).
template <typename T, int ND>
__global__ void k_beta(Grid g, const T* __restrict__ psi, In3<T> V, const T* __restrict__ G, bool unit,
                       const T* __restrict__ mx, const T* __restrict__ mn, T* __restrict__ bu,
                       T* __restrict__ bd) {
  FOR_CELLS(g) {
  const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});
  const long long i = nb.i;
  const T p = psi[i];
  T in = T(0), out = T(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const long long ip = nb.at(d, +1);
    const long long im = nb.at(d, -1);
    const T Fp = flux(p, psi[ip], V.p[d][nb.face(d, 0)], unit);
    const T Fm = flux(psi[im], p, V.p[d][nb.face(d, -1)], unit);
    in = in + (posp(Fm) - negp(Fp));
    out = out + (posp(Fp) - negp(Fm));
  }
  const T Gi = G ? G[i] : T(1);
  bu[i] = factor_sum(in) ? qdiv(Gi * posp(mx[i] - p), in) : T(1);
  bd[i] = factor_sum(out) ? qdiv(Gi * posp(p - mn[i]), out) : T(1);
  }
}

// Limited advector: V min(1, beta_dn_i, beta_up_{i+e_d}) if the unlimited flux leaves
// cell i (F > 0, or F = 0 with V > 0), else V min(1, beta_up_i, beta_dn_{i+e_d}).
template <typename T, int ND>
__global__ void k_limit(Grid g, const T* __restrict__ psi, In3<T> Vu, bool unit,
                        const T* __restrict__ bu, const T* __restrict__ bd, Out3<T> Vout) {
  FOR_CELLS(g) {
  const Nbr<ND> nb(g, Coord{{c0_, c1_, c2_}});
  const long long i = nb.i;
  const T p = psi[i];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const long long ip = nb.at(d, +1);
    const T V = Vu.p[d][i];
    const T F = flux(p, psi[ip], V, unit);
    const bool right = goes_right(F, V);
    const T a = right ? bd[i] : bu[i];
    const T b = right ? bu[ip] : bd[ip];
    T m = T(1);
    m = mine(a, m);
    m = mine(b, m);
    Vout.p[d][i] = V * m;
  }
  }
}

// Every step of a call for a 1D field small enough for shared memory: one block holds the
// field and all intermediates in shared memory and runs the sub-steps above (same
// expressions, same order) as passes over the field separated by block barriers, so the
// call is one launch instead of several per step.  Advector scale 1 (no per-step factors).
constexpr int kSteps1dThreads = 1024;
constexpr int kSteps1dArrays = 13;  // state, psi^(0), two levels, gc, two advectors, unlimited, bounds, factors, G, R

template <typename T>
__global__ void __launch_bounds__(kSteps1dThreads) k_steps1d(int n, int n_steps, Opts o, const T* __restrict__ psi_in,
                                                             T* __restrict__ psi_out, const T* __restrict__ gc,
                                                             const T* __restrict__ Gin, const T* __restrict__ Rin,
                                                             T dt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const sm = reinterpret_cast<T*>(smem_raw);
  T* st = sm;          // state psi^n
  T* p0 = sm + n;      // psi^n + dt R (euler_b)
  T* lev[2] = {sm + 2 * n, sm + 3 * n};
  T* v0 = sm + 4 * n;  // the advector
  T* vl[2] = {sm + 5 * n, sm + 6 * n};
  T* vu = sm + 7 * n;
  T* mx = sm + 8 * n;
  T* mn = sm + 9 * n;
  T* bu = sm + 10 * n;
  T* bd = sm + 11 * n;
  T* Gs = sm + 12 * n;
  const T* G = o.nug ? Gs : nullptr;
  const int K = o.n_iters;
  auto L = [&](int i) { return i == 0 ? n - 1 : i - 1; };
  auto Rt = [&](int i) { return i == n - 1 ? 0 : i + 1; };
  auto R2 = [&](int i) { int j = i + 2; if (j >= n) j -= n; if (j >= n) j -= n; return j; };
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    st[i] = psi_in[i];
    v0[i] = gc[i];
    if (o.nug) Gs[i] = Gin[i];
  }
  __syncthreads();
  // donor-cell pass of k_donor: src with advector v (flux of psi unless unit), to dst
  auto donor = [&](const T* src, const T* v, bool unit, bool post, T* dst) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const T p = src[i];
      T s = p, comp = T(0);
      const T Gi = G ? G[i] : T(1);
      const int ip = Rt(i), im = L(i);
      const T vp = v[i], vm = v[im];
      const T Fp = flux(p, src[ip], vp, unit);
      const T Fm = flux(src[im], p, vm, unit);
      const T t0 = G ? -qdiv(Fp, Gi) : -Fp;
      const T t1 = G ? qdiv(Fm, Gi) : Fm;
      if (o.kahan) {
        T y = t0 - comp;
        T u = s + y;
        comp = (u - s) - y;
        s = u;
        y = t1 - comp;
        u = s + y;
        comp = (u - s) - y;
        s = u;
      } else {
        s = s + t0;
        s = s + t1;
      }
      if (post) s = s + dt * Rin[i];
      dst[i] = s;
    }
  };
  for (int step = 0; step < n_steps; ++step) {
    const T* q0 = st;
    if (o.rhs_b) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) p0[i] = st[i] + dt * Rin[i];
      q0 = p0;
      __syncthreads();
    }
    T* dst1 = K == 1 ? st : lev[0];  // with one pass the result is the new state
    if (K == 1 && !o.rhs_b) dst1 = lev[0];
    donor(q0, v0, false, K == 1 && o.rhs_a, dst1);
    __syncthreads();
    if (K == 1) {
      if (dst1 != st) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) st[i] = dst1[i];
        __syncthreads();
      }
      continue;
    }
    if (o.fct) {  // k_bounds
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T hi = q0[i] > lev[0][i] ? q0[i] : lev[0][i];
        T lo = q0[i] < lev[0][i] ? q0[i] : lev[0][i];
        const int js[2] = {L(i), Rt(i)};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const T a = q0[js[t]], b = lev[0][js[t]];
          hi = maxe(a, hi);
          hi = maxe(b, hi);
          lo = mine(a, lo);
          lo = mine(b, lo);
        }
        mx[i] = hi;
        mn[i] = lo;
      }
    }
    const T* prev = lev[0];
    const T* vprev = v0;
    for (int k = 2; k <= K; ++k) {
      T* lim = vl[k % 2];
      T* vk = o.fct ? vu : lim;
      // k_antidiff (1D: no cross terms; third-order D_dd term)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T pp0 = prev[i];
        const int ip = Rt(i);
        const T rGb = G ? qdiv(T(1), T(0.5) * (G[i] + G[ip])) : T(1);
        const T V = vprev[i];
        const T p1 = prev[ip];
        const T A = o.iga ? (p1 - pp0) * T(0.5) : fracg(p1 - pp0, pp0 + p1);
        T out = (absv(V) - V * V * rGb) * A;
        if (o.tot) {
          const T pm = prev[L(i)];
          const T p2 = prev[R2(i)];
          const T num = ((p2 - p1) - pp0) + pm;
          const T D = o.iga ? num * T(0.25) : fracg(num, ((p2 + p1) + pp0) + pm);
          out = out + ((T(3) * V * absv(V)) * rGb - (T(2) * V * V * V) * (rGb * rGb) - V) * T(1.0 / 3.0) * D;
        }
        vk[i] = out;
      }
      __syncthreads();
      const T* vuse = vk;
      if (o.fct) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {  // k_beta
          const T p = prev[i];
          T in = T(0), ou = T(0);
          const int ip = Rt(i), im = L(i);
          const T Fp = flux(p, prev[ip], vk[i], o.iga);
          const T Fm = flux(prev[im], p, vk[im], o.iga);
          in = in + (posp(Fm) - negp(Fp));
          ou = ou + (posp(Fp) - negp(Fm));
          const T Gi = G ? G[i] : T(1);
          bu[i] = factor_sum(in) ? qdiv(Gi * posp(mx[i] - p), in) : T(1);
          bd[i] = factor_sum(ou) ? qdiv(Gi * posp(p - mn[i]), ou) : T(1);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {  // k_limit
          const T p = prev[i];
          const int ip = Rt(i);
          const T V = vk[i];
          const T F = flux(p, prev[ip], V, o.iga);
          const bool right = goes_right(F, V);
          const T a = right ? bd[i] : bu[i];
          const T b = right ? bu[ip] : bd[ip];
          T m = T(1);
          m = mine(a, m);
          m = mine(b, m);
          lim[i] = V * m;
        }
        __syncthreads();
        vuse = lim;
      }
      T* dst = k == K ? st : (prev == lev[0] ? lev[1] : lev[0]);
      donor(prev, vuse, o.iga, k == K && o.rhs_a, dst);
      __syncthreads();
      prev = dst;
      vprev = vuse;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) psi_out[i] = st[i];
}

template <typename T>
size_t steps1d_smem(long long n) { return static_cast<size_t>(kSteps1dArrays) * static_cast<size_t>(n) * sizeof(T); }

template <typename T, bool ABS>
void launch_antidiff3_t(const Grid& g, const T* psi, In3<T> v, T vscale, const T* G, bool iga, bool tot, Out3<T> out,
                        cudaStream_t st) {
  static PerDevice<bool> attr;
  attr.get([](int) {
    return cudaFuncSetAttribute(k_antidiff3<T, ABS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(antidiff3_smem<T>())) == cudaSuccess;
  });
  k_antidiff3<T, ABS><<<march3_grid(g), dim3(kAx, kAy), antidiff3_smem<T>(), st>>>(g, psi, v, vscale, G, iga, tot, out);
}

template <typename T>
void launch_antidiff3(const Grid& g, const T* psi, In3<T> v, T vscale, const T* G, bool iga, bool tot, bool abs_psi,
                      Out3<T> out, cudaStream_t st) {
  if (abs_psi) launch_antidiff3_t<T, true>(g, psi, v, vscale, G, iga, tot, out, st);
  else launch_antidiff3_t<T, false>(g, psi, v, vscale, G, iga, tot, out, st);
}

template <typename T>
void launch_p1b3(const Grid& g, const T* psi, In3<T> v, T vscale, const T* G, bool kahan, T* p1, T* mx, T* mn,
                 cudaStream_t st) {
  static PerDevice<bool> attr;
  attr.get([](int) {
    return cudaFuncSetAttribute(k_p1b3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(p1b3_smem<T>())) == cudaSuccess;
  });
  k_p1b3<T><<<march3_grid(g), dim3(kAx, kAy), p1b3_smem<T>(), st>>>(g, psi, v, vscale, G, kahan, p1, mx, mn);
}

template <typename T>
void launch_corr3(const Grid& g, const T* psi, In3<T> vu, const T* G, bool unit, bool kahan, const T* mx,
                  const T* mn, const T* R, T dt, bool post, Out3<T> lim, T* out, cudaStream_t st) {
  static PerDevice<bool> attr;  // the FP64 rings exceed the default 48 KB of dynamic shared memory
  attr.get([](int) {
    return cudaFuncSetAttribute(k_corr3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(corr3_smem<T>())) == cudaSuccess;
  });
  k_corr3<T><<<march3_grid(g), dim3(kAx, kAy), corr3_smem<T>(), st>>>(g, psi, vu, G, unit, kahan, mx, mn, R, dt,
                                                                      post, lim, out);
}

template <typename T, int ND>
cudaError_t staged_nd(const Grid& g, const Opts& o, const StepArgs<T>& a, const StagedScratch<T>& s,
                      cudaStream_t st) {
  const int bs = 256;
  const unsigned nb = static_cast<unsigned>((g.N + bs - 1) / bs);
  const int K = o.n_iters;
  const T* G = o.nug ? a.g : nullptr;
  const T* p0 = a.psi_in;
  if (o.rhs_b) {
    k_pre<T><<<nb, bs, 0, st>>>(g.N, a.psi_in, a.r, a.dt, s.p0);
    p0 = s.p0;
  }
  In3<T> gc{{a.gc[0], a.gc[1], a.gc[2]}};
  // pass 1
  const bool inplace1 = (a.psi_out == a.psi_in) && !o.rhs_b;
  T* dst1 = (K == 1 && !inplace1) ? a.psi_out : s.pa;
  // FP32: pass 1 and the bounds in one z-march (FP64 is arithmetic-bound and the z-march
  // recomputes pass 1 on a one-cell halo)
  if (ND == 3 && K >= 2 && o.fct && sizeof(T) == 4 && !o.open) {
    bool done = false;
    if constexpr (sizeof(T) == 4) done = p1b3_vec(g, p0, gc.p, a.gc_scale, G, o.kahan, s.pa, s.mx, s.mn, st);
    if (!done) launch_p1b3<T>(g, p0, gc, a.gc_scale, G, o.kahan, s.pa, s.mx, s.mn, st);
  } else {
    k_donor<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, p0, gc, a.gc_scale, false, G, o.kahan, a.r, a.dt,
                                      K == 1 && o.rhs_a, dst1);
    if (K == 1) {
      if (dst1 != a.psi_out)
        return cudaMemcpyAsync(a.psi_out, dst1, sizeof(T) * g.N, cudaMemcpyDeviceToDevice, st);
      return cudaGetLastError();
    }
    if (o.fct) k_bounds<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, p0, s.pa, s.mx, s.mn);
  }
  const T* prev = s.pa;
  In3<T> vprev = gc;
  T vscale = a.gc_scale;
  for (int k = 2; k <= K; ++k) {
    T* const* lim = (k % 2 == 0) ? s.va : s.vb;
    Out3<T> vk{{o.fct ? s.vu[0] : lim[0], o.fct ? s.vu[1] : lim[1], o.fct ? s.vu[2] : lim[2]}};
    if (ND == 3 && !o.dfl && !o.open) {
      bool done = false;
      if constexpr (sizeof(T) == 4)
        done = antidiff3_vec(g, prev, vprev.p, vscale, G, o.iga, o.tot, o.abs, vk.p, st);
      if (!done) launch_antidiff3<T>(g, prev, vprev, vscale, G, o.iga, o.tot, o.abs, vk, st);
    } else {
      k_antidiff<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, prev, vprev, vscale, G, o.iga, o.tot, o.abs, o.dfl,
                                                         vk);
    }
    In3<T> vuse{{vk.p[0], vk.p[1], vk.p[2]}};
    // FP32: factors, limiter and donor pass in one z-march (it limits each face from both sides
    // and forms the factors on a one-cell halo: cheaper than the array traffic it saves in
    // FP32, dearer in FP64, which the arithmetic bounds); lanes of 4 cells (march3.cu) where
    // the field allows, else one cell per thread
    if (ND == 3 && o.fct && sizeof(T) == 4 && !o.open) {
      T* dst = (k == K) ? a.psi_out : (prev == s.pa ? s.pb : s.pa);
      Out3<T> lk{{nullptr, nullptr, nullptr}};
      if (k < K) lk = Out3<T>{{lim[0], lim[1], lim[2]}};
      bool done = false;
      if constexpr (sizeof(T) == 4)
        done = corr3_vec(g, prev, vuse.p, G, o.iga, o.kahan, s.mx, s.mn, k == K && o.rhs_a, lk.p, dst, st);
      if (!done)
        launch_corr3<T>(g, prev, vuse, G, o.iga, o.kahan, s.mx, s.mn, a.r, a.dt, k == K && o.rhs_a, lk, dst, st);
      prev = dst;
      vprev = In3<T>{{lim[0], lim[1], lim[2]}};
      vscale = T(1);
      continue;
    }
    if (o.fct) {
      k_beta<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, prev, vuse, G, o.iga, s.mx, s.mn, s.bu, s.bd);
      Out3<T> vl{{lim[0], lim[1], lim[2]}};
      k_limit<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, prev, vuse, o.iga, s.bu, s.bd, vl);
      vuse = In3<T>{{lim[0], lim[1], lim[2]}};
    }
    T* dst = (k == K) ? a.psi_out : (prev == s.pa ? s.pb : s.pa);
    k_donor<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, prev, vuse, T(1), o.iga, G, o.kahan, a.r, a.dt,
                                      k == K && o.rhs_a, dst);
    prev = dst;
    vprev = vuse;
    vscale = T(1);
  }
  return cudaGetLastError();
}

template <typename T, int ND>
cudaError_t tape_nd(const Grid& g, const Opts& o, const T* const* gc, const T* G, const Tape<T>& tp,
                    T* const* levels, T* psi_next, cudaStream_t st) {
  const int bs = 256;
  const int K = o.n_iters;
  In3<T> v1{{gc[0], gc[1], gc[2]}};
  if (K == 1 && psi_next)
    k_donor<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[0], v1, T(1), false, G, o.kahan, nullptr, T(0), false, psi_next);
  if (K >= 2) {
    if (ND == 3 && o.fct && sizeof(T) == 4) {
      launch_p1b3<T>(g, tp.psi[0], v1, T(1), G, o.kahan, levels[1], tp.mx, tp.mn, st);
    } else {
      k_donor<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[0], v1, T(1), false, G, o.kahan, nullptr, T(0), false,
                                                      levels[1]);
      if (o.fct) k_bounds<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[0], tp.psi[1], tp.mx, tp.mn);
    }
  }
  for (int k = 2; k <= K; ++k) {
    In3<T> vprev{{tp.vh[k - 1][0], tp.vh[k - 1][1], tp.vh[k - 1][2]}};
    Out3<T> vk{{tp.v[k][0], tp.v[k][1], tp.v[k][2]}};
    if (ND == 3 && !o.dfl) {  // the z-march leaves the divergent-flow term to the generic kernel
      launch_antidiff3<T>(g, tp.psi[k - 1], vprev, T(1), G, o.iga, o.tot, o.abs, vk, st);
    } else {
      k_antidiff<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[k - 1], vprev, T(1), G, o.iga, o.tot, o.abs,
                                                         o.dfl, vk);
    }
    In3<T> vu{{tp.v[k][0], tp.v[k][1], tp.v[k][2]}};
    if (o.fct) {
      k_beta<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[k - 1], vu, G, o.iga, tp.mx, tp.mn, tp.bu[k], tp.bd[k]);
      Out3<T> vl{{const_cast<T*>(tp.vh[k][0]), const_cast<T*>(tp.vh[k][1]), const_cast<T*>(tp.vh[k][2])}};
      k_limit<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[k - 1], vu, o.iga, tp.bu[k], tp.bd[k], vl);
    }
    T* const dst = k < K ? levels[k] : psi_next;  // the last pass only when the step's result is wanted
    if (dst) {
      In3<T> vh{{tp.vh[k][0], tp.vh[k][1], tp.vh[k][2]}};
      k_donor<T, ND><<<cell_grid(g, bs), bs, 0, st>>>(g, tp.psi[k - 1], vh, T(1), o.iga, G, o.kahan, nullptr, T(0), false,
                                        dst);
    }
  }
  return cudaGetLastError();
}

}  // namespace

template <typename T>
StagedScratch<T> carve_staged(void* base, long long n_max) {
  T* p = static_cast<T*>(base);
  StagedScratch<T> s;
  auto take = [&]() { T* q = p; p += n_max; return q; };
  s.p0 = take();
  s.pa = take();
  s.pb = take();
  for (int d = 0; d < 3; ++d) s.va[d] = take();
  for (int d = 0; d < 3; ++d) s.vb[d] = take();
  for (int d = 0; d < 3; ++d) s.vu[d] = take();
  s.mx = take();
  s.mn = take();
  s.bu = take();
  s.bd = take();
  return s;
}

template <typename T>
cudaError_t staged_step(const Grid& g, const Opts& o, const StepArgs<T>& a, const StagedScratch<T>& s,
                        cudaStream_t st) {
  switch (g.nd) {
    case 1: return staged_nd<T, 1>(g, o, a, s, st);
    case 2: return staged_nd<T, 2>(g, o, a, s, st);
    case 3: return staged_nd<T, 3>(g, o, a, s, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t staged_forward_tape(const Grid& g, const Opts& o, const T* const* gc, const T* G, const Tape<T>& tp,
                                T* const* levels, T* psi_next, cudaStream_t st) {
  switch (g.nd) {
    case 1: return tape_nd<T, 1>(g, o, gc, G, tp, levels, psi_next, st);
    case 2: return tape_nd<T, 2>(g, o, gc, G, tp, levels, psi_next, st);
    case 3: return tape_nd<T, 3>(g, o, gc, G, tp, levels, psi_next, st);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t staged_forward_tape<float>(const Grid&, const Opts&, const float* const*, const float*,
                                                const Tape<float>&, float* const*, float*, cudaStream_t);
template cudaError_t staged_forward_tape<double>(const Grid&, const Opts&, const double* const*, const double*,
                                                 const Tape<double>&, double* const*, double*, cudaStream_t);
template StagedScratch<float> carve_staged<float>(void*, long long);
template StagedScratch<double> carve_staged<double>(void*, long long);
template <typename T>
int steps1d(const Grid& g, const Opts& o, const T* psi_in, T* psi_out, const T* gc, const T* G, const T* R, T dt,
            int n_steps, cudaStream_t st) {
  if (g.nd != 1 || o.n_iters > 64 || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  const size_t smem = steps1d_smem<T>(g.N);
  static PerDevice<int> max_smem_of;
  const int max_smem = max_smem_of.get([](int dev) {
    int m = 0;
    cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(k_steps1d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
    return m;
  });
  if (smem > static_cast<size_t>(max_smem)) return MPDATA_EUNSUPPORTED;
  k_steps1d<T><<<1, kSteps1dThreads, smem, st>>>(static_cast<int>(g.N), n_steps, o, psi_in, psi_out, gc, G, R, dt);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template int steps1d<float>(const Grid&, const Opts&, const float*, float*, const float*, const float*,
                            const float*, float, int, cudaStream_t);
template int steps1d<double>(const Grid&, const Opts&, const double*, double*, const double*, const double*,
                             const double*, double, int, cudaStream_t);

template cudaError_t staged_step<float>(const Grid&, const Opts&, const StepArgs<float>&,
                                        const StagedScratch<float>&, cudaStream_t);
template cudaError_t staged_step<double>(const Grid&, const Opts&, const StepArgs<double>&,
                                         const StagedScratch<double>&, cudaStream_t);

}  // namespace mpd
