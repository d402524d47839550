// Fused 2D MPDATA step: the donor-cell pass, the FCT bounds, the antidiffusive
// pseudo-advector (Eq. 6 with its cross term), the FCT limiting factors and the
// corrective donor-cell pass of one time step in one kernel, with no
// intermediate written to global memory.  Covers 2D fields with n_iters = 2 and
// every option except the third-order terms (those run on the staged path).
//
// Work decomposition ("warp march"): a warp owns a strip of 64 columns (two per
// lane) and walks down TY rows.  Vertical neighbours stay in per-thread register
// windows (one row of each quantity per iteration), horizontal neighbours are
// exchanged with warp shuffles.  A step's stencil reaches 3 cells (two passes
// plus the limiter), so each strip recomputes a 3-column halo on both sides and
// stores the 56 columns in its middle; the strips' starts are 4 columns left of
// their first output so every lane's pair of columns is 8/16-byte aligned.
// Input rows are prefetched kPF rows ahead into a per-warp shared-memory ring
// with cp.async (each lane copies and later reads only its own two elements).
//
// Row lags at iteration t (row x = R0 - 3 + t loaded):
//   pass 1 at row x-1; bounds, pseudo-advectors, unlimited fluxes and limiting
//   factors at row x-2; limited fluxes and pass 2 at row x-3 (stored).
#include <cuda_runtime.h>

#include "kernels.h"

namespace mpd {
namespace {

constexpr int kCols = 64;    // columns computed per warp
constexpr int kStride = 56;  // output columns per strip
constexpr int kLead = 4;     // computed columns left of the strip's first output column
constexpr int kPF = 4;       // rows in flight
constexpr int kSlots = kPF + 1;
constexpr int kArr = 5;      // psi, gc0, gc1, G, R
constexpr int kWarps = 4;    // warps per block
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct F2Params {
  const T* psi;
  T* out;
  const T* gc0;
  const T* gc1;
  const T* G;
  const T* R;
  int n0, n1, strips, rowtiles, ty;
  T dt, scale;
  int iga, kahan, rhs_a, rhs_b, vec;
};

__device__ __forceinline__ int wrapi(int c, int n) {
  int r = c % n;
  return r < 0 ? r + n : r;
}

template <typename T> __device__ __forceinline__ T fdiv(T a, T b);
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }

template <typename T> __device__ __forceinline__ T posp(T x) { return x > T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T negp(T x) { return x < T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T absv(T x) { return x < T(0) ? -x : x; }
template <typename T> __device__ __forceinline__ T maxv(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T minv(T a, T b) { return a < b ? a : b; }
// donor-cell flux (Eq. 5) in advector units
template <typename T> __device__ __forceinline__ T flux(T L, T R, T V) { return posp(V) * L + negp(V) * R; }
// psi-fraction of Eq. 6 with the zero-denominator guard
template <typename T> __device__ __forceinline__ T ratio(T n, T d) { return d != T(0) ? fdiv(n, d) : T(0); }

// value of the column left of this lane's first column / right of its second
template <typename T> __device__ __forceinline__ T from_left(const T (&a)[2]) { return __shfl_up_sync(kFull, a[1], 1); }
template <typename T> __device__ __forceinline__ T from_right(const T (&a)[2]) { return __shfl_down_sync(kFull, a[0], 1); }

template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ void copy_pair(T* dst, const T* row, int c0, int c1, bool vec) {
  if (vec) {
    cp_async<2 * sizeof(T)>(dst, row + c0);
  } else {
    cp_async<sizeof(T)>(dst, row + c0);
    cp_async<sizeof(T)>(dst + 1, row + c1);
  }
}

template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& comp, T t) {
  const T y = t - comp;
  const T u = s + y;
  comp = (u - s) - y;
  s = u;
}

// donor-cell sum psi - Fp0/G + Fm0/G - Fp1/G + Fm1/G (dimension 0 first), rG = 1/G
template <typename T, bool NUG>
__device__ __forceinline__ T donor(T p, T Fp0, T Fm0, T Fp1, T Fm1, T rG, bool kahan) {
  if (NUG) {
    Fp0 *= rG;
    Fm0 *= rG;
    Fp1 *= rG;
    Fm1 *= rG;
  }
  if (kahan) {
    T s = p, comp = T(0);
    kahan_add(s, comp, -Fp0);
    kahan_add(s, comp, Fm0);
    kahan_add(s, comp, -Fp1);
    kahan_add(s, comp, Fm1);
    return s;
  }
  return (((p - Fp0) + Fm0) - Fp1) + Fm1;
}

template <typename T, bool FCT, bool NUG>
__global__ void __launch_bounds__(kWarps * 32) k_fused2d(const F2Params<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long wid = static_cast<long long>(blockIdx.x) * kWarps + wib;
  if (wid >= static_cast<long long>(p.strips) * p.rowtiles) return;  // whole warp
  const int strip = static_cast<int>(wid % p.strips);
  const int R0 = static_cast<int>(wid / p.strips) * p.ty;
  const int lc0 = 2 * lane;
  const int cs = strip * kStride - kLead;
  const int c0 = wrapi(cs + lc0, p.n1), c1 = wrapi(cs + lc0 + 1, p.n1);
  T* ring = reinterpret_cast<T*>(smem_raw) + static_cast<size_t>(wib) * kSlots * kArr * kCols;
  const int nt = p.ty + 6;

  auto issue = [&](int t) {
    if (t < nt) {
      const long long base = static_cast<long long>(wrapi(R0 - 3 + t, p.n0)) * p.n1;
      T* slot = ring + (t % kSlots) * kArr * kCols + lc0;
      copy_pair(slot, p.psi + base, c0, c1, p.vec);
      copy_pair(slot + kCols, p.gc0 + base, c0, c1, p.vec);
      copy_pair(slot + 2 * kCols, p.gc1 + base, c0, c1, p.vec);
      if (NUG) copy_pair(slot + 3 * kCols, p.G + base, c0, c1, p.vec);
      if (p.rhs_b) copy_pair(slot + 4 * kCols, p.R + base, c0, c1, p.vec);
    }
    cp_commit();
  };
#pragma unroll
  for (int t = 0; t < kPF; ++t) issue(t);

  // register windows, [row][column of the lane]; row 0 is the oldest
  T ps[4][2], v0[3][2], v1[3][2], gg[4][2];
  T p1[4][2], p1r[3];
  T hi[3][2], lo[3][2];
  T pv0[2][2], f0c[2];
  T a0[2][2], u0[2][2], a1[2][2], u1[2][2], bu[2][2], bd[2][2], h0c[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
#pragma unroll
    for (int k = 0; k < 4; ++k) { ps[k][c] = T(0); gg[k][c] = T(1); p1[k][c] = T(0); }
#pragma unroll
    for (int k = 0; k < 3; ++k) { v0[k][c] = v1[k][c] = hi[k][c] = lo[k][c] = T(0); }
#pragma unroll
    for (int k = 0; k < 2; ++k) { pv0[k][c] = a0[k][c] = u0[k][c] = a1[k][c] = u1[k][c] = T(0); bu[k][c] = bd[k][c] = T(1); }
    f0c[c] = h0c[c] = T(0);
  }
  p1r[0] = p1r[1] = p1r[2] = T(0);
  const bool iga = p.iga, kahan = p.kahan;

  for (int t = 0; t < nt; ++t) {
    // ---- load row x = R0 - 3 + t
    cp_wait<kPF - 1>();
    {
      const T* slot = ring + (t % kSlots) * kArr * kCols + lc0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        ps[0][c] = ps[1][c]; ps[1][c] = ps[2][c]; ps[2][c] = ps[3][c];
        v0[0][c] = v0[1][c]; v0[1][c] = v0[2][c];
        v1[0][c] = v1[1][c]; v1[1][c] = v1[2][c];
        T x = slot[c];
        if (p.rhs_b) x = x + p.dt * slot[4 * kCols + c];
        ps[3][c] = x;
        v0[2][c] = slot[kCols + c] * p.scale;
        v1[2][c] = slot[2 * kCols + c] * p.scale;
        if (NUG) { gg[0][c] = gg[1][c]; gg[1][c] = gg[2][c]; gg[2][c] = gg[3][c]; gg[3][c] = slot[3 * kCols + c]; }
      }
    }
    issue(t + kPF);

    // ---- pass 1 (Eqs. 4-5) at row r = x-1
    T fnew[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) fnew[c] = flux(ps[2][c], ps[3][c], v0[1][c]);  // face (x-1)+1/2
    if (t >= 2) {
      const T psR = from_right(ps[2]);
      T F1[2];
      F1[0] = flux(ps[2][0], ps[2][1], v1[1][0]);
      F1[1] = flux(ps[2][1], psR, v1[1][1]);
      const T F1L = from_left(F1);
      T np1[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T rG = NUG ? fdiv(T(1), gg[2][c]) : T(1);
        np1[c] = donor<T, NUG>(ps[2][c], fnew[c], f0c[c], F1[c], c == 0 ? F1L : F1[0], rG, kahan);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        p1[0][c] = p1[1][c]; p1[1][c] = p1[2][c]; p1[2][c] = p1[3][c]; p1[3][c] = np1[c];
        if (FCT) {
          hi[0][c] = hi[1][c]; hi[1][c] = hi[2][c]; hi[2][c] = maxv(ps[2][c], np1[c]);
          lo[0][c] = lo[1][c]; lo[1][c] = lo[2][c]; lo[2][c] = minv(ps[2][c], np1[c]);
        }
      }
      p1r[0] = p1r[1]; p1r[1] = p1r[2]; p1r[2] = from_right(p1[3]);
    }
    f0c[0] = fnew[0];
    f0c[1] = fnew[1];

    // ---- row r = x-2: pseudo-advectors (Eq. 6 + cross term), unlimited fluxes, FCT factors
    if (t >= 3) {
      // dimension-0 faces between rows r and r+1
      const T v0R = from_right(v0[0]);
      T S0[2], PV1[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) { S0[c] = p1[2][c] + p1[3][c]; PV1[c] = v1[0][c] + v1[1][c]; }
      const T S0L = from_left(S0), S0R = from_right(S0), PV1L = from_left(PV1);
      T na0[2], nu0[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T V = v0[0][c];
        const T Gb = NUG ? T(0.5) * (gg[1][c] + gg[2][c]) : T(1);
        const T d = p1[3][c] - p1[2][c];
        const T A = iga ? d * T(0.5) : ratio(d, S0[c]);
        const T Tt = c == 0 ? S0[1] : S0R, Bt = c == 0 ? S0L : S0[0];
        const T B = iga ? (Tt - Bt) * T(0.25) : ratio(Tt - Bt, Tt + Bt);
        const T Vq = T(0.25) * (PV1[c] + (c == 0 ? PV1L : PV1[0]));
        const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
        const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
        na0[c] = out;
        nu0[c] = iga ? out : flux(p1[2][c], p1[3][c], out);
      }
      T npv[2] = {v0[0][0] + v0[0][1], v0[0][1] + v0R};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        pv0[0][c] = pv0[1][c]; pv0[1][c] = npv[c];
        a0[0][c] = a0[1][c]; a0[1][c] = na0[c];
        u0[0][c] = u0[1][c]; u0[1][c] = nu0[c];
      }
    }
    if (t >= 4) {
      // dimension-1 faces (r, j+1/2)
      T Sm[2], Sc[2], Sp[2];
      Sm[0] = p1[1][0] + p1[1][1]; Sm[1] = p1[1][1] + p1r[0];
      Sc[0] = p1[2][0] + p1[2][1]; Sc[1] = p1[2][1] + p1r[1];
      Sp[0] = p1[3][0] + p1[3][1]; Sp[1] = p1[3][1] + p1r[2];
      const T gR = NUG ? from_right(gg[1]) : T(1);
      T na1[2], nu1[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T V = v1[0][c];
        const T Gb = NUG ? T(0.5) * (gg[1][c] + (c == 0 ? gg[1][1] : gR)) : T(1);
        const T q0 = p1[2][c], q1 = c == 0 ? p1[2][1] : p1r[1];
        const T A = iga ? (q1 - q0) * T(0.5) : ratio(q1 - q0, Sc[c]);
        const T B = iga ? (Sp[c] - Sm[c]) * T(0.25) : ratio(Sp[c] - Sm[c], Sp[c] + Sm[c]);
        const T Vq = T(0.25) * (pv0[1][c] + pv0[0][c]);
        const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
        const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
        na1[c] = out;
        nu1[c] = iga ? out : flux(q0, q1, out);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        a1[0][c] = a1[1][c]; a1[1][c] = na1[c];
        u1[0][c] = u1[1][c]; u1[1][c] = nu1[c];
      }
      if (FCT) {
        // bounds (extrema of psi^n and psi^(1) over the cell and its face neighbours)
        const T hL = from_left(hi[1]), hR = from_right(hi[1]);
        const T lL = from_left(lo[1]), lR = from_right(lo[1]);
        const T u1L = from_left(u1[1]);
        T nbu[2], nbd[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T mx = maxv(maxv(maxv(hi[1][c], hi[0][c]), maxv(hi[2][c], c == 0 ? hL : hi[1][0])),
                            c == 0 ? hi[1][1] : hR);
          const T mn = minv(minv(minv(lo[1][c], lo[0][c]), minv(lo[2][c], c == 0 ? lL : lo[1][0])),
                            c == 0 ? lo[1][1] : lR);
          const T Fm0 = u0[0][c], Fp0 = u0[1][c];
          const T Fp1 = u1[1][c], Fm1 = c == 0 ? u1L : u1[1][0];
          const T in = (posp(Fm0) - negp(Fp0)) + (posp(Fm1) - negp(Fp1));
          const T ou = (posp(Fp0) - negp(Fm0)) + (posp(Fp1) - negp(Fm1));
          const T Gi = NUG ? gg[1][c] : T(1);
          const T q = p1[2][c];
          nbu[c] = in > T(0) ? minv(T(1), fdiv(Gi * posp(mx - q), in)) : T(1);
          nbd[c] = ou > T(0) ? minv(T(1), fdiv(Gi * posp(q - mn), ou)) : T(1);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          bu[0][c] = bu[1][c]; bu[1][c] = nbu[c];
          bd[0][c] = bd[1][c]; bd[1][c] = nbd[c];
        }
      }
    }

    // ---- row r = x-3: limited fluxes and pass 2
    if (t >= 5) {
      T h0[2], h1[2];
      if (FCT) {
        const T buR = from_right(bu[0]), bdR = from_right(bd[0]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          {  // face (r+1/2, c) between rows r and r+1
            const T V = a0[0][c], F = u0[0][c];
            const bool right = F > T(0) || (F == T(0) && V > T(0));
            const T m = minv(right ? bd[0][c] : bu[0][c], right ? bu[1][c] : bd[1][c]);
            h0[c] = F * m;
          }
          {  // face (r, c+1/2)
            const T V = a1[0][c], F = u1[0][c];
            const bool right = F > T(0) || (F == T(0) && V > T(0));
            const T a = right ? bd[0][c] : bu[0][c];
            const T b = right ? (c == 0 ? bu[0][1] : buR) : (c == 0 ? bd[0][1] : bdR);
            h1[c] = F * minv(a, b);
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c) { h0[c] = u0[0][c]; h1[c] = u1[0][c]; }
      }
      if (t >= 6) {
        const T h1L = from_left(h1);
        const int row = R0 + t - 6;
        T np2[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T rG = NUG ? fdiv(T(1), gg[0][c]) : T(1);
          np2[c] = donor<T, NUG>(p1[1][c], h0[c], h0c[c], h1[c], c == 0 ? h1L : h1[0], rG, kahan);
        }
        if (row < p.n0) {
          const int col = strip * kStride + lc0 - kLead;
          const bool ok0 = lc0 >= kLead && lc0 < kLead + kStride && col < p.n1;
          const bool ok1 = lc0 + 1 >= kLead && lc0 + 1 < kLead + kStride && col + 1 < p.n1;
          const long long o = static_cast<long long>(row) * p.n1 + col;
          if (p.rhs_a) {
            if (ok0) np2[0] = np2[0] + p.dt * p.R[o];
            if (ok1) np2[1] = np2[1] + p.dt * p.R[o + 1];
          }
          if (p.vec && ok0 && ok1) {
            if constexpr (sizeof(T) == 4) {
              *reinterpret_cast<float2*>(p.out + o) = make_float2(np2[0], np2[1]);
            } else {
              *reinterpret_cast<double2*>(p.out + o) = make_double2(np2[0], np2[1]);
            }
          } else {
            if (ok0) p.out[o] = np2[0];
            if (ok1) p.out[o + 1] = np2[1];
          }
        }
      }
      h0c[0] = h0[0];
      h0c[1] = h0[1];
    }
  }
  cp_wait<0>();
}

template <typename T, bool FCT, bool NUG>
void launch(const F2Params<T>& p, cudaStream_t st) {
  const long long warps = static_cast<long long>(p.strips) * p.rowtiles;
  const unsigned blocks = static_cast<unsigned>((warps + kWarps - 1) / kWarps);
  const size_t smem = static_cast<size_t>(kWarps) * kSlots * kArr * kCols * sizeof(T);
  static bool attr_set = false;  // FP64 rings exceed the default 48 KB of dynamic shared memory
  if (!attr_set) {
    cudaFuncSetAttribute(k_fused2d<T, FCT, NUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    attr_set = true;
  }
  k_fused2d<T, FCT, NUG><<<blocks, kWarps * 32, smem, st>>>(p);
}

bool al(const void* q, size_t a) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) % a) == 0; }

}  // namespace

template <typename T>
int fused_step(const Grid& g, const Opts& o, const StepArgs<T>& a, T*, cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot) return MPDATA_EUNSUPPORTED;
  if (a.psi_out == a.psi_in) return MPDATA_EUNSUPPORTED;
  F2Params<T> p;
  p.psi = a.psi_in;
  p.out = a.psi_out;
  p.gc0 = a.gc[0];
  p.gc1 = a.gc[1];
  p.G = o.nug ? a.g : nullptr;
  p.R = a.r;
  p.n0 = g.n[1];
  p.n1 = g.n[2];
  p.strips = (p.n1 + kStride - 1) / kStride;
  p.ty = 8;
  for (int ty : {64, 32, 16}) {
    if (static_cast<long long>(p.strips) * ((p.n0 + ty - 1) / ty) >= 152LL * 8) { p.ty = ty; break; }
  }
  p.rowtiles = (p.n0 + p.ty - 1) / p.ty;
  p.dt = a.dt;
  p.scale = a.gc_scale;
  p.iga = o.iga;
  p.kahan = o.kahan;
  p.rhs_a = o.rhs_a;
  p.rhs_b = o.rhs_b;
  const size_t va = 2 * sizeof(T);
  p.vec = (p.n1 % 2 == 0) && al(p.psi, va) && al(p.out, va) && al(p.gc0, va) && al(p.gc1, va) &&
          al(p.G, va) && al(p.R, va);
  if (o.fct) {
    if (o.nug) launch<T, true, true>(p, st); else launch<T, true, false>(p, st);
  } else {
    if (o.nug) launch<T, false, true>(p, st); else launch<T, false, false>(p, st);
  }
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template int fused_step<float>(const Grid&, const Opts&, const StepArgs<float>&, float*, cudaStream_t);
template int fused_step<double>(const Grid&, const Opts&, const StepArgs<double>&, double*, cudaStream_t);

}  // namespace mpd
