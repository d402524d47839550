// Temporal blocking of the 2D step: S MPDATA steps per launch (the fusion depth).
//
// A step's result at a cell depends on the step's input within 3 cells (pass 1 reaches 1, the
// bounds and the pseudo-advector 1 more, the limiting factors and the limited fluxes of the
// corrective pass 1 more), so S steps of a tile need its input with a 3S-cell halo.  A block
// loads that region of psi and of both advector components into shared memory once, runs the S
// steps there -- each sub-step (pass 1; antidiffusive fluxes; factors; limiting; pass 2) a loop
// over its region separated by block barriers, the regions shrinking by 3 cells per step -- and
// writes the tile.  Global traffic per S steps: the haloed input once and the tile once; the
// price is the recomputed halo and every neighbour read going through shared memory.
//
// The arithmetic is that of the warp march (Eqs. 4-6 with the cross term, FCT of Sect. 3.1.4,
// infinite gauge of Sect. 3.1.5), the same expressions in the same order, so a depth-S launch
// and S warp-march steps agree to rounding.  Covers 2D fields with n_iters = 2, FCT or not,
// infinite gauge or not, G = 1, no sources, periodic edges; one advector scale per step (a flow
// evaluated at n + 1/2).
#include <cuda_runtime.h>

#include "kernels.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

using namespace dev;

constexpr int kTile = 32;  // output tile side
constexpr int kTbThreads = 256;
constexpr int kTbMaxDepth = kTblockMaxDepth;
constexpr int kTbArrays = 8;

struct TbScales { double s[kTbMaxDepth]; };

template <typename T>
struct TbParams {
  const T* psi;
  T* out;
  const T* gc0;
  const T* gc1;
  int n0, n1, depth;
  TbScales scale;
};

template <typename T>
constexpr size_t tb_smem(int depth) {
  const size_t L = kTile + 6 * depth;
  return sizeof(T) * kTbArrays * L * L;
}

// f(r, c) over the rows [r0, r1) x columns [c0, c1) of the region, the cells numbered row by
// row and dealt to the threads in turn (every lane busy whatever the region's width)
template <class F>
__device__ __forceinline__ void region_for(int r0, int r1, int c0, int c1, F&& f) {
  const int W = c1 - c0, n = (r1 - r0) * W;
  if (n <= 0) return;
  const int t = static_cast<int>(threadIdx.x);
  int r = r0 + t / W, c = c0 + t % W;
  const int dr = kTbThreads / W, dc = kTbThreads % W;
  for (int k = t; k < n; k += kTbThreads) {
    f(r, c);
    r += dr;
    c += dc;
    if (c >= c1) {
      c -= W;
      ++r;
    }
  }
}

template <typename T, bool FCT, bool IGA>
__global__ void __launch_bounds__(kTbThreads) k_tblock2d(const TbParams<T> p) {
  const int S = p.depth;
  const int H = 3 * S, L = kTile + 2 * H, A = L * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const P = reinterpret_cast<T*>(smem_raw);  // psi of the current step, then its result
  T* const Q = P + A;                           // psi^(1)
  T* const G0 = Q + A;                          // input advector, dimension 0 (rows)
  T* const G1 = G0 + A;                         // input advector, dimension 1 (columns)
  T* const F0 = G1 + A;                         // antidiffusive flux, dimension-0 faces
  T* const F1 = F0 + A;                         // the same, dimension-1 faces
  T* const BU = F1 + A;                         // FCT factors
  T* const BD = BU + A;
  const int x0 = static_cast<int>(blockIdx.y) * kTile - H;  // region origin: row
  const int y0 = static_cast<int>(blockIdx.x) * kTile - H;  // region origin: column
  // load the region (periodic wrap); consecutive threads take consecutive columns of a row
  region_for(0, L, 0, L, [&](int r, int c) {
    int gr = x0 + r, gc = y0 + c;
    while (gr < 0) gr += p.n0;
    while (gr >= p.n0) gr -= p.n0;
    while (gc < 0) gc += p.n1;
    while (gc >= p.n1) gc -= p.n1;
    const long long gi = static_cast<long long>(gr) * p.n1 + gc;
    const int li = r * L + c;
    P[li] = p.psi[gi];
    G0[li] = p.gc0[gi];
    G1[li] = p.gc1[gi];
  });
  __syncthreads();
  for (int k = 0; k < S; ++k) {
    double skd = p.scale.s[0];  // (selected, not indexed: the parameters stay out of local memory)
#pragma unroll
    for (int j = 1; j < kTbMaxDepth; ++j)
      if (k == j) skd = p.scale.s[j];
    const T sc = static_cast<T>(skd);
    const int e = 3 * (S - 1 - k);  // this step's result is needed on the tile plus e cells
    // pass 1 (Eqs. 4-5) on margin e + 2
    {
      const int lo = H - e - 2, hi = H + kTile + e + 2;
      region_for(lo, hi, lo, hi, [&](int r, int c) {
        const int i = r * L + c;
        const T pc = P[i];
        const T Fp0 = flux(pc, P[i + L], G0[i] * sc), Fm0 = flux(P[i - L], pc, G0[i - L] * sc);
        const T Fp1 = flux(pc, P[i + 1], G1[i] * sc), Fm1 = flux(P[i - 1], pc, G1[i - 1] * sc);
        Q[i] = donor<T, false, false>(pc, Fp0, Fm0, Fp1, Fm1, T(1));
      });
    }
    __syncthreads();
    const int lo = H - e - 1, hi = H + kTile + e + 1;  // margin e + 1: factors
    // antidiffusive fluxes (Eq. 6 with the cross term, then Eq. 5) at the faces of the margin-
    // (e + 1) cells: dimension 0 on rows [lo-1, hi) x columns [lo, hi), dimension 1 on rows
    // [lo, hi) x columns [lo-1, hi)
    region_for(lo - 1, hi, lo - 1, hi, [&](int r, int c) {
      const int i = r * L + c;
      const T q0 = Q[i];
      if (c >= lo) {  // face between rows r and r+1
        const int ip = i + L;
        const T V = G0[i] * sc;
        const T q1 = Q[ip];
        const T Av = IGA ? (q1 - q0) * T(0.5) : ratio(q1 - q0, q0 + q1);
        const T Tt = Q[i + 1] + Q[ip + 1], Bt = Q[i - 1] + Q[ip - 1];
        const T B = IGA ? (Tt - Bt) * T(0.25) : ratio(Tt - Bt, Tt + Bt);
        const T Vq = T(0.25) * ((G1[i] * sc + G1[ip] * sc) + (G1[i - 1] * sc + G1[ip - 1] * sc));
        const T v = (absv(V) - V * V) * Av - T(0.5) * V * Vq * B;
        F0[i] = IGA ? v : flux(q0, q1, v);
      }
      if (r >= lo) {  // face between columns c and c+1
        const int ip = i + 1;
        const T V = G1[i] * sc;
        const T q1 = Q[ip];
        const T Av = IGA ? (q1 - q0) * T(0.5) : ratio(q1 - q0, q0 + q1);
        const T Sp = Q[i + L] + Q[ip + L], Sm = Q[i - L] + Q[ip - L];
        const T B = IGA ? (Sp - Sm) * T(0.25) : ratio(Sp - Sm, Sp + Sm);
        const T Vq = T(0.25) * ((G0[i] * sc + G0[ip] * sc) + (G0[i - L] * sc + G0[ip - L] * sc));
        const T v = (absv(V) - V * V) * Av - T(0.5) * V * Vq * B;
        F1[i] = IGA ? v : flux(q0, q1, v);
      }
    });
    __syncthreads();
    const int lo2 = H - e, hi2 = H + kTile + e;  // margin e: this step's result
    if (FCT) {
      // factors on margin e + 1 (Sect. 3.1.4): bounds from psi^n and psi^(1) over the cell and
      // its face neighbours, in/out sums of the unlimited fluxes
      region_for(lo, hi, lo, hi, [&](int r, int c) {
        const int i = r * L + c;
        const T q = Q[i];
        T mx = maxv(P[i], q), mn = minv(P[i], q);
        const int nb[4] = {i - L, i + L, i - 1, i + 1};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T a = P[nb[j]], b = Q[nb[j]];
          mx = maxv(mx, maxv(a, b));
          mn = minv(mn, minv(a, b));
        }
        const T Fp0 = F0[i], Fm0 = F0[i - L], Fp1 = F1[i], Fm1 = F1[i - 1];
        const T pFm0 = posp(Fm0), nFp0 = negp(Fp0), pFm1 = posp(Fm1), nFp1 = negp(Fp1);
        const T in = (pFm0 - nFp0) + (pFm1 - nFp1);
        const T ou = ((Fp0 - nFp0) - (Fm0 - pFm0)) + ((Fp1 - nFp1) - (Fm1 - pFm1));
        // min(1, x / |s|) is 1 for s = 0 (x/0 is inf or NaN, and min ignores NaN)
        BU[i] = min1(fdiv(posp(mx - q), absv(in)));
        BD[i] = min1(fdiv(posp(q - mn), absv(ou)));
      });
      __syncthreads();
      // limited fluxes at the faces of the margin-e cells, in place: F min(beta_dn of the
      // upwind cell, beta_up of the downwind cell) (a zero flux stays zero)
      region_for(lo2 - 1, hi2, lo2 - 1, hi2, [&](int r, int c) {
        const int i = r * L + c;
        if (c >= lo2) {
          const T F = F0[i];
          const bool right = F > T(0);
          F0[i] = F * minv(right ? BD[i] : BU[i], right ? BU[i + L] : BD[i + L]);
        }
        if (r >= lo2) {
          const T F = F1[i];
          const bool right = F > T(0);
          F1[i] = F * minv(right ? BD[i] : BU[i], right ? BU[i + 1] : BD[i + 1]);
        }
      });
      __syncthreads();
    }
    // pass 2 (Eq. 4 with the antidiffusive fluxes) on margin e into P
    region_for(lo2, hi2, lo2, hi2, [&](int r, int c) {
      const int i = r * L + c;
      P[i] = donor<T, false, false>(Q[i], F0[i], F0[i - L], F1[i], F1[i - 1], T(1));
    });
    __syncthreads();
  }
  // the tile
  region_for(H, H + kTile, H, H + kTile, [&](int r, int c) {
    const int gr = static_cast<int>(blockIdx.y) * kTile + (r - H);
    const int gc = static_cast<int>(blockIdx.x) * kTile + (c - H);
    if (gr < p.n0 && gc < p.n1) p.out[static_cast<long long>(gr) * p.n1 + gc] = P[r * L + c];
  });
}

// the deepest S whose shared-memory region fits the opt-in limit (227 KB)
template <typename T>
int max_depth() {
  int s = kTbMaxDepth;
  while (s > 1 && tb_smem<T>(s) > static_cast<size_t>(227) * 1024) --s;
  return s;
}

template <typename T, bool FCT, bool IGA>
int launch_tb(const TbParams<T>& p, cudaStream_t st) {
  static PerDevice<bool> attr;
  const bool ok = attr.get([](int) {
    return cudaFuncSetAttribute(k_tblock2d<T, FCT, IGA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(tb_smem<T>(max_depth<T>()))) == cudaSuccess;
  });
  if (!ok) return MPDATA_ECUDA;
  const dim3 grid(static_cast<unsigned>((p.n1 + kTile - 1) / kTile), static_cast<unsigned>((p.n0 + kTile - 1) / kTile));
  k_tblock2d<T, FCT, IGA><<<grid, kTbThreads, tb_smem<T>(p.depth), st>>>(p);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

}  // namespace

template <typename T>
bool tblock_covers(const Grid& g, const Opts& o, int depth) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open || o.nug || o.kahan || o.rhs_a || o.rhs_b)
    return false;
  // the launch grid's y extent is limited to 65535 row tiles
  return depth >= 1 && depth <= max_depth<T>() && g.n[1] <= 65535 * kTile;
}
template bool tblock_covers<float>(const Grid&, const Opts&, int);
template bool tblock_covers<double>(const Grid&, const Opts&, int);

template <typename T>
int tblock_steps(const Grid& g, const Opts& o, const T* psi_in, T* psi_out, const T* gc0, const T* gc1, int depth,
                 const double* scales, cudaStream_t st) {
  if (!tblock_covers<T>(g, o, depth) || psi_in == psi_out) return MPDATA_EUNSUPPORTED;
  TbParams<T> p;
  p.psi = psi_in;
  p.out = psi_out;
  p.gc0 = gc0;
  p.gc1 = gc1;
  p.n0 = g.n[1];
  p.n1 = g.n[2];
  p.depth = depth;
  for (int k = 0; k < kTbMaxDepth; ++k) p.scale.s[k] = (scales && k < depth) ? scales[k] : 1.0;
  if (o.fct) return o.iga ? launch_tb<T, true, true>(p, st) : launch_tb<T, true, false>(p, st);
  return o.iga ? launch_tb<T, false, true>(p, st) : launch_tb<T, false, false>(p, st);
}

template int tblock_steps<float>(const Grid&, const Opts&, const float*, float*, const float*, const float*, int,
                                 const double*, cudaStream_t);
template int tblock_steps<double>(const Grid&, const Opts&, const double*, double*, const double*, const double*,
                                  int, const double*, cudaStream_t);

}  // namespace mpd
