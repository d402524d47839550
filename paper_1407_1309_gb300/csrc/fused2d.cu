// Fused 2D MPDATA step: the donor-cell pass, the FCT bounds, the antidiffusive
// pseudo-advector (Eq. 6 with its cross term), the FCT limiting factors and the
// corrective donor-cell pass of one time step in one kernel, with no
// intermediate written to global memory.  Covers 2D fields with n_iters = 2 and
// every option except the third-order terms (those run on the staged path).
//
// Work decomposition ("warp march"): a warp owns a strip of 32*NC columns (NC
// adjacent columns per lane) and walks down TY rows.  Vertical neighbours stay
// in per-thread register windows (one row of each quantity per iteration),
// horizontal neighbours inside a lane are registers and across lanes come from
// warp shuffles.  A step's stencil reaches 3 cells (two passes plus the
// limiter), so each strip recomputes a 3-column halo on both sides and stores
// the 32*NC - 8 columns in its middle; strips start 4 columns left of their
// first output, so every lane's NC columns are aligned and the copies are
// vectorised.  Input rows are prefetched kPF rows ahead into a per-warp
// shared-memory ring with cp.async (each lane copies and later reads only its
// own elements, so no barrier is involved).
//
// Row lags at iteration t (row x = R0 - 3 + t loaded):
//   pass 1 at row x-1; bounds, pseudo-advectors, unlimited fluxes and limiting
//   factors at row x-2; limited fluxes and pass 2 at row x-3 (stored).
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

using namespace dev;

constexpr int kLead = 4;     // computed columns left of the strip's first output column
constexpr int kPF = 4;       // rows in flight
constexpr int kSlots = kPF + 1;
// arrays in a ring slot: psi, gc0, gc1, G, R [, lo of the compensated state]
template <bool COMP> constexpr int arrs() { return COMP ? 6 : 5; }
constexpr int kWarps = 4;    // warps per block

template <int NC> constexpr int cols() { return 32 * NC; }
template <int NC> constexpr int stride() { return 32 * NC - 2 * kLead; }

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
  int rhs_a, rhs_b, vec;
  const T* lo;   // compensated state: low parts in / out (COMP only)
  T* lo_out;
  T* tape;       // adjoint tape (TAPE only): arrays of tape_n elements
  long long tape_n;
};

// One warp marches one tile: the strip `strip` (columns strip*kStride - kLead ...) from
// row R0 down ty rows of the field described by p; `ring` is the warp's shared-memory ring.
// COMP: the state is the pair psi = hi + lo (hi in p.psi, lo in p.lo); every stencil
// quantity is formed from the hi parts, both donor passes add their flux divergence to hi with
// an error-free two-sum (donor_comp), the first pass also moves the low parts with their own
// donor-cell fluxes
// (the corrective pass's low-part fluxes are of the order of FP32 rounding and omitted),
// and both parts are stored.
// TAPE: the step also writes, for the tile's own rows, what the reverse step reads: psi^(1)
// (tape array 0), the pseudo-advectors of both dimensions (1, 2) and under FCT the bounds
// (5, 6) and the factors (7, 8); the limited advectors (3, 4) are left to the reverse step,
// which re-derives them from these.
template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN, bool COMP, bool TAPE = false>
__device__ __forceinline__ void march_tile(const F2Params<T>& p, const int strip, const int R0, T* ring_warp,
                                           const int lane) {
  constexpr int kArr = arrs<COMP>();
  constexpr int kCols = cols<NC>();
  constexpr int kStride = stride<NC>();
  const int lc0 = NC * lane;
  const int cs = strip * kStride - kLead;
  int col[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) col[c] = wrapi(cs + lc0 + c, p.n1);
  T* ring = ring_warp + lc0;
  const int nt = p.ty + 6;
  // one row of tape array j, own rows and columns only
  auto tape_store = [&](const int j, const int row, const T (&v)[NC]) {
    if (!TAPE || row < R0 || row >= R0 + p.ty || row >= p.n0) return;
    const int gcol = strip * kStride + lc0 - kLead;
    T* q = p.tape + j * p.tape_n + static_cast<long long>(row) * p.n1 + gcol;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (lc0 + c >= kLead && lc0 + c < kLead + kStride && gcol + c < p.n1) q[c] = v[c];
  };
  const T* src[6] = {p.psi, p.gc0, p.gc1, NUG ? p.G : nullptr, p.rhs_b ? p.R : nullptr, COMP ? p.lo : nullptr};
  // prefetch cursor: next row to copy, its element offset and ring slot
  int pf_t = 0, pf_row = wrapi(R0 - 3, p.n0), pf_slot = 0;
  long long pf_off = static_cast<long long>(pf_row) * p.n1;

  auto issue = [&]() {
    if (pf_t < nt) {
      T* slot = ring + pf_slot * kArr * kCols;
#pragma unroll
      for (int a = 0; a < kArr; ++a) {
        if (a == 3 && !NUG) continue;
        if (a == 4 && !p.rhs_b) continue;
        const T* q = src[a] + pf_off;
        if (p.vec) {
          constexpr int bytes = NC * static_cast<int>(sizeof(T));
          if constexpr (bytes <= 16) {
            cp_async<bytes>(slot + a * kCols, q + col[0]);
          } else {
            constexpr int per = 16 / static_cast<int>(sizeof(T));
#pragma unroll
            for (int h = 0; h < bytes / 16; ++h) cp_async<16>(slot + a * kCols + h * per, q + col[0] + h * per);
          }
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) cp_async<sizeof(T)>(slot + a * kCols + c, q + col[c]);
        }
      }
      ++pf_t;
      pf_slot = pf_slot + 1 == kSlots ? 0 : pf_slot + 1;
      pf_row = pf_row + 1 == p.n0 ? 0 : pf_row + 1;
      pf_off = static_cast<long long>(pf_row) * p.n1;
    }
    cp_commit();
  };
#pragma unroll
  for (int t = 0; t < kPF; ++t) issue();
  int rd_slot = 0;

  // register windows, [row][column of the lane]; row 0 is the oldest
  T ps[4][NC], v0[3][NC], v1[3][NC], gg[4][NC];
  T p1[4][NC], p1r[3];
  T hi[3][NC], lo[3][NC];
  T pv0[2][NC], f0c[NC];
  T a0[2][NC], u0[2][NC], a1[2][NC], u1[2][NC], bu[2][NC], bd[2][NC], h0c[NC];
  // COMP: lo of the loaded rows x-2 .. x, the low-part flux through face (x-2)+1/2, and lo of
  // pass 1's rows x-3 .. x-1
  T lw[3][NC], flc[NC], l1[3][NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
#pragma unroll
    for (int k = 0; k < 4; ++k) { ps[k][c] = T(0); gg[k][c] = T(1); p1[k][c] = T(0); }
#pragma unroll
    for (int k = 0; k < 3; ++k) { v0[k][c] = v1[k][c] = hi[k][c] = lo[k][c] = T(0); }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      pv0[k][c] = a0[k][c] = u0[k][c] = a1[k][c] = u1[k][c] = T(0);
      bu[k][c] = bd[k][c] = T(1);
    }
    f0c[c] = h0c[c] = T(0);
    lw[0][c] = lw[1][c] = lw[2][c] = flc[c] = l1[0][c] = l1[1][c] = l1[2][c] = T(0);
  }
  p1r[0] = p1r[1] = p1r[2] = T(0);

  // One iteration of the march: load row x = R0 - 3 + t and advance every stage by one
  // row.  In the six ramp iterations (steady = false) a stage only runs once the rows it
  // reads exist; afterwards every stage runs every iteration.
  auto body = [&](const int t, auto steady) {
    constexpr bool S = decltype(steady)::value;
    // ---- load row x = R0 - 3 + t
    cp_wait<kPF - 1>();
    {
      const T* slot = ring + rd_slot * kArr * kCols;
      rd_slot = rd_slot + 1 == kSlots ? 0 : rd_slot + 1;
      copy_row(ps[0], ps[1]); copy_row(ps[1], ps[2]); copy_row(ps[2], ps[3]);
      copy_row(v0[0], v0[1]); copy_row(v0[1], v0[2]);
      copy_row(v1[0], v1[1]); copy_row(v1[1], v1[2]);
      if (NUG) { copy_row(gg[0], gg[1]); copy_row(gg[1], gg[2]); copy_row(gg[2], gg[3]); }
      if (COMP) { copy_row(lw[0], lw[1]); copy_row(lw[1], lw[2]); }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T x = slot[c];
        if (COMP) {
          T e = slot[5 * kCols + c];
          if (p.rhs_b) two_sum_acc(x, e, p.dt * slot[4 * kCols + c]);
          lw[2][c] = e;
        } else if (p.rhs_b) {
          x = x + p.dt * slot[4 * kCols + c];
        }
        ps[3][c] = x;
        v0[2][c] = slot[kCols + c] * p.scale;
        v1[2][c] = slot[2 * kCols + c] * p.scale;
        if (NUG) gg[3][c] = slot[3 * kCols + c];
      }
    }
    issue();

    // ---- pass 1 (Eqs. 4-5) at row r = x-1
    T fnew[NC], flnew[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      fnew[c] = flux(ps[2][c], ps[3][c], v0[1][c]);  // face (x-1)+1/2
      if (COMP) flnew[c] = flux(lw[1][c], lw[2][c], v0[1][c]);  // the low parts through it
    }
    if (S || t >= 2) {
      const T psR = from_right(ps[2]);
      T F1[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) F1[c] = flux(ps[2][c], right_of(ps[2], c, psR), v1[1][c]);
      const T F1L = from_left(F1);
      T np1[NC], nl1[NC], FL1[NC];
      T FL1L = T(0);
      if (COMP) {  // low-part fluxes through the faces (x-1, c+1/2)
        const T loR = from_right(lw[1]);
#pragma unroll
        for (int c = 0; c < NC; ++c) FL1[c] = flux(lw[1][c], right_of(lw[1], c, loR), v1[1][c]);
        FL1L = from_left(FL1);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T rG = NUG ? fdiv(T(1), gg[2][c]) : T(1);
        if (COMP) {
          const T lo_div = (flc[c] - flnew[c]) + (left_of(FL1, c, FL1L) - FL1[c]);
          np1[c] = donor_comp<T, NUG>(ps[2][c], lw[1][c], fnew[c], f0c[c], F1[c], left_of(F1, c, F1L), rG, lo_div,
                                      nl1[c]);
        } else {
          np1[c] = donor<T, NUG, KAHAN>(ps[2][c], fnew[c], f0c[c], F1[c], left_of(F1, c, F1L), rG);
        }
      }
      tape_store(0, R0 - 4 + t, np1);
      copy_row(p1[0], p1[1]); copy_row(p1[1], p1[2]); copy_row(p1[2], p1[3]); copy_row(p1[3], np1);
      if (COMP) { copy_row(l1[0], l1[1]); copy_row(l1[1], l1[2]); copy_row(l1[2], nl1); }
      if (FCT) {
        copy_row(hi[0], hi[1]); copy_row(hi[1], hi[2]);
        copy_row(lo[0], lo[1]); copy_row(lo[1], lo[2]);
#pragma unroll
        for (int c = 0; c < NC; ++c) { hi[2][c] = maxv(ps[2][c], np1[c]); lo[2][c] = minv(ps[2][c], np1[c]); }
      }
      p1r[0] = p1r[1]; p1r[1] = p1r[2]; p1r[2] = from_right(p1[3]);
    }
    copy_row(f0c, fnew);
    if (COMP) copy_row(flc, flnew);

    // ---- row r = x-2: pseudo-advectors (Eq. 6 + cross term), unlimited fluxes, FCT factors
    if (S || t >= 3) {
      // dimension-0 faces between rows r and r+1
      const T v0R = from_right(v0[0]);
      T S0[NC], PV1[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) { S0[c] = p1[2][c] + p1[3][c]; PV1[c] = v1[0][c] + v1[1][c]; }
      const T S0L = from_left(S0), S0R = from_right(S0), PV1L = from_left(PV1);
      T na0[NC], nu0[NC], npv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T V = v0[0][c];
        const T Gb = NUG ? T(0.5) * (gg[1][c] + gg[2][c]) : T(1);
        const T d = p1[3][c] - p1[2][c];
        const T A = IGA ? d * T(0.5) : ratio(d, S0[c]);
        const T Tt = right_of(S0, c, S0R), Bt = left_of(S0, c, S0L);
        const T B = IGA ? (Tt - Bt) * T(0.25) : ratio(Tt - Bt, Tt + Bt);
        const T Vq = T(0.25) * (PV1[c] + left_of(PV1, c, PV1L));
        const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
        const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
        na0[c] = out;
        nu0[c] = IGA ? out : flux(p1[2][c], p1[3][c], out);
        npv[c] = v0[0][c] + right_of(v0[0], c, v0R);
      }
      tape_store(1, R0 - 5 + t, na0);
      copy_row(pv0[0], pv0[1]); copy_row(pv0[1], npv);
      copy_row(a0[0], a0[1]); copy_row(a0[1], na0);
      copy_row(u0[0], u0[1]); copy_row(u0[1], nu0);
    }
    if (S || t >= 4) {
      // dimension-1 faces (r, j+1/2); S1 = psi1_j + psi1_{j+1} on rows r-1, r, r+1
      T Sm[NC], Sc[NC], Sp[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        Sm[c] = p1[1][c] + right_of(p1[1], c, p1r[0]);
        Sc[c] = p1[2][c] + right_of(p1[2], c, p1r[1]);
        Sp[c] = p1[3][c] + right_of(p1[3], c, p1r[2]);
      }
      const T gR = NUG ? from_right(gg[1]) : T(1);
      T na1[NC], nu1[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T V = v1[0][c];
        const T Gb = NUG ? T(0.5) * (gg[1][c] + right_of(gg[1], c, gR)) : T(1);
        const T q0 = p1[2][c], q1 = right_of(p1[2], c, p1r[1]);
        const T A = IGA ? (q1 - q0) * T(0.5) : ratio(q1 - q0, Sc[c]);
        const T B = IGA ? (Sp[c] - Sm[c]) * T(0.25) : ratio(Sp[c] - Sm[c], Sp[c] + Sm[c]);
        const T Vq = T(0.25) * (pv0[1][c] + pv0[0][c]);
        const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
        const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
        na1[c] = out;
        nu1[c] = IGA ? out : flux(q0, q1, out);
      }
      tape_store(2, R0 - 5 + t, na1);
      copy_row(a1[0], a1[1]); copy_row(a1[1], na1);
      copy_row(u1[0], u1[1]); copy_row(u1[1], nu1);
      if (FCT) {
        // bounds (extrema of psi^n and psi^(1) over the cell and its face neighbours)
        const T hL = from_left(hi[1]), hR = from_right(hi[1]);
        const T lL = from_left(lo[1]), lR = from_right(lo[1]);
        const T u1L = from_left(u1[1]);
        T nbu[NC], nbd[NC], tmx[NC], tmn[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T mx = maxv(maxv(maxv(hi[1][c], hi[0][c]), maxv(hi[2][c], left_of(hi[1], c, hL))),
                            right_of(hi[1], c, hR));
          const T mn = minv(minv(minv(lo[1][c], lo[0][c]), minv(lo[2][c], left_of(lo[1], c, lL))),
                            right_of(lo[1], c, lR));
          const T Fm0 = u0[0][c], Fp0 = u0[1][c];
          const T Fp1 = u1[1][c], Fm1 = left_of(u1[1], c, u1L);
          // [x]- = x - [x]+ and [x]+ = x - [x]- hold exactly in floating point, so the
          // outflow sum reuses the inflow sum's four extrema (adds instead of min/max)
          const T pFm0 = posp(Fm0), nFp0 = negp(Fp0), pFm1 = posp(Fm1), nFp1 = negp(Fp1);
          const T in = (pFm0 - nFp0) + (pFm1 - nFp1);
          const T ou = ((Fp0 - nFp0) - (Fm0 - pFm0)) + ((Fp1 - nFp1) - (Fm1 - pFm1));
          const T Gi = NUG ? gg[1][c] : T(1);
          const T q = p1[2][c];
          // min(1, x / |s|) is 1 for s = 0 (x/0 is inf or NaN, and min ignores NaN)
          nbu[c] = min1(fdiv(Gi * posp(mx - q), absv(in)));
          nbd[c] = min1(fdiv(Gi * posp(q - mn), absv(ou)));
          tmx[c] = mx;
          tmn[c] = mn;
        }
        tape_store(5, R0 - 5 + t, tmx);
        tape_store(6, R0 - 5 + t, tmn);
        tape_store(7, R0 - 5 + t, nbu);
        tape_store(8, R0 - 5 + t, nbd);
        copy_row(bu[0], bu[1]); copy_row(bu[1], nbu);
        copy_row(bd[0], bd[1]); copy_row(bd[1], nbd);
      }
    }

    // ---- row r = x-3: limited fluxes and pass 2
    if (S || t >= 5) {
      T h0[NC], h1[NC];
      if (FCT) {
        const T buR = from_right(bu[0]), bdR = from_right(bd[0]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          // With two passes only the limited flux F*m is used, so a zero flux needs no
          // factor: m = min(beta_dn of the upwind cell, beta_up of the downwind cell).
          {  // face (r+1/2, c) between rows r and r+1
            const T F = u0[0][c];
            const bool right = gt0(F);
            h0[c] = F * minv(right ? bd[0][c] : bu[0][c], right ? bu[1][c] : bd[1][c]);
          }
          {  // face (r, c+1/2)
            const T F = u1[0][c];
            const bool right = gt0(F);
            const T a = right ? bd[0][c] : bu[0][c];
            const T b = right ? right_of(bu[0], c, buR) : right_of(bd[0], c, bdR);
            h1[c] = F * minv(a, b);
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) { h0[c] = u0[0][c]; h1[c] = u1[0][c]; }
      }
      if (S || t >= 6) {
        const T h1L = from_left(h1);
        const int row = R0 + t - 6;
        T np2[NC], nl2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T rG = NUG ? fdiv(T(1), gg[0][c]) : T(1);
          if (COMP) {
            np2[c] = donor_comp<T, NUG>(p1[1][c], l1[0][c], h0[c], h0c[c], h1[c], left_of(h1, c, h1L), rG, T(0),
                                        nl2[c]);
          } else {
            np2[c] = donor<T, NUG, KAHAN>(p1[1][c], h0[c], h0c[c], h1[c], left_of(h1, c, h1L), rG);
          }
        }
        if (row < p.n0) {
          const int gcol = strip * kStride + lc0 - kLead;
          const long long o = static_cast<long long>(row) * p.n1 + gcol;
          bool ok[NC];
          bool all = true;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            ok[c] = lc0 + c >= kLead && lc0 + c < kLead + kStride && gcol + c < p.n1;
            all = all && ok[c];
            if (p.rhs_a && ok[c]) {
              if (COMP) {
                T e = nl2[c];
                two_sum_acc(np2[c], e, p.dt * p.R[o + c]);
                const T h = np2[c] + e;  // renormalise
                const T bp = h - np2[c];
                nl2[c] = (np2[c] - (h - bp)) + (e - bp);
                np2[c] = h;
              } else {
                np2[c] = np2[c] + p.dt * p.R[o + c];
              }
            }
            if (COMP && ok[c]) p.lo_out[o + c] = nl2[c];
          }
          if (p.vec && all) {
            if constexpr (sizeof(T) == 4 && NC == 4) {
              *reinterpret_cast<float4*>(p.out + o) = make_float4(np2[0], np2[1], np2[2], np2[3]);
            } else if constexpr (sizeof(T) == 4 && NC == 2) {
              *reinterpret_cast<float2*>(p.out + o) = make_float2(np2[0], np2[1]);
            } else if constexpr (sizeof(T) == 8 && NC == 2) {
              *reinterpret_cast<double2*>(p.out + o) = make_double2(np2[0], np2[1]);
            } else {
#pragma unroll
              for (int c = 0; c < NC; ++c) p.out[o + c] = np2[c];
            }
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c)
              if (ok[c]) p.out[o + c] = np2[c];
          }
        }
      }
      copy_row(h0c, h0);
    }
  };
#pragma unroll
  for (int t = 0; t < 6; ++t) body(t, std::false_type{});
#pragma unroll 2
  for (int t = 6; t < nt; ++t) body(t, std::true_type{});
  cp_wait<0>();
}

template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN, bool COMP, bool TAPE = false>
__global__ void __launch_bounds__(kWarps * 32) k_fused2d(const F2Params<T> p) {
  constexpr int kArr = arrs<COMP>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long wid = static_cast<long long>(blockIdx.x) * kWarps + wib;
  if (wid >= static_cast<long long>(p.strips) * p.rowtiles) return;  // whole warp
  const int strip = static_cast<int>(wid % p.strips);
  const int R0 = static_cast<int>(wid / p.strips) * p.ty;
  T* ring = reinterpret_cast<T*>(smem_raw) + static_cast<size_t>(wib) * kSlots * kArr * cols<NC>();
  march_tile<T, NC, FCT, NUG, IGA, KAHAN, COMP, TAPE>(p, strip, R0, ring, lane);
}

// Ensemble of fields: a persistent grid walks a table of (field, strip, row tile) items.
template <typename T>
struct BatchParams {
  const T* psi;
  T* out;
  const T* gc0;
  const T* gc1;
  const T* G;
  const T* R;
  const BatchField* fields;
  const int* item_field;  // field of every work item
  int n_items, ty;
  T dt, scale;
  int rhs_a, rhs_b, vec_ok;
};

template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN>
__global__ void __launch_bounds__(kWarps * 32) k_fused2d_batched(const BatchParams<T> b) {
  constexpr int kArr = arrs<false>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* ring = reinterpret_cast<T*>(smem_raw) + static_cast<size_t>(wib) * kSlots * kArr * cols<NC>();
  const int total = gridDim.x * kWarps;
  for (int item = blockIdx.x * kWarps + wib; item < b.n_items; item += total) {
    const BatchField fd = b.fields[b.item_field[item]];
    const int local = item - fd.item_base;
    F2Params<T> p;
    p.psi = b.psi + fd.offset;
    p.out = b.out + fd.offset;
    p.gc0 = b.gc0 + fd.offset;
    p.gc1 = b.gc1 + fd.offset;
    p.G = NUG ? b.G + fd.offset : nullptr;
    p.R = b.R ? b.R + fd.offset : nullptr;
    p.n0 = fd.n0;
    p.n1 = fd.n1;
    p.strips = fd.strips;
    p.rowtiles = 0;
    p.ty = b.ty;
    p.dt = b.dt;
    p.scale = b.scale;
    p.rhs_a = b.rhs_a;
    p.rhs_b = b.rhs_b;
    p.vec = fd.vec && b.vec_ok;
    p.lo = nullptr;
    p.lo_out = nullptr;
    p.tape = nullptr;
    p.tape_n = 0;
    march_tile<T, NC, FCT, NUG, IGA, KAHAN, false>(p, local % fd.strips, (local / fd.strips) * b.ty, ring, lane);
  }
}

template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN, bool COMP = false, bool TAPE = false>
void launch(const F2Params<T>& p, cudaStream_t st) {
  const long long warps = static_cast<long long>(p.strips) * p.rowtiles;
  const unsigned blocks = static_cast<unsigned>((warps + kWarps - 1) / kWarps);
  const size_t smem = static_cast<size_t>(kWarps) * kSlots * arrs<COMP>() * cols<NC>() * sizeof(T);
  static PerDevice<bool> attr;  // large rings exceed the default 48 KB of dynamic shared memory
  attr.get([&](int) {
    return cudaFuncSetAttribute(k_fused2d<T, NC, FCT, NUG, IGA, KAHAN, COMP, TAPE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) == cudaSuccess;
  });
  k_fused2d<T, NC, FCT, NUG, IGA, KAHAN, COMP, TAPE><<<blocks, kWarps * 32, smem, st>>>(p);
}

template <typename T, int NC, bool FCT, bool NUG>
void launch_mode(const F2Params<T>& p, bool iga, bool kahan, cudaStream_t st) {
  if (iga) {
    if (kahan) launch<T, NC, FCT, NUG, true, true>(p, st); else launch<T, NC, FCT, NUG, true, false>(p, st);
  } else {
    if (kahan) launch<T, NC, FCT, NUG, false, true>(p, st); else launch<T, NC, FCT, NUG, false, false>(p, st);
  }
}

template <typename T, int NC>
void launch_all(const F2Params<T>& p, const Opts& o, cudaStream_t st) {
  if (o.fct) {
    if (o.nug) launch_mode<T, NC, true, true>(p, o.iga, o.kahan, st);
    else launch_mode<T, NC, true, false>(p, o.iga, o.kahan, st);
  } else {
    if (o.nug) launch_mode<T, NC, false, true>(p, o.iga, o.kahan, st);
    else launch_mode<T, NC, false, false>(p, o.iga, o.kahan, st);
  }
}

bool al(const void* q, size_t a) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) % a) == 0; }

template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN>
void launch_b(const BatchParams<T>& b, cudaStream_t st) {
  const size_t smem = static_cast<size_t>(kWarps) * kSlots * arrs<false>() * cols<NC>() * sizeof(T);
  static PerDevice<int> grid_of;  // persistent grid: every block that fits on the GPU at once
  const int grid = grid_of.get([&](int dev) {
    cudaFuncSetAttribute(k_fused2d_batched<T, NC, FCT, NUG, IGA, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2d_batched<T, NC, FCT, NUG, IGA, KAHAN>,
                                                  kWarps * 32, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  });
  const int need = (b.n_items + kWarps - 1) / kWarps;
  k_fused2d_batched<T, NC, FCT, NUG, IGA, KAHAN><<<need < grid ? need : grid, kWarps * 32, smem, st>>>(b);
}

template <typename T, int NC, bool FCT, bool NUG>
void launch_b_mode(const BatchParams<T>& b, bool iga, bool kahan, cudaStream_t st) {
  if (iga) {
    if (kahan) launch_b<T, NC, FCT, NUG, true, true>(b, st); else launch_b<T, NC, FCT, NUG, true, false>(b, st);
  } else {
    if (kahan) launch_b<T, NC, FCT, NUG, false, true>(b, st); else launch_b<T, NC, FCT, NUG, false, false>(b, st);
  }
}

}  // namespace

template <typename T>
int fused_batched_columns() { return sizeof(T) == 4 ? 4 : 2; }
template int fused_batched_columns<float>();
template int fused_batched_columns<double>();

int fused_strip_stride(int nc) { return 32 * nc - 2 * kLead; }

namespace {

template <typename T, int NC>
int batched_launch(const BatchTable& tab, const Opts& o, const T* psi_in, T* psi_out, const T* gc0, const T* gc1,
                   const T* G, const T* R, T dt, T scale, cudaStream_t st) {
  BatchParams<T> b;
  b.psi = psi_in;
  b.out = psi_out;
  b.gc0 = gc0;
  b.gc1 = gc1;
  b.G = o.nug ? G : nullptr;
  b.R = R;
  b.fields = tab.fields;
  b.item_field = tab.item_field;
  b.n_items = tab.n_items;
  b.ty = tab.ty;
  b.dt = dt;
  b.scale = scale;
  b.rhs_a = o.rhs_a;
  b.rhs_b = o.rhs_b;
  const size_t va = NC * sizeof(T) <= 16 ? NC * sizeof(T) : 16;
  b.vec_ok = al(psi_in, va) && al(psi_out, va) && al(gc0, va) && al(gc1, va) && al(b.G, va) && al(R, va);
  if (o.fct) {
    if (o.nug) launch_b_mode<T, NC, true, true>(b, o.iga, o.kahan, st);
    else launch_b_mode<T, NC, true, false>(b, o.iga, o.kahan, st);
  } else {
    if (o.nug) launch_b_mode<T, NC, false, true>(b, o.iga, o.kahan, st);
    else launch_b_mode<T, NC, false, false>(b, o.iga, o.kahan, st);
  }
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

}  // namespace

template <typename T>
int fused_batched_step(const BatchTable& tab, const Opts& o, const T* psi_in, T* psi_out, const T* gc0,
                       const T* gc1, const T* G, const T* R, T dt, T scale, cudaStream_t st, int nc) {
  if (o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  if (sizeof(T) == 4 && nc == 2)
    return batched_launch<T, 2>(tab, o, psi_in, psi_out, gc0, gc1, G, R, dt, scale, st);
  if (nc != fused_batched_columns<T>()) return MPDATA_EINVAL;
  return batched_launch<T, sizeof(T) == 4 ? 4 : 2>(tab, o, psi_in, psi_out, gc0, gc1, G, R, dt, scale, st);
}

template int fused_batched_step<float>(const BatchTable&, const Opts&, const float*, float*, const float*,
                                       const float*, const float*, const float*, float, float, cudaStream_t, int);
template int fused_batched_step<double>(const BatchTable&, const Opts&, const double*, double*, const double*,
                                        const double*, const double*, const double*, double, double, cudaStream_t,
                                        int);

namespace {

// Warp-march parameters of one step of one field; *band is set when the automatic choice is
// the band march.  NC columns per lane: FP32 lanes own 4 (16-byte copies) or, with
// MPDATA_TUNE_KERNEL = 3, 2 (twice the strips, so twice the warps on a small field), FP64
// lanes 2 (register budget).
template <typename T, int NC = (sizeof(T) == 4 ? 4 : 2)>
F2Params<T> warp_params(const Grid& g, const Opts& o, const StepArgs<T>& a, bool* band) {
  F2Params<T> p;
  p.psi = a.psi_in;
  p.out = a.psi_out;
  p.gc0 = a.gc[0];
  p.gc1 = a.gc[1];
  p.G = o.nug ? a.g : nullptr;
  p.R = a.r;
  p.n0 = g.n[1];
  p.n1 = g.n[2];
  p.strips = (p.n1 + stride<NC>() - 1) / stride<NC>();
  // the tallest tile that still gives ~7.5 warps per SM (152 SMs), at least 8 rows
  // (measured on the rotation workload: 8 rows at 1024^2, 32 at 2048^2, 48-64 at 4096^2)
  auto warps = [&](int ty) { return static_cast<long long>(p.strips) * ((p.n0 + ty - 1) / ty); };
  int auto_ty = 8;
  for (int ty : {64, 48, 32, 24, 16, 12}) {
    if (warps(ty) >= 1140) { auto_ty = ty; break; }
  }
  // Where the warp march cannot fill the GPU even with 8-row tiles (FP32: fewer than ~4
  // warps per SM), or in FP64 (arithmetic-bound: every recomputed halo row costs FP64
  // issue slots) with tiles of 16 rows or less, one front per block of warps (band
  // march) is faster.
  *band = sizeof(T) == 4 ? warps(8) < 608 : auto_ty <= 16;
  p.ty = o.tile_rows > 0 ? o.tile_rows : auto_ty;
  p.rowtiles = (p.n0 + p.ty - 1) / p.ty;
  p.dt = a.dt;
  p.scale = a.gc_scale;
  p.rhs_a = o.rhs_a;
  p.rhs_b = o.rhs_b;
  const size_t va = NC * sizeof(T) <= 16 ? NC * sizeof(T) : 16;
  p.vec = (p.n1 % NC == 0) && al(p.psi, va) && al(p.out, va) && al(p.gc0, va) && al(p.gc1, va) &&
          al(p.G, va) && al(p.R, va);
  p.lo = nullptr;
  p.lo_out = nullptr;
  p.tape = nullptr;
  p.tape_n = 0;
  return p;
}

template <bool FCT, bool NUG, int NC = 4>
void launch_comp(const F2Params<float>& p, bool iga, cudaStream_t st) {
  if (iga) launch<float, NC, FCT, NUG, true, false, true>(p, st);
  else launch<float, NC, FCT, NUG, false, false, true>(p, st);
}

}  // namespace

template <typename T>
int fused_step(const Grid& g, const Opts& o, const StepArgs<T>& a, T*, cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  if (a.psi_out == a.psi_in) return MPDATA_EUNSUPPORTED;
  constexpr int NC = sizeof(T) == 4 ? 4 : 2;
  bool band_auto = false;
  if (o.kernel == 3 && sizeof(T) == 4) {  // narrow lanes (FP32)
    launch_all<T, 2>(warp_params<T, 2>(g, o, a, &band_auto), o, st);
    return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
  }
  const F2Params<T> p = warp_params(g, o, a, &band_auto);
  if (o.kernel == 2 || (o.kernel == 0 && band_auto)) return band_step<T>(g, o, a, st);
  launch_all<T, NC>(p, o, st);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

int fused_step_comp(const Grid& g, const Opts& o, const StepArgs<float>& a, const float* lo_in, float* lo_out,
                    cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  if (a.psi_out == a.psi_in || lo_out == lo_in) return MPDATA_EUNSUPPORTED;
  bool band_auto = false;
  if (o.kernel == 3 && o.fct && !o.nug) {  // narrow lanes, the common case
    F2Params<float> p = warp_params<float, 2>(g, o, a, &band_auto);
    p.lo = lo_in;
    p.lo_out = lo_out;
    p.vec = p.vec && al(lo_in, 8) && al(lo_out, 8);
    launch_comp<true, false, 2>(p, o.iga, st);
    return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
  }
  F2Params<float> p = warp_params(g, o, a, &band_auto);  // the warp march carries the low parts
  p.lo = lo_in;
  p.lo_out = lo_out;
  p.vec = p.vec && al(lo_in, 16) && al(lo_out, 16);
  if (o.fct) {
    if (o.nug) launch_comp<true, true>(p, o.iga, st); else launch_comp<true, false>(p, o.iga, st);
  } else {
    if (o.nug) launch_comp<false, true>(p, o.iga, st); else launch_comp<false, false>(p, o.iga, st);
  }
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template <typename T>
int fused_tape(const Grid& g, const Opts& o, const StepArgs<T>& a, T* tape, cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open || o.kahan || o.nug || o.iga || o.rhs_a || o.rhs_b)
    return MPDATA_EUNSUPPORTED;
  if (a.psi_out == nullptr || a.psi_out == a.psi_in) return MPDATA_EUNSUPPORTED;
  constexpr int NC = sizeof(T) == 4 ? 4 : 2;
  bool band_auto = false;
  F2Params<T> p = warp_params(g, o, a, &band_auto);
  if (o.kernel == 2 || (o.kernel == 0 && band_auto)) return band_tape<T>(g, o, a, tape, st);
  p.tape = tape;
  p.tape_n = g.N;
  if (o.fct) launch<T, NC, true, false, false, false, false, true>(p, st);
  else launch<T, NC, false, false, false, false, false, true>(p, st);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template int fused_tape<float>(const Grid&, const Opts&, const StepArgs<float>&, float*, cudaStream_t);
template int fused_tape<double>(const Grid&, const Opts&, const StepArgs<double>&, double*, cudaStream_t);

template int fused_step<float>(const Grid&, const Opts&, const StepArgs<float>&, float*, cudaStream_t);
template int fused_step<double>(const Grid&, const Opts&, const StepArgs<double>&, double*, cudaStream_t);

}  // namespace mpd
