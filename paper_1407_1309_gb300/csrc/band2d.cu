// Band-march 2D MPDATA step: the same fused step as fused2d.cu (donor-cell pass,
// FCT bounds, antidiffusive pseudo-advector of Eq. 6 with its cross term,
// limiting factors, corrective donor-cell pass; n_iters = 2) with a different
// decomposition.
//
// A block of W warps owns a strip of 32*NC columns (NC adjacent columns per lane,
// horizontal neighbours from warp shuffles, a 4-column recomputed halo on both
// sides, exactly as in the warp march) and a band of H rows.  The block walks down
// the band in chunks of W rows with one marching front: in every chunk each warp
// loads one input row and advances every stage by one row, with stage lags
//   pass 1 at row x-1; pseudo-advectors, bounds and limiting factors at x-2;
//   limited fluxes and pass 2 at x-3          (x = the row the warp loads),
// separated by block barriers.  Rows of every input and intermediate live in
// shared-memory rings indexed by row, so a row's vertical neighbours computed by
// other warps are read back from the rings, and a warp keeps the rows it reuses
// itself in registers.  Only the band's first and last rows carry the stencil's
// 3-row halo, so a tall band recomputes little while W warps share one front.
// Input rows are prefetched kDepth chunks ahead with cp.async.  Pass 2 of one
// chunk shares a barrier interval with pass 1 of the next (they touch disjoint
// data), so a chunk costs three block barriers.
#include <cuda_runtime.h>

#include "kernels.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

using namespace dev;

constexpr int kLeadB = 4;     // computed columns left of the strip's first output column
constexpr int kInRing = 32;   // rows kept of every input array (>= (kDepth + 1) * W + 3)
constexpr int kMidRing = 16;  // rows kept of every intermediate (>= W + 3)
constexpr int kDepth = 2;     // chunks of input rows in flight
constexpr int kBandWarps = 8;

template <typename T>
struct BandParams {
  const T* psi;
  T* out;
  const T* gc0;
  const T* gc1;
  const T* G;
  const T* R;
  int n0, n1, strips, H;
  T dt, scale;
  int rhs_a, rhs_b, vec;
  T* tape;  // adjoint tape (TAPE only): arrays of tape_n elements
  long long tape_n;
  int tape_vec;  // tape rows may be written as 16-byte vectors
};

// NC values of one lane from / to a shared-memory row (16-byte vectors where they fit)
template <typename T, int NC>
__device__ __forceinline__ void lds(T (&d)[NC], const T* q) {
  if constexpr (sizeof(T) == 4 && NC == 4) {
    const float4 v = *reinterpret_cast<const float4*>(q);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else if constexpr (sizeof(T) == 8 && NC == 2) {
    const double2 v = *reinterpret_cast<const double2*>(q);
    d[0] = v.x; d[1] = v.y;
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) d[c] = q[c];
  }
}
template <typename T, int NC>
__device__ __forceinline__ void sts(T* q, const T (&s)[NC]) {
  if constexpr (sizeof(T) == 4 && NC == 4) {
    *reinterpret_cast<float4*>(q) = make_float4(s[0], s[1], s[2], s[3]);
  } else if constexpr (sizeof(T) == 8 && NC == 2) {
    *reinterpret_cast<double2*>(q) = make_double2(s[0], s[1]);
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) q[c] = s[c];
  }
}

// TAPE: the step also writes, for the band's own rows, what the reverse step reads: psi^(1)
// (tape array 0), the pseudo-advectors of both dimensions (1, 2) and under FCT the bounds
// (5, 6) and the factors (7, 8); the limited advectors (3, 4) are left to the reverse step,
// which re-derives them from these.
template <typename T, int NC, int W, bool FCT, bool NUG, bool IGA, bool KAHAN, bool TAPE = false>
__global__ void __launch_bounds__(W * 32, 2) k_band2d(const BandParams<T> p) {
  constexpr int kCols = 32 * NC;
  constexpr int kStride = kCols - 2 * kLeadB;
  constexpr int kIn = kInRing * kCols, kMid = kMidRing * kCols;
  static_assert(kInRing >= (kDepth + 1) * W + 3 && kMidRing >= W + 3, "rings too short for the chunk");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int lc0 = NC * lane;
  const int strip = blockIdx.x % p.strips;
  const int R0 = (blockIdx.x / p.strips) * p.H;
  const int Hb = min(p.H, p.n0 - R0);
  const int Rs = R0 - 3;        // global row of local row 0 (the first row loaded)
  const int n_load = Hb + 6;    // local rows 0 .. Hb+5 are loaded

  // rings: inputs psi, gc0, gc1 [, G] [, R], then psi^(1), the unlimited fluxes and
  // the two limiting factors; every pointer is already offset to this lane's columns
  T* const s_psi = reinterpret_cast<T*>(smem_raw) + lc0;
  T* const s_v0 = s_psi + kIn;
  T* const s_v1 = s_v0 + kIn;
  T* const s_g = s_v1 + kIn;
  T* const s_r = s_g + (NUG ? kIn : 0);
  T* const s_p1 = s_r + (p.rhs_b ? kIn : 0);
  T* const s_u0 = s_p1 + kMid;
  T* const s_u1 = s_u0 + kMid;
  T* const s_bu = s_u1 + kMid;
  T* const s_bd = s_bu + kMid;
  auto in_row = [](T* base, int lr) { return base + (lr & (kInRing - 1)) * kCols; };
  auto mid_row = [](T* base, int lr) { return base + (lr & (kMidRing - 1)) * kCols; };

  const int cs = strip * kStride - kLeadB;
  int col[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) col[c] = wrapi(cs + lc0 + c, p.n1);
  const int gcol = cs + lc0;  // first global column of this lane (unwrapped)
  bool ok[NC];
  bool all_ok = true;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    ok[c] = lc0 + c >= kLeadB && lc0 + c < kLeadB + kStride && gcol + c < p.n1;
    all_ok = all_ok && ok[c];
  }

  // one row (local row L) of tape array j, own rows and columns only
  auto tape_row = [&](const int j, const int L, const T (&v)[NC]) {
    if (!TAPE || L < 3 || L > Hb + 2) return;
    T* q = p.tape + j * p.tape_n + static_cast<long long>(Rs + L) * p.n1 + gcol;
    if (p.tape_vec && all_ok) {
      sts(q, v);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (ok[c]) q[c] = v[c];
    }
  };

  auto copy_in = [&](T* dst, const T* src_row) {
    if (p.vec) {
      constexpr int bytes = NC * static_cast<int>(sizeof(T));
      if constexpr (bytes <= 16) {
        cp_async<bytes>(dst, src_row + col[0]);
      } else {
        constexpr int per = 16 / static_cast<int>(sizeof(T));
#pragma unroll
        for (int h = 0; h < bytes / 16; ++h) cp_async<16>(dst + h * per, src_row + col[0] + h * per);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) cp_async<sizeof(T)>(dst + c, src_row + col[c]);
    }
  };
  // local row lr of every input array, issued by this warp; one commit group per call.
  // The warp's load rows advance by W per chunk: their global row is kept wrapped
  // incrementally (the first one with a modulo).
  int g_row = wrapi(Rs + w, p.n0);
  auto load_row = [&](int lr) {
    if (lr < n_load) {
      const long long off = static_cast<long long>(g_row) * p.n1;
      g_row += W;
      while (g_row >= p.n0) g_row -= p.n0;
      copy_in(in_row(s_psi, lr), p.psi + off);
      copy_in(in_row(s_v0, lr), p.gc0 + off);
      copy_in(in_row(s_v1, lr), p.gc1 + off);
      if (NUG) copy_in(in_row(s_g, lr), p.G + off);
      if (p.rhs_b) copy_in(in_row(s_r, lr), p.R + off);
    }
    cp_commit();
  };

#pragma unroll
  for (int j = 0; j < kDepth; ++j) load_row(j * W + w);
  const bool fix = p.rhs_b || p.scale != T(1);
  // euler_b source and advector scale on a row this warp loaded itself
  auto fix_row = [&](int lr) {
    if (fix && lr < n_load) {
      T* q = in_row(s_psi, lr);
      T* q0 = in_row(s_v0, lr);
      T* q1 = in_row(s_v1, lr);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (p.rhs_b) q[c] = q[c] + p.dt * in_row(s_r, lr)[c];
        q0[c] = q0[c] * p.scale;
        q1[c] = q1[c] * p.scale;
      }
    }
  };
  const int n_chunks = (n_load + W - 1) / W;
  cp_wait<kDepth - 1>();
  fix_row(w);
  __syncthreads();

  // Per chunk, three barrier-separated stages: A = pass 2 of the previous chunk and
  // pass 1 of this one (disjoint data), B = pseudo-advectors, C = limiting factors.
  // Carried from the previous chunk's stages B and C into its pass 2:
  T q_m[NC], u0m[NC], bun[NC], bdn[NC];
  for (int j = 0; j <= n_chunks; ++j) {
    // ---- stage A, first half: limited fluxes and pass 2 of the previous chunk at local
    // row r = (j-1)*W + w - 3, from the registers its pseudo-advector and factor stages left
    const int r = (j - 1) * W + w - 3;
    if (r >= 3 && r <= Hb + 2) {
      T u0mm[NC], u1c[NC], h0[NC], h0c[NC], h1[NC];
      lds(u0mm, mid_row(s_u0, r - 1));  // face r-1/2; face r+1/2 is u0m
      lds(u1c, mid_row(s_u1, r));
      if (FCT) {
        T bu_m[NC], bd_m[NC], bu_c[NC], bd_c[NC];
        lds(bu_m, mid_row(s_bu, r - 1));
        lds(bd_m, mid_row(s_bd, r - 1));
        lds(bu_c, mid_row(s_bu, r));
        lds(bd_c, mid_row(s_bd, r));
        const T buR = from_right(bu_c), bdR = from_right(bd_c);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          // With two passes only the limited flux F*m is used, so a zero flux needs no
          // factor: m = min(beta_dn of the upwind cell, beta_up of the downwind cell).
          {  // face (r+1/2, c)
            const T F = u0m[c];
            const bool right = gt0(F);
            h0[c] = F * minv(right ? bd_c[c] : bu_c[c], right ? bun[c] : bdn[c]);
          }
          {  // face (r-1/2, c)
            const T F = u0mm[c];
            const bool right = gt0(F);
            h0c[c] = F * minv(right ? bd_m[c] : bu_m[c], right ? bu_c[c] : bd_c[c]);
          }
          {  // face (r, c+1/2)
            const T F = u1c[c];
            const bool right = gt0(F);
            const T x = right ? bd_c[c] : bu_c[c];
            const T y = right ? right_of(bu_c, c, buR) : right_of(bd_c, c, bdR);
            h1[c] = F * minv(x, y);
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) { h0[c] = u0m[c]; h0c[c] = u0mm[c]; h1[c] = u1c[c]; }
      }
      T g_r[NC];
      if (NUG) lds(g_r, in_row(s_g, r));
      const T h1L = from_left(h1);
      T np2[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T rG = NUG ? fdiv(T(1), g_r[c]) : T(1);
        np2[c] = donor<T, NUG, KAHAN>(q_m[c], h0[c], h0c[c], h1[c], left_of(h1, c, h1L), rG);
      }
      const long long o = static_cast<long long>(Rs + r) * p.n1 + gcol;
      if (p.rhs_a) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (ok[c]) np2[c] = np2[c] + p.dt * p.R[o + c];
      }
      if (p.vec && all_ok) {
        if constexpr (sizeof(T) == 4 && NC == 4) {
          *reinterpret_cast<float4*>(p.out + o) = make_float4(np2[0], np2[1], np2[2], np2[3]);
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
    if (j == n_chunks) break;

    // ---- stage A, second half: pass 1 (Eqs. 4-5) of this chunk at local row a
    const int a = j * W + w - 1;
    const bool do_p1 = a >= 1 && a <= Hb + 4;
    T pn_m[NC], pn_c[NC], v0_m[NC], v1_c[NC], g_c[NC], p1_c[NC];
    if (do_p1) {
      T pn_p[NC], v0_c[NC];
      lds(pn_m, in_row(s_psi, a - 1));
      lds(pn_c, in_row(s_psi, a));
      lds(pn_p, in_row(s_psi, a + 1));
      lds(v0_m, in_row(s_v0, a - 1));
      lds(v0_c, in_row(s_v0, a));
      lds(v1_c, in_row(s_v1, a));
      if (NUG) lds(g_c, in_row(s_g, a));
      const T psR = from_right(pn_c);
      T F1[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) F1[c] = flux(pn_c[c], right_of(pn_c, c, psR), v1_c[c]);
      const T F1L = from_left(F1);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T rG = NUG ? fdiv(T(1), g_c[c]) : T(1);
        const T Fp0 = flux(pn_c[c], pn_p[c], v0_c[c]);  // face a+1/2
        const T Fm0 = flux(pn_m[c], pn_c[c], v0_m[c]);  // face a-1/2
        p1_c[c] = donor<T, NUG, KAHAN>(pn_c[c], Fp0, Fm0, F1[c], left_of(F1, c, F1L), rG);
      }
      sts(mid_row(s_p1, a), p1_c);
      tape_row(0, a, p1_c);
    }
    __syncthreads();
    load_row((j + kDepth) * W + w);  // after the barrier: the slots it refills are no longer read

    // ---- local row b = a - 1: pseudo-advectors (Eq. 6 + cross term) and unlimited fluxes.
    // The face between rows b and b+1 needs psi^(1) on rows b, b+1 only and is computed
    // from the band's second row on; the faces along the row and the bounds need rows
    // b-1 .. b+1 and start one row later.
    const int b = a - 1;
    const bool do_ad = b >= 1 && b <= Hb + 3;
    const bool do_x = do_ad && b >= 2;
    T q_c[NC], g_b[NC], u0n[NC], u1n[NC], mx[NC], mn[NC];
    if (do_ad) {
      // row b of psi^(1) from the ring, row b+1 = a is this warp's pass-1 output
      T w1_c[NC];
      lds(q_c, mid_row(s_p1, b));
      lds(w1_c, in_row(s_v1, b));  // row b; row b+1 is v1_c
      if (NUG) lds(g_b, in_row(s_g, b));
      // dimension-0 face between rows b and b+1
      const T v0R = from_right(v0_m);
      T S0[NC], PV1[NC], pvp[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) { S0[c] = q_c[c] + p1_c[c]; PV1[c] = w1_c[c] + v1_c[c]; }
      const T S0L = from_left(S0), S0R = from_right(S0), PV1L = from_left(PV1);
      T na0[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T V = v0_m[c];
        const T Gb = NUG ? T(0.5) * (g_b[c] + g_c[c]) : T(1);
        const T d = p1_c[c] - q_c[c];
        const T A = IGA ? d * T(0.5) : ratio(d, S0[c]);
        const T Tt = right_of(S0, c, S0R), Bt = left_of(S0, c, S0L);
        const T B = IGA ? (Tt - Bt) * T(0.25) : ratio(Tt - Bt, Tt + Bt);
        const T Vq = T(0.25) * (PV1[c] + left_of(PV1, c, PV1L));
        const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
        const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
        u0n[c] = IGA ? out : flux(q_c[c], p1_c[c], out);
        na0[c] = out;
        pvp[c] = v0_m[c] + right_of(v0_m, c, v0R);
      }
      sts(mid_row(s_u0, b), u0n);
      tape_row(1, b, na0);
      if (do_x) {
        // dimension-1 faces (b, c+1/2)
        T w0_m[NC];
        lds(q_m, mid_row(s_p1, b - 1));
        lds(w0_m, in_row(s_v0, b - 1));  // face b-1/2; face b+1/2 is v0_m
        const T w0R = from_right(w0_m);
        const T rm = from_right(q_m), rc = from_right(q_c), rp = from_right(p1_c);
        const T gR = NUG ? from_right(g_b) : T(1);
        T na1[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T V = w1_c[c];
          const T Gb = NUG ? T(0.5) * (g_b[c] + right_of(g_b, c, gR)) : T(1);
          const T Sm = q_m[c] + right_of(q_m, c, rm);
          const T Sc = q_c[c] + right_of(q_c, c, rc);
          const T Sp = p1_c[c] + right_of(p1_c, c, rp);
          const T q0 = q_c[c], q1 = right_of(q_c, c, rc);
          const T A = IGA ? (q1 - q0) * T(0.5) : ratio(q1 - q0, Sc);
          const T B = IGA ? (Sp - Sm) * T(0.25) : ratio(Sp - Sm, Sp + Sm);
          const T pvm = w0_m[c] + right_of(w0_m, c, w0R);
          const T Vq = T(0.25) * (pvp[c] + pvm);
          const T rGb = NUG ? fdiv(T(1), Gb) : T(1);
          const T out = (absv(V) - V * V * rGb) * A - T(0.5) * V * Vq * rGb * B;
          u1n[c] = IGA ? out : flux(q0, q1, out);
          na1[c] = out;
        }
        sts(mid_row(s_u1, b), u1n);
        tape_row(2, b, na1);
        if (FCT) {
          // extrema of psi^n and psi^(1) over the cell and its face neighbours
          T pn_mm[NC], hi_m[NC], hi_c[NC], hi_p[NC], lo_m[NC], lo_c[NC], lo_p[NC];
          lds(pn_mm, in_row(s_psi, b - 1));
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            hi_m[c] = maxv(pn_mm[c], q_m[c]); lo_m[c] = minv(pn_mm[c], q_m[c]);
            hi_c[c] = maxv(pn_m[c], q_c[c]);  lo_c[c] = minv(pn_m[c], q_c[c]);
            hi_p[c] = maxv(pn_c[c], p1_c[c]); lo_p[c] = minv(pn_c[c], p1_c[c]);
          }
          const T hL = from_left(hi_c), hR = from_right(hi_c);
          const T lL = from_left(lo_c), lR = from_right(lo_c);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            mx[c] = maxv(maxv(maxv(hi_c[c], hi_m[c]), maxv(hi_p[c], left_of(hi_c, c, hL))),
                         right_of(hi_c, c, hR));
            mn[c] = minv(minv(minv(lo_c[c], lo_m[c]), minv(lo_p[c], left_of(lo_c, c, lL))),
                         right_of(lo_c, c, lR));
          }
          tape_row(5, b, mx);
          tape_row(6, b, mn);
        }
      }
    }
    __syncthreads();

    // ---- limiting factors at row b (the flux through face b-1/2 comes from the ring)
    if (do_x) {
      lds(u0m, mid_row(s_u0, b - 1));
      if (FCT) {
        const T u1L = from_left(u1n);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T Fm0 = u0m[c], Fp0 = u0n[c];
          const T Fp1 = u1n[c], Fm1 = left_of(u1n, c, u1L);
          // [x]- = x - [x]+ and [x]+ = x - [x]- hold exactly in floating point, so the
          // outflow sum reuses the inflow sum's four extrema (adds instead of min/max)
          const T pFm0 = posp(Fm0), nFp0 = negp(Fp0), pFm1 = posp(Fm1), nFp1 = negp(Fp1);
          const T in = (pFm0 - nFp0) + (pFm1 - nFp1);
          const T ou = ((Fp0 - nFp0) - (Fm0 - pFm0)) + ((Fp1 - nFp1) - (Fm1 - pFm1));
          const T Gi = NUG ? g_b[c] : T(1);
          const T q = q_c[c];
          // min(1, x / |s|) is 1 for s = 0 (x/0 is inf or NaN, and min ignores NaN)
          bun[c] = min1(fdiv(Gi * posp(mx[c] - q), absv(in)));
          bdn[c] = min1(fdiv(Gi * posp(q - mn[c]), absv(ou)));
        }
        sts(mid_row(s_bu, b), bun);
        sts(mid_row(s_bd, b), bdn);
        tape_row(7, b, bun);
        tape_row(8, b, bdn);
      }
    }
    // next chunk's input rows
    cp_wait<kDepth - 1>();
    fix_row((j + 1) * W + w);
    __syncthreads();
  }
  cp_wait<0>();
}

template <typename T>
constexpr size_t band_smem(int n_in, bool fct) {
  return static_cast<size_t>(n_in * kInRing + (fct ? 5 : 3) * kMidRing) * 32 * (sizeof(T) == 4 ? 4 : 2) *
         sizeof(T);
}

template <typename T, int NC, bool FCT, bool NUG, bool IGA, bool KAHAN, bool TAPE = false>
void launch_band(BandParams<T> p, int tile_rows, cudaStream_t st) {
  constexpr int W = kBandWarps;
  auto kern = k_band2d<T, NC, W, FCT, NUG, IGA, KAHAN, TAPE>;
  static PerDevice<int> slots_of;  // blocks resident on the whole GPU at the largest ring layout
  const int slots = slots_of.get([&](int dev) {
    const size_t most = band_smem<T>(5, FCT);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(most));
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, band_smem<T>(3 + (NUG ? 1 : 0), FCT));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  });
  if (tile_rows > 0) {
    p.H = tile_rows;
  } else {  // one band per resident block: as few, tall bands as fill the GPU once
    const int bands = slots / p.strips > 1 ? slots / p.strips : 1;
    p.H = (p.n0 + bands - 1) / bands;
    if (p.H < 8) p.H = 8;
  }
  const long long blocks = static_cast<long long>(p.strips) * ((p.n0 + p.H - 1) / p.H);
  const size_t smem = band_smem<T>(3 + (NUG ? 1 : 0) + (p.rhs_b ? 1 : 0), FCT);
  kern<<<static_cast<unsigned>(blocks), W * 32, smem, st>>>(p);
}

template <typename T, int NC, bool FCT, bool NUG>
void band_mode(const BandParams<T>& p, int rows, bool iga, bool kahan, cudaStream_t st) {
  if (iga) {
    if (kahan) launch_band<T, NC, FCT, NUG, true, true>(p, rows, st);
    else launch_band<T, NC, FCT, NUG, true, false>(p, rows, st);
  } else {
    if (kahan) launch_band<T, NC, FCT, NUG, false, true>(p, rows, st);
    else launch_band<T, NC, FCT, NUG, false, false>(p, rows, st);
  }
}

bool aligned_to(const void* q, size_t a) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) % a) == 0; }

}  // namespace

template <typename T>
int band_step(const Grid& g, const Opts& o, const StepArgs<T>& a, cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  if (a.psi_out == a.psi_in) return MPDATA_EUNSUPPORTED;
  constexpr int NC = sizeof(T) == 4 ? 4 : 2;
  BandParams<T> p;
  p.psi = a.psi_in;
  p.out = a.psi_out;
  p.gc0 = a.gc[0];
  p.gc1 = a.gc[1];
  p.G = o.nug ? a.g : nullptr;
  p.R = a.r;
  p.n0 = g.n[1];
  p.n1 = g.n[2];
  p.strips = (p.n1 + 32 * NC - 2 * kLeadB - 1) / (32 * NC - 2 * kLeadB);
  p.H = 0;
  p.dt = a.dt;
  p.scale = a.gc_scale;
  p.rhs_a = o.rhs_a;
  p.rhs_b = o.rhs_b;
  const size_t va = NC * sizeof(T) <= 16 ? NC * sizeof(T) : 16;
  p.vec = (p.n1 % NC == 0) && aligned_to(p.psi, va) && aligned_to(p.out, va) && aligned_to(p.gc0, va) &&
          aligned_to(p.gc1, va) && aligned_to(p.G, va) && aligned_to(p.R, va);
  p.tape = nullptr;
  p.tape_n = 0;
  p.tape_vec = 0;
  if (o.fct) {
    if (o.nug) band_mode<T, NC, true, true>(p, o.tile_rows, o.iga, o.kahan, st);
    else band_mode<T, NC, true, false>(p, o.tile_rows, o.iga, o.kahan, st);
  } else {
    if (o.nug) band_mode<T, NC, false, true>(p, o.tile_rows, o.iga, o.kahan, st);
    else band_mode<T, NC, false, false>(p, o.tile_rows, o.iga, o.kahan, st);
  }
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template <typename T>
int band_tape(const Grid& g, const Opts& o, const StepArgs<T>& a, T* tape, cudaStream_t st) {
  if (g.nd != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open || o.kahan || o.nug || o.iga || o.rhs_a || o.rhs_b)
    return MPDATA_EUNSUPPORTED;
  if (a.psi_out == nullptr || a.psi_out == a.psi_in) return MPDATA_EUNSUPPORTED;
  constexpr int NC = sizeof(T) == 4 ? 4 : 2;
  BandParams<T> p;
  p.psi = a.psi_in;
  p.out = a.psi_out;
  p.gc0 = a.gc[0];
  p.gc1 = a.gc[1];
  p.G = nullptr;
  p.R = nullptr;
  p.n0 = g.n[1];
  p.n1 = g.n[2];
  p.strips = (p.n1 + 32 * NC - 2 * kLeadB - 1) / (32 * NC - 2 * kLeadB);
  p.H = 0;
  p.dt = T(0);
  p.scale = a.gc_scale;
  p.rhs_a = 0;
  p.rhs_b = 0;
  p.vec = (p.n1 % NC == 0) && aligned_to(p.psi, 16) && aligned_to(p.out, 16) && aligned_to(p.gc0, 16) &&
          aligned_to(p.gc1, 16);
  p.tape = tape;
  p.tape_n = g.N;
  p.tape_vec = p.vec && aligned_to(tape, 16);
  if (o.fct) launch_band<T, NC, true, false, false, false, true>(p, o.tile_rows, st);
  else launch_band<T, NC, false, false, false, false, true>(p, o.tile_rows, st);
  return cudaGetLastError() == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

template int band_tape<float>(const Grid&, const Opts&, const StepArgs<float>&, float*, cudaStream_t);
template int band_tape<double>(const Grid&, const Opts&, const StepArgs<double>&, double*, cudaStream_t);
template int band_step<float>(const Grid&, const Opts&, const StepArgs<float>&, cudaStream_t);
template int band_step<double>(const Grid&, const Opts&, const StepArgs<double>&, cudaStream_t);

}  // namespace mpd
