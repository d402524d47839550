// Vectorised 3D z-march kernels (FP32) for fields of at least 128 columns whose x extent is a
// multiple of 4: the pseudo-advector of Eq. 6 with its multi-dimensional cross terms and
// third-order terms (Sect. 3.1.1-3.1.2; infinite gauge and |psi| of Sect. 3.1.5) of a corrective
// pass, pass 1 (Eqs. 4-5) with the FCT bounds (Sect. 3.1.4), and the FCT corrective pass
// (factors, limiter and donor pass).  The corrective pass keeps in shared memory only what
// neighbouring rows read (psi, the x and y advector components, the factors) and takes the
// values only the cell itself reads into registers, so that two blocks fit on an SM.
//
// Work decomposition: a block of warps owns a tile of 32*NC (x) by 8 (y) cells and walks a
// chunk of z-planes.  Lane l of warp w owns the NC adjacent cells x0 + NC*l .. x0 + NC*l + NC-1
// of one row, so one 16-byte (NC = 4) shared-memory load brings a row segment of all its cells,
// and two more loads the neighbours just outside the segment.  The
// planes the march reads are staged in shared-memory rings, row by row with four halo cells on
// each side in x so that every 16-byte chunk of a row is aligned in global and shared memory;
// each chunk is one cp.async, issued for the next step while this one computes.  The chunks wrap
// periodically as whole chunks, which needs the x extent to be a multiple of 4.  The options are
// template parameters, so no branch separates the arithmetic of the cells and faces.
#include <cuda_runtime.h>

#include <cstdlib>

#include "internal.h"
#include "stencil2d.cuh"

namespace mpd {
namespace {

using namespace dev;

constexpr int kRows = 8;     // tile rows, one warp each
constexpr int kZc = 16;      // z-planes per block
constexpr int kThreads = 32 * kRows;
template <int NC> constexpr int row_w() { return 32 * NC + 8; }  // row with 4 halo cells each side

__device__ __forceinline__ int wrapi3(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// Copy plan of a plane region of R rows starting at row ylo for a block of NT threads: this
// thread copies the 16-byte chunks tid, tid + NT, ...; chunk c is row c / (W/4), columns
// x0 - 4 + 4 (c % (W/4)) + 0..3.
template <int NC, int R, int NT = kThreads>
struct Plan {
  static constexpr int kPerRow = row_w<NC>() / 4;
  static constexpr int kChunks = R * kPerRow;
  static constexpr int kPer = (kChunks + NT - 1) / NT;
  int off[kPer];
  __device__ __forceinline__ void init(int tid, int x0, int ylo, int nx, int ny) {
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int c = tid + NT * j;
      const int r = c / kPerRow, k = c - r * kPerRow;
      off[j] = c < kChunks ? wrapi3(ylo + r, ny) * nx + wrapi3(x0 - 4 + 4 * k, nx) : -1;
    }
  }
  __device__ __forceinline__ void copy(float* dst, const float* src, int tid) const {
#pragma unroll
    for (int j = 0; j < kPer; ++j)
      if (off[j] >= 0) cp_async<16>(dst + 4 * (tid + NT * j), src + off[j]);
  }
  // multiply this thread's chunks by s (after its own copies have landed)
  __device__ __forceinline__ void scale(float* dst, int tid, float s) const {
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (off[j] >= 0) {
        float4* q = reinterpret_cast<float4*>(dst + 4 * (tid + NT * j));
        float4 v = *q;
        v.x *= s; v.y *= s; v.z *= s; v.w *= s;
        *q = v;
      }
    }
  }
};

// Row segment of this lane: w[i + 1] is the cell x + i, i = -1 .. NC + 1 (x the lane's first cell),
// read straight from the staged row (its halo cells included): three loads and no shuffles,
// lane-edge branches or selects (measured 11 % faster over the 3D step than taking the outer
// values from the neighbouring lanes by shuffles, for about a third more shared-memory wavefronts)
template <int NC>
__device__ __forceinline__ void fetch(const float* row, int lane, float (&w)[NC + 3]) {
  const float* p = row + 4 + NC * lane;
  w[0] = p[-1];
  if constexpr (NC == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[1] = v.x; w[2] = v.y; w[3] = v.z; w[4] = v.w;
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    w[1] = v.x; w[2] = v.y;
  }
  const float2 r = *reinterpret_cast<const float2*>(p + NC);
  w[NC + 1] = r.x;
  w[NC + 2] = r.y;
}

// The lane's NC cells of a staged row (no neighbours)
template <int NC>
__device__ __forceinline__ void center(const float* row, int lane, float (&w)[NC]) {
  const float* p = row + 4 + NC * lane;
  if constexpr (NC == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    w[0] = v.x; w[1] = v.y;
  }
}
template <int NC>
__device__ __forceinline__ void put(float* dst, const float (&v)[NC]) {
  if constexpr (NC == 4) *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
}

__device__ __forceinline__ float frac1(float n, float d) { return divisible(d) ? __fdividef(n, d) : 0.0f; }
// n1/d and n2/d with one guard and one approximate reciprocal (0 when d == 0)
__device__ __forceinline__ void frac2v(float n1, float n2, float d, float& r1, float& r2) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(d));
  r1 = divisible(d) ? n1 * r : 0.0f;
  r2 = divisible(d) ? n2 * r : 0.0f;
}

// One face of Eq. 6 with the cross terms of the two transverse dimensions q1, q2 (in the
// order z, y, x skipping the face's own dimension) and the third-order terms:
//   (|V| - V^2/Gb) A - sum_q 0.5 V Vq/Gb B_q
//   + tot: Gb(3C|C| - 2C^3 - C)/3 D_dd + sum_q Gb|C|C_q(1 - 2|C|) D_dq - (2/3) Gb C C_q1 C_q2 D_q1q2
// psi values (|psi| under ABS): p0 = psi_i, p1 = psi_{i+e_d}, pm = psi_{i-e_d}, p2 = psi_{i+2e_d};
// per q: a = psi_{i+e_q}, b = psi_{i+e_q+e_d}, e = psi_{i-e_q}, f = psi_{i-e_q+e_d}; pr = the
// pairs psi_j + psi_{j+e_d} at j = i +-e_q1 +-e_q2 in the order (+,+), (+,-), (-,+), (-,-).
template <bool IGA, bool TOT>
__device__ __forceinline__ float face(float p0, float p1, float pm, float p2, float rGb, float V,
                                      float vq1, float a1, float b1, float e1, float f1,
                                      float vq2, float a2, float b2, float e2, float f2,
                                      float pr0, float pr1, float pr2, float pr3) {
  constexpr bool iga = IGA;
  const float A = iga ? (p1 - p0) * 0.5f : frac1(p1 - p0, p0 + p1);
  float out = (fabsf(V) - V * V * rGb) * A;
  float B1, D1, B2, D2;
  {
    const float Tp = a1 + b1, Bt = e1 + f1;
    if constexpr (iga) { B1 = (Tp - Bt) * 0.25f; D1 = ((b1 - a1) - (f1 - e1)) * 0.25f; }
    else frac2v(Tp - Bt, (b1 - a1) - (f1 - e1), Tp + Bt, B1, D1);
    out = out - 0.5f * V * vq1 * rGb * B1;
  }
  {
    const float Tp = a2 + b2, Bt = e2 + f2;
    if constexpr (iga) { B2 = (Tp - Bt) * 0.25f; D2 = ((b2 - a2) - (f2 - e2)) * 0.25f; }
    else frac2v(Tp - Bt, (b2 - a2) - (f2 - e2), Tp + Bt, B2, D2);
    out = out - 0.5f * V * vq2 * rGb * B2;
  }
  if constexpr (TOT) {
    const float num = ((p2 - p1) - p0) + pm;
    const float D = iga ? num * 0.25f : frac1(num, ((p2 + p1) + p0) + pm);
    out = out + ((3.0f * V * fabsf(V)) * rGb - (2.0f * V * V * V) * (rGb * rGb) - V) * (1.0f / 3.0f) * D;
    const float c2 = fabsf(V) * rGb * (1.0f - 2.0f * fabsf(V) * rGb);
    out = out + c2 * vq1 * D1;
    out = out + c2 * vq2 * D2;
    const float n3 = (pr0 - pr1) - (pr2 - pr3);
    const float D3 = iga ? n3 * 0.125f : frac1(n3, (pr0 + pr1) + (pr2 + pr3));
    out = out - (2.0f / 3.0f) * V * vq1 * vq2 * (rGb * rGb) * D3;
  }
  return out;
}

struct V3 { const float* p[3]; };
struct O3 { float* p[3]; };

// psi ring: 5 planes of 11 rows (y0-1 .. y0+9); advector components and G: 3 planes of 10 rows
// (y0-1 .. y0+8); the spare slot of each ring takes the next step's plane.
constexpr int kPsiRing = 5, kVRing = 3, kPsiRows = kRows + 3, kVRows = kRows + 2;
template <int NC>
constexpr size_t antidiff3v_smem() {
  return sizeof(float) * row_w<NC>() * (kPsiRing * kPsiRows + 4 * kVRing * kVRows);
}

// NC cells per lane; MINB resident blocks per SM requested from the register allocator; the
// options are compile-time so that the cells' and faces' arithmetic has no branch between it
template <int NC, int MINB, bool ABS, bool IGA, bool TOT, bool NUG>
__global__ void __launch_bounds__(kThreads, MINB) k_antidiff3v(Grid g, const float* __restrict__ psi, V3 Vin,
                                                         float vscale, const float* __restrict__ G, O3 Vout) {
  constexpr int W = row_w<NC>();
  constexpr int nP = kPsiRows * W, nV = kVRows * W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const sP = reinterpret_cast<float*>(smem_raw);  // [kPsiRing][nP]
  float* const sZ = sP + kPsiRing * nP;                   // [kVRing][nV] z component
  float* const sY = sZ + kVRing * nV;                     // y component
  float* const sX = sY + kVRing * nV;                     // x component
  float* const sG = sX + kVRing * nV;                     // G
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
  const int x0 = blockIdx.x * 32 * NC, y0 = blockIdx.y * kRows;
  const int zb = blockIdx.z * kZc;
  const int ze = zb + kZc < nz ? zb + kZc : nz;
  const long long plane = static_cast<long long>(ny) * nx;
  Plan<NC, kPsiRows> pp;
  Plan<NC, kVRows> pv;
  pp.init(tid, x0, y0 - 1, nx, ny);
  pv.init(tid, x0, y0 - 1, nx, ny);
  auto zoff = [&](int z) { return static_cast<long long>(wrapi3(z, nz)) * plane; };
  auto rot = [](int s, int j, int n) { const int v = s + j; return v >= n ? v - n : v; };
  // ring slots at step z: psi planes z-1 .. z+2 in cp .. cp+3; z component planes z-1, z in
  // cz, cz+1; y, x components and G planes z, z+1 in cq, cq+1
  int cp = 0, cz = 0, cq = 0;
  {  // prologue
    for (int j = 0; j < 4; ++j) pp.copy(sP + j * nP, psi + zoff(zb - 1 + j), tid);
    pv.copy(sZ, Vin.p[0] + zoff(zb - 1), tid);
    pv.copy(sZ + nV, Vin.p[0] + zoff(zb), tid);
    for (int j = 0; j < 2; ++j) {
      const long long zo = zoff(zb + j);
      pv.copy(sY + j * nV, Vin.p[1] + zo, tid);
      pv.copy(sX + j * nV, Vin.p[2] + zo, tid);
      if (NUG) pv.copy(sG + j * nV, G + zo, tid);
    }
    cp_commit();
    cp_wait<0>();
    if (vscale != 1.0f) {
      for (int j = 0; j < 2; ++j) {
        pv.scale(sZ + j * nV, tid, vscale);
        pv.scale(sY + j * nV, tid, vscale);
        pv.scale(sX + j * nV, tid, vscale);
      }
    }
  }
  const int y = y0 + wy;
  const bool row_in = y < ny;
  const int xl = x0 + NC * lane;
  for (int z = zb; z < ze; ++z) {
    __syncthreads();
    const int fp = rot(cp, 4, kPsiRing), fz = rot(cz, 2, kVRing), fq = rot(cq, 2, kVRing);
    if (z + 1 < ze) {
      pp.copy(sP + fp * nP, psi + zoff(z + 3), tid);
      pv.copy(sZ + fz * nV, Vin.p[0] + zoff(z + 1), tid);
      const long long zo = zoff(z + 2);
      pv.copy(sY + fq * nV, Vin.p[1] + zo, tid);
      pv.copy(sX + fq * nV, Vin.p[2] + zo, tid);
      if (NUG) pv.copy(sG + fq * nV, G + zo, tid);
    }
    cp_commit();
    if (row_in) {
      // plane pointers: psi planes z-1 .. z+2; z component z-1, z; the others and G z, z+1
      const float* P[4] = {sP + cp * nP, sP + rot(cp, 1, kPsiRing) * nP, sP + rot(cp, 2, kPsiRing) * nP,
                           sP + rot(cp, 3, kPsiRing) * nP};
      const int cq1 = rot(cq, 1, kVRing);
      const float* Zp[2] = {sZ + cz * nV, sZ + rot(cz, 1, kVRing) * nV};
      const float* Yp[2] = {sY + cq * nV, sY + cq1 * nV};
      const float* Xp[2] = {sX + cq * nV, sX + cq1 * nV};
      const float* Gp[2] = {sG + cq * nV, sG + cq1 * nV};
      // row segment of psi at plane z + dz, row y + dy (|psi| under ABS)
      auto Pw = [&](int dz, int dy, float (&w)[NC + 3]) {
        fetch<NC>(P[dz + 1] + (wy + 1 + dy) * W, lane, w);
        if constexpr (ABS) {
#pragma unroll
          for (int i = 0; i < NC + 3; ++i) w[i] = fabsf(w[i]);
        }
      };
      auto Vw = [&](const float* pl, int dy, float (&w)[NC + 3]) { fetch<NC>(pl + (wy + 1 + dy) * W, lane, w); };
      float res[3][NC];
      {  // faces along x (d = 2); transverse z then y
        float p00[NC + 3], pz1[NC + 3], pzm[NC + 3], py1[NC + 3], pym[NC + 3];
        float ppp[NC + 3], ppm[NC + 3], pmp[NC + 3], pmm[NC + 3];
        Pw(0, 0, p00); Pw(1, 0, pz1); Pw(-1, 0, pzm); Pw(0, 1, py1); Pw(0, -1, pym);
        Pw(1, 1, ppp); Pw(1, -1, ppm); Pw(-1, 1, pmp); Pw(-1, -1, pmm);
        float vx[NC + 3], vy0[NC + 3], vym[NC + 3], vz0[NC + 3], vzm[NC + 3], g0[NC + 3];
        Vw(Xp[0], 0, vx); Vw(Yp[0], 0, vy0); Vw(Yp[0], -1, vym); Vw(Zp[1], 0, vz0); Vw(Zp[0], 0, vzm);
        if (NUG) Vw(Gp[0], 0, g0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int i = c + 1;
          const float rGb = NUG ? __fdividef(1.0f, 0.5f * (g0[i] + g0[i + 1])) : 1.0f;
          const float vqz = 0.25f * ((vz0[i] + vz0[i + 1]) + (vzm[i] + vzm[i + 1]));
          const float vqy = 0.25f * ((vy0[i] + vy0[i + 1]) + (vym[i] + vym[i + 1]));
          res[2][c] = face<IGA, TOT>(p00[i], p00[i + 1], p00[i - 1], p00[i + 2], rGb, vx[i],
                           vqz, pz1[i], pz1[i + 1], pzm[i], pzm[i + 1],
                           vqy, py1[i], py1[i + 1], pym[i], pym[i + 1],
                           ppp[i] + ppp[i + 1], ppm[i] + ppm[i + 1], pmp[i] + pmp[i + 1], pmm[i] + pmm[i + 1]);
        }
      }
      {  // faces along y (d = 1); transverse z then x
        float p00[NC + 3], p01[NC + 3], p0m[NC + 3], p02[NC + 3], pz0[NC + 3], pz1[NC + 3], pm0[NC + 3],
            pm1[NC + 3];
        Pw(0, 0, p00); Pw(0, 1, p01); Pw(0, -1, p0m); Pw(0, 2, p02);
        Pw(1, 0, pz0); Pw(1, 1, pz1); Pw(-1, 0, pm0); Pw(-1, 1, pm1);
        float vy[NC + 3], vx0[NC + 3], vx1[NC + 3], vz00[NC + 3], vz01[NC + 3], vzm0[NC + 3], vzm1[NC + 3];
        float g0[NC + 3], g1[NC + 3];
        Vw(Yp[0], 0, vy); Vw(Xp[0], 0, vx0); Vw(Xp[0], 1, vx1);
        Vw(Zp[1], 0, vz00); Vw(Zp[1], 1, vz01); Vw(Zp[0], 0, vzm0); Vw(Zp[0], 1, vzm1);
        if (NUG) { Vw(Gp[0], 0, g0); Vw(Gp[0], 1, g1); }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int i = c + 1;
          const float rGb = NUG ? __fdividef(1.0f, 0.5f * (g0[i] + g1[i])) : 1.0f;
          const float vqz = 0.25f * ((vz00[i] + vz01[i]) + (vzm0[i] + vzm1[i]));
          const float vqx = 0.25f * ((vx0[i] + vx1[i]) + (vx0[i - 1] + vx1[i - 1]));
          res[1][c] = face<IGA, TOT>(p00[i], p01[i], p0m[i], p02[i], rGb, vy[i],
                           vqz, pz0[i], pz1[i], pm0[i], pm1[i],
                           vqx, p00[i + 1], p01[i + 1], p00[i - 1], p01[i - 1],
                           pz0[i + 1] + pz1[i + 1], pz0[i - 1] + pz1[i - 1], pm0[i + 1] + pm1[i + 1],
                           pm0[i - 1] + pm1[i - 1]);
        }
      }
      {  // faces along z (d = 0); transverse y then x
        float p00[NC + 3], p10[NC + 3], pm0[NC + 3], p20[NC + 3], p01[NC + 3], p11[NC + 3], p0m[NC + 3],
            p1m[NC + 3];
        Pw(0, 0, p00); Pw(1, 0, p10); Pw(-1, 0, pm0); Pw(2, 0, p20);
        Pw(0, 1, p01); Pw(1, 1, p11); Pw(0, -1, p0m); Pw(1, -1, p1m);
        float vz[NC + 3], vy0[NC + 3], vy1[NC + 3], vy0m[NC + 3], vy1m[NC + 3], vx0[NC + 3], vx1[NC + 3];
        float g0[NC + 3], g1[NC + 3];
        Vw(Zp[1], 0, vz); Vw(Yp[0], 0, vy0); Vw(Yp[1], 0, vy1); Vw(Yp[0], -1, vy0m); Vw(Yp[1], -1, vy1m);
        Vw(Xp[0], 0, vx0); Vw(Xp[1], 0, vx1);
        if (NUG) { Vw(Gp[0], 0, g0); Vw(Gp[1], 0, g1); }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int i = c + 1;
          const float rGb = NUG ? __fdividef(1.0f, 0.5f * (g0[i] + g1[i])) : 1.0f;
          const float vqy = 0.25f * ((vy0[i] + vy1[i]) + (vy0m[i] + vy1m[i]));
          const float vqx = 0.25f * ((vx0[i] + vx1[i]) + (vx0[i - 1] + vx1[i - 1]));
          res[0][c] = face<IGA, TOT>(p00[i], p10[i], pm0[i], p20[i], rGb, vz[i],
                           vqy, p01[i], p11[i], p0m[i], p1m[i],
                           vqx, p00[i + 1], p10[i + 1], p00[i - 1], p10[i - 1],
                           p01[i + 1] + p11[i + 1], p01[i - 1] + p11[i - 1], p0m[i + 1] + p1m[i + 1],
                           p0m[i - 1] + p1m[i - 1]);
        }
      }
      // stores: the lane's NC cells of row y (vectorised when all are inside)
      const long long o = static_cast<long long>(z) * plane + static_cast<long long>(y) * nx + xl;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (xl + NC <= nx) {
          if constexpr (NC == 4) *reinterpret_cast<float4*>(Vout.p[d] + o) = make_float4(res[d][0], res[d][1], res[d][2], res[d][3]);
          else *reinterpret_cast<float2*>(Vout.p[d] + o) = make_float2(res[d][0], res[d][1]);
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (xl + c < nx) Vout.p[d][o + c] = res[d][c];
        }
      }
    }
    cp_wait<0>();
    if (z + 1 < ze && vscale != 1.0f) {  // only planes copied in this step are scaled
      pv.scale(sZ + fz * nV, tid, vscale);
      pv.scale(sY + fq * nV, tid, vscale);
      pv.scale(sX + fq * nV, tid, vscale);
    }
    cp = rot(cp, 1, kPsiRing);
    cz = rot(cz, 1, kVRing);
    cq = rot(cq, 1, kVRing);
  }
}

constexpr int kCWarps = kRows + 2;  // rows y0-1 .. y0+8, one warp each
constexpr int kCThreads = 32 * kCWarps;

// donor-cell flux of Eq. 5 in advector units; psi -> 1 under infinite gauge
template <bool UNIT>
__device__ __forceinline__ float fluxv(float L, float R, float V) {
  if constexpr (UNIT) return V;
  else return posp(V) * L + negp(V) * R;
}
// ---------------------------------------------------------------- pass 1 and the FCT bounds
// Pass 1 (Eqs. 4-5) and the FCT bounds (Sect. 3.1.4: extrema of psi^n and psi^(1) over the cell
// and its face neighbours) as one z-march (the work of k_donor and k_bounds): at step z warp w
// forms psi^(1) of row y0 - 1 + w of plane z (lanes 0 and 31 also the halo columns) into a ring
// of three planes, then warps 1 .. kRows form the bounds of their row of plane z-1 and write
// psi^(1), the bounds' maximum and minimum.  The advector is scaled at use.
constexpr int kBPsiRing = 5, kBVqRing = 2, kBVzRing = 3, kB1Ring = 3;
constexpr int kBPsiRows = kRows + 4;  // psi^n, y0-2 .. y0+9
constexpr int kBVxRows = kRows + 2;   // y0-1 .. y0+8
constexpr int kBVyRows = kRows + 3;   // y0-2 .. y0+8
constexpr int kBVzRows = kRows + 2;   // y0-1 .. y0+8
constexpr int kB1Rows = kRows + 2;    // psi^(1), y0-1 .. y0+8
template <int NC>
constexpr size_t p1b3v_smem() {
  return sizeof(float) * row_w<NC>() *
         (kBPsiRing * kBPsiRows + kBVqRing * (kBVxRows + kBVyRows) + kBVzRing * kBVzRows + kB1Ring * kB1Rows);
}

// donor-cell pass (Eq. 4) of one cell from its neighbours and face advectors, dimensions z, y, x,
// psi - F_{i+1/2}/G + F_{i-1/2}/G per dimension (with compensated summation under KAHAN)
template <bool KAHAN>
__device__ __forceinline__ float donor1(float p, const float (&np)[3], const float (&nm)[3], const float (&vp)[3],
                                        const float (&vm)[3], float Gi, bool nug) {
  float s = p, comp = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float Fp = fluxv<false>(p, np[d], vp[d]);
    const float Fm = fluxv<false>(nm[d], p, vm[d]);
    const float t0 = nug ? -__fdividef(Fp, Gi) : -Fp;
    const float t1 = nug ? __fdividef(Fm, Gi) : Fm;
    if constexpr (KAHAN) {
      float yk = t0 - comp;
      float u = s + yk;
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
  return s;
}

template <int NC, bool KAHAN, bool NUG>
__global__ void __launch_bounds__(kCThreads) k_p1b3v(Grid g, const float* __restrict__ psi, V3 V, float vscale,
                                                     const float* __restrict__ G, float* __restrict__ p1,
                                                     float* __restrict__ mx, float* __restrict__ mn) {
  constexpr int W = row_w<NC>();
  constexpr int nP = kBPsiRows * W, nX = kBVxRows * W, nY = kBVyRows * W, nZ = kBVzRows * W, n1 = kB1Rows * W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const sN = reinterpret_cast<float*>(smem_raw);  // [5][nP] psi^n
  float* const sX = sN + kBPsiRing * nP;                  // [2][nX]
  float* const sY = sX + kBVqRing * nX;                   // [2][nY]
  float* const sZ = sY + kBVqRing * nY;                   // [3][nZ]
  float* const s1 = sZ + kBVzRing * nZ;                   // [3][n1] psi^(1)
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int x0 = blockIdx.x * 32 * NC, y0 = blockIdx.y * kRows;
  const int zb = blockIdx.z * kZc;
  const int ze = zb + kZc < nz ? zb + kZc : nz;
  const long long plane = static_cast<long long>(ny) * nx;
  Plan<NC, kBPsiRows, kCThreads> pn;
  Plan<NC, kBVxRows, kCThreads> px;
  Plan<NC, kBVyRows, kCThreads> py;
  Plan<NC, kBVzRows, kCThreads> pz;
  pn.init(tid, x0, y0 - 2, nx, ny);
  px.init(tid, x0, y0 - 1, nx, ny);
  py.init(tid, x0, y0 - 2, nx, ny);
  pz.init(tid, x0, y0 - 1, nx, ny);
  auto zoff = [&](int z) { return static_cast<long long>(wrapi3(z, nz)) * plane; };
  auto rj = [](int k, int j, int n) { const int v = k + j; return v >= n ? v - n : (v < 0 ? v + n : v); };
  // ring slots of plane z at step z: psi^n j = -2 .. 1 (+2 in flight), x/y components j = 0
  // (+1 in flight), z component j = -1 .. 0 (+1 in flight), psi^(1) j = -2 .. 0
  int kn = 0, kq = 0, kz = 0, k1 = 0;
  auto Np = [&](int j) { return sN + rj(kn, j, kBPsiRing) * nP; };
  auto Xp = [&](int j) { return sX + rj(kq, j, kBVqRing) * nX; };
  auto Yp = [&](int j) { return sY + rj(kq, j, kBVqRing) * nY; };
  auto Zp = [&](int j) { return sZ + rj(kz, j, kBVzRing) * nZ; };
  auto Qp = [&](int j) { return s1 + rj(k1, j, kB1Ring) * n1; };
  {  // prologue (step zb-1): psi^n planes zb-2 .. zb, z component zb-2, zb-1, x and y components zb-1
    for (int j = -1; j <= 1; ++j) pn.copy(Np(j), psi + zoff(zb - 1 + j), tid);
    pz.copy(Zp(-1), V.p[0] + zoff(zb - 2), tid);
    pz.copy(Zp(0), V.p[0] + zoff(zb - 1), tid);
    px.copy(Xp(0), V.p[2] + zoff(zb - 1), tid);
    py.copy(Yp(0), V.p[1] + zoff(zb - 1), tid);
    cp_commit();
    cp_wait<0>();
  }
  const int yb = y0 - 1 + w;
  const long long yoff = static_cast<long long>(wrapi3(yb, ny)) * nx;
  const int xl = x0 + NC * lane;
  const int xw = wrapi3(xl, nx);
  constexpr bool nug = NUG;
  // psi^(1) of the cell in column col of this warp's row of plane z, element by element
  auto pass1_col = [&](int col, float Gi) {
    const float* N0 = Np(0) + (w + 1) * W;
    const float* X0 = Xp(0) + w * W;
    const float* Y0 = Yp(0);
    const float np[3] = {Np(1)[(w + 1) * W + col], N0[W + col], N0[col + 1]};
    const float nm[3] = {Np(-1)[(w + 1) * W + col], N0[col - W], N0[col - 1]};
    const float vp[3] = {Zp(0)[w * W + col] * vscale, Y0[(w + 1) * W + col] * vscale, X0[col] * vscale};
    const float vm[3] = {Zp(-1)[w * W + col] * vscale, Y0[w * W + col] * vscale, X0[col - 1] * vscale};
    return donor1<KAHAN>(N0[col], np, nm, vp, vm, Gi, nug);
  };
  // G of the lane's cells in this warp's row, and (lanes 0 and 31) of the cell left (right) of the
  // tile, loaded one plane ahead
  const int hcol = lane == 0 ? 3 : 4 + 32 * NC;  // ring column of the edge lanes' extra cell
  const long long hoff = yoff + wrapi3(x0 - 4 + hcol, nx);
  float g_n[NC], gh_n = 1.0f;
  auto load_g = [&](long long zo) {
    if constexpr (NUG) {
      const long long gb = zo + yoff + xw;
      if constexpr (NC == 4) {
        const float4 c = __ldg(reinterpret_cast<const float4*>(G + gb));
        g_n[0] = c.x; g_n[1] = c.y; g_n[2] = c.z; g_n[3] = c.w;
      } else {
        const float2 c = __ldg(reinterpret_cast<const float2*>(G + gb));
        g_n[0] = c.x; g_n[1] = c.y;
      }
      if (lane == 0 || lane == 31) gh_n = __ldg(G + zo + hoff);
    }
  };
#pragma unroll
  for (int c = 0; c < NC; ++c) g_n[c] = 1.0f;
  load_g(zoff(zb - 1));
  for (int z = zb - 1; z <= ze; ++z) {
    __syncthreads();  // step z's planes are in (each thread waited for its own copies)
    float gi[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) gi[c] = g_n[c];
    const float gh = gh_n;
    if (z + 1 <= ze) {
      pn.copy(Np(2), psi + zoff(z + 2), tid);
      const long long zo = zoff(z + 1);
      pz.copy(Zp(1), V.p[0] + zo, tid);
      px.copy(Xp(1), V.p[2] + zo, tid);
      py.copy(Yp(1), V.p[1] + zo, tid);
      load_g(zo);
    }
    cp_commit();
    {  // psi^(1) of plane z, row yb
      float n0[NC + 3], vx[NC + 3], nu[NC], nd[NC], nzp[NC], nzm[NC], vy[NC], vym[NC], vz[NC], vzm[NC];
      fetch<NC>(Np(0) + (w + 1) * W, lane, n0);
      fetch<NC>(Xp(0) + w * W, lane, vx);
      center<NC>(Np(0) + (w + 2) * W, lane, nu);
      center<NC>(Np(0) + w * W, lane, nd);
      center<NC>(Np(1) + (w + 1) * W, lane, nzp);
      center<NC>(Np(-1) + (w + 1) * W, lane, nzm);
      center<NC>(Yp(0) + (w + 1) * W, lane, vy);
      center<NC>(Yp(0) + w * W, lane, vym);
      center<NC>(Zp(0) + w * W, lane, vz);
      center<NC>(Zp(-1) + w * W, lane, vzm);
      float r[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = c + 1;
        const float np[3] = {nzp[c], nu[c], n0[i + 1]}, nm[3] = {nzm[c], nd[c], n0[i - 1]};
        const float vp[3] = {vz[c] * vscale, vy[c] * vscale, vx[i] * vscale};
        const float vm[3] = {vzm[c] * vscale, vym[c] * vscale, vx[i - 1] * vscale};
        r[c] = donor1<KAHAN>(n0[i], np, nm, vp, vm, nug ? gi[c] : 1.0f, nug);
      }
      put<NC>(Qp(0) + w * W + 4 + NC * lane, r);
      if (lane == 0 || lane == 31) Qp(0)[w * W + hcol] = pass1_col(hcol, gh);
    }
    // no barrier here: of plane z the bounds below read only the thread's own cells, written
    // just above; what they read of other rows and lanes is plane z-1's, written at the
    // previous step, before this step's barrier
    const int q = z - 1;
    if (w >= 1 && w <= kRows && q >= zb && yb < ny) {  // bounds of plane q, row yb
      float a0[NC + 3], b0[NC + 3], au[NC], ad[NC], azp[NC], azm[NC], bu[NC], bd[NC], bzp[NC], bzm[NC];
      fetch<NC>(Np(-1) + (w + 1) * W, lane, a0);
      fetch<NC>(Qp(-1) + w * W, lane, b0);
      center<NC>(Np(-1) + (w + 2) * W, lane, au);
      center<NC>(Np(-1) + w * W, lane, ad);
      center<NC>(Np(0) + (w + 1) * W, lane, azp);
      center<NC>(Np(-2) + (w + 1) * W, lane, azm);
      center<NC>(Qp(-1) + (w + 1) * W, lane, bu);
      center<NC>(Qp(-1) + (w - 1) * W, lane, bd);
      center<NC>(Qp(0) + w * W, lane, bzp);
      center<NC>(Qp(-2) + w * W, lane, bzm);
      float hi[NC], lo[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = c + 1;
        float h = a0[i] > b0[i] ? a0[i] : b0[i];
        float l = a0[i] < b0[i] ? a0[i] : b0[i];
        // neighbours in the order z-1, z+1, y-1, y+1, x-1, x+1; psi^n before psi^(1)
        const float ca[6] = {azm[c], azp[c], ad[c], au[c], a0[i - 1], a0[i + 1]};
        const float cb[6] = {bzm[c], bzp[c], bd[c], bu[c], b0[i - 1], b0[i + 1]};
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          h = ca[j] > h ? ca[j] : h;
          h = cb[j] > h ? cb[j] : h;
          l = ca[j] < l ? ca[j] : l;
          l = cb[j] < l ? cb[j] : l;
        }
        hi[c] = h;
        lo[c] = l;
      }
      const long long o = static_cast<long long>(q) * plane + static_cast<long long>(yb) * nx + xl;
      if (xl + NC <= nx) {
        if constexpr (NC == 4) {
          *reinterpret_cast<float4*>(p1 + o) = make_float4(b0[1], b0[2], b0[3], b0[4]);
          *reinterpret_cast<float4*>(mx + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4*>(mn + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          *reinterpret_cast<float2*>(p1 + o) = make_float2(b0[1], b0[2]);
          *reinterpret_cast<float2*>(mx + o) = make_float2(hi[0], hi[1]);
          *reinterpret_cast<float2*>(mn + o) = make_float2(lo[0], lo[1]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (xl + c < nx) {
            p1[o + c] = b0[c + 1];
            mx[o + c] = hi[c];
            mn[o + c] = lo[c];
          }
        }
      }
    }
    cp_wait<0>();
    kn = rj(kn, 1, kBPsiRing);
    kq = rj(kq, 1, kBVqRing);
    kz = rj(kz, 1, kBVzRing);
    k1 = rj(k1, 1, kB1Ring);
  }
}

// ---------------------------------------------------------------- FCT corrective pass
// One FCT corrective pass (Sect. 3.1.4: the factors beta_up and beta_dn, the limited advector
// V min(1, beta, beta), then the donor-cell pass of Eqs. 4-5 with it) as one z-march with lanes
// of NC cells: the work of the scalar k_corr3 (staged.cu), the same expressions in the same
// order.  At step s every warp forms the factors of plane s on its row (rows y0-1 .. y0+8) into
// a ring of three planes; then warps 1 .. kRows limit and advance their row of plane s-1, while
// warps 0 and kRows+1 form the factors of plane s in the columns just left and right of the
// tile, which the limiter reads at the next step.  psi and the x and y components of the
// unlimited advector are staged in shared-memory rings (cp.async, one step ahead); the values
// that only the cell itself reads (the z component, the bounds and G) come from global memory
// into registers, also one step ahead (those of the cells beside the tile into a small ring).
constexpr int kKPsiRing = 5, kKVRing = 3, kKBRing = 3;
constexpr int kKPsiRows = kRows + 4;  // psi: rows y0-2 .. y0+9
constexpr int kKVRows = kRows + 3;    // x and y components: rows y0-2 .. y0+8
constexpr int kKBRows = kRows + 2;    // factors: rows y0-1 .. y0+8
// the z component, the bounds and G of the cells just left and right of the tile (rows y0 ..
// y0+7), whose factors warps 0 and kRows+1 form: a ring of three planes, 4 arrays each
constexpr int kKHRing = 3, kKHCells = 2 * kRows;
template <int NC>
constexpr size_t corr3v_smem() {
  return sizeof(float) * (row_w<NC>() * (kKPsiRing * kKPsiRows + 2 * kKVRing * kKVRows + 2 * kKBRing * kKBRows) +
                           kKHRing * 4 * kKHCells);
}

// The FCT factors of one cell: in/out sums of the unlimited fluxes through its six faces
// (dimensions z, y, x: the neighbours and face advectors on the + and - side), then
// beta_up = G[psi_max - psi]+ / in and beta_dn = G[psi - psi_min]+ / out, 1 where the sum is not
// positive
template <bool UNIT>
__device__ __forceinline__ void factors1(float p, float pzp, float pzm, float pyp, float pym, float pxp, float pxm,
                                         float vzp, float vzm, float vyp, float vym, float vxp, float vxm, float Gi,
                                         float mxi, float mni, float& bu, float& bd) {
  float in = 0.0f, ou = 0.0f;
  {
    const float Fp = fluxv<UNIT>(p, pzp, vzp), Fm = fluxv<UNIT>(pzm, p, vzm);
    in = in + (posp(Fm) - negp(Fp));
    ou = ou + (posp(Fp) - negp(Fm));
  }
  {
    const float Fp = fluxv<UNIT>(p, pyp, vyp), Fm = fluxv<UNIT>(pym, p, vym);
    in = in + (posp(Fm) - negp(Fp));
    ou = ou + (posp(Fp) - negp(Fm));
  }
  {
    const float Fp = fluxv<UNIT>(p, pxp, vxp), Fm = fluxv<UNIT>(pxm, p, vxm);
    in = in + (posp(Fm) - negp(Fp));
    ou = ou + (posp(Fp) - negp(Fm));
  }
  bu = in > 0.0f ? __fdividef(Gi * posp(mxi - p), in) : 1.0f;
  bd = ou > 0.0f ? __fdividef(Gi * posp(p - mni), ou) : 1.0f;
}

// The limited advector V min(1, a, b) of a face between L and R: the upwind side's outflow
// factor and the downwind side's inflow factor (by the direction of the unlimited flux)
template <bool UNIT>
__device__ __forceinline__ float limited(float L, float R, float V, float buL, float bdL, float buR, float bdR) {
  const float F = fluxv<UNIT>(L, R, V);
  const bool right = F > 0.0f || (F == 0.0f && V > 0.0f);
  const float a = right ? bdL : buL;
  const float b = right ? buR : bdR;
  float m = 1.0f;
  m = minv(a, m);
  m = minv(b, m);
  return V * m;
}

template <int NC, bool NUG, bool UNIT, bool LIM>
__global__ void __launch_bounds__(kCThreads, 2) k_corr3v(Grid g, const float* __restrict__ psi, V3 Vu,
                                                         const float* __restrict__ G, const float* __restrict__ mxg,
                                                         const float* __restrict__ mng, O3 lim,
                                                         float* __restrict__ out) {
  constexpr int W = row_w<NC>();
  constexpr int nP = kKPsiRows * W, nV = kKVRows * W, nB = kKBRows * W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const sP = reinterpret_cast<float*>(smem_raw);  // [5][nP] psi
  float* const sX = sP + kKPsiRing * nP;                  // [3][nV] x component
  float* const sY = sX + kKVRing * nV;                    // [3][nV] y component
  float* const sU = sY + kKVRing * nV;                    // [3][nB] beta_up
  float* const sD = sU + kKBRing * nB;                    // [3][nB] beta_dn
  float* const sH = sD + kKBRing * nB;                    // [3][4][kKHCells] halo cells' vz, mx, mn, G
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int x0 = blockIdx.x * 32 * NC, y0 = blockIdx.y * kRows;
  const int zb = blockIdx.z * kZc;
  const int ze = zb + kZc < nz ? zb + kZc : nz;
  const long long plane = static_cast<long long>(ny) * nx;
  Plan<NC, kKPsiRows, kCThreads> pp;
  Plan<NC, kKVRows, kCThreads> pv;
  pp.init(tid, x0, y0 - 2, nx, ny);
  pv.init(tid, x0, y0 - 2, nx, ny);
  auto zoff = [&](int z) { return static_cast<long long>(wrapi3(z, nz)) * plane; };
  auto rot = [](int s, int j, int n) { const int v = s + j; return v >= n ? v - n : v; };
  // this warp's row y0 - 1 + w and the lane's first column, wrapped, for the register loads
  const int y = y0 - 1 + w;
  const long long yo = static_cast<long long>(wrapi3(y, ny)) * nx;
  const int xl = x0 + NC * lane;
  const int xw = wrapi3(xl, nx);
  auto ld = [&](const float* a, long long zo, float (&r)[NC]) {
    const float* q = a + zo + yo + xw;
    if constexpr (NC == 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(q));
      r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else {
      const float2 v = __ldg(reinterpret_cast<const float2*>(q));
      r[0] = v.x; r[1] = v.y;
    }
  };
  // ring slots at step s: psi plane s+j (j = -2 .. 2) in rot(kp, j + 2, 5); the x and y
  // components of plane s+j (j = -1 .. 1) in rot(kv, j + 1, 3); the factors of plane s+j
  // (j = -2 .. 0) in rot(kb, j + 2, 3).  Registers: the z component of planes s+1 (loading),
  // s, s-1, s-2; the bounds of plane s+1 (loading); G of planes s+1 (loading), s, s-1.
  int kp = 0, kv = 0, kb = 0, kh = 0;
  // halo-cell arrays of plane s+j (j = -1 .. 1) in ring slot rot(kh, j + 1, 3); thread tid <
  // 4 kKHCells copies array ha (the z component, the bounds, G) of cell hk (the left column for
  // hk < kRows; field row y0 + hk % kRows)
  auto copy_h = [&](int slot, long long zo) {
    const int ha = tid / kKHCells, hk = tid - ha * kKHCells;
    if (tid < 4 * kKHCells && (ha < 3 || NUG)) {
      const float* src = ha == 0 ? Vu.p[0] : (ha == 1 ? mxg : (ha == 2 ? mng : G));
      const long long off = static_cast<long long>(wrapi3(y0 + hk % kRows, ny)) * nx +
                            wrapi3(hk < kRows ? x0 - 1 : x0 + 32 * NC, nx);
      cp_async<4>(sH + (slot * 4 + ha) * kKHCells + hk, src + zo + off);
    }
  };
  float vz_n[NC], vz_c[NC], vz_m[NC], vz_mm[NC], mx_n[NC], mn_n[NC], g_n[NC], g_c[NC], g_m[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) { vz_m[c] = 0.0f; g_c[c] = 1.0f; g_n[c] = 1.0f; }
  {  // prologue (step zb-1): psi planes zb-2 .. zb, components of plane zb-1
    pp.copy(sP + 1 * nP, psi + zoff(zb - 2), tid);
    pp.copy(sP + 2 * nP, psi + zoff(zb - 1), tid);
    pp.copy(sP + 3 * nP, psi + zoff(zb), tid);
    pv.copy(sX + 1 * nV, Vu.p[2] + zoff(zb - 1), tid);
    pv.copy(sY + 1 * nV, Vu.p[1] + zoff(zb - 1), tid);
    copy_h(1, zoff(zb - 1));
    cp_commit();
    ld(Vu.p[0], zoff(zb - 2), vz_c);
    const long long zo = zoff(zb - 1);
    ld(Vu.p[0], zo, vz_n);
    ld(mxg, zo, mx_n);
    ld(mng, zo, mn_n);
    if (NUG) ld(G, zo, g_n);
    cp_wait<0>();
  }
  for (int s = zb - 1; s <= ze; ++s) {
    __syncthreads();  // step s's planes are in (each thread waited for its own copies)
    float mx_c[NC], mn_c[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      vz_mm[c] = vz_m[c]; vz_m[c] = vz_c[c]; vz_c[c] = vz_n[c];
      g_m[c] = g_c[c]; g_c[c] = g_n[c];
      mx_c[c] = mx_n[c]; mn_c[c] = mn_n[c];
    }
    if (s + 1 <= ze) {
      pp.copy(sP + rot(kp, 4, kKPsiRing) * nP, psi + zoff(s + 2), tid);
      const long long zo = zoff(s + 1);
      pv.copy(sX + rot(kv, 2, kKVRing) * nV, Vu.p[2] + zo, tid);
      pv.copy(sY + rot(kv, 2, kKVRing) * nV, Vu.p[1] + zo, tid);
      copy_h(rot(kh, 2, kKHRing), zo);
      ld(Vu.p[0], zo, vz_n);
      ld(mxg, zo, mx_n);
      ld(mng, zo, mn_n);
      if (NUG) ld(G, zo, g_n);
    }
    cp_commit();
    const float* P0 = sP + rot(kp, 2, kKPsiRing) * nP;  // psi of plane s
    const float* Pp = sP + rot(kp, 3, kKPsiRing) * nP;  // s+1
    const float* Pm = sP + rot(kp, 1, kKPsiRing) * nP;  // s-1
    const float* X0 = sX + rot(kv, 1, kKVRing) * nV;    // components of plane s
    const float* Y0 = sY + rot(kv, 1, kKVRing) * nV;
    float* const U0 = sU + rot(kb, 2, kKBRing) * nB;    // factors of plane s
    float* const D0 = sD + rot(kb, 2, kKBRing) * nB;
    {  // factors of plane s, row y0 - 1 + w (psi and component row w + 1, factor row w)
      float pc[NC + 3], vx[NC + 3], pu[NC], pd[NC], pzp[NC], pzm[NC], vy[NC], vym[NC];
      fetch<NC>(P0 + (w + 1) * W, lane, pc);
      fetch<NC>(X0 + (w + 1) * W, lane, vx);
      center<NC>(P0 + (w + 2) * W, lane, pu);
      center<NC>(P0 + w * W, lane, pd);
      center<NC>(Pp + (w + 1) * W, lane, pzp);
      center<NC>(Pm + (w + 1) * W, lane, pzm);
      center<NC>(Y0 + (w + 1) * W, lane, vy);
      center<NC>(Y0 + w * W, lane, vym);
      float bu[NC], bd[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = c + 1;
        factors1<UNIT>(pc[i], pzp[c], pzm[c], pu[c], pd[c], pc[i + 1], pc[i - 1], vz_c[c], vz_m[c], vy[c], vym[c],
                       vx[i], vx[i - 1], NUG ? g_c[c] : 1.0f, mx_c[c], mn_c[c], bu[c], bd[c]);
      }
      put<NC>(U0 + w * W + 4 + NC * lane, bu);
      put<NC>(D0 + w * W + 4 + NC * lane, bd);
    }
    // no barrier here: of plane s the limiter below reads only the thread's own factors, written
    // just above; the factors of other rows and lanes it reads are plane s-1's, written at the
    // previous step (the edge warps' columns included), before this step's barrier
    const int q = s - 1;
    if (w >= 1 && w <= kRows) {
      if (q >= zb && y < ny) {  // limit and advance row y of plane q = s - 1
        const float* Q0 = Pm;                                  // psi of plane q
        const float* Qm = sP + kp * nP;                        // q - 1
        const float* XQ = sX + kv * nV;                        // components of plane q
        const float* YQ = sY + kv * nV;
        const float* UQ = sU + rot(kb, 1, kKBRing) * nB;       // factors of plane q
        const float* DQ = sD + rot(kb, 1, kKBRing) * nB;
        const float* UQm = sU + kb * nB;                       // q - 1
        const float* DQm = sD + kb * nB;
        // the cells' psi and factors; the donor sum and the limited advectors, dimension by
        // dimension (z, y, x) so that only one dimension's neighbours are live at a time
        float p[NC], bu[NC], bd[NC], acc[NC], hz[NC], hy[NC], hx[NC];
        center<NC>(Q0 + (w + 1) * W, lane, p);
        center<NC>(UQ + w * W, lane, bu);
        center<NC>(DQ + w * W, lane, bd);
        float Gc[NC];  // G of the cells (the divisor of the donor terms)
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[c] = p[c]; Gc[c] = NUG ? g_m[c] : 1.0f; }
        // the donor terms of one dimension: -F+/G then +F-/G, added in that order
        auto donor_d = [&](int c, float Fp, float Fm) {
          const float t0 = NUG ? -__fdividef(Fp, Gc[c]) : -Fp;
          const float t1 = NUG ? __fdividef(Fm, Gc[c]) : Fm;
          acc[c] = acc[c] + t0;
          acc[c] = acc[c] + t1;
        };
        {  // z
          float nzp[NC], nzm[NC], uzp[NC], dzp[NC], uzm[NC], dzm[NC];
          center<NC>(P0 + (w + 1) * W, lane, nzp);
          center<NC>(Qm + (w + 1) * W, lane, nzm);
          center<NC>(U0 + w * W, lane, uzp);
          center<NC>(D0 + w * W, lane, dzp);
          center<NC>(UQm + w * W, lane, uzm);
          center<NC>(DQm + w * W, lane, dzm);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float hp = limited<UNIT>(p[c], nzp[c], vz_m[c], bu[c], bd[c], uzp[c], dzp[c]);
            const float hm = limited<UNIT>(nzm[c], p[c], vz_mm[c], uzm[c], dzm[c], bu[c], bd[c]);
            donor_d(c, fluxv<UNIT>(p[c], nzp[c], hp), fluxv<UNIT>(nzm[c], p[c], hm));
            hz[c] = hp;
          }
        }
        {  // y
          float nyp[NC], nym[NC], vy[NC], vym[NC], uu[NC], du[NC], ud[NC], dd[NC];
          center<NC>(Q0 + (w + 2) * W, lane, nyp);
          center<NC>(Q0 + w * W, lane, nym);
          center<NC>(YQ + (w + 1) * W, lane, vy);
          center<NC>(YQ + w * W, lane, vym);
          center<NC>(UQ + (w + 1) * W, lane, uu);
          center<NC>(DQ + (w + 1) * W, lane, du);
          center<NC>(UQ + (w - 1) * W, lane, ud);
          center<NC>(DQ + (w - 1) * W, lane, dd);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float hp = limited<UNIT>(p[c], nyp[c], vy[c], bu[c], bd[c], uu[c], du[c]);
            const float hm = limited<UNIT>(nym[c], p[c], vym[c], ud[c], dd[c], bu[c], bd[c]);
            donor_d(c, fluxv<UNIT>(p[c], nyp[c], hp), fluxv<UNIT>(nym[c], p[c], hm));
            hy[c] = hp;
          }
        }
        {  // x: the row segments with their outer neighbours
          float pc[NC + 3], vx[NC + 3], uc[NC + 3], dc[NC + 3];
          fetch<NC>(Q0 + (w + 1) * W, lane, pc);
          fetch<NC>(XQ + (w + 1) * W, lane, vx);
          fetch<NC>(UQ + w * W, lane, uc);
          fetch<NC>(DQ + w * W, lane, dc);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int i = c + 1;
            const float hp = limited<UNIT>(p[c], pc[i + 1], vx[i], bu[c], bd[c], uc[i + 1], dc[i + 1]);
            const float hm = limited<UNIT>(pc[i - 1], p[c], vx[i - 1], uc[i - 1], dc[i - 1], bu[c], bd[c]);
            donor_d(c, fluxv<UNIT>(p[c], pc[i + 1], hp), fluxv<UNIT>(pc[i - 1], p[c], hm));
            hx[c] = hp;
          }
        }
        const long long o = static_cast<long long>(q) * plane + static_cast<long long>(y) * nx + xl;
        if (xl + NC <= nx) {
          put<NC>(out + o, acc);
          if constexpr (LIM) {
            put<NC>(lim.p[0] + o, hz);
            put<NC>(lim.p[1] + o, hy);
            put<NC>(lim.p[2] + o, hx);
          }
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (xl + c < nx) {
              out[o + c] = acc[c];
              if constexpr (LIM) {
                lim.p[0][o + c] = hz[c];
                lim.p[1][o + c] = hy[c];
                lim.p[2][o + c] = hx[c];
              }
            }
          }
        }
      }
    } else if (s >= zb && s < ze && lane < kRows) {
      // warps 0 and kRows+1: the factors of plane s in the column left (right) of the tile, factor
      // row r = lane + 1 (field row y0 + lane), for the limiter of the next step
      const int r = lane + 1;
      const int cix = w == 0 ? 3 : 4 + 32 * NC;  // ring column of x0 - 1 (x0 + 32 NC)
      const int pr = (r + 1) * W + cix;          // psi and component ring index of the cell
      const float* Hs = sH + rot(kh, 1, kKHRing) * 4 * kKHCells + (w == 0 ? 0 : kRows) + lane;  // plane s
      const float* Hm = sH + kh * 4 * kKHCells + (w == 0 ? 0 : kRows) + lane;                   // s - 1
      float bu, bd;
      factors1<UNIT>(P0[pr], Pp[pr], Pm[pr], P0[pr + W], P0[pr - W], P0[pr + 1], P0[pr - 1], Hs[0], Hm[0], Y0[pr],
                     Y0[pr - W], X0[pr], X0[pr - 1], NUG ? Hs[3 * kKHCells] : 1.0f, Hs[kKHCells],
                     Hs[2 * kKHCells], bu, bd);
      U0[r * W + cix] = bu;
      D0[r * W + cix] = bd;
    }
    cp_wait<0>();
    kp = rot(kp, 1, kKPsiRing);
    kv = rot(kv, 1, kKVRing);
    kb = rot(kb, 1, kKBRing);
    kh = rot(kh, 1, kKHRing);
  }
}

template <int NC, int MINB, bool ABS, bool IGA, bool TOT, bool NUG>
void launch_v(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, float* const* out,
              cudaStream_t st) {
  static PerDevice<bool> attr;
  attr.get([](int) {
    return cudaFuncSetAttribute(k_antidiff3v<NC, MINB, ABS, IGA, TOT, NUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(antidiff3v_smem<NC>())) == cudaSuccess;
  });
  const dim3 grid(static_cast<unsigned>((g.n[2] + 32 * NC - 1) / (32 * NC)),
                  static_cast<unsigned>((g.n[1] + kRows - 1) / kRows), static_cast<unsigned>((g.n[0] + kZc - 1) / kZc));
  V3 vin{{v[0], v[1], v[2]}};
  O3 vo{{out[0], out[1], out[2]}};
  k_antidiff3v<NC, MINB, ABS, IGA, TOT, NUG><<<grid, dim3(32, kRows), antidiff3v_smem<NC>(), st>>>(g, psi, vin, vscale,
                                                                                                  G, vo);
}

template <int NC, bool KAHAN, bool NUG>
void launch_b(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, float* p1,
              float* mx, float* mn, cudaStream_t st) {
  static PerDevice<bool> attr;
  attr.get([](int) {
    return cudaFuncSetAttribute(k_p1b3v<NC, KAHAN, NUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(p1b3v_smem<NC>())) == cudaSuccess;
  });
  const dim3 grid(static_cast<unsigned>((g.n[2] + 32 * NC - 1) / (32 * NC)),
                  static_cast<unsigned>((g.n[1] + kRows - 1) / kRows), static_cast<unsigned>((g.n[0] + kZc - 1) / kZc));
  V3 vv{{v[0], v[1], v[2]}};
  k_p1b3v<NC, KAHAN, NUG><<<grid, dim3(32, kCWarps), p1b3v_smem<NC>(), st>>>(g, psi, vv, vscale, G, p1, mx, mn);
}

template <int NC, bool NUG, bool UNIT, bool LIM>
void launch_k(const Grid& g, const float* psi, const float* const* vu, const float* G, const float* mx,
              const float* mn, float* const* lim, float* out, cudaStream_t st) {
  static PerDevice<bool> attr;
  attr.get([](int) {
    return cudaFuncSetAttribute(k_corr3v<NC, NUG, UNIT, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(corr3v_smem<NC>())) == cudaSuccess;
  });
  const dim3 grid(static_cast<unsigned>((g.n[2] + 32 * NC - 1) / (32 * NC)),
                  static_cast<unsigned>((g.n[1] + kRows - 1) / kRows), static_cast<unsigned>((g.n[0] + kZc - 1) / kZc));
  V3 vv{{vu[0], vu[1], vu[2]}};
  O3 lo{{lim[0], lim[1], lim[2]}};
  k_corr3v<NC, NUG, UNIT, LIM><<<grid, dim3(32, kCWarps), corr3v_smem<NC>(), st>>>(g, psi, vv, G, mx, mn, lo, out);
}

// The vectorised z-march runs with lanes of 4 cells on fields of at least 128 columns; narrower
// fields take the scalar z-march of staged.cu (measured at 256^3: lanes of 2 cells gain nothing
// over it).  MPDATA_MARCH3=0 in the environment selects the scalar z-march everywhere.
bool use_vec(const Grid& g) {
  static const bool off = [] {
    const char* e = std::getenv("MPDATA_MARCH3");
    return e && std::atoi(e) == 0;
  }();
  return !off && g.n[2] >= 128;
}

bool al16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// The vectorised pseudo-advector z-march for FP32 3D fields whose x extent is a multiple of 4
// with 16-byte aligned arrays; false (nothing launched) otherwise.
bool antidiff3_vec(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, bool iga,
                   bool tot, bool abs_psi, float* const* out, cudaStream_t st) {
  if (g.nd != 3 || g.n[2] % 4 != 0 || g.any_open()) return false;
  if (!al16(psi) || !al16(G) || !al16(v[0]) || !al16(v[1]) || !al16(v[2]) || !al16(out[0]) || !al16(out[1]) ||
      !al16(out[2]) || !use_vec(g))
    return false;
  const bool nug = G != nullptr;
#define MPD_V(A, I, T, N) launch_v<4, 2, A, I, T, N>(g, psi, v, vscale, G, out, st)
#define MPD_VN(A, I, T) \
  do { if (nug) MPD_V(A, I, T, true); else MPD_V(A, I, T, false); } while (0)
#define MPD_VT(A, I) \
  do { if (tot) MPD_VN(A, I, true); else MPD_VN(A, I, false); } while (0)
  if (abs_psi) MPD_VT(true, false);
  else if (iga) MPD_VT(false, true);
  else MPD_VT(false, false);
#undef MPD_VT
#undef MPD_VN
#undef MPD_V
  return true;
}

// The vectorised pass-1-and-bounds z-march (FP32, same conditions as antidiff3_vec).
bool p1b3_vec(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, bool kahan,
              float* p1, float* mx, float* mn, cudaStream_t st) {
  if (g.nd != 3 || g.n[2] % 4 != 0 || g.any_open()) return false;
  if (!al16(psi) || !al16(G) || !al16(v[0]) || !al16(v[1]) || !al16(v[2]) || !al16(p1) || !al16(mx) || !al16(mn) ||
      !use_vec(g))
    return false;
  const bool nug = G != nullptr;
#define MPD_B(K)                                                             \
  do {                                                                       \
    if (nug) launch_b<4, K, true>(g, psi, v, vscale, G, p1, mx, mn, st);     \
    else launch_b<4, K, false>(g, psi, v, vscale, G, p1, mx, mn, st);        \
  } while (0)
  if (kahan) MPD_B(true); else MPD_B(false);
#undef MPD_B
  return true;
}

// The vectorised FCT corrective pass (FP32; same conditions as antidiff3_vec, and neither the
// Kahan summation nor a source term); false (nothing launched) otherwise.
bool corr3_vec(const Grid& g, const float* psi, const float* const* vu, const float* G, bool iga, bool kahan,
               const float* mx, const float* mn, bool post, float* const* lim, float* out, cudaStream_t st) {
  if (g.nd != 3 || g.n[2] % 4 != 0 || g.any_open() || kahan || post) return false;
  if (!al16(psi) || !al16(G) || !al16(vu[0]) || !al16(vu[1]) || !al16(vu[2]) || !al16(mx) || !al16(mn) ||
      !al16(out) || !al16(lim[0]) || !al16(lim[1]) || !al16(lim[2]) || !use_vec(g))
    return false;
  const bool nug = G != nullptr, lm = lim[0] != nullptr;
#define MPD_K(N, U, L) launch_k<4, N, U, L>(g, psi, vu, G, mx, mn, lim, out, st)
#define MPD_KL(N, U) \
  do { if (lm) MPD_K(N, U, true); else MPD_K(N, U, false); } while (0)
#define MPD_KU(N) \
  do { if (iga) MPD_KL(N, true); else MPD_KL(N, false); } while (0)
  if (nug) MPD_KU(true);
  else MPD_KU(false);
#undef MPD_KU
#undef MPD_KL
#undef MPD_K
  return true;
}

}  // namespace mpd
