/*
 * MPDATA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of one MPDATA time step for the
 * generalised transport equation d_t(G psi) + div(G u psi) = G R
 * (libmpdata++ 0.1 paper, Sect. 1, Eq. 1; homogeneous form Sect. 3.1, Eq. 3)
 * on a periodic Arakawa-C grid (Sect. 2.3), plus its tangent-linear and adjoint.
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline
 * leg may load this library.  The CUDA library shares no code, header, table or
 * constant with it, and neither side includes or links the other.
 *
 * Layout: row-major, last dimension fastest (Sect. 3.2.5).  A field of shape
 * (n_0, ..., n_{D-1}) has N cells; cell i and the advector component d stored
 * at index i describe the face between cell i and cell i + e_d (periodic).
 *
 * One step (Sect. 3.1.1 and 4.1; readings of passages the paper leaves to
 * other papers are listed beside each function):
 *   psi0 = psi (+ dt R if euler_b)
 *   psi1 = donor(psi0, GC)                                   Eqs. 4-5
 *   for k = 2..n_iters:
 *     V^k    = antidiffusive advector from V^{k-1}, psi^{k-1}  Eq. 6 (+ multi-D, tot, dfl;
 *              |psi| in its psi-fractions with abs)
 *     V^k    = FCT-limited V^k (if fct)                      Sect. 3.1.4
 *     psi^k  = donor(psi^{k-1}, V^k)                         Eqs. 4-5
 *   psi^{n+1} = psi^{n_iters} (+ dt R if euler_a)
 *
 * Every sub-step is one loop over output elements calling a small local
 * formula written once as a template over the number type.  Instantiated with
 * double it is the forward step; instantiated with a dual number it yields the
 * local partial derivatives, which the tangent-linear sweep gathers and the
 * adjoint sweep scatters (the exact transpose of the same Jacobian entries).
 *
 * Non-differentiable points: [x]+ and [x]- have derivative 1/2 at x = 0 (so
 * |x| has derivative 0 there); max/min selections pass the derivative of the
 * first candidate, in the stated candidate order, that attains the extremum.
 *
 * Build: g++ -std=c++17 -O2 -ffp-contract=off -fopenmp -shared -fPIC
 * (no fused multiply-add contraction, so x86-64 and aarch64 hosts agree bit for bit).
 */
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

/* Option bits of the oracle (the same values the library interface defines). */
constexpr unsigned O_FCT = 1u, O_TOT = 2u, O_IGA = 4u, O_NUG = 8u, O_KAHAN = 16u,
                   O_RHS_A = 32u, O_RHS_B = 64u, O_ABS = 256u, O_DFL = 512u;
/* open edges (Sect. 2.4, bcond::open) along dimension d: bit O_OPEN0 << d */
constexpr unsigned O_OPEN0 = 1024u;

/* ------------------------------------------------------------------ grid */

struct Grid {
  int nd = 1;                 /* number of dimensions, 1..3 */
  long n[3] = {1, 1, 1};      /* extents on three internal axes; leading unused axes have extent 1 */
  long N = 1;
  bool open[3] = {false, false, false};  /* open edges on an internal axis (else periodic) */
  int ax(int d) const { return 3 - nd + d; }  /* internal axis of dimension d */
};

struct Cell { long c[3]; };

inline long wrapc(long c, long n) { long r = c % n; return r < 0 ? r + n : r; }

/* cell x shifted by s cells along dimension d: periodic, or, with open edges (Sect. 2.4,
 * bcond::open), clamped to the edge cell -- the halo cells beyond an open edge hold the edge
 * value (zero gradient) */
inline Cell sh(const Grid& g, Cell x, int d, long s) {
  int a = g.ax(d);
  long v = x.c[a] + s;
  if (g.open[a]) x.c[a] = v < 0 ? 0 : (v > g.n[a] - 1 ? g.n[a] - 1 : v);
  else x.c[a] = wrapc(v, g.n[a]);
  return x;
}
inline long lin(const Grid& g, const Cell& x) { return (x.c[0] * g.n[1] + x.c[1]) * g.n[2] + x.c[2]; }
inline Cell cell_of(const Grid& g, long i) {
  Cell x;
  x.c[2] = i % g.n[2];
  long r = i / g.n[2];
  x.c[1] = r % g.n[1];
  x.c[0] = r / g.n[1];
  return x;
}
inline long nbr(const Grid& g, long i, int d, long s) { return lin(g, sh(g, cell_of(g, i), d, s)); }

/* Storage index of a face of a vector field along d: the face s faces from face i+1/2 of
 * cell i.  Periodic: n faces, wrapped.  Open edges (Sect. 2.4: a zero-divergence condition on
 * the domain edges): the n-1 faces between the cells are interior (indices 0 .. n-2, the
 * advector of Sect. 3.2.5 is one shorter than the field along its own dimension), and the two
 * boundary faces -1/2 and n-1/2 take the value of the adjacent interior face, so that every
 * vector field -- the advector and each pass's pseudo-velocity -- has zero divergence along d
 * in the edge cells.  The entry n-1 of a component along an open dimension is never read. */
inline long fc(const Grid& g, long i, int d, long s) {
  Cell x = cell_of(g, i);
  const int a = g.ax(d);
  long f = x.c[a] + s;
  if (g.open[a]) x.c[a] = f < 0 ? 0 : (f > g.n[a] - 2 ? g.n[a] - 2 : f);
  else x.c[a] = wrapc(f, g.n[a]);
  return lin(g, x);
}

/* ------------------------------------------------------------ dual numbers */

constexpr int NSLOT = 64;

struct Dual {
  double v;
  double d[NSLOT];
  Dual() : v(0.0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }  // NOLINT: implicit on purpose
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r; r.v = a.v + b.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r; r.v = a.v - b.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) { Dual r; r.v = -a.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r; r.v = a.v * b.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r; r.v = a.v / b.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v; return r; }
inline Dual operator*(double a, const Dual& b) { Dual r; r.v = a * b.v; for (int k = 0; k < NSLOT; ++k) r.d[k] = a * b.d[k]; return r; }
inline Dual operator*(const Dual& a, double b) { Dual r; r.v = a.v * b; for (int k = 0; k < NSLOT; ++k) r.d[k] = a.d[k] * b; return r; }
inline Dual operator/(const Dual& a, double b) { Dual r; r.v = a.v / b; for (int k = 0; k < NSLOT; ++k) r.d[k] = a.d[k] / b; return r; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

/* [x]+ = max(x, 0) and [x]- = min(x, 0) (Eq. 5); derivative 1/2 at x = 0 */
template <class T> T pos(const T& x) { if (val(x) > 0) return x; if (val(x) < 0) return T(0.0); return 0.5 * x; }
template <class T> T neg(const T& x) { if (val(x) < 0) return x; if (val(x) > 0) return T(0.0); return 0.5 * x; }
template <class T> T absv(const T& x) { if (val(x) > 0) return x; if (val(x) < 0) return -x; return 0.0 * x; }
/* psi-fraction with the zero-denominator guard: n/d, or 0 when d == 0 */
template <class T> T frac(const T& n, const T& d) { if (val(d) != 0.0) return n / d; return T(0.0); }

/* --------------------------------------------------------------- the tape */

/* Each array of one step is written exactly once (single assignment), so the
 * adjoint sweep can consume an array's adjoint right after its producer. */
struct Ids {
  int K = 1;
  int in() const { return 0; }                        /* step input psi^n */
  int psi(int k) const { return 1 + k; }              /* psi^(k), k = 0..K */
  int out() const { return K + 2; }                   /* psi^{n+1} */
  int mx() const { return K + 3; }
  int mn() const { return K + 4; }
  int base() const { return K + 5; }
  int v(int k, int d) const { return base() + (k * 3 + d) * 4 + 0; }   /* antidiffusive (k>=2) or input (k=1) advector */
  int vh(int k, int d) const { return base() + (k * 3 + d) * 4 + 1; }  /* FCT-limited advector */
  int f(int k, int d) const { return base() + (k * 3 + d) * 4 + 2; }   /* unlimited flux (FCT only) */
  int fh(int k, int d) const { return base() + (k * 3 + d) * 4 + 3; }  /* flux used by the donor pass */
  int bu(int k) const { return base() + (K + 1) * 12 + 2 * k; }
  int bd(int k) const { return base() + (K + 1) * 12 + 2 * k + 1; }
  int count() const { return base() + (K + 1) * 12 + 2 * (K + 1); }
};

struct Ctx {
  Grid g;
  Ids id;
  int K = 1;
  bool fct = false, tot = false, iga = false, kahan = false, rhs_a = false, rhs_b = false;
  bool abs = false;  /* |psi| in every psi-fraction of the pseudo-velocity (Sect. 3.1.5) */
  bool dfl = false;  /* divergent-flow term of the pseudo-velocity (Sect. 3.1.3) */
  const double* G = nullptr;  /* NULL => G = 1 */
  const double* R = nullptr;
  double dt = 0.0;
  std::vector<std::vector<double>>* A = nullptr;  /* tape values */
  double Gc(long i) const { return G ? G[i] : 1.0; }
  double raw(int a, long i) const { return (*A)[a][i]; }
  /* advector that drives pass k: the input advector for k = 1, the limited one under FCT */
  int adv(int k, int d) const { return (k == 1 || !fct) ? id.v(k, d) : id.vh(k, d); }
};

/* --------------------------------------------------------- local formulas */

/* euler_b: psi^(0) = psi^n + dt R^n before advection (Sect. 4.1, euler_b scheme) */
template <class T, class Get> T f_pre(const Ctx& c, long i, Get get) {
  T p = get(c.id.in(), i);
  if (c.rhs_b) return p + T(c.dt * c.R[i]);
  return p;
}

/* euler_a: psi^{n+1} = ADV(psi^n) + dt R^n after advection (Sect. 4.1, euler_a scheme) */
template <class T, class Get> T f_post(const Ctx& c, long i, Get get) {
  T p = get(c.id.psi(c.K), i);
  if (c.rhs_a) return p + T(c.dt * c.R[i]);
  return p;
}

/* Donor-cell flux through face i+1/2 of dimension d in pass k, Eq. 5 in Courant
 * units: F(L, R, V) = [V]+ L + [V]- R with V = G*C the advector.  In the
 * corrective passes of the infinite-gauge variant psi is replaced by 1 (the
 * limit of MPDATA on psi + c for c -> infinity, Sect. 3.1.5), so F = V. */
template <class T, class Get> T f_flux_at(const Ctx& c, int k, int d, long i, long s, bool limited, Get get) {
  T V = get(limited ? c.adv(k, d) : c.id.v(k, d), fc(c.g, i, d, s));
  if (k >= 2 && c.iga) return V;
  T L = get(c.id.psi(k - 1), nbr(c.g, i, d, s));
  T R = get(c.id.psi(k - 1), nbr(c.g, i, d, s + 1));
  return pos(V) * L + neg(V) * R;
}
template <class T, class Get> T f_flux(const Ctx& c, int k, int d, long i, bool limited, Get get) {
  return f_flux_at<T>(c, k, d, i, 0, limited, get);
}
/* Flux through face i-1/2 along d: the stored flux of face (i-1)+1/2, except at an open
 * left edge, where face -1/2 is a boundary face (no storage): its flux is formed here, with
 * the halo value psi_0 on both sides and the advector of face 1/2. */
template <class T, class Get> T f_flux_m(const Ctx& c, int k, int d, long i, bool limited, Get get) {
  const int a = c.g.ax(d);
  if (c.g.open[a] && cell_of(c.g, i).c[a] == 0) return f_flux_at<T>(c, k, d, i, -1, limited, get);
  return get(limited ? c.id.fh(k, d) : c.id.f(k, d), nbr(c.g, i, d, -1));
}

/* Donor-cell pass, Eq. 4: psi_i - (1/G_i) sum_d [F_{i+1/2} - F_{i-1/2}], summed
 * as psi_i - F_{i+1/2}/G_i + F_{i-1/2}/G_i, dimension 0 first.  With the Kahan
 * option the same terms are added with compensated summation (Sect. 3.1.1). */
template <class T, class Get> T f_donor(const Ctx& c, int k, long i, Get get) {
  T s = get(c.id.psi(k - 1), i);
  T comp = 0.0;
  const double Gi = c.Gc(i);
  for (int d = 0; d < c.g.nd; ++d) {
    T Fp = get(c.id.fh(k, d), i);
    T Fm = f_flux_m<T>(c, k, d, i, true, get);
    T terms[2] = {-Fp / Gi, Fm / Gi};
    for (const T& t : terms) {
      if (c.kahan) {
        T y = t - comp;
        T u = s + y;
        comp = (u - s) - y;
        s = u;
      } else {
        s = s + t;
      }
    }
  }
  return s;
}

/* FCT bounds (Sect. 3.1.4; Smolarkiewicz & Grabowski 1990): extremum over the
 * cell and its +-e_d neighbours of psi^n and psi^(1).  Candidate order: the cell,
 * then for d = 0.. the -e_d and +e_d neighbours; psi^n before psi^(1). */
template <class T, class Get> T f_bound(const Ctx& c, long i, bool upper, Get get) {
  long loc[7];
  int nl = 0;
  loc[nl++] = i;
  for (int d = 0; d < c.g.nd; ++d) {
    loc[nl++] = nbr(c.g, i, d, -1);
    loc[nl++] = nbr(c.g, i, d, +1);
  }
  T best = get(c.id.psi(0), loc[0]);
  for (int j = 0; j < nl; ++j) {
    for (int a = 0; a < 2; ++a) {
      T v = get(c.id.psi(a), loc[j]);
      if (upper ? val(v) > val(best) : val(v) < val(best)) best = v;
    }
  }
  return best;
}

/* Third-order terms of the pseudo-velocity at face i+1/2 along d (Sect. 3.1.2;
 * the formulae are cited there to Smolarkiewicz & Margolin 1998, Eq. 36, and
 * not reproduced in the paper).  Reading, derived from the requirement that
 * one step of the linear (infinite-gauge) two-pass scheme with constant
 * Courant numbers C be exact on every cubic polynomial of cell means, then
 * normalised like the second-order terms (each difference divided by the sum
 * of the psi values it uses; divided by their count under infinite gauge):
 *   + Gb (3 C|C| - 2 C^3 - C)/3                * D_dd
 *   + sum_{q != d} Gb |C| C_q (1 - 2|C|)         * D_dq
 *   - (2/3) Gb C C_q1 C_q2                       * D_q1q2     (3D only)
 * with C = V/Gb, C_q = Vq_bar/Gb and
 *   D_dd   = frac(psi_{i+2} - psi_{i+1} - psi_i + psi_{i-1}, their sum)    (along d),
 *   D_dq   = frac((psi_{i+e_d+e_q} - psi_{i+e_q}) - (psi_{i+e_d-e_q} - psi_{i-e_q}), their sum),
 *   D_q1q2 = frac(pairs at (+q1+q2) - (+q1-q2) - (-q1+q2) + (-q1-q2), their sum),
 *            a pair being psi_j + psi_{j+e_d}. */
template <class T, class Get>
T f_tot(const Ctx& c, int k, int d, long i, const T& V, const T* Vq, double Gb, Get get_psi) {
  const Grid& g = c.g;
  const int P = c.id.psi(k - 1);
  /* variable-sign option: the psi values of the fractions enter as |psi| */
  auto get = [&](int a, long j) { return c.abs ? absv(get_psi(a, j)) : get_psi(a, j); };
  const Cell x = cell_of(g, i);
  T pm = get(P, nbr(g, i, d, -1));
  T p0 = get(P, i);
  T p1 = get(P, nbr(g, i, d, +1));
  T p2 = get(P, nbr(g, i, d, +2));
  T num = ((p2 - p1) - p0) + pm;
  T D = c.iga ? num * 0.25 : frac(num, ((p2 + p1) + p0) + pm);
  T out = ((3.0 * V * absv(V)) / Gb - (2.0 * V * V * V) / (Gb * Gb) - V) / 3.0 * D;
  int qs[2], nq = 0;
  for (int q = 0; q < g.nd; ++q) {
    if (q == d) continue;
    qs[nq++] = q;
    const Cell xp = sh(g, x, q, +1), xm = sh(g, x, q, -1);
    T a = get(P, lin(g, xp)), b = get(P, lin(g, sh(g, xp, d, +1)));
    T e = get(P, lin(g, xm)), f = get(P, lin(g, sh(g, xm, d, +1)));
    T n2 = (b - a) - (f - e);
    T D2 = c.iga ? n2 * 0.25 : frac(n2, (a + b) + (e + f));
    out = out + absv(V) * Vq[q] / Gb * (1.0 - 2.0 * absv(V) / Gb) * D2;
  }
  if (nq == 2) {
    auto pair = [&](long s1, long s2) {
      const Cell y = sh(g, sh(g, x, qs[0], s1), qs[1], s2);
      return get(P, lin(g, y)) + get(P, lin(g, sh(g, y, d, +1)));
    };
    T ppp = pair(+1, +1), ppm = pair(+1, -1), pmp = pair(-1, +1), pmm = pair(-1, -1);
    T n3 = (ppp - ppm) - (pmp - pmm);
    T D3 = c.iga ? n3 * 0.125 : frac(n3, (ppp + ppm) + (pmp + pmm));
    out = out - (2.0 / 3.0) * V * Vq[qs[0]] * Vq[qs[1]] / (Gb * Gb) * D3;
  }
  return out;
}

/* Antidiffusive pseudo-velocity of pass k at face i+1/2 along d (Sect. 3.1.1,
 * Eq. 6 in 1D; the multi-D cross terms are cited there to Smolarkiewicz &
 * Margolin 1998, Sect. 2.2):
 *   V^k = (|V| - V^2/Gb) A  -  sum_{q != d} 0.5 V Vq_bar / Gb * B_q   [+ tot]
 * V = V^{k-1} at this face, Gb = (G_i + G_{i+e_d})/2,
 * A   = frac(psi_{i+e_d} - psi_i, psi_{i+e_d} + psi_i),
 * Vq_bar = mean of V_q^{k-1} on the four q-faces touching cells i and i+e_d,
 * B_q = frac(T - Bt, T + Bt), T = psi_{i+e_q} + psi_{i+e_d+e_q}, Bt = psi_{i-e_q} + psi_{i+e_d-e_q}.
 * The cross term is the flux form of the -dt u v psi_xy part of the donor-cell
 * truncation error, split evenly between the two directions.
 * Infinite gauge (Sect. 3.1.5, limit of psi + c, c -> infinity, with the
 * pseudo-velocity rescaled by c): A = (psi_{i+e_d} - psi_i)/2, B_q = (T - Bt)/4. */
template <class T, class Get> T f_antidiff(const Ctx& c, int k, int d, long i, Get get) {
  const Grid& g = c.g;
  const int P = c.id.psi(k - 1);
  const Cell x = cell_of(g, i);
  const long ip = lin(g, sh(g, x, d, +1));
  const double Gb = 0.5 * (c.Gc(i) + c.Gc(ip));
  T V = get(c.adv(k - 1, d), fc(g, i, d, 0));
  /* variable-sign option (Sect. 3.1.5): psi enters every psi-fraction as |psi| */
  auto psi = [&](long j) { return c.abs ? absv(get(P, j)) : get(P, j); };
  T p0 = psi(i), p1 = psi(ip);
  T A = c.iga ? (p1 - p0) * 0.5 : frac(p1 - p0, p0 + p1);
  T out = (absv(V) - V * V / Gb) * A;
  T Vq[3];
  for (int q = 0; q < g.nd; ++q) {
    if (q == d) continue;
    const int Q = c.adv(k - 1, q);
    const Cell xp = sh(g, x, q, +1), xm = sh(g, x, q, -1);
    const long iqp = lin(g, xp), idqp = lin(g, sh(g, xp, d, +1));
    const long iqm = lin(g, xm), idqm = lin(g, sh(g, xm, d, +1));
    /* the q-faces q+1/2 and q-1/2 of cells i and i+e_d */
    Vq[q] = 0.25 * ((get(Q, fc(g, i, q, 0)) + get(Q, fc(g, ip, q, 0))) +
                    (get(Q, fc(g, i, q, -1)) + get(Q, fc(g, ip, q, -1))));
    T Tp = psi(iqp) + psi(idqp);
    T Bt = psi(iqm) + psi(idqm);
    T B = c.iga ? (Tp - Bt) * 0.25 : frac(Tp - Bt, Tp + Bt);
    out = out - 0.5 * V * Vq[q] / Gb * B;
  }
  if (c.tot) out = out + f_tot<T>(c, k, d, i, V, Vq, Gb, get);
  if (c.dfl) {
    /* Divergent-flow term (Sect. 3.1.3, cited there to Smolarkiewicz & Margolin 1998; the
     * formula is not reproduced in the paper).  Reading, from the donor-cell scheme's
     * first-order error -dt/2 G psi_tt, whose flux part -dt/2 (V/G) psi div(V) is not
     * cancelled by the terms above when the advector is divergent:
     *   - 1/4 V (div_i + div_{i+e_d}) / Gb,  div_j = sum_q (V_q at face j+1/2 - at face j-1/2),
     * with the advector of the previous pass (1D: -1/4 V_{i+1/2} (V_{i+3/2} - V_{i-1/2})). */
    auto div = [&](const Cell& y) {
      T s = 0.0;
      for (int q = 0; q < g.nd; ++q) {
        const int Q = c.adv(k - 1, q);
        s = s + (get(Q, fc(g, lin(g, y), q, 0)) - get(Q, fc(g, lin(g, y), q, -1)));
      }
      return s;
    };
    out = out - 0.25 * V * (div(x) + div(sh(g, x, d, +1))) / Gb;
  }
  return out;
}

/* FCT limiting factors of pass k at cell i (Sect. 3.1.4; Zalesak-type limiter of
 * Smolarkiewicz & Grabowski 1990).  With F the unlimited donor fluxes of the pass,
 *   in_i  = sum_d [F_{i-1/2}]+ - [F_{i+1/2}]-,   out_i = sum_d [F_{i+1/2}]+ - [F_{i-1/2}]-,
 *   beta_up_i = G_i [psi_max_i - psi_i]+ / in_i,   beta_dn_i = G_i [psi_i - psi_min_i]+ / out_i,
 * and beta = 1 where the denominator is zero. */
template <class T, class Get> T f_beta(const Ctx& c, int k, long i, bool up, Get get) {
  T in = 0.0, out = 0.0;
  for (int d = 0; d < c.g.nd; ++d) {
    T Fp = get(c.id.f(k, d), i);
    T Fm = f_flux_m<T>(c, k, d, i, false, get);
    in = in + (pos(Fm) - neg(Fp));
    out = out + (pos(Fp) - neg(Fm));
  }
  T p = get(c.id.psi(k - 1), i);
  const double Gi = c.Gc(i);
  if (up) {
    if (val(in) > 0) return Gi * pos(get(c.id.mx(), i) - p) / in;
    return T(1.0);
  }
  if (val(out) > 0) return Gi * pos(p - get(c.id.mn(), i)) / out;
  return T(1.0);
}

/* Limited advector at face i+1/2 along d: V * min(1, beta_dn_i, beta_up_{i+e_d})
 * when the unlimited flux leaves cell i (F > 0, or F = 0 with V > 0), else
 * V * min(1, beta_up_i, beta_dn_{i+e_d}). */
template <class T, class Get> T f_limit(const Ctx& c, int k, int d, long i, Get get) {
  const long ip = nbr(c.g, i, d, +1);
  T V = get(c.id.v(k, d), i);
  const double F = c.raw(c.id.f(k, d), i);
  const bool right = F > 0 || (F == 0 && val(V) > 0);
  T a = right ? get(c.id.bd(k), i) : get(c.id.bu(k), i);
  T b = right ? get(c.id.bu(k), ip) : get(c.id.bd(k), ip);
  T m = T(1.0);
  if (val(a) < val(m)) m = a;
  if (val(b) < val(m)) m = b;
  return V * m;
}

/* ------------------------------------------------------------ primitives */

enum Kind { PRE, FLUX, FLUXU, DONOR, BOUND_UP, BOUND_DN, ANTIDIFF, BETA_UP, BETA_DN, LIMIT, POST };
struct Prim { Kind kind; int out; int k; int d; };

template <class T, class Get> T eval(const Ctx& c, const Prim& p, long i, Get get) {
  switch (p.kind) {
    case PRE: return f_pre<T>(c, i, get);
    case FLUX: return f_flux<T>(c, p.k, p.d, i, true, get);
    case FLUXU: return f_flux<T>(c, p.k, p.d, i, false, get);
    case DONOR: return f_donor<T>(c, p.k, i, get);
    case BOUND_UP: return f_bound<T>(c, i, true, get);
    case BOUND_DN: return f_bound<T>(c, i, false, get);
    case ANTIDIFF: return f_antidiff<T>(c, p.k, p.d, i, get);
    case BETA_UP: return f_beta<T>(c, p.k, i, true, get);
    case BETA_DN: return f_beta<T>(c, p.k, i, false, get);
    case LIMIT: return f_limit<T>(c, p.k, p.d, i, get);
    case POST: return f_post<T>(c, i, get);
  }
  return T(0.0);
}

/* The sub-steps of one time step, in execution order. */
std::vector<Prim> program(const Ctx& c) {
  std::vector<Prim> P;
  const Ids& id = c.id;
  const int D = c.g.nd;
  P.push_back({PRE, id.psi(0), 0, 0});
  for (int d = 0; d < D; ++d) P.push_back({FLUX, id.fh(1, d), 1, d});
  P.push_back({DONOR, id.psi(1), 1, 0});
  if (c.fct && c.K >= 2) {
    P.push_back({BOUND_UP, id.mx(), 0, 0});
    P.push_back({BOUND_DN, id.mn(), 0, 0});
  }
  for (int k = 2; k <= c.K; ++k) {
    for (int d = 0; d < D; ++d) P.push_back({ANTIDIFF, id.v(k, d), k, d});
    if (c.fct) {
      for (int d = 0; d < D; ++d) P.push_back({FLUXU, id.f(k, d), k, d});
      P.push_back({BETA_UP, id.bu(k), k, 0});
      P.push_back({BETA_DN, id.bd(k), k, 0});
      for (int d = 0; d < D; ++d) P.push_back({LIMIT, id.vh(k, d), k, d});
    }
    for (int d = 0; d < D; ++d) P.push_back({FLUX, id.fh(k, d), k, d});
    P.push_back({DONOR, id.psi(k), k, 0});
  }
  P.push_back({POST, id.out(), 0, 0});
  return P;
}

/* Records which tape elements a local formula reads and seeds one dual slot each. */
struct Recorder {
  const std::vector<std::vector<double>>* A;
  int arr[NSLOT];
  long idx[NSLOT];
  int n = 0;
  Dual get(int a, long i) {
    int s = 0;
    while (s < n && !(arr[s] == a && idx[s] == i)) ++s;
    if (s == n) {
      if (n == NSLOT) { std::fprintf(stderr, "mpdata oracle: dual slots exhausted\n"); std::abort(); }
      arr[n] = a; idx[n] = i; ++n;
    }
    Dual r((*A)[a][i]);
    r.d[s] = 1.0;
    return r;
  }
};

/* ------------------------------------------------------------- step setup */

int setup(Ctx& c, int nd, const int64_t* shape, const double* const* gc, const double* g,
          const double* r, double dt, int n_iters, unsigned opts) {
  if (nd < 1 || nd > 3 || !shape || n_iters < 1) return 1;
  if ((opts & O_IGA) && n_iters != 2) return 1;
  if ((opts & O_IGA) && (opts & O_ABS)) return 1;  /* two alternative variable-sign options */
  if ((opts & O_IGA) && (opts & O_DFL)) return 1;  /* the divergent-flow flux scales with psi */
  if ((opts & O_RHS_A) && (opts & O_RHS_B)) return 1;
  if (((opts & (O_RHS_A | O_RHS_B)) != 0) != (r != nullptr)) return 1;
  if (((opts & O_NUG) != 0) != (g != nullptr)) return 1;
  c.g.nd = nd;
  long N = 1;
  if (opts & ~((O_OPEN0 << nd) - 1u) & ~1023u) return 1;  /* open bits of absent dimensions */
  for (int d = 0; d < nd; ++d) {
    if (shape[d] < 1) return 1;
    c.g.n[c.g.ax(d)] = shape[d];
    c.g.open[c.g.ax(d)] = (opts & (O_OPEN0 << d)) != 0;
    if (c.g.open[c.g.ax(d)] && shape[d] < 2) return 1;  /* an open dimension needs an interior face */
    N *= shape[d];
  }
  c.g.N = N;
  for (int d = 0; d < nd; ++d) if (!gc[d]) return 1;
  c.K = n_iters;
  c.id.K = n_iters;
  c.fct = opts & O_FCT;
  c.tot = opts & O_TOT;
  c.iga = opts & O_IGA;
  c.abs = opts & O_ABS;
  c.dfl = opts & O_DFL;
  c.kahan = opts & O_KAHAN;
  c.rhs_a = opts & O_RHS_A;
  c.rhs_b = opts & O_RHS_B;
  c.G = (opts & O_NUG) ? g : nullptr;
  c.R = r;
  c.dt = dt;
  return 0;
}

/* Runs the forward step on the tape; arrays of finished passes are released
 * unless keep is set (the derivative sweeps need all of them). */
void forward(Ctx& c, std::vector<std::vector<double>>& A, const double* psi, const double* const* gc, bool keep) {
  const long N = c.g.N;
  A.assign(c.id.count(), {});
  c.A = &A;
  A[c.id.in()].assign(psi, psi + N);
  for (int d = 0; d < c.g.nd; ++d) A[c.id.v(1, d)].assign(gc[d], gc[d] + N);
  auto rawget = [&](int a, long i) -> double { return A[a][i]; };
  for (const Prim& p : program(c)) {
    std::vector<double>& o = A[p.out];
    o.assign(N, 0.0);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) o[i] = eval<double>(c, p, i, rawget);
    if (!keep && p.kind == DONOR) {
      /* pass p.k is done: everything it read except the bounds and the advector the next pass needs */
      const int k = p.k;
      for (int d = 0; d < c.g.nd; ++d) {
        A[c.id.fh(k, d)] = {};
        A[c.id.f(k, d)] = {};
        if (k >= 2) A[c.adv(k - 1, d)] = {};
      }
      if (k >= 2) { A[c.id.psi(k - 1)] = {}; A[c.id.bu(k)] = {}; A[c.id.bd(k)] = {}; }
      if (k >= 2 && c.fct) for (int d = 0; d < c.g.nd; ++d) A[c.id.v(k, d)] = {};
    }
  }
}

}  // namespace

/* ================================================================ C ABI */
extern "C" {

/* Advances psi (in place) by n_steps MPDATA steps.  gc0..gc2: advector
 * components (unused ones NULL); g: G field (NULL unless the NUG bit is set);
 * r: source term (NULL unless an RHS bit is set).  If mx/mn are non-NULL they
 * receive the FCT bounds of the last step.  Returns 0, or 1 on invalid input. */
int mpo_step_ex(int nd, const int64_t* shape, double* psi, const double* gc0, const double* gc1,
                const double* gc2, const double* g, const double* r, double dt, int n_iters,
                unsigned opts, int64_t n_steps, double* mx, double* mn) {
  const double* gc[3] = {gc0, gc1, gc2};
  Ctx c;
  if (setup(c, nd, shape, gc, g, r, dt, n_iters, opts) != 0 || n_steps < 0) return 1;
  std::vector<std::vector<double>> A;
  for (int64_t s = 0; s < n_steps; ++s) {
    const bool last = s + 1 == n_steps;
    forward(c, A, psi, gc, false);
    std::memcpy(psi, A[c.id.out()].data(), sizeof(double) * c.g.N);
    if (last && mx && !A[c.id.mx()].empty()) std::memcpy(mx, A[c.id.mx()].data(), sizeof(double) * c.g.N);
    if (last && mn && !A[c.id.mn()].empty()) std::memcpy(mn, A[c.id.mn()].data(), sizeof(double) * c.g.N);
  }
  return 0;
}

int mpo_step(int nd, const int64_t* shape, double* psi, const double* gc0, const double* gc1,
             const double* gc2, const double* g, const double* r, double dt, int n_iters,
             unsigned opts, int64_t n_steps) {
  return mpo_step_ex(nd, shape, psi, gc0, gc1, gc2, g, r, dt, n_iters, opts, n_steps, nullptr, nullptr);
}

/* Tangent-linear of one step at state psi: dpsi_out = d psi^{n+1} [dpsi, dgc]. */
int mpo_tl_step(int nd, const int64_t* shape, const double* psi, const double* gc0, const double* gc1,
                const double* gc2, const double* g, const double* r, double dt, int n_iters,
                unsigned opts, const double* dpsi, const double* dgc0, const double* dgc1,
                const double* dgc2, double* dpsi_out) {
  const double* gc[3] = {gc0, gc1, gc2};
  const double* dgc[3] = {dgc0, dgc1, dgc2};
  Ctx c;
  if (setup(c, nd, shape, gc, g, r, dt, n_iters, opts) != 0) return 1;
  std::vector<std::vector<double>> A;
  forward(c, A, psi, gc, true);
  const long N = c.g.N;
  std::vector<std::vector<double>> Tn(A.size());
  Tn[c.id.in()].assign(dpsi, dpsi + N);
  for (int d = 0; d < nd; ++d) {
    if (dgc[d]) Tn[c.id.v(1, d)].assign(dgc[d], dgc[d] + N);
    else Tn[c.id.v(1, d)].assign(N, 0.0);
  }
  for (const Prim& p : program(c)) {
    std::vector<double>& o = Tn[p.out];
    o.assign(N, 0.0);
    for (long i = 0; i < N; ++i) {
      Recorder rec{&A};
      Dual y = eval<Dual>(c, p, i, [&](int a, long j) { return rec.get(a, j); });
      double t = 0.0;
      for (int s = 0; s < rec.n; ++s) t += y.d[s] * Tn[rec.arr[s]][rec.idx[s]];
      o[i] = t;
    }
  }
  std::memcpy(dpsi_out, Tn[c.id.out()].data(), sizeof(double) * N);
  return 0;
}

/* Adjoint of one step at state psi: on entry psi_bar = dL/dpsi^{n+1}, on exit
 * dL/dpsi^n; gc_bar_d (nullable) are incremented by dL/dgc_d. */
int mpo_adj_step(int nd, const int64_t* shape, const double* psi, const double* gc0, const double* gc1,
                 const double* gc2, const double* g, const double* r, double dt, int n_iters,
                 unsigned opts, double* psi_bar, double* gcb0, double* gcb1, double* gcb2) {
  const double* gc[3] = {gc0, gc1, gc2};
  double* gcb[3] = {gcb0, gcb1, gcb2};
  Ctx c;
  if (setup(c, nd, shape, gc, g, r, dt, n_iters, opts) != 0) return 1;
  std::vector<std::vector<double>> A;
  forward(c, A, psi, gc, true);
  const long N = c.g.N;
  std::vector<std::vector<double>> B(A.size());
  for (size_t a = 0; a < A.size(); ++a) if (!A[a].empty()) B[a].assign(N, 0.0);
  B[c.id.out()].assign(psi_bar, psi_bar + N);
  std::vector<Prim> prog = program(c);
  for (auto it = prog.rbegin(); it != prog.rend(); ++it) {
    const Prim& p = *it;
    for (long i = 0; i < N; ++i) {
      const double ob = B[p.out][i];
      if (ob == 0.0) continue;
      Recorder rec{&A};
      Dual y = eval<Dual>(c, p, i, [&](int a, long j) { return rec.get(a, j); });
      for (int s = 0; s < rec.n; ++s) B[rec.arr[s]][rec.idx[s]] += y.d[s] * ob;
    }
  }
  std::memcpy(psi_bar, B[c.id.in()].data(), sizeof(double) * N);
  for (int d = 0; d < nd; ++d)
    if (gcb[d]) for (long i = 0; i < N; ++i) gcb[d][i] += B[c.id.v(1, d)][i];
  return 0;
}

/* Total mass sum_i G_i psi_i (G = 1 when g is NULL), plain sequential FP64 sum. */
double mpo_mass(int nd, const int64_t* shape, const double* psi, const double* g) {
  long N = 1;
  for (int d = 0; d < nd; ++d) N *= shape[d];
  double s = 0.0;
  for (long i = 0; i < N; ++i) s += (g ? g[i] : 1.0) * psi[i];
  return s;
}

int mpo_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // extern "C"
