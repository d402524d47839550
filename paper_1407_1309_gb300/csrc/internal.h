// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/mpdata.h"

namespace mpd {

constexpr uint32_t kOpenBits = MPDATA_OPEN0 | MPDATA_OPEN1 | MPDATA_OPEN2;

// A value computed once per device (a kernel's opt-in shared-memory attribute, a persistent
// grid size): get() returns the value cached for the current device, computing it with
// init(device) under a lock on the first call there, so threads that launch on several
// devices each see their own device's set-up, and none launches before it is complete.
// Devices past the 64th are not cached (init runs on every call, under the lock).
template <typename V>
class PerDevice {
 public:
  template <class F>
  V get(F&& init) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    const bool cached = dev >= 0 && dev < 64;
    const uint64_t bit = cached ? (uint64_t{1} << dev) : 0;
    if (cached && (ready_.load(std::memory_order_acquire) & bit)) return val_[dev];
    std::lock_guard<std::mutex> lock(mu_);
    if (!cached) return init(dev);
    if (!(ready_.load(std::memory_order_relaxed) & bit)) {
      val_[dev] = init(dev);
      ready_.fetch_or(bit, std::memory_order_release);
    }
    return val_[dev];
  }

 private:
  std::mutex mu_;
  std::atomic<uint64_t> ready_{0};
  V val_[64] = {};
};

// Grid of one field on three internal axes: dimension d of an nd-dimensional
// field lives on axis 3 - nd + d; unused leading axes have extent 1.
struct Grid {
  int nd;
  int n[3];
  long long N;
  // open edges (MPDATA_OPEN0 << d) on each internal axis; periodic where false
  bool open[3];
  bool any_open() const { return open[0] || open[1] || open[2]; }
};

inline Grid make_grid(int nd, const int64_t* shape, uint32_t opts = 0) {
  Grid g;
  g.nd = nd;
  g.n[0] = g.n[1] = g.n[2] = 1;
  g.open[0] = g.open[1] = g.open[2] = false;
  g.N = 1;
  for (int d = 0; d < nd; ++d) {
    g.n[3 - nd + d] = static_cast<int>(shape[d]);
    g.open[3 - nd + d] = (opts & (MPDATA_OPEN0 << d)) != 0;
    g.N *= shape[d];
  }
  return g;
}

// Option bits a handle accepts for nd dimensions; checks shared by mpdata_create and
// mpdata_step_noalloc.
inline bool valid_open_bits(int nd, uint32_t opts, const int64_t* shape) {
  // bits 0 .. 9, the open bits of the nd dimensions, the trapezoidal source scheme and the
  // shallow-water system
  const uint32_t all = ((MPDATA_OPEN0 << nd) - 1u) | MPDATA_RHS_TRAPEZ | MPDATA_SW;
  if (opts & ~all) return false;
  for (int d = 0; d < nd; ++d)
    if ((opts & (MPDATA_OPEN0 << d)) && shape[d] < 2) return false;
  return true;
}

// Run-time options of one step.
struct Opts {
  bool fct, tot, iga, nug, kahan, rhs_a, rhs_b, staged;
  bool abs;  // |psi| in the psi-fractions of the pseudo-velocity (variable-sign fields)
  bool dfl;  // divergent-flow term of the pseudo-velocity
  bool open; // open edges along some dimension (staged kernels only)
  int n_iters;
  int tile_rows;  // fused 2D kernels: rows per warp tile / per block band (0 = automatic)
  int kernel;     // fused 2D kernel family: 0 automatic, 1 warp march, 2 band march
};

inline Opts make_opts(uint32_t o, int n_iters) {
  Opts p;
  p.fct = o & MPDATA_FCT;
  p.tot = o & MPDATA_TOT;
  p.iga = o & MPDATA_IGA;
  p.nug = o & MPDATA_NUG;
  p.kahan = o & MPDATA_KAHAN;
  p.rhs_a = o & MPDATA_RHS_EULER_A;
  p.rhs_b = o & MPDATA_RHS_EULER_B;
  p.staged = o & MPDATA_STAGED;
  p.abs = o & MPDATA_ABS;
  p.dfl = o & MPDATA_DFL;
  p.open = (o & kOpenBits) != 0;
  p.n_iters = n_iters;
  p.tile_rows = 0;
  p.kernel = 0;
  return p;
}

// Pointers of one field for one step.
template <typename T>
struct StepArgs {
  const T* psi_in;
  T* psi_out;
  const T* gc[3];
  const T* g;    // NULL unless nug
  const T* r;    // NULL unless an rhs bit
  T dt;
  T gc_scale;    // advector multiplier of this step
};

// Scratch of the staged path: 16 arrays of n_max elements.
template <typename T>
struct StagedScratch {
  T* p0;          // psi^(0) when euler_b
  T* pa;          // psi^(k) ping
  T* pb;          // psi^(k) pong
  T* va[3];       // advector ping
  T* vb[3];       // advector pong
  T* vu[3];       // unlimited antidiffusive advector (FCT)
  T* mx;
  T* mn;
  T* bu;
  T* bd;
};
constexpr int kStagedArrays = 16;

template <typename T>
StagedScratch<T> carve_staged(void* base, long long n_max);

// One step of one field with one kernel per sub-step; returns a cudaError_t.
template <typename T>
cudaError_t staged_step(const Grid& g, const Opts& o, const StepArgs<T>& a,
                        const StagedScratch<T>& s, cudaStream_t st);

// Every step of a call for a 1D field in one launch of one block, when the field and its
// intermediates fit in shared memory (13 arrays of n); MPDATA_EUNSUPPORTED otherwise.
template <typename T>
int steps1d(const Grid& g, const Opts& o, const T* psi_in, T* psi_out, const T* gc, const T* G, const T* R, T dt,
            int n_steps, cudaStream_t st);

// Intermediates of one forward step kept for the adjoint (n_iters <= kTapeMax).
constexpr int kTapeMax = 4;
template <typename T>
struct Tape {
  const T* psi[kTapeMax];          // psi^(k), k = 0..K-1 (psi[0] is the step input)
  T* v[kTapeMax + 1][3];           // unlimited antidiffusive advector of pass k >= 2
  const T* vh[kTapeMax + 1][3];    // advector that drives pass k (gc for k = 1; limited under FCT)
  T* mx;
  T* mn;
  T* bu[kTapeMax + 1];
  T* bd[kTapeMax + 1];
};

// Forward step on the staged kernels keeping every pass's intermediates (no sources).
// Writes psi^(1..K-1), the pseudo-advectors, the FCT bounds and factors into the tape, and
// the step's result psi^(K) into psi_next unless it is null.
template <typename T>
cudaError_t staged_forward_tape(const Grid& g, const Opts& o, const T* const* gc, const T* G,
                                const Tape<T>& tp, T* const* psi_out_levels, T* psi_next, cudaStream_t st);

// Trapezoidal source scheme (rhs.cu) for a system of E <= kTrapezMax equations of n cells each,
// stored field after field: pre writes psi + dt/2 (A psi + b) into out; post turns the advected
// fields into psi^{n+1} = Minv (psi* + dt/2 b) in place, Minv = (I - dt/2 A)^{-1}.
constexpr int kTrapezMax = 8;
struct TrapezMat {
  int E;
  double A[kTrapezMax * kTrapezMax];
  double Minv[kTrapezMax * kTrapezMax];
};
// Minv of I - dt/2 A by Gauss-Jordan elimination with partial pivoting; false if singular.
bool trapez_matrix(TrapezMat& m, const double* A, int E, double dt);
template <typename T>
cudaError_t trapez_pre(const TrapezMat& m, long long n, T dt, const T* psi, const T* b, T* out, cudaStream_t st);
template <typename T>
cudaError_t trapez_post(const TrapezMat& m, long long n, T dt, const T* b, T* psi, cudaStream_t st);

// Vectorised FP32 pseudo-advector z-march for 3D fields (march3.cu): launched, and true
// returned, when the x extent is a multiple of 4 and at least 128, no edge is open and every
// array is 16-byte aligned; false (nothing launched) otherwise.
bool antidiff3_vec(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, bool iga,
                   bool tot, bool abs_psi, float* const* out, cudaStream_t st);

// Vectorised FP32 pass-1-and-bounds z-march (march3.cu), same conditions.
bool p1b3_vec(const Grid& g, const float* psi, const float* const* v, float vscale, const float* G, bool kahan,
              float* p1, float* mx, float* mn, cudaStream_t st);

// Vectorised FP32 FCT corrective pass (march3.cu): factors, limiter and donor pass as one z-march,
// same conditions, and neither the Kahan summation nor a source term (post); lim[0] null when the
// limited advector is not wanted.
bool corr3_vec(const Grid& g, const float* psi, const float* const* vu, const float* G, bool iga, bool kahan,
               const float* mx, const float* mn, bool post, float* const* lim, float* out, cudaStream_t st);

// Prognosed velocity and shallow-water sources (vip.cu).  state: h then the momenta q_d, n cells
// each.  vip_advector: the advector of the step (adv, nd arrays) from the velocities q/h (h > eps)
// extrapolated to n + 1/2 (ext: nd scratch arrays; uprev: u^{n-1} in, u^n out, ignored when
// first) and interpolated to the walls, times courant = dt/dx.  sw_force: q_d += half_dt R_d,
// R_d = -h dh/dx_d by centred differences.
template <typename T>
cudaError_t vip_advector(const Grid& g, const T* state, T* uprev, T* ext, T* adv, bool first, T eps, T courant,
                         cudaStream_t st);
template <typename T>
cudaError_t sw_force(const Grid& g, T* state, T half_dt, T dx, cudaStream_t st);

// FP64 reductions (reduce.cu).  partial: device scratch of at least
// kRedBlocks * n_fields doubles per output.
constexpr int kRedBlocks = 256;
struct FieldSpan {
  long long offset;
  long long n;
};
template <typename T>
cudaError_t reduce_mass(const T* psi, const T* g, const FieldSpan* d_spans, int n_fields,
                        double* d_partial, double* d_out, cudaStream_t st);
template <typename T>
cudaError_t reduce_diff(const T* a, const T* b, const FieldSpan* d_spans, int n_fields,
                        double* d_partial, double* d_out, cudaStream_t st);
template <typename T>
cudaError_t reduce_courant(const Grid* grids, const long long* offsets, int n_fields, const T* const* gc,
                           const T* g, double* d_partial, double* d_out, cudaStream_t st);

}  // namespace mpd
