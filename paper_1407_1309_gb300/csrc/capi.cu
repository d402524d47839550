// C ABI of the library (include/mpdata.h): handle management, argument
// validation, dispatch to the fused / batched / staged kernels, reductions.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "kernels.h"

struct mpdata_s {
  int nd = 0, n_fields = 0, dtype = 0, n_iters = 0;
  uint32_t opts = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<mpd::Grid> grids;
  std::vector<long long> offsets;
  long long total = 0, n_max = 0;
  size_t esize = 4;
  void* staged = nullptr;            // staged-path scratch
  void* pingpong = nullptr;          // out-of-place buffer for the fused paths (total elements)
  void* pingpong_lo = nullptr;       // its low-part twin for the compensated state (on first use)
  void* adj = nullptr;               // adjoint scratch
  mpd::FieldSpan* d_spans = nullptr;
  double* d_partial = nullptr;       // 2 * kRedBlocks * n_fields
  double* d_out = nullptr;           // 2 * n_fields
  double* h_out = nullptr;           // pinned, 2 * n_fields
  int* d_status = nullptr;           // device-side error word (bounded waits)
  void* batch = nullptr;             // batched-kernel tables
  int tile_rows = 0;                 // MPDATA_TUNE_TILE_ROWS
  int kernel = 0;                    // MPDATA_TUNE_KERNEL
  int steps_per_launch = 0;          // MPDATA_TUNE_STEPS_PER_LAUNCH
  std::atomic<int> stop{0};
  // trapezoidal source scheme: R = A psi + b over the fields (mpdata_set_rhs_linear)
  bool rhs_lin = false;
  std::vector<double> rhs_A;
  const void* rhs_b = nullptr;
  void* trapez_buf = nullptr;        // psi^n + dt/2 R^n (total elements, on first use)
  // shallow-water system: u^{n-1}, extrapolated velocities, advector (3 x nd arrays, first use)
  void* sw_buf = nullptr;
  bool sw_first = true;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T>
int run_advance(mpdata_s* h, const T* psi_in, T* psi_out, const void* const* gcv, const T* g, const T* r,
                double dt, int n_steps, const double* gc_scale, bool inner = false);

// The trapezoidal source scheme (Sect. 4.1): per step the sources' first half is added (all
// equations at once, R^n = A psi^n + b), the fields are advected by one ordinary step (any
// kernel family), and the implicit second half is solved per cell.
template <typename T>
int run_trapez(mpdata_s* h, const T* psi_in, T* psi_out, const void* const* gcv, const T* g, double dt,
               int n_steps, const double* gc_scale) {
  if (!h->rhs_lin) return MPDATA_EINVAL;
  mpd::TrapezMat m;
  if (!mpd::trapez_matrix(m, h->rhs_A.data(), h->n_fields, dt)) return MPDATA_EINVAL;
  if (!h->trapez_buf && cudaMalloc(&h->trapez_buf, static_cast<size_t>(h->total) * sizeof(T)) != cudaSuccess) {
    h->trapez_buf = nullptr;
    return MPDATA_ENOMEM;
  }
  const long long n = h->grids[0].N;
  T* S = static_cast<T*>(h->trapez_buf);
  const T* b = static_cast<const T*>(h->rhs_b);
  for (int s = 0; s < n_steps; ++s) {
    if (h->stop.load(std::memory_order_relaxed)) return MPDATA_ESTOPPED;
    if (mpd::trapez_pre<T>(m, n, static_cast<T>(dt), s == 0 ? psi_in : psi_out, b, S, h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    const int rc = run_advance<T>(h, S, psi_out, gcv, g, nullptr, dt, 1, gc_scale ? gc_scale + s : nullptr, true);
    if (rc != MPDATA_OK) return rc;
    if (mpd::trapez_post<T>(m, n, static_cast<T>(dt), b, psi_out, h->stream) != cudaSuccess) return MPDATA_ECUDA;
  }
  return MPDATA_OK;
}

template <typename T>
int run_advance(mpdata_s* h, const T* psi_in, T* psi_out, const void* const* gcv, const T* g, const T* r,
                double dt, int n_steps, const double* gc_scale, bool inner) {
  if (!inner && (h->opts & MPDATA_RHS_TRAPEZ)) return run_trapez<T>(h, psi_in, psi_out, gcv, g, dt, n_steps, gc_scale);
  mpd::Opts o = mpd::make_opts(h->opts, h->n_iters);
  o.tile_rows = h->tile_rows;
  o.kernel = h->kernel;
  const T* gc[3] = {static_cast<const T*>(gcv[0]), h->nd > 1 ? static_cast<const T*>(gcv[1]) : nullptr,
                    h->nd > 2 ? static_cast<const T*>(gcv[2]) : nullptr};
  const mpd::StagedScratch<T> ss = mpd::carve_staged<T>(h->staged, h->n_max);
  // Every step reads one buffer and writes another: the result alternates between
  // psi_out and the handle's ping-pong buffer so that the last step lands in psi_out.
  // In place with an odd step count, psi is first copied to the ping-pong buffer.
  // a small 1D field runs every step of the call in one launch of one block (it reads the
  // whole field before writing, so in place needs no copy)
  if (h->nd == 1 && h->n_fields == 1 && !o.staged && !gc_scale) {
    const int rc = mpd::steps1d<T>(h->grids[0], o, psi_in, psi_out, gc[0], g, r, static_cast<T>(dt), n_steps,
                                   h->stream);
    if (rc != MPDATA_EUNSUPPORTED) return rc;
  }
  T* X = psi_out;
  T* P = static_cast<T*>(h->pingpong);
  const T* cur = psi_in;
  // temporal blocking: groups of up to steps_per_launch steps, one launch each, the results
  // alternating between psi_out and the ping-pong buffer as for single steps
  const int depth = h->steps_per_launch;
  if (depth > 1 && h->n_fields == 1 && !o.staged && n_steps > 1 && mpd::tblock_covers<T>(h->grids[0], o, depth)) {
    const int n_groups = (n_steps + depth - 1) / depth;
    if (psi_in == psi_out && n_groups % 2 == 1) {
      if (cudaMemcpyAsync(P, X, sizeof(T) * h->total, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return MPDATA_ECUDA;
      cur = P;
    }
    for (int k = 0, s = 0; k < n_groups; ++k, s += depth) {
      if (h->stop.load(std::memory_order_relaxed)) return MPDATA_ESTOPPED;
      const int d = n_steps - s < depth ? n_steps - s : depth;
      T* dst = ((n_groups - 1 - k) % 2 == 0) ? X : P;
      const int rc = mpd::tblock_steps<T>(h->grids[0], o, cur, dst, gc[0], gc[1], d, gc_scale ? gc_scale + s : nullptr,
                                          h->stream);
      if (rc != MPDATA_OK) return rc;
      cur = dst;
    }
    return cuda_status(cudaGetLastError());
  }
  if (psi_in == psi_out && n_steps % 2 == 1) {
    if (cudaMemcpyAsync(P, X, sizeof(T) * h->total, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    cur = P;
  }
  for (int s = 0; s < n_steps; ++s) {
    if (h->stop.load(std::memory_order_relaxed)) return MPDATA_ESTOPPED;
    const T scale = gc_scale ? static_cast<T>(gc_scale[s]) : T(1);
    T* dst = ((n_steps - 1 - s) % 2 == 0) ? X : P;
    if (h->n_fields > 1 && !o.staged) {
      int rc = mpd::batched_step<T>(h, cur, dst, gc, g, r, static_cast<T>(dt), scale, o);
      if (rc != MPDATA_EUNSUPPORTED) {
        if (rc != MPDATA_OK) return rc;
        cur = dst;
        continue;
      }
    }
    for (int f = 0; f < h->n_fields; ++f) {
      const long long off = h->offsets[f];
      const mpd::Grid& gr = h->grids[f];
      mpd::StepArgs<T> a;
      a.psi_in = cur + off;
      a.psi_out = dst + off;
      for (int d = 0; d < 3; ++d) a.gc[d] = (d < h->nd) ? gc[d] + off : nullptr;
      a.g = g ? g + off : nullptr;
      a.r = r ? r + off : nullptr;
      a.dt = static_cast<T>(dt);
      a.gc_scale = scale;
      int rc = o.staged ? MPDATA_EUNSUPPORTED : mpd::fused_step<T>(gr, o, a, nullptr, h->stream);
      if (rc == MPDATA_EUNSUPPORTED) rc = cuda_status(mpd::staged_step<T>(gr, o, a, ss, h->stream));
      if (rc != MPDATA_OK) return rc;
    }
    cur = dst;
  }
  return cuda_status(cudaGetLastError());
}

int validate_fields(mpdata_s* h, const void* psi, const void* const* gc, const void* g, const void* r) {
  if (!psi || !gc) return MPDATA_EINVAL;
  if (!aligned(psi, h->esize)) return MPDATA_EINVAL;
  for (int d = 0; d < h->nd; ++d)
    if (!gc[d] || !aligned(gc[d], h->esize)) return MPDATA_EINVAL;
  const bool nug = h->opts & MPDATA_NUG;
  if (nug != (g != nullptr)) return MPDATA_EINVAL;
  if (g && !aligned(g, h->esize)) return MPDATA_EINVAL;
  const bool rhs = h->opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B);
  if (rhs != (r != nullptr)) return MPDATA_EINVAL;
  if (r && !aligned(r, h->esize)) return MPDATA_EINVAL;
  if ((h->opts & MPDATA_RHS_TRAPEZ) && !h->rhs_lin) return MPDATA_EINVAL;
  return MPDATA_OK;
}

int sync_status(mpdata_s* h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  int st = 0;
  e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  if (st != 0) {
    cudaMemset(h->d_status, 0, sizeof(int));
    return st;
  }
  return MPDATA_OK;
}

void free_all(mpdata_s* h) {
  cudaFree(h->staged);
  cudaFree(h->pingpong);
  cudaFree(h->pingpong_lo);
  cudaFree(h->trapez_buf);
  cudaFree(h->sw_buf);
  mpd::adjoint_free(h);
  cudaFree(h->d_spans);
  cudaFree(h->d_partial);
  cudaFree(h->d_out);
  cudaFree(h->d_status);
  cudaFreeHost(h->h_out);
  mpd::batched_free(h);
}

}  // namespace

namespace mpd {
int handle_nd(const mpdata_s* h) { return h->nd; }
int handle_fields(const mpdata_s* h) { return h->n_fields; }
const Grid* handle_grids(const mpdata_s* h) { return h->grids.data(); }
const long long* handle_offsets(const mpdata_s* h) { return h->offsets.data(); }
long long handle_total(const mpdata_s* h) { return h->total; }
cudaStream_t handle_stream(const mpdata_s* h) { return h->stream; }
int* handle_status(const mpdata_s* h) { return h->d_status; }
void** handle_batch(mpdata_s* h) { return &h->batch; }
void** handle_adj(mpdata_s* h) { return &h->adj; }
int handle_n_iters(const mpdata_s* h) { return h->n_iters; }
uint32_t handle_opts(const mpdata_s* h) { return h->opts; }
void handle_tuning(const mpdata_s* h, int* kernel, int* tile_rows) {
  *kernel = h->kernel;
  *tile_rows = h->tile_rows;  // as mpdata_advance passes them
}
}  // namespace mpd

namespace {

// The shallow-water system (Sect. 5): per step the prognosed advector, the first half of the
// momentum sources, one MPDATA step of every field with that advector (any kernel family), the
// second half with the new depth.  The result alternates between the state and the handle's
// ping-pong buffer so that the last step lands in the state.
template <typename T>
int run_sw(mpdata_s* h, T* state, double dt, double dx, double eps, int n_steps) {
  const mpd::Grid& gr = h->grids[0];
  const long long n = gr.N;
  const int nd = h->nd;
  if (!h->sw_buf && cudaMalloc(&h->sw_buf, static_cast<size_t>(3 * nd) * n * sizeof(T)) != cudaSuccess) {
    h->sw_buf = nullptr;
    return MPDATA_ENOMEM;
  }
  T* uprev = static_cast<T*>(h->sw_buf);
  T* ext = uprev + static_cast<long long>(nd) * n;
  T* adv = ext + static_cast<long long>(nd) * n;
  mpd::Opts o = mpd::make_opts(h->opts, h->n_iters);
  o.tile_rows = h->tile_rows;
  o.kernel = h->kernel;
  const mpd::StagedScratch<T> ss = mpd::carve_staged<T>(h->staged, h->n_max);
  T* X = state;
  T* P = static_cast<T*>(h->pingpong);
  T* cur = X;
  if (n_steps % 2 == 1) {
    if (cudaMemcpyAsync(P, X, sizeof(T) * h->total, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    cur = P;
  }
  for (int s = 0; s < n_steps; ++s) {
    if (h->stop.load(std::memory_order_relaxed)) return MPDATA_ESTOPPED;
    T* dst = ((n_steps - 1 - s) % 2 == 0) ? X : P;
    if (mpd::vip_advector<T>(gr, cur, uprev, ext, adv, h->sw_first, static_cast<T>(eps), static_cast<T>(dt / dx),
                             h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    h->sw_first = false;
    if (mpd::sw_force<T>(gr, cur, static_cast<T>(0.5 * dt), static_cast<T>(dx), h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    for (int f = 0; f <= nd; ++f) {
      mpd::StepArgs<T> a;
      a.psi_in = cur + static_cast<long long>(f) * n;
      a.psi_out = dst + static_cast<long long>(f) * n;
      for (int d = 0; d < 3; ++d) a.gc[d] = d < nd ? adv + static_cast<long long>(d) * n : nullptr;
      a.g = nullptr;
      a.r = nullptr;
      a.dt = static_cast<T>(dt);
      a.gc_scale = T(1);
      int rc = o.staged ? MPDATA_EUNSUPPORTED : mpd::fused_step<T>(gr, o, a, nullptr, h->stream);
      if (rc == MPDATA_EUNSUPPORTED) rc = cuda_status(mpd::staged_step<T>(gr, o, a, ss, h->stream));
      if (rc != MPDATA_OK) return rc;
    }
    if (mpd::sw_force<T>(gr, dst, static_cast<T>(0.5 * dt), static_cast<T>(dx), h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    cur = dst;
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

int mpdata_create(mpdata_t* out, int ndims, int n_fields, const int64_t* shapes, int dtype, int n_iters,
                  uint32_t opts, void* cuda_stream) {
  if (!out || !shapes) return MPDATA_EINVAL;
  *out = nullptr;
  if (ndims < 1 || ndims > 3 || n_fields < 1 || n_iters < 1) return MPDATA_EINVAL;
  if (dtype != MPDATA_F32 && dtype != MPDATA_F64) return MPDATA_EINVAL;
  if ((opts & MPDATA_IGA) && n_iters != 2) return MPDATA_EINVAL;
  if ((opts & MPDATA_IGA) && (opts & (MPDATA_ABS | MPDATA_DFL))) return MPDATA_EINVAL;
  if ((opts & MPDATA_RHS_EULER_A) && (opts & MPDATA_RHS_EULER_B)) return MPDATA_EINVAL;
  if ((opts & MPDATA_RHS_TRAPEZ) && (opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B))) return MPDATA_EINVAL;
  if (opts & MPDATA_SW) {  // h and one momentum per dimension, of one shape, G = 1, no other sources
    if (n_fields != ndims + 1 ||
        (opts & (MPDATA_NUG | MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B | MPDATA_RHS_TRAPEZ)))
      return MPDATA_EINVAL;
    for (int f = 1; f < n_fields; ++f)
      for (int d = 0; d < ndims; ++d)
        if (shapes[static_cast<long long>(f) * ndims + d] != shapes[d]) return MPDATA_EINVAL;
  }
  for (long long i = 0; i < static_cast<long long>(n_fields) * ndims; ++i)
    if (shapes[i] < 1 || shapes[i] > (int64_t(1) << 30)) return MPDATA_EINVAL;
  for (int f = 0; f < n_fields; ++f)
    if (!mpd::valid_open_bits(ndims, opts, shapes + static_cast<long long>(f) * ndims)) return MPDATA_EINVAL;
  mpdata_s* h = new (std::nothrow) mpdata_s;
  if (!h) return MPDATA_ENOMEM;
  h->nd = ndims;
  h->n_fields = n_fields;
  h->dtype = dtype;
  h->n_iters = n_iters;
  h->opts = opts;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->esize = dtype == MPDATA_F32 ? 4 : 8;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return MPDATA_ECUDA; }
  std::vector<mpd::FieldSpan> spans(n_fields);
  for (int f = 0; f < n_fields; ++f) {
    mpd::Grid g = mpd::make_grid(ndims, shapes + static_cast<long long>(f) * ndims, opts);
    h->grids.push_back(g);
    h->offsets.push_back(h->total);
    spans[f] = {h->total, g.N};
    h->total += g.N;
    if (g.N > h->n_max) h->n_max = g.N;
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chk(cudaMalloc(&h->staged, static_cast<size_t>(mpd::kStagedArrays) * h->n_max * h->esize));
  chk(cudaMalloc(&h->pingpong, static_cast<size_t>(h->total) * h->esize));
  chk(cudaMalloc(&h->d_spans, sizeof(mpd::FieldSpan) * n_fields));
  chk(cudaMalloc(&h->d_partial, sizeof(double) * 2 * mpd::kRedBlocks * n_fields));
  chk(cudaMalloc(&h->d_out, sizeof(double) * 2 * n_fields));
  chk(cudaMalloc(&h->d_status, sizeof(int)));
  chk(cudaMallocHost(&h->h_out, sizeof(double) * 2 * n_fields));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_spans, spans.data(), sizeof(mpd::FieldSpan) * n_fields, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? MPDATA_ENOMEM : MPDATA_ECUDA;
  }
  *out = h;
  return MPDATA_OK;
}

int mpdata_advance(mpdata_t h, const void* psi_in, void* psi_out, const void* const* gc, const void* g,
                   const void* r, double dt, int n_steps, const double* gc_scale) {
  if (!h || n_steps < 1 || !psi_out) return MPDATA_EINVAL;
  int rc = validate_fields(h, psi_in, gc, g, r);
  if (rc != MPDATA_OK) return rc;
  if (!aligned(psi_out, h->esize)) return MPDATA_EINVAL;
  if (h->stop.load()) return MPDATA_ESTOPPED;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32)
    return run_advance<float>(h, static_cast<const float*>(psi_in), static_cast<float*>(psi_out), gc,
                              static_cast<const float*>(g), static_cast<const float*>(r), dt, n_steps, gc_scale);
  return run_advance<double>(h, static_cast<const double*>(psi_in), static_cast<double*>(psi_out), gc,
                             static_cast<const double*>(g), static_cast<const double*>(r), dt, n_steps, gc_scale);
}

int mpdata_advance_compensated(mpdata_t h, const void* psi_in, const void* lo_in, void* psi_out, void* lo_out,
                               const void* const* gc, const void* g, const void* r, double dt, int n_steps,
                               const double* gc_scale) {
  if (!h || n_steps < 1 || !psi_out || !lo_in || !lo_out) return MPDATA_EINVAL;
  int rc = validate_fields(h, psi_in, gc, g, r);
  if (rc != MPDATA_OK) return rc;
  if (!aligned(psi_out, h->esize) || !aligned(lo_in, h->esize) || !aligned(lo_out, h->esize)) return MPDATA_EINVAL;
  if ((psi_in == psi_out) != (lo_in == lo_out)) return MPDATA_EINVAL;
  if (h->dtype != MPDATA_F32 || h->n_fields != 1 || h->nd != 2 || h->n_iters != 2 || (h->opts & MPDATA_TOT) ||
      (h->opts & (MPDATA_STAGED | MPDATA_RHS_TRAPEZ | mpd::kOpenBits)))
    return MPDATA_EUNSUPPORTED;
  if (h->stop.load()) return MPDATA_ESTOPPED;
  DeviceGuard dg(h->device);
  if (!h->pingpong_lo && cudaMalloc(&h->pingpong_lo, static_cast<size_t>(h->total) * sizeof(float)) != cudaSuccess) {
    h->pingpong_lo = nullptr;
    return MPDATA_ENOMEM;
  }
  mpd::Opts o = mpd::make_opts(h->opts, h->n_iters);
  o.tile_rows = h->kernel != 2 ? h->tile_rows : 0;  // band heights do not apply
  o.kernel = h->kernel == 3 ? 3 : 0;
  const float* gcf[3] = {static_cast<const float*>(gc[0]), static_cast<const float*>(gc[1]), nullptr};
  // as in mpdata_advance: the result alternates between the outputs and the ping-pong
  // pair so that the last step lands in (psi_out, lo_out)
  float* X = static_cast<float*>(psi_out);
  float* XL = static_cast<float*>(lo_out);
  float* P = static_cast<float*>(h->pingpong);
  float* PL = static_cast<float*>(h->pingpong_lo);
  const float* cur = static_cast<const float*>(psi_in);
  const float* curl = static_cast<const float*>(lo_in);
  const size_t bytes = static_cast<size_t>(h->total) * sizeof(float);
  if (psi_in == psi_out && n_steps % 2 == 1) {
    if (cudaMemcpyAsync(P, X, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(PL, XL, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return MPDATA_ECUDA;
    cur = P;
    curl = PL;
  }
  for (int s = 0; s < n_steps; ++s) {
    if (h->stop.load(std::memory_order_relaxed)) return MPDATA_ESTOPPED;
    const bool last_parity = (n_steps - 1 - s) % 2 == 0;
    float* dst = last_parity ? X : P;
    float* dstl = last_parity ? XL : PL;
    mpd::StepArgs<float> a;
    a.psi_in = cur;
    a.psi_out = dst;
    a.gc[0] = gcf[0];
    a.gc[1] = gcf[1];
    a.gc[2] = nullptr;
    a.g = static_cast<const float*>(g);
    a.r = static_cast<const float*>(r);
    a.dt = static_cast<float>(dt);
    a.gc_scale = gc_scale ? static_cast<float>(gc_scale[s]) : 1.0f;
    rc = mpd::fused_step_comp(h->grids[0], o, a, curl, dstl, h->stream);
    if (rc != MPDATA_OK) return rc;
    cur = dst;
    curl = dstl;
  }
  return cuda_status(cudaGetLastError());
}

int mpdata_sw_advance(mpdata_t h, void* state, double dt, double dx, double eps, int n_steps) {
  if (!h || !state || n_steps < 1 || !(h->opts & MPDATA_SW) || !(dt > 0.0) || !(dx > 0.0) || !(eps >= 0.0))
    return MPDATA_EINVAL;
  if (!aligned(state, h->esize)) return MPDATA_EINVAL;
  if (h->stop.load()) return MPDATA_ESTOPPED;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32) return run_sw<float>(h, static_cast<float*>(state), dt, dx, eps, n_steps);
  return run_sw<double>(h, static_cast<double*>(state), dt, dx, eps, n_steps);
}

int mpdata_sw_reset(mpdata_t h) {
  if (!h || !(h->opts & MPDATA_SW)) return MPDATA_EINVAL;
  h->sw_first = true;
  return MPDATA_OK;
}

int mpdata_set_rhs_linear(mpdata_t h, const double* A, const void* b) {
  if (!h || !A || !(h->opts & MPDATA_RHS_TRAPEZ)) return MPDATA_EINVAL;
  if (h->n_fields > mpd::kTrapezMax) return MPDATA_EINVAL;
  for (int f = 1; f < h->n_fields; ++f)
    for (int a = 0; a < 3; ++a)
      if (h->grids[f].n[a] != h->grids[0].n[a]) return MPDATA_EINVAL;
  if (b && !aligned(b, h->esize)) return MPDATA_EINVAL;
  h->rhs_A.assign(A, A + static_cast<size_t>(h->n_fields) * h->n_fields);
  h->rhs_b = b;
  h->rhs_lin = true;
  return MPDATA_OK;
}

int mpdata_step(mpdata_t h, void* psi, const void* const* gc, const void* g, const void* r, double dt,
                int n_steps) {
  return mpdata_advance(h, psi, psi, gc, g, r, dt, n_steps, nullptr);
}

int mpdata_adjoint_step(mpdata_t h, const void* psi_n, const void* const* gc, const void* g, void* psi_bar,
                        void* const* gc_bar) {
  if (!h || !psi_bar) return MPDATA_EINVAL;
  if (h->opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B | MPDATA_RHS_TRAPEZ | MPDATA_SW | mpd::kOpenBits))
    return MPDATA_EUNSUPPORTED;
  int rc = validate_fields(h, psi_n, gc, g, nullptr);
  if (rc != MPDATA_OK) return rc;
  if (!aligned(psi_bar, h->esize)) return MPDATA_EINVAL;
  if (gc_bar)
    for (int d = 0; d < h->nd; ++d)
      if (gc_bar[d] && !aligned(gc_bar[d], h->esize)) return MPDATA_EINVAL;
  if (h->n_fields != 1) return MPDATA_EUNSUPPORTED;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32)
    return mpd::adjoint_step<float>(h, static_cast<const float*>(psi_n), gc, static_cast<const float*>(g),
                                    static_cast<float*>(psi_bar), gc_bar);
  return mpd::adjoint_step<double>(h, static_cast<const double*>(psi_n), gc, static_cast<const double*>(g),
                                   static_cast<double*>(psi_bar), gc_bar);
}

int mpdata_adjoint_step_rhs(mpdata_t h, const void* psi_n, const void* const* gc, const void* g, const void* r,
                            double dt, void* psi_bar, void* const* gc_bar, void* r_bar) {
  if (!h || !psi_bar || !r) return MPDATA_EINVAL;
  if (!(h->opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B))) return MPDATA_EUNSUPPORTED;
  if (h->opts & (MPDATA_RHS_TRAPEZ | MPDATA_SW | mpd::kOpenBits)) return MPDATA_EUNSUPPORTED;
  int rc = validate_fields(h, psi_n, gc, g, r);
  if (rc != MPDATA_OK) return rc;
  if (!aligned(psi_bar, h->esize) || !aligned(r_bar, h->esize)) return MPDATA_EINVAL;
  if (gc_bar)
    for (int d = 0; d < h->nd; ++d)
      if (gc_bar[d] && !aligned(gc_bar[d], h->esize)) return MPDATA_EINVAL;
  if (h->n_fields != 1) return MPDATA_EUNSUPPORTED;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32)
    return mpd::adjoint_step_rhs<float>(h, static_cast<const float*>(psi_n), gc, static_cast<const float*>(g),
                                        static_cast<const float*>(r), static_cast<float>(dt),
                                        static_cast<float*>(psi_bar), gc_bar, static_cast<float*>(r_bar));
  return mpd::adjoint_step_rhs<double>(h, static_cast<const double*>(psi_n), gc, static_cast<const double*>(g),
                                       static_cast<const double*>(r), dt, static_cast<double*>(psi_bar), gc_bar,
                                       static_cast<double*>(r_bar));
}

// Checks shared by the reverse-step entry points: options, fields, a single-field handle.
static int adjoint_checks(mpdata_t h, const void* psi_n, const void* const* gc, const void* g) {
  if (!h) return MPDATA_EINVAL;
  if (h->opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B | MPDATA_RHS_TRAPEZ | MPDATA_SW | mpd::kOpenBits))
    return MPDATA_EUNSUPPORTED;
  int rc = validate_fields(h, psi_n, gc, g, nullptr);
  if (rc != MPDATA_OK) return rc;
  if (h->n_fields != 1) return MPDATA_EUNSUPPORTED;
  if (h->n_iters > 4) return MPDATA_EUNSUPPORTED;
  return MPDATA_OK;
}

int mpdata_adjoint_tape_bytes(mpdata_t h, size_t* bytes) {
  if (!h || !bytes) return MPDATA_EINVAL;
  if (h->opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B | MPDATA_RHS_TRAPEZ | MPDATA_SW | mpd::kOpenBits))
    return MPDATA_EUNSUPPORTED;
  if (h->n_fields != 1 || h->n_iters > 4) return MPDATA_EUNSUPPORTED;
  *bytes = mpd::adjoint_tape_bytes(h, h->esize);
  return MPDATA_OK;
}

int mpdata_adjoint_record(mpdata_t h, const void* psi_n, const void* const* gc, const void* g, void* tape,
                          void* psi_next) {
  int rc = adjoint_checks(h, psi_n, gc, g);
  if (rc != MPDATA_OK) return rc;
  if (!aligned(tape, h->esize) || (psi_next && (!aligned(psi_next, h->esize) || psi_next == psi_n)))
    return MPDATA_EINVAL;
  if (!tape && mpd::adjoint_tape_bytes(h, h->esize) > 0) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32)
    return mpd::adjoint_record<float>(h, static_cast<const float*>(psi_n), gc, static_cast<const float*>(g),
                                      static_cast<float*>(tape), static_cast<float*>(psi_next));
  return mpd::adjoint_record<double>(h, static_cast<const double*>(psi_n), gc, static_cast<const double*>(g),
                                     static_cast<double*>(tape), static_cast<double*>(psi_next));
}

int mpdata_adjoint_replay(mpdata_t h, const void* psi_n, const void* const* gc, const void* g, const void* tape,
                          void* psi_bar, void* const* gc_bar) {
  int rc = adjoint_checks(h, psi_n, gc, g);
  if (rc != MPDATA_OK) return rc;
  if (!psi_bar || !aligned(psi_bar, h->esize) || !aligned(tape, h->esize)) return MPDATA_EINVAL;
  if (!tape && mpd::adjoint_tape_bytes(h, h->esize) > 0) return MPDATA_EINVAL;
  if (gc_bar)
    for (int d = 0; d < h->nd; ++d)
      if (gc_bar[d] && !aligned(gc_bar[d], h->esize)) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  if (h->dtype == MPDATA_F32)
    return mpd::adjoint_replay<float>(h, static_cast<const float*>(psi_n), gc, static_cast<const float*>(g),
                                      static_cast<const float*>(tape), static_cast<float*>(psi_bar), gc_bar);
  return mpd::adjoint_replay<double>(h, static_cast<const double*>(psi_n), gc, static_cast<const double*>(g),
                                     static_cast<const double*>(tape), static_cast<double*>(psi_bar), gc_bar);
}

int mpdata_reduce(mpdata_t h, const void* psi, const void* g, double* mass_out) {
  if (!h || !psi || !mass_out) return MPDATA_EINVAL;
  if (!aligned(psi, h->esize) || (g && !aligned(g, h->esize))) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  cudaError_t e = h->dtype == MPDATA_F32
                      ? mpd::reduce_mass<float>(static_cast<const float*>(psi), static_cast<const float*>(g),
                                                h->d_spans, h->n_fields, h->d_partial, h->d_out, h->stream)
                      : mpd::reduce_mass<double>(static_cast<const double*>(psi), static_cast<const double*>(g),
                                                 h->d_spans, h->n_fields, h->d_partial, h->d_out, h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  e = cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * h->n_fields, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  int rc = sync_status(h);
  std::memcpy(mass_out, h->h_out, sizeof(double) * h->n_fields);
  return rc;
}

int mpdata_diff_norms(mpdata_t h, const void* a, const void* b, double* l2sq_out, double* linf_out) {
  if (!h || !a || !b) return MPDATA_EINVAL;
  if (!aligned(a, h->esize) || !aligned(b, h->esize)) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  cudaError_t e = h->dtype == MPDATA_F32
                      ? mpd::reduce_diff<float>(static_cast<const float*>(a), static_cast<const float*>(b),
                                                h->d_spans, h->n_fields, h->d_partial, h->d_out, h->stream)
                      : mpd::reduce_diff<double>(static_cast<const double*>(a), static_cast<const double*>(b),
                                                 h->d_spans, h->n_fields, h->d_partial, h->d_out, h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  e = cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * 2 * h->n_fields, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  int rc = sync_status(h);
  if (l2sq_out) std::memcpy(l2sq_out, h->h_out, sizeof(double) * h->n_fields);
  if (linf_out) std::memcpy(linf_out, h->h_out + h->n_fields, sizeof(double) * h->n_fields);
  return rc;
}

int mpdata_check_courant(mpdata_t h, const void* const* gc, const void* g, double* max_out) {
  if (!h || !gc) return MPDATA_EINVAL;
  for (int d = 0; d < h->nd; ++d)
    if (!gc[d] || !aligned(gc[d], h->esize)) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  cudaError_t e;
  if (h->dtype == MPDATA_F32) {
    const float* p[3] = {static_cast<const float*>(gc[0]), h->nd > 1 ? static_cast<const float*>(gc[1]) : nullptr,
                         h->nd > 2 ? static_cast<const float*>(gc[2]) : nullptr};
    e = mpd::reduce_courant<float>(h->grids.data(), h->offsets.data(), h->n_fields, p,
                                   static_cast<const float*>(g), h->d_partial, h->d_out, h->stream);
  } else {
    const double* p[3] = {static_cast<const double*>(gc[0]), h->nd > 1 ? static_cast<const double*>(gc[1]) : nullptr,
                          h->nd > 2 ? static_cast<const double*>(gc[2]) : nullptr};
    e = mpd::reduce_courant<double>(h->grids.data(), h->offsets.data(), h->n_fields, p,
                                    static_cast<const double*>(g), h->d_partial, h->d_out, h->stream);
  }
  if (e != cudaSuccess) return MPDATA_ECUDA;
  e = cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * h->n_fields, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return MPDATA_ECUDA;
  int rc = sync_status(h);
  if (rc != MPDATA_OK) return rc;
  double m = 0.0;
  for (int f = 0; f < h->n_fields; ++f) m = h->h_out[f] > m ? h->h_out[f] : m;
  if (max_out) *max_out = m;
  return m > 1.0 ? MPDATA_ECOURANT : MPDATA_OK;
}

int mpdata_tune(mpdata_t h, int knob, int value) {
  if (!h) return MPDATA_EINVAL;
  if (knob == MPDATA_TUNE_TILE_ROWS) {
    if (value != 0 && (value < 4 || value > 65536)) return MPDATA_EINVAL;
    h->tile_rows = value;
    return MPDATA_OK;
  }
  if (knob == MPDATA_TUNE_KERNEL) {
    if (value < 0 || value > 3) return MPDATA_EINVAL;
    h->kernel = value;
    return MPDATA_OK;
  }
  if (knob == MPDATA_TUNE_STEPS_PER_LAUNCH) {
    if (value < 0 || value > mpd::kTblockMaxDepth) return MPDATA_EINVAL;
    h->steps_per_launch = value;
    return MPDATA_OK;
  }
  return MPDATA_EINVAL;
}

int mpdata_request_stop(mpdata_t h) {
  if (!h) return MPDATA_EINVAL;
  h->stop.store(1);
  return MPDATA_OK;
}

int mpdata_clear_stop(mpdata_t h) {
  if (!h) return MPDATA_EINVAL;
  h->stop.store(0);
  return MPDATA_OK;
}

int mpdata_set_stream(mpdata_t h, void* cuda_stream) {
  if (!h) return MPDATA_EINVAL;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return MPDATA_OK;
}

int mpdata_sync(mpdata_t h) {
  if (!h) return MPDATA_EINVAL;
  DeviceGuard dg(h->device);
  return sync_status(h);
}

int mpdata_destroy(mpdata_t h) {
  if (!h) return MPDATA_EINVAL;
  {
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
  }
  delete h;
  return MPDATA_OK;
}

const char* mpdata_strerror(int code) {
  switch (code) {
    case MPDATA_OK: return "ok";
    case MPDATA_EINVAL: return "invalid argument";
    case MPDATA_EUNSUPPORTED: return "unsupported configuration";
    case MPDATA_ECUDA: return "CUDA runtime error";
    case MPDATA_ECOURANT: return "Courant condition violated (sum of outflow advectors / G > 1)";
    case MPDATA_ETIMEOUT: return "bounded device wait timed out";
    case MPDATA_ESTOPPED: return "stopped on request";
    case MPDATA_ENOMEM: return "out of memory";
  }
  return "unknown status";
}

const char* mpdata_version(void) { return "mpdata-gb300 0.1 (sm_103a)"; }

}  // extern "C"
