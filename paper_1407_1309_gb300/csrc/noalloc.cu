// Allocation-free entry point: one MPDATA step of one field on the staged
// kernels, with the scratch those kernels need taken from a fixed array that
// is part of the library image instead of from cudaMalloc.
//
// Why: some callers may not allocate device memory at the point where they
// advance a field -- for example a host that hands the library a fixed memory
// budget and forbids any allocation after start-up (a framework whose caching
// allocator owns the device memory), or a latency-critical loop that cannot
// afford cudaMalloc / cudaFree, which may synchronise the whole device.  Such
// callers cannot create a handle (mpdata_create allocates the handle's
// scratch).  mpdata_step_noalloc needs no handle and calls no allocating
// routine; the caller still provides every input and output buffer.
//
// The array below is held by every GPU that loads this library, until the
// process exits.  All calls share it, so calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it; serialise them.
// It keeps the previous call's contents; nothing in it has to start at zero,
// because each staged sub-step writes every scratch element before any later
// sub-step of the same call reads it.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

// Size of the static scratch array (MPDATA_NOALLOC_SCRATCH_BYTES in include/mpdata.h).
constexpr size_t kNoallocBytes = static_cast<size_t>(16) << 20;
static_assert(kNoallocBytes == MPDATA_NOALLOC_SCRATCH_BYTES, "header and library disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, called once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPDATA_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return MPDATA_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MPDATA_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MPDATA_OK;
}

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T>
int run(const mpd::Grid& g, const mpd::Opts& o, const void* psi_in, void* psi_out, const void* const* gc,
        const void* gf, const void* r, double dt, void* scratch, cudaStream_t st) {
  mpd::StepArgs<T> a;
  a.psi_in = static_cast<const T*>(psi_in);
  a.psi_out = static_cast<T*>(psi_out);
  for (int d = 0; d < 3; ++d) a.gc[d] = d < g.nd ? static_cast<const T*>(gc[d]) : nullptr;
  a.g = static_cast<const T*>(gf);
  a.r = static_cast<const T*>(r);
  a.dt = static_cast<T>(dt);
  a.gc_scale = T(1);
  const mpd::StagedScratch<T> s = mpd::carve_staged<T>(scratch, g.N);
  return mpd::staged_step<T>(g, o, a, s, st) == cudaSuccess ? MPDATA_OK : MPDATA_ECUDA;
}

}  // namespace

extern "C" int mpdata_step_noalloc(int ndims, const int64_t* shape, int dtype, int n_iters, uint32_t opts,
                                   const void* psi_in, void* psi_out, const void* const* gc, const void* g,
                                   const void* r, double dt, void* cuda_stream) {
  if (!shape || !psi_in || !psi_out || !gc) return MPDATA_EINVAL;
  if (ndims < 1 || ndims > 3 || n_iters < 1) return MPDATA_EINVAL;
  if (dtype != MPDATA_F32 && dtype != MPDATA_F64) return MPDATA_EINVAL;
  if ((opts & MPDATA_IGA) && n_iters != 2) return MPDATA_EINVAL;
  if ((opts & MPDATA_IGA) && (opts & (MPDATA_ABS | MPDATA_DFL))) return MPDATA_EINVAL;
  if ((opts & MPDATA_RHS_EULER_A) && (opts & MPDATA_RHS_EULER_B)) return MPDATA_EINVAL;
  const bool nug = opts & MPDATA_NUG;
  const bool rhs = opts & (MPDATA_RHS_EULER_A | MPDATA_RHS_EULER_B);
  if (nug != (g != nullptr) || rhs != (r != nullptr)) return MPDATA_EINVAL;
  long long n = 1;
  for (int d = 0; d < ndims; ++d) {
    if (shape[d] < 1 || shape[d] > (int64_t(1) << 30)) return MPDATA_EINVAL;
    n *= shape[d];
    if (n > (1LL << 40)) return MPDATA_EINVAL;
  }
  if (!mpd::valid_open_bits(ndims, opts, shape) || (opts & MPDATA_RHS_TRAPEZ)) return MPDATA_EINVAL;
  const size_t es = dtype == MPDATA_F32 ? 4 : 8;
  // the staged sub-steps use kStagedArrays arrays of n elements
  if (static_cast<unsigned long long>(n) * mpd::kStagedArrays * es > kNoallocBytes) return MPDATA_EINVAL;
  if (!aligned_to(psi_in, es) || !aligned_to(psi_out, es) || (g && !aligned_to(g, es)) || (r && !aligned_to(r, es)))
    return MPDATA_EINVAL;
  for (int d = 0; d < ndims; ++d)
    if (!gc[d] || !aligned_to(gc[d], es)) return MPDATA_EINVAL;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != MPDATA_OK) return rc;
  const mpd::Grid gr = mpd::make_grid(ndims, shape, opts);
  const mpd::Opts o = mpd::make_opts(opts, n_iters);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (dtype == MPDATA_F32) return run<float>(gr, o, psi_in, psi_out, gc, g, r, dt, scratch, st);
  return run<double>(gr, o, psi_in, psi_out, gc, g, r, dt, scratch, st);
}
