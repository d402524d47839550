// Entry points of the kernel families, called by the C ABI (capi.cu).
#pragma once

#include "internal.h"

namespace mpd {

// accessors of the opaque handle (capi.cu)
int handle_nd(const mpdata_s* h);
int handle_fields(const mpdata_s* h);
const Grid* handle_grids(const mpdata_s* h);
const long long* handle_offsets(const mpdata_s* h);
long long handle_total(const mpdata_s* h);
cudaStream_t handle_stream(const mpdata_s* h);
int* handle_status(const mpdata_s* h);
void** handle_batch(mpdata_s* h);
void** handle_adj(mpdata_s* h);
int handle_n_iters(const mpdata_s* h);
uint32_t handle_opts(const mpdata_s* h);
// the handle's MPDATA_TUNE_KERNEL and MPDATA_TUNE_TILE_ROWS settings
void handle_tuning(const mpdata_s* h, int* kernel, int* tile_rows);

// Fused tile kernel for one field and one step (fused2d.cu).  Returns
// MPDATA_EUNSUPPORTED when the field / options are not covered, so the caller
// runs the staged path.  tmp: device buffer of the field's size, used when the
// step is in place.
// Temporal blocking (tblock2d.cu): `depth` steps of one 2D field (n_iters = 2, FCT and infinite
// gauge or not, G = 1, no sources, periodic) in one launch, psi_in -> psi_out (distinct
// buffers), scales[k] the advector factor of step k (nullptr: 1).  tblock_covers says whether
// the field, options and depth are covered; tblock_steps returns MPDATA_EUNSUPPORTED where not.
constexpr int kTblockMaxDepth = 4;
template <typename T>
bool tblock_covers(const Grid& g, const Opts& o, int depth);
template <typename T>
int tblock_steps(const Grid& g, const Opts& o, const T* psi_in, T* psi_out, const T* gc0, const T* gc1, int depth,
                 const double* scales, cudaStream_t st);

template <typename T>
int fused_step(const Grid& g, const Opts& o, const StepArgs<T>& a, T* tmp, cudaStream_t st);

// One 2D step (n_iters = 2, no third-order terms, Kahan summation, G, infinite gauge or
// sources) by the warp march that also writes the adjoint tape (psi^(1), pseudo-advectors
// and, under FCT, bounds and factors, in the layout of mpdata_adjoint_record; the limited
// advectors are left unwritten, the reverse step re-derives them) into `tape`;
// MPDATA_EUNSUPPORTED for other cases.  It hands over to band_tape where fused_step would
// run the band march.
template <typename T>
int fused_tape(const Grid& g, const Opts& o, const StepArgs<T>& a, T* tape, cudaStream_t st);
// The same by the band march (band2d.cu).
template <typename T>
int band_tape(const Grid& g, const Opts& o, const StepArgs<T>& a, T* tape, cudaStream_t st);

// The fused 2D step on a compensated FP32 state psi = hi + lo (fused2d.cu, warp march):
// hi in a.psi_in / a.psi_out, lo in lo_in / lo_out.  MPDATA_EUNSUPPORTED outside 2D,
// n_iters = 2, no tot, out of place.
int fused_step_comp(const Grid& g, const Opts& o, const StepArgs<float>& a, const float* lo_in, float* lo_out,
                    cudaStream_t st);

// The same step with one marching front per block of warps (band2d.cu).
template <typename T>
int band_step(const Grid& g, const Opts& o, const StepArgs<T>& a, cudaStream_t st);

// Work table of the batched fused kernel: one item per (field, strip, row tile).
struct BatchField {
  long long offset;  // first cell of the field in the concatenated arrays
  int n0, n1, strips, item_base, vec;
};
struct BatchTable {
  BatchField* fields;  // device
  int* item_field;     // device, field of every item
  int n_items, ty;
};
template <typename T>
int fused_batched_columns();
int fused_strip_stride(int nc);
template <typename T>
int fused_batched_step(const BatchTable& tab, const Opts& o, const T* psi_in, T* psi_out, const T* gc0,
                       const T* gc1, const T* G, const T* R, T dt, T scale, cudaStream_t st, int nc);

// One step of all fields of a batched handle in one persistent launch
// (batched.cu); MPDATA_EUNSUPPORTED when not covered.
template <typename T>
int batched_step(mpdata_s* h, const T* psi_in, T* psi_out, const T* const* gc, const T* g, const T* r, T dt,
                 T gc_scale, const Opts& o);
void batched_free(mpdata_s* h);

// Reverse of one step of a single-field handle (adjoint.cu).
template <typename T>
int adjoint_step(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, T* psi_bar,
                 void* const* gc_bar);
// The same with the Euler source terms: R (r, dt of the step) added after (euler_a) or before
// (euler_b) the advection; r_bar (nullable) accumulates dL/dR.
template <typename T>
int adjoint_step_rhs(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, const T* r, T dt, T* psi_bar,
                     void* const* gc_bar, T* r_bar);
void adjoint_free(mpdata_s* h);
// The reverse step split in two: the forward tape of one step recorded into a caller buffer of
// adjoint_tape_bytes (plus the step's result when psi_next is not null), and the reverse sweep
// that reads it.
size_t adjoint_tape_bytes(mpdata_s* h, size_t esize);
template <typename T>
int adjoint_record(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, T* tape, T* psi_next);
template <typename T>
int adjoint_replay(mpdata_s* h, const T* psi_n, const void* const* gc, const T* g, const T* tape, T* psi_bar,
                   void* const* gc_bar);

}  // namespace mpd
