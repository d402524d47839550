// Batched step: every field of an ensemble handle (independent 2D fields of
// uneven sizes, concatenated) advanced by one launch of the fused kernel whose
// persistent grid walks a table of (field, strip, row tile) work items.  The
// table is built on the host once per handle and tile height and kept on the
// device with the handle.
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"

namespace mpd {
namespace {

struct TableHolder {
  BatchTable tab{};
  int nc = 0;
};

constexpr int kDefaultBatchRows = 32;

}  // namespace

void batched_free(mpdata_s* h) {
  void** slot = handle_batch(h);
  auto* th = static_cast<TableHolder*>(*slot);
  if (th) {
    cudaFree(th->tab.fields);
    cudaFree(th->tab.item_field);
    delete th;
    *slot = nullptr;
  }
}

template <typename T>
int batched_step(mpdata_s* h, const T* psi_in, T* psi_out, const T* const* gc, const T* g, const T* r, T dt,
                 T gc_scale, const Opts& o) {
  if (handle_nd(h) != 2 || o.n_iters != 2 || o.tot || o.abs || o.dfl || o.open) return MPDATA_EUNSUPPORTED;
  // lanes of 2 columns for FP32 when the handle asks for them (MPDATA_TUNE_KERNEL = 3)
  const int nc = (o.kernel == 3 && sizeof(T) == 4) ? 2 : fused_batched_columns<T>();
  const int ty = o.tile_rows > 0 ? o.tile_rows : kDefaultBatchRows;
  void** slot = handle_batch(h);
  auto* th = static_cast<TableHolder*>(*slot);
  if (th == nullptr || th->tab.ty != ty || th->nc != nc) {
    batched_free(h);
    const int nf = handle_fields(h);
    const Grid* grids = handle_grids(h);
    const long long* offs = handle_offsets(h);
    const int stride = fused_strip_stride(nc);
    std::vector<BatchField> fields(nf);
    std::vector<int> item_field;
    for (int f = 0; f < nf; ++f) {
      BatchField& b = fields[f];
      b.offset = offs[f];
      b.n0 = grids[f].n[1];
      b.n1 = grids[f].n[2];
      b.strips = (b.n1 + stride - 1) / stride;
      b.item_base = static_cast<int>(item_field.size());
      b.vec = (b.n1 % nc == 0) && (b.offset % nc == 0);
      const long long items = static_cast<long long>(b.strips) * ((b.n0 + ty - 1) / ty);
      if (item_field.size() + items > (1LL << 30)) return MPDATA_EUNSUPPORTED;
      item_field.insert(item_field.end(), static_cast<size_t>(items), f);
    }
    th = new TableHolder;
    th->nc = nc;
    th->tab.ty = ty;
    th->tab.n_items = static_cast<int>(item_field.size());
    if (cudaMalloc(&th->tab.fields, sizeof(BatchField) * nf) != cudaSuccess ||
        cudaMalloc(&th->tab.item_field, sizeof(int) * item_field.size()) != cudaSuccess) {
      cudaFree(th->tab.fields);
      delete th;
      return MPDATA_ENOMEM;
    }
    cudaMemcpy(th->tab.fields, fields.data(), sizeof(BatchField) * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(th->tab.item_field, item_field.data(), sizeof(int) * item_field.size(), cudaMemcpyHostToDevice);
    *slot = th;
  }
  return fused_batched_step<T>(th->tab, o, psi_in, psi_out, gc[0], gc[1], g, r, dt, gc_scale, handle_stream(h),
                               th->nc);
}

template int batched_step<float>(mpdata_s*, const float*, float*, const float* const*, const float*, const float*,
                                 float, float, const Opts&);
template int batched_step<double>(mpdata_s*, const double*, double*, const double* const*, const double*,
                                  const double*, double, double, const Opts&);

}  // namespace mpd
