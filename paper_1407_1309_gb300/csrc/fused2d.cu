#include "kernels.h"
namespace mpd {
template <typename T>
int fused_step(const Grid&, const Opts&, const StepArgs<T>&, T*, cudaStream_t) { return MPDATA_EUNSUPPORTED; }
template int fused_step<float>(const Grid&, const Opts&, const StepArgs<float>&, float*, cudaStream_t);
template int fused_step<double>(const Grid&, const Opts&, const StepArgs<double>&, double*, cudaStream_t);
}
