#include "kernels.h"
namespace mpd {
template <typename T>
int batched_step(mpdata_s*, const T*, T*, const T* const*, const T*, const T*, T, T, const Opts&) { return MPDATA_EUNSUPPORTED; }
void batched_free(mpdata_s*) {}
template int batched_step<float>(mpdata_s*, const float*, float*, const float* const*, const float*, const float*, float, float, const Opts&);
template int batched_step<double>(mpdata_s*, const double*, double*, const double* const*, const double*, const double*, double, double, const Opts&);
}
