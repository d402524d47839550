#include "kernels.h"
namespace mpd {
template <typename T>
int adjoint_step(mpdata_s*, const T*, const void* const*, const T*, T*, void* const*) { return MPDATA_EUNSUPPORTED; }
template int adjoint_step<float>(mpdata_s*, const float*, const void* const*, const float*, float*, void* const*);
template int adjoint_step<double>(mpdata_s*, const double*, const void* const*, const double*, double*, void* const*);
}
