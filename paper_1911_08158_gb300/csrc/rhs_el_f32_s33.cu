// rhs_el_f32_s33.cu -- instantiation of the elastic K1 launches (float, 33-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_el_seg<float, kSegAlt>(int, const RhsArgs<float> &, const RhsElas<float> &, cudaStream_t);
}
