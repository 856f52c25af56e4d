// rhs_el_f32_s44.cu -- instantiation of the elastic K1 launches (float, 44-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_el_seg<float, kSegLong>(int, const RhsArgs<float> &, const RhsElas<float> &, cudaStream_t);
}
