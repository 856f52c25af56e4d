// rhs_el_f32.cu -- instantiation of the elastic K1 launches (float, 32-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_el_seg<float, kSeg>(int, const RhsArgs<float> &, const RhsElas<float> &, cudaStream_t);
}
