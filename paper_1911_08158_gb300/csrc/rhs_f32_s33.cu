// rhs_f32_s33.cu -- instantiation of the K1 launches (float, 33-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<float, kSegAlt>(int, const RhsArgs<float> *, int, cudaStream_t);
}
