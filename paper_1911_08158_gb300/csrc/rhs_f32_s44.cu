// rhs_f32_s44.cu -- instantiation of the K1 launches (float, 44-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<float, kSegLong>(int, const RhsArgs<float> *, int, cudaStream_t);
}
