// rhs_f32.cu -- instantiation of the K1 launches (float, 32-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<float, kSeg>(int, const RhsArgs<float> *, int, cudaStream_t);
}
