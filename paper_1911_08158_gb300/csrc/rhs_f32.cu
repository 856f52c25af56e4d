// rhs_f32.cu -- instantiation of the K1 launches (float).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_group<float>(int, const RhsArgs<float> *, int, cudaStream_t);
}
