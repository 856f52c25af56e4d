// rhs_f64.cu -- instantiation of the K1 launches (double, 32-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<double, kSeg>(int, const RhsArgs<double> *, int, cudaStream_t);
}
