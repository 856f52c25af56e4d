// rhs_f64_s44.cu -- instantiation of the K1 launches (double, 44-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<double, kSegLong>(int, const RhsArgs<double> *, int, cudaStream_t);
}
