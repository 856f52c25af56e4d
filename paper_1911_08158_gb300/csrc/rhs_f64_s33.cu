// rhs_f64_s33.cu -- instantiation of the K1 launches (double, 33-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_seg<double, kSegAlt>(int, const RhsArgs<double> *, int, cudaStream_t);
}
