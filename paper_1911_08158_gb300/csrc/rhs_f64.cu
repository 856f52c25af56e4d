// rhs_f64.cu -- instantiation of the K1 launches (double).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_group<double>(int, const RhsArgs<double> *, int, cudaStream_t);
}
