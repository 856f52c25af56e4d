// rhs_el_f64_s33.cu -- instantiation of the elastic K1 launches (double, 33-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_el_seg<double, kSegAlt>(int, const RhsArgs<double> &, const RhsElas<double> &, cudaStream_t);
}
