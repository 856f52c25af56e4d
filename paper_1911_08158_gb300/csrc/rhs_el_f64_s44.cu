// rhs_el_f64_s44.cu -- instantiation of the elastic K1 launches (double, 44-row segments).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_rhs_el_seg<double, kSegLong>(int, const RhsArgs<double> &, const RhsElas<double> &, cudaStream_t);
}
