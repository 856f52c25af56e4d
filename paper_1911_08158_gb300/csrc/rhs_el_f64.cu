// rhs_el_f64.cu -- instantiation of the elastic K1 launches (double, every segment length).
#include "sweep.cuh"

namespace ads {
template <>
cudaError_t launch_rhs_el<double>(int p, const RhsArgs<double> &a, const RhsElas<double> &el, cudaStream_t s)
{
    return launch_rhs_el_impl<double>(p, a, el, s);
}
}  // namespace ads
