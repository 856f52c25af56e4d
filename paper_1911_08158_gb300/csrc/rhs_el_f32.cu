// rhs_el_f32.cu -- instantiation of the elastic K1 launches (float, every segment length).
#include "sweep.cuh"

namespace ads {
template <>
cudaError_t launch_rhs_el<float>(int p, const RhsArgs<float> &a, const RhsElas<float> &el, cudaStream_t s)
{
    return launch_rhs_el_impl<float>(p, a, el, s);
}
}  // namespace ads
