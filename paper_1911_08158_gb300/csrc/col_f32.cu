// col_f32.cu -- instantiation of the K2/K3 launches (float).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_col_group<float>(int, const ColArgs<float> *, const ColMaps *, int, cudaStream_t);
}
