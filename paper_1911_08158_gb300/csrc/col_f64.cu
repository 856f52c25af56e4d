// col_f64.cu -- instantiation of the K2/K3 launches (double).
#include "sweep.cuh"

namespace ads {
template cudaError_t launch_col_group<double>(int, const ColArgs<double> *, const ColMaps *, int, cudaStream_t);
}
