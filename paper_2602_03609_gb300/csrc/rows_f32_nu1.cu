// Row kernels, float arithmetic, Matern order code 1 (0, 1, 2 = nu 0.5, 1.5, 2.5).
#include <algorithm>

#include "rows_launch.cuh"

namespace vst {
template cudaError_t launch_rows_tn<float, 1>(int, int, const RowArgs&, cudaStream_t, int64_t*);
}  // namespace vst
