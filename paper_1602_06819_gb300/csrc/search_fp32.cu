// search_fp32.cu -- iGNNS search kernels over the fp32 copy of the rows.
#include "search.cuh"

namespace knn {
KNN_DEFINE_SEARCH_LAUNCHER(launch_search_fp32, ST_FP32)
}  // namespace knn
