// search_fp8.cu -- iGNNS search kernels over the fp8 copy of the rows.
#include "search.cuh"

namespace knn {
KNN_DEFINE_SEARCH_LAUNCHER(launch_search_fp8, ST_FP8)
}  // namespace knn
