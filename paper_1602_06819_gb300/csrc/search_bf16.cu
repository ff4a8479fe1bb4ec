// search_bf16.cu -- iGNNS search kernels over the bf16 copy of the rows.
#include "search.cuh"

namespace knn {
KNN_DEFINE_SEARCH_LAUNCHER(launch_search_bf16, ST_BF16)
}  // namespace knn
