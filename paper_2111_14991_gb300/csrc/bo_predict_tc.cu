// Tensor-core prediction pass (tcgen05): not built yet.
#include "bo_internal.h"

namespace bo {
int launch_predict_tc(const DevView&, int, int64_t, cudaStream_t) { return -1; }
}  // namespace bo
