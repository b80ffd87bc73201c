// Placeholder until the tensor-core engine lands: every mixed request is
// rejected with PINV_ERR_ARG (there is no fallback to another precision).
#include "mixed.h"
#include "../../include/pinv.h"

namespace pinv {
struct MixedEngine { int unused; };
MixedEngine* mixed_create() { return new MixedEngine{}; }
void mixed_destroy(MixedEngine* e) { delete e; }
size_t mixed_workspace_bytes(int, int) { return 0; }
int mixed_begin(MixedEngine*, int, int, int, const double*, int, int, cudaStream_t, MixedSchedule*) {
    return PINV_ERR_ARG;
}
int mixed_loop_precision(const MixedSchedule*, int, double) { return 0; }
int mixed_pm_loop(MixedEngine*, const MixedSchedule*, int, const double*, double*, double*, cudaStream_t) {
    return -1;
}
int mixed_last_kernels(const MixedEngine*) { return 0; }
}  // namespace pinv
