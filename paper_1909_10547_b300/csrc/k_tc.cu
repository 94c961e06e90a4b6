// Tensor-core path (tcgen05): placeholder until the kernel lands.
#include "fk_internal.h"

namespace fk {
int tc_build(fk_table *, const double *) { return fail(FK_EUNSUPPORTED, "tensor-core modes not built yet"); }
int fwd_tc(const fk_table *, const float *, int, float *, int, int, cudaStream_t) {
    return fail(FK_EUNSUPPORTED, "tensor-core modes not built yet");
}
void tc_free(fk_table *) {}
}  // namespace fk
