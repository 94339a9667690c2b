// update_limb.cu -- trailing update on the integer tensor pipe (placeholder
// until the limb kernel lands).
#include "linac_host.h"
#include "update.cuh"

namespace linac {

linac_status launch_update_limb(uint32_t*, int64_t, int64_t, int64_t, int, const Field&, const DenseState*,
                                const int32_t*, int64_t, const int32_t*, int64_t, const LimbScratch*,
                                cudaStream_t) {
    return LINAC_ERR_UNSUPPORTED;
}

}  // namespace linac
