// Bulk-copy (TMA) engine: placeholder until the engine lands.
#include "me_internal.h"

namespace me {
bool bulk_available() { return false; }
bool bulk_eligible(const Geo &, const void *) { return false; }
cudaError_t launch_bulk(const Geo &, uint32_t *, const me_tile_cfg &, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace me
