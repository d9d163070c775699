// Serving engine: placeholder until the engine lands.
#include "me_internal.h"

extern "C" {
int me_serve_open(const me_serve_cfg *c, me_server **o) {
    return (c && o) ? ME_ERR_UNSUPPORTED : ME_ERR_ARG;
}
int me_serve_submit(me_server *s, const uint32_t *, int32_t, int32_t, int32_t, int32_t,
                    uint64_t *) { return s ? ME_ERR_UNSUPPORTED : ME_ERR_ARG; }
int me_serve_poll(me_server *s, uint64_t, uint32_t *, int64_t, me_timing *) {
    return s ? ME_ERR_UNSUPPORTED : ME_ERR_ARG;
}
int me_serve_stats(me_server *s, int64_t *, int64_t *, int64_t *, int64_t *) {
    return s ? ME_ERR_UNSUPPORTED : ME_ERR_ARG;
}
int me_serve_close(me_server *s, int64_t) { return s ? ME_ERR_UNSUPPORTED : ME_ERR_ARG; }
}
