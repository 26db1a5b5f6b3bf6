// Serving loop (continuous batching of refinement requests): fr_server_* in flowref.h.
#include "api_internal.h"

struct fr_server {
    int dummy;
};

extern "C" fr_status fr_server_create(fr_server **srv, const fr_server_config *cfg) {
    (void)cfg;
    if (srv) *srv = nullptr;
    return FR_ERR_INVALID_ARG;
}
extern "C" fr_status fr_server_add_graph(fr_server *, int32_t, int32_t, const int32_t *, const int32_t *,
                                         const int32_t *, const int32_t *, int32_t *) { return FR_ERR_INVALID_ARG; }
extern "C" fr_status fr_server_submit(fr_server *, const fr_request *) { return FR_ERR_INVALID_ARG; }
extern "C" fr_status fr_server_next(fr_server *, fr_response *, int32_t *, int32_t, int32_t) { return FR_ERR_INVALID_ARG; }
extern "C" fr_status fr_server_stats(fr_server *, int64_t *, int64_t *, int64_t *, int32_t *) { return FR_ERR_INVALID_ARG; }
extern "C" fr_status fr_server_destroy(fr_server *) { return FR_ERR_INVALID_ARG; }
