// Serving loop (placeholder until the continuous-batching server lands).
#include "gb300bfs.h"
#include "internal.h"

extern "C" {

gb_status server_create(const gb_graph *const *, int, size_t, gb_server **out)
{
    if (out) *out = nullptr;
    gb::set_error("server_create: not built yet");
    return GB_ERR_UNIMPLEMENTED;
}
gb_status server_submit(gb_server *, int, int64_t, int64_t *) { return GB_ERR_UNIMPLEMENTED; }
gb_status server_poll(gb_server *, int64_t, const int32_t **, const int32_t **) { return GB_ERR_UNIMPLEMENTED; }
gb_status server_release(gb_server *, int64_t) { return GB_ERR_UNIMPLEMENTED; }
gb_status server_run_trace(gb_server *, int64_t, const double *, const int32_t *, const int64_t *, int,
                           double *)
{
    return GB_ERR_UNIMPLEMENTED;
}
gb_status server_destroy(gb_server *) { return GB_OK; }

}  // extern "C"
