// duwp_server.cu -- continuous-batching server over one engine (see include/duwp.h).
#include <cstring>

#include "duwp_engine.h"

extern "C" {

struct duwp_server;

int duwp_server_create(const duwp_server_cfg *cfg, duwp_alloc_fn alloc, duwp_free_fn free_fn, void *alloc_ctx,
                       duwp_server **out)
{
    (void)cfg; (void)alloc; (void)free_fn; (void)alloc_ctx;
    if (out) *out = nullptr;
    return DUWP_EINVAL;
}

int duwp_submit(duwp_server *s, const duwp_params *params, int32_t n_steps, uint64_t *req_id)
{
    (void)s; (void)params; (void)n_steps; (void)req_id;
    return DUWP_EINVAL;
}

int duwp_poll(duwp_server *s, uint64_t req_id, duwp_result *out)
{
    (void)s; (void)req_id; (void)out;
    return DUWP_EINVAL;
}

int duwp_server_destroy(duwp_server *s)
{
    (void)s;
    return DUWP_EINVAL;
}

}  // extern "C"
