// cfpq_server.cu -- continuous-batching server (placeholder until implemented).
#include "cfpq_engine.cuh"

struct cfpq_server {};

extern "C" {
int cfpq_server_create(cfpq_server **out, const cfpq_options *, void *, uint32_t, uint32_t, size_t, const uint32_t *,
                       const uint32_t *, const uint32_t *) {
    if (out) *out = nullptr;
    return CFPQ_ERR_UNSUPPORTED;
}
int cfpq_server_destroy(cfpq_server *) { return CFPQ_OK; }
int cfpq_submit(cfpq_server *, const cfpq_rsm *, uint64_t *) { return CFPQ_ERR_UNSUPPORTED; }
int cfpq_server_step(cfpq_server *, uint32_t *, uint32_t *) { return CFPQ_ERR_UNSUPPORTED; }
int cfpq_poll(cfpq_server *, uint64_t, int *) { return CFPQ_ERR_UNSUPPORTED; }
int cfpq_result_reachable_bits(cfpq_server *, uint64_t, uint32_t, uint64_t *) { return CFPQ_ERR_UNSUPPORTED; }
int cfpq_release(cfpq_server *, uint64_t) { return CFPQ_ERR_UNSUPPORTED; }
}
