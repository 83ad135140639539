// lpp_serve.cu -- serving loop (placeholder until the continuous-batching
// server is built): every call reports that the server is not available.
#include "lpp_engine.h"

extern "C" {
lpp_status lpp_server_create(size_t, const lpp_opts *, lpp_server **srv) {
    if (srv) *srv = nullptr;
    return LPP_ERR_INVALID;
}
lpp_status lpp_server_submit(lpp_server *, const lpp_lp *, uint64_t *) { return LPP_ERR_INVALID; }
lpp_status lpp_server_take(lpp_server *, uint64_t, int32_t, lpp_reduced **, lpp_postsolve **) {
    return LPP_ERR_INVALID;
}
lpp_status lpp_server_stats_get(lpp_server *, lpp_server_stats *) { return LPP_ERR_INVALID; }
void lpp_server_destroy(lpp_server *) {}
}
