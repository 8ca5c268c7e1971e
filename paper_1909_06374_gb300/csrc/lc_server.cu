// lc_server.cu -- continuous-batching server entry points of the C ABI.
#include "lc_internal.h"

using namespace lc;

extern "C" {

lc_status lc_server_create(int, size_t, lc_precision, lc_server* out)
{
    if (out) *out = nullptr;
    set_error("server not available");
    return LC_ERR_INVALID;
}
lc_status lc_submit(lc_server, const lc_job*, lc_ticket*) { set_error("server not available"); return LC_ERR_INVALID; }
lc_status lc_poll(lc_server, lc_ticket, void*, uint64_t*) { set_error("server not available"); return LC_ERR_INVALID; }
lc_status lc_server_stats(lc_server, uint64_t*, uint64_t*, uint64_t*) { set_error("server not available"); return LC_ERR_INVALID; }
lc_status lc_server_destroy(lc_server) { set_error("server not available"); return LC_ERR_INVALID; }

}
