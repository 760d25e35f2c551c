// bls_server.cpp -- serving entry points (placeholder until the scheduler lands).
#include "bls_plan.h"

using namespace blsgpu;

namespace blsgpu {
struct Server {};
void server_destroy(bls_plan_impl* P) { delete P->server; P->server = nullptr; }
}  // namespace blsgpu

extern "C" {
bls_status bls_submit(bls_plan*, const bls_curve*, uint64_t*) { return set_error(BLS_ERR_INVALID, "serving not built"); }
bls_status bls_poll(bls_plan*, uint64_t, bls_peak*, int) { return set_error(BLS_ERR_INVALID, "serving not built"); }
bls_status bls_cancel(bls_plan*, uint64_t) { return set_error(BLS_ERR_INVALID, "serving not built"); }
bls_status bls_server_stats_get(bls_plan*, bls_server_stats*) { return set_error(BLS_ERR_INVALID, "serving not built"); }
}
