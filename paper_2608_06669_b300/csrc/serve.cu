// Continuous-batching server (placeholder until the scheduler lands).
#include "common.h"

extern "C" {
int cc_server_create(cc_server** srv, int, size_t, int) { if (srv) *srv = nullptr; return CC_ERR_INVALID; }
void cc_server_destroy(cc_server*) {}
int cc_serve_submit(cc_server*, int, int, int, const double*, const double*, const cc_solve_opts*, uint64_t*) { return CC_ERR_INVALID; }
int cc_serve_poll(cc_server*, uint64_t, cc_report*, double*, double*) { return CC_ERR_INVALID; }
int cc_serve_times(cc_server*, uint64_t, double*, double*, double*) { return CC_ERR_INVALID; }
}
