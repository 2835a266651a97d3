// Link stand-ins for the solver entry points the request server calls in
// its GPU mode, so that the server (csrc/server.cu) can be built alone for
// the host sanitizers. A server made by trm_server_create_fn never calls
// them; each returns an error if it ever is.
#include <string>

#include "solver.cuh"

namespace trm {
void set_global_error(const std::string&) {}
size_t Solver::footprint(int64_t N, int m) { return (size_t)N * m * 92; }
}  // namespace trm

extern "C" {
trm_status trm_create_stencil(trm_handle*, int, int, int, int, double,
                              const double*, int, double,
                              const trm_options*) {
  return TRM_ECUDA;
}
trm_status trm_solve(trm_handle, double*, double*, double*, int,
                     const double*, trm_stats*) {
  return TRM_ECUDA;
}
trm_status trm_destroy(trm_handle) { return TRM_OK; }
const char* trm_last_error(trm_handle) { return "stub"; }
const char* trm_last_global_error(void) { return "stub"; }
}
