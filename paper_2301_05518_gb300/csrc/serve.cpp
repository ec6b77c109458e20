// serve.cpp -- continuous-batching server (placeholder until the scheduler lands).
#include "api_internal.h"

namespace tls {
void serve_shutdown(tls_ctx *) {}
}  // namespace tls

using namespace tls;

extern "C" {
tls_status tls_serve_start(tls_ctx *, const tls_serve_opts *) { return fail(TLS_ERR_UNSUPPORTED, "serving not built"); }
tls_status tls_serve_stop(tls_ctx *) { return fail(TLS_ERR_UNSUPPORTED, "serving not built"); }
tls_status tls_serve_submit(tls_ctx *, const tls_job *, uint64_t *) { return fail(TLS_ERR_UNSUPPORTED, "serving not built"); }
tls_status tls_serve_poll(tls_ctx *, uint64_t, int *) { return fail(TLS_ERR_UNSUPPORTED, "serving not built"); }
tls_status tls_serve_wait(tls_ctx *, uint64_t, double, tls_job_result *) { return fail(TLS_ERR_UNSUPPORTED, "serving not built"); }
}
