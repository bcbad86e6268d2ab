// Serving loop (continuous batching of propagator requests).
#include "lqcd_impl.h"

using namespace lqcd;

extern "C" {

int lqcd_serve_create(int, size_t, int, lqcd_server *out)
{
    if (out) *out = nullptr;
    return fail(LQCD_ENOTIMPL, "serving loop not built yet");
}
int lqcd_serve_gauge(lqcd_server, const int *, const double *, int *) { return fail(LQCD_ENOTIMPL, "serving loop not built yet"); }
int lqcd_serve_submit(lqcd_server, int, const lqcd_dirac_params *, const lqcd_solver_params *, const int *, uint64_t *)
{
    return fail(LQCD_ENOTIMPL, "serving loop not built yet");
}
int lqcd_serve_poll(lqcd_server, uint64_t, double *, lqcd_solve_info *, double *, int)
{
    return fail(LQCD_ENOTIMPL, "serving loop not built yet");
}
int lqcd_serve_destroy(lqcd_server) { return LQCD_OK; }

}  // extern "C"
