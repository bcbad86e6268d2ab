// The C ABI (include/lqcd.h): argument checks, host/device buffer handling,
// error reporting.  No call aborts: every failure becomes a status code with
// a thread-local message.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "lqcd_impl.h"

namespace lqcd {

static thread_local std::string g_error;

void set_error(const std::string &msg) { g_error = msg; }

int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

// Makes the lattice's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        LQCD_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

static int check_params(const lqcd_dirac_params *dp)
{
    if (!dp) return fail(LQCD_EINVAL, "null dirac params");
    if (!(dp->kappa >= 0.0) || !std::isfinite(dp->kappa)) return fail(LQCD_EINVAL, "kappa must be finite and >= 0");
    if (!std::isfinite(dp->csw)) return fail(LQCD_EINVAL, "csw must be finite");
    if (!std::isfinite(dp->mu)) return fail(LQCD_EINVAL, "mu must be finite");
    if (dp->bc != LQCD_BC_PERIODIC && dp->bc != LQCD_BC_OPEN && dp->bc != LQCD_BC_SF)
        return fail(LQCD_EINVAL, "unknown boundary condition");
    if (dp->bc != LQCD_BC_PERIODIC && !std::isfinite(dp->cF)) return fail(LQCD_EINVAL, "cF must be finite");
    if (dp->bc == LQCD_BC_SF && dp->mu != 0.0) return fail(LQCD_EINVAL, "SF boundaries are built for mu = 0");
    for (int m = 0; m < 4; ++m)
        if (!std::isfinite(dp->theta_re[m]) || !std::isfinite(dp->theta_im[m]))
            return fail(LQCD_EINVAL, "theta must be finite");
    return LQCD_OK;
}

static int check_solver(const lqcd_solver_params *sp)
{
    if (!sp) return fail(LQCD_EINVAL, "null solver params");
    if (!(sp->tol > 0.0) || !(sp->tol < 1.0)) return fail(LQCD_EINVAL, "tol must be in (0, 1)");
    if (sp->maxiter < 1) return fail(LQCD_EINVAL, "maxiter must be >= 1");
    if (sp->precision < LQCD_PREC_FP64 || sp->precision > LQCD_PREC_MIXED_FP16)
        return fail(LQCD_EINVAL, "unknown precision");
    if (sp->inner_tol < 0.0 || sp->inner_tol >= 1.0) return fail(LQCD_EINVAL, "inner_tol must be in [0, 1)");
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

#define API_TRY try {
#define API_CATCH                                                                                   \
    }                                                                                               \
    catch (const Error &e) { return fail(e.code, e.msg); }                                          \
    catch (const std::bad_alloc &) { return fail(LQCD_ENOMEM, "host allocation failed"); }          \
    catch (...) { return fail(LQCD_ECUDA, "unexpected exception"); }

extern "C" {

const char *lqcd_last_error(void) { return g_error.c_str(); }

int lqcd_abi_version(void) { return LQCD_ABI_VERSION; }

int lqcd_lattice_create(const int dims[4], int device, lqcd_lattice *out)
{
    if (!dims || !out) return fail(LQCD_EINVAL, "null argument");
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2 != 0)
            return fail(LQCD_EINVAL, "every extent must be even and >= 2 (even-odd preconditioning)");
        V *= dims[m];
        if (V > (1L << 40)) return fail(LQCD_EINVAL, "lattice too large");
    }
    if (V / 2 >= (1L << 31) / 24) return fail(LQCD_EINVAL, "lattice too large for 32-bit site indexing");
    API_TRY
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(LQCD_ECUDA, "no such CUDA device");
    DeviceGuard dg(device);
    auto *lat = new lqcd_lattice_s();
    std::memcpy(lat->dims, dims, sizeof lat->dims);
    lat->device = device;
    lat->V = V;
    lat->vh = V / 2;
    lat->stride = (lat->vh + 63) / 64 * 64;
    for (int m = 0; m < 4; ++m) lat->geom.L[m] = dims[m];
    lat->geom.Lxh = dims[0] / 2;
    lat->geom.vh = int(lat->vh);
    lat->geom.stride = lat->stride;
    *out = lat;
    return LQCD_OK;
    API_CATCH
}

int lqcd_lattice_destroy(lqcd_lattice lat)
{
    if (!lat) return LQCD_OK;
    API_TRY
    {
        DeviceGuard dg(lat->device);
        cudaDeviceSynchronize();
        delete lat;
    }
    return LQCD_OK;
    API_CATCH
}

int lqcd_gauge_upload(lqcd_lattice lat, const double *U, int *gauge_id)
{
    if (!lat || !U || !gauge_id) return fail(LQCD_EINVAL, "null argument");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    const size_t bytes = sizeof(double) * 72 * (size_t)lat->V;
    lat->staging.ensure(bytes);
    LQCD_CUDA(cudaMemcpy(lat->staging.p, U, bytes, cudaMemcpyHostToDevice));
    auto g = std::make_unique<GaugeSet>();
    gauge_repack(lat, *g, lat->staging.as<const double>(), 0);
    LQCD_CUDA(cudaDeviceSynchronize());
    int id = lat->next_gauge++;
    lat->gauges.emplace(id, std::move(g));
    *gauge_id = id;
    return LQCD_OK;
    API_CATCH
}

int lqcd_gauge_free(lqcd_lattice lat, int gauge_id)
{
    if (!lat) return fail(LQCD_EINVAL, "null lattice");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    LQCD_CUDA(cudaDeviceSynchronize());
    lat->gauges.erase(it);
    return LQCD_OK;
    API_CATCH
}

int lqcd_gauge_flow(lqcd_lattice lat, int gauge_id, double eps, int nsteps, void *stream)
{
    if (!lat) return fail(LQCD_EINVAL, "null lattice");
    if (!(eps > 0.0) || !std::isfinite(eps) || nsteps < 0) return fail(LQCD_EINVAL, "eps must be > 0, nsteps >= 0");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    gauge_flow(lat, *it->second, eps, nsteps, static_cast<cudaStream_t>(stream));
    return LQCD_OK;
    API_CATCH
}

int lqcd_fermion_flow(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, double *psi, int nrhs,
                      double eps, int nsteps, int flags, void *stream)
{
    if (!lat || !dp || !psi) return fail(LQCD_EINVAL, "null argument");
    if (!(eps > 0.0) || !std::isfinite(eps) || nsteps < 0) return fail(LQCD_EINVAL, "eps must be > 0, nsteps >= 0");
    if (nrhs < 1) return fail(LQCD_EINVAL, "nrhs must be >= 1");
    if (int rc = check_params(dp)) return rc;
    if (dp->bc != LQCD_BC_PERIODIC) return fail(LQCD_EINVAL, "the flow is built for periodic boundaries only");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * 24 * (size_t)lat->V * nrhs;
    double *d = psi;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, psi, bytes, cudaMemcpyHostToDevice, st));
        d = lat->staging.as<double>();
    }
    fermion_flow(lat, *it->second, *dp, d, nrhs, eps, nsteps, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(psi, d, bytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_fermion_backflow(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, double *eta, int nrhs,
                          double eps, int nsteps, int nsave, int flags, void *stream)
{
    if (!lat || !dp || !eta) return fail(LQCD_EINVAL, "null argument");
    if (!(eps > 0.0) || !std::isfinite(eps) || nsteps < 0) return fail(LQCD_EINVAL, "eps must be > 0, nsteps >= 0");
    if (nrhs < 1 || nsave < 1) return fail(LQCD_EINVAL, "nrhs and nsave must be >= 1");
    if (int rc = check_params(dp)) return rc;
    if (dp->bc != LQCD_BC_PERIODIC) return fail(LQCD_EINVAL, "the flow is built for periodic boundaries only");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * 24 * (size_t)lat->V * nrhs;
    double *d = eta;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, eta, bytes, cudaMemcpyHostToDevice, st));
        d = lat->staging.as<double>();
    }
    fermion_backflow(lat, *it->second, *dp, d, nrhs, eps, nsteps, nsave, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(eta, d, bytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_gauge_observables(lqcd_lattice lat, int gauge_id, double *plaq, double *Eplaq, double *Eclov, double *Q,
                           void *stream)
{
    if (!lat) return fail(LQCD_EINVAL, "null lattice");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = lat->dims[3];
    DevBuf out;
    out.ensure(sizeof(double) * 4 * T);
    gauge_observables(lat, *it->second, out.as<double>(), st);
    std::vector<double> h(4 * T);
    LQCD_CUDA(cudaMemcpyAsync(h.data(), out.p, sizeof(double) * 4 * T, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    if (plaq) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += h[t];
        *plaq = s / (6.0 * double(lat->V));
    }
    for (int t = 0; t < T; ++t) {
        if (Eplaq) Eplaq[t] = h[T + t];
        if (Eclov) Eclov[t] = h[2 * T + t];
        if (Q) Q[t] = h[3 * T + t];
    }
    return LQCD_OK;
    API_CATCH
}

int lqcd_hmc_trajectory(lqcd_lattice lat, int gauge_id, double beta, double eps, int nsteps, const double *mom,
                        double u, double *dH, int *accepted, void *stream)
{
    if (!lat || !mom || !dH || !accepted) return fail(LQCD_EINVAL, "null argument");
    if (!(beta > 0.0) || !std::isfinite(beta) || !(eps > 0.0) || !std::isfinite(eps) || nsteps < 1)
        return fail(LQCD_EINVAL, "beta and eps must be > 0, nsteps >= 1");
    if (!(u > 0.0 && u < 1.0)) return fail(LQCD_EINVAL, "u must be in (0, 1)");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * 32 * (size_t)lat->V;
    lat->staging.ensure(bytes);
    LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, mom, bytes, cudaMemcpyHostToDevice, st));
    *accepted = hmc_trajectory(lat, *it->second, beta, eps, nsteps, lat->staging.as<const double>(), u, dH, st);
    return LQCD_OK;
    API_CATCH
}

int lqcd_gauge_download(lqcd_lattice lat, int gauge_id, double *U, int flags, void *stream)
{
    if (!lat || !U) return fail(LQCD_EINVAL, "null argument");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * 72 * (size_t)lat->V;
    double *Ud = U;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        Ud = lat->staging.as<double>();
    }
    gauge_download(lat, *it->second, Ud, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(U, Ud, bytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_dirac_apply(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, const double *psi_in,
                     double *psi_out, int flags, void *stream)
{
    if (!lat || !psi_in || !psi_out) return fail(LQCD_EINVAL, "null argument");
    if (int rc = check_params(dp)) return rc;
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    const size_t bytes = sizeof(double) * 24 * (size_t)lat->V;
    const double *in = psi_in;
    double *out = psi_out;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        lat->staging2.ensure(bytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, psi_in, bytes, cudaMemcpyHostToDevice, st));
        in = lat->staging.as<const double>();
        out = lat->staging2.as<double>();
    }
    dirac_apply_dev(lat, *it->second, *dp, in, out, (flags & LQCD_DAG) != 0, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(psi_out, out, bytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_schur_apply(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, int precision, const double *in,
                     double *out, int nrhs, int repeat, int flags, void *stream)
{
    if (!lat || !in || !out) return fail(LQCD_EINVAL, "null argument");
    if (nrhs < 1 || repeat < 1) return fail(LQCD_EINVAL, "nrhs and repeat must be >= 1");
    if (precision < LQCD_PREC_FP64 || precision > LQCD_PREC_MIXED_FP16) return fail(LQCD_EINVAL, "unknown precision");
    if (int rc = check_params(dp)) return rc;
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto it = lat->gauges.find(gauge_id);
    if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
    const size_t bytes = sizeof(double) * 24 * (size_t)lat->V * nrhs;
    const double *id = in;
    double *od = out;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        lat->staging2.ensure(bytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, in, bytes, cudaMemcpyHostToDevice, st));
        id = lat->staging.as<const double>();
        od = lat->staging2.as<double>();
    }
    schur_apply_dev(lat, *it->second, *dp, precision, id, od, nrhs, repeat, (flags & LQCD_DAG) != 0, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(out, od, bytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_cg_solve(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, const lqcd_solver_params *sp,
                  const double *b, double *x, int nrhs, lqcd_solve_info *info, int flags, void *stream)
{
    if (!lat || !b || !x) return fail(LQCD_EINVAL, "null argument");
    if (nrhs < 1) return fail(LQCD_EINVAL, "nrhs must be >= 1");
    if (int rc = check_params(dp)) return rc;
    if (int rc = check_solver(sp)) return rc;
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * 24 * (size_t)lat->V * nrhs;
    const double *bd = b;
    double *xd = x;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(bytes);
        lat->staging2.ensure(bytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, b, bytes, cudaMemcpyHostToDevice, st));
        if (flags & LQCD_GUESS) LQCD_CUDA(cudaMemcpyAsync(lat->staging2.p, x, bytes, cudaMemcpyHostToDevice, st));
        bd = lat->staging.as<const double>();
        xd = lat->staging2.as<double>();
    }
    int failed = solve(lat, gauge_id, *dp, *sp, bd, xd, nullptr, nrhs, info, nullptr, st, (flags & LQCD_GUESS) != 0);
    if (!(flags & LQCD_DEVICE_PTRS)) {
        LQCD_CUDA(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, st));
        LQCD_CUDA(cudaStreamSynchronize(st));
    }
    if (failed) return fail(LQCD_ENOCONV, std::to_string(failed) + " right-hand side(s) did not converge");
    return LQCD_OK;
    API_CATCH
}

int lqcd_pion_corr(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, const lqcd_solver_params *sp,
                   const int src[4], double *corr, double *prop, lqcd_solve_info *info, int flags, void *stream)
{
    if (!lat || !src || !corr) return fail(LQCD_EINVAL, "null argument");
    for (int m = 0; m < 4; ++m)
        if (src[m] < 0 || src[m] >= lat->dims[m]) return fail(LQCD_EINVAL, "source outside the lattice");
    if (int rc = check_params(dp)) return rc;
    if (int rc = check_solver(sp)) return rc;
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = lat->dims[3];
    const size_t pbytes = sizeof(double) * 24 * (size_t)lat->V * 12;
    double *corr_d = corr, *prop_d = prop;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(sizeof(double) * T);
        corr_d = lat->staging.as<double>();
        if (prop) {
            lat->staging2.ensure(pbytes);
            prop_d = lat->staging2.as<double>();
        }
    }
    int failed = solve(lat, gauge_id, *dp, *sp, nullptr, prop_d, src, 12, info, corr_d, st);
    if (!(flags & LQCD_DEVICE_PTRS)) {
        LQCD_CUDA(cudaMemcpyAsync(corr, corr_d, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
        if (prop) LQCD_CUDA(cudaMemcpyAsync(prop, prop_d, pbytes, cudaMemcpyDeviceToHost, st));
        LQCD_CUDA(cudaStreamSynchronize(st));
    }
    if (failed) return fail(LQCD_ENOCONV, std::to_string(failed) + " column(s) did not converge");
    return LQCD_OK;
    API_CATCH
}

int lqcd_boundary_corr(lqcd_lattice lat, int gauge_id, const lqcd_dirac_params *dp, const lqcd_solver_params *sp,
                       double *fP, double *fA, double *H, lqcd_solve_info *info, int flags, void *stream)
{
    if (!lat || !fP || !fA) return fail(LQCD_EINVAL, "null argument");
    if (int rc = check_params(dp)) return rc;
    if (int rc = check_solver(sp)) return rc;
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = lat->dims[3];
    const size_t cbytes = sizeof(double) * 24 * (size_t)lat->V * 6;
    lat->staging.ensure(cbytes);  // the six wall sources
    double *H_d = H;
    if (!(flags & LQCD_DEVICE_PTRS) || !H) {
        lat->staging2.ensure(cbytes);
        H_d = lat->staging2.as<double>();
    }
    DevBuf fbuf;  // fP then fA on the device
    fbuf.ensure(sizeof(double) * 2 * T);
    double *f_d = fbuf.as<double>();
    if (dp->bc == LQCD_BC_SF) {
        auto it = lat->gauges.find(gauge_id);
        if (it == lat->gauges.end()) return fail(LQCD_EINVAL, "unknown gauge id");
        wall_sources_sf(lat, *it->second, lat->staging.as<double>(), st);
    } else {
        wall_sources_p_plus(lat, lat->staging.as<double>(), st);
    }
    int failed = solve(lat, gauge_id, *dp, *sp, lat->staging.as<const double>(), H_d, nullptr, 6, info, nullptr, st);
    const long nchunk = (lat->V / T + kBlock - 1) / kBlock;
    lat->red_partial.ensure(sizeof(double) * 2 * (size_t)T * nchunk);
    if (lat->red_counter.bytes < sizeof(unsigned) * (size_t)std::max(2 * T, 4096)) {
        lat->red_counter.ensure(sizeof(unsigned) * (size_t)std::max(2 * T, 4096));
        LQCD_CUDA(cudaMemsetAsync(lat->red_counter.p, 0, lat->red_counter.bytes, st));
    }
    boundary_contract(lat, H_d, f_d, f_d + T, lat->red_partial.as<double>(), lat->red_counter.as<unsigned>(), st);
    const cudaMemcpyKind k = (flags & LQCD_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LQCD_CUDA(cudaMemcpyAsync(fP, f_d, sizeof(double) * T, k, st));
    LQCD_CUDA(cudaMemcpyAsync(fA, f_d + T, sizeof(double) * T, k, st));
    if (H && !(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(H, H_d, cbytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    if (failed) return fail(LQCD_ENOCONV, std::to_string(failed) + " column(s) did not converge");
    return LQCD_OK;
    API_CATCH
}

int lqcd_pion_corr_batch(lqcd_pion_job *jobs, int njobs, const lqcd_solver_params *sp, int chunk, void *stream)
{
    if (!jobs || njobs < 1) return fail(LQCD_EINVAL, "no jobs");
    if (int rc = check_solver(sp)) return rc;
    if (chunk < 0 || chunk > 1024) return fail(LQCD_EINVAL, "chunk must be in 0..1024");
    std::vector<lqcd_lattice_s *> lats;
    for (int k = 0; k < njobs; ++k) {
        const lqcd_pion_job &j = jobs[k];
        if (!j.lat || !j.corr) return fail(LQCD_EINVAL, "null lattice or corr in job " + std::to_string(k));
        if (int rc = check_params(&j.dp)) return rc;
        for (int m = 0; m < 4; ++m)
            if (j.src[m] < 0 || j.src[m] >= j.lat->dims[m])
                return fail(LQCD_EINVAL, "source outside the lattice in job " + std::to_string(k));
        if (j.lat->device != jobs[0].lat->device) return fail(LQCD_EINVAL, "all jobs must use the same device");
        lats.push_back(j.lat);
    }
    std::sort(lats.begin(), lats.end());
    lats.erase(std::unique(lats.begin(), lats.end()), lats.end());
    API_TRY
    std::vector<std::unique_lock<std::mutex>> locks;
    for (lqcd_lattice_s *l : lats) locks.emplace_back(l->mu);  // address order: no lock-order inversion
    DeviceGuard dg(jobs[0].lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t origin = nullptr;
    LQCD_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    int failed = 0;
    try {
        LQCD_CUDA(cudaStreamSynchronize(st));
        failed = pion_batch(jobs, njobs, *sp, chunk ? chunk : 8, origin);
    } catch (...) {
        cudaStreamDestroy(origin);
        throw;
    }
    cudaStreamDestroy(origin);
    if (failed) return fail(LQCD_ENOCONV, std::to_string(failed) + " job(s) had a column that did not converge");
    return LQCD_OK;
    API_CATCH
}

int lqcd_pion_contract(lqcd_lattice lat, const double *prop, int src_t, double *corr, int flags, void *stream)
{
    if (!lat || !prop || !corr) return fail(LQCD_EINVAL, "null argument");
    if (src_t < 0 || src_t >= lat->dims[3]) return fail(LQCD_EINVAL, "source time outside the lattice");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = lat->dims[3];
    const size_t pbytes = sizeof(double) * 24 * (size_t)lat->V * 12;
    const double *pd = prop;
    double *cd = corr;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(pbytes);
        lat->staging2.ensure(sizeof(double) * T);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, prop, pbytes, cudaMemcpyHostToDevice, st));
        pd = lat->staging.as<const double>();
        cd = lat->staging2.as<double>();
    }
    const long nchunk = (lat->V / T * 12 + kBlock * 4 - 1) / (kBlock * 4);
    lat->red_partial.ensure(sizeof(double) * (size_t)T * nchunk);
    if (lat->red_counter.bytes < sizeof(unsigned) * (size_t)std::max(T, 4096)) {
        lat->red_counter.ensure(sizeof(unsigned) * (size_t)std::max(T, 4096));
        LQCD_CUDA(cudaMemsetAsync(lat->red_counter.p, 0, lat->red_counter.bytes, st));
    }
    pion_contract_aos(lat, pd, src_t, cd, lat->red_partial.as<double>(), lat->red_counter.as<unsigned>(), st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(corr, cd, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

int lqcd_meson_contract(lqcd_lattice lat, const double *prop, int src_t, const double *gammas, int ng, double *corr,
                        int flags, void *stream)
{
    if (!lat || !prop || !gammas || !corr) return fail(LQCD_EINVAL, "null argument");
    if (src_t < 0 || src_t >= lat->dims[3]) return fail(LQCD_EINVAL, "source time outside the lattice");
    if (ng < 1 || ng > LQCD_MESON_MAX_GAMMAS) return fail(LQCD_EINVAL, "ng must be in 1..LQCD_MESON_MAX_GAMMAS");
    for (int k = 0; k < 32 * ng; ++k)
        if (!std::isfinite(gammas[k])) return fail(LQCD_EINVAL, "gammas must be finite");
    API_TRY
    std::lock_guard<std::mutex> lk(lat->mu);
    DeviceGuard dg(lat->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = lat->dims[3];
    const size_t pbytes = sizeof(double) * 24 * (size_t)lat->V * 12;
    const size_t cbytes = sizeof(double) * 2 * (size_t)ng * T;
    const double *pd = prop;
    double *cd = corr;
    if (!(flags & LQCD_DEVICE_PTRS)) {
        lat->staging.ensure(pbytes);
        lat->staging2.ensure(cbytes);
        LQCD_CUDA(cudaMemcpyAsync(lat->staging.p, prop, pbytes, cudaMemcpyHostToDevice, st));
        pd = lat->staging.as<const double>();
        cd = lat->staging2.as<double>();
    }
    meson_contract(lat, pd, src_t, gammas, ng, cd, st);
    if (!(flags & LQCD_DEVICE_PTRS)) LQCD_CUDA(cudaMemcpyAsync(corr, cd, cbytes, cudaMemcpyDeviceToHost, st));
    LQCD_CUDA(cudaStreamSynchronize(st));
    return LQCD_OK;
    API_CATCH
}

}  // extern "C"
