// Serving loop: continuous batching of point-source propagator requests.
//
// Requests (gauge field, kappa, csw, source, solver parameters) are queued by
// lqcd_serve_submit and admitted in arrival order whenever a slot is free
// and the HBM budget holds the request's clover field and solver workspace.
// Each slot is a host thread with its own CUDA stream; admitted requests run
// concurrently on the device (their kernels overlap across streams) and
// each one retires on its own as soon as its 12 columns have converged,
// releasing its slot and memory for the next arrival.  Device memory of a
// request is allocated stream-ordered (cudaMallocAsync / cudaFreeAsync), so
// admitting or retiring one request never synchronizes the others.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>

#include "lqcd_impl.h"

namespace lqcd {

struct ServeRequest {
    uint64_t ticket = 0;
    int gauge = -1;
    lqcd_dirac_params dp{};
    lqcd_solver_params sp{};
    int src[4] = {0, 0, 0, 0};
    double ts[4] = {0, 0, 0, 0};  // arrive, admit, start, finish
    size_t bytes = 0;
    bool done = false;
    int status = LQCD_EBUSY;
    std::string err;
    std::vector<double> corr;
    lqcd_solve_info info[12]{};
};

struct ServeGauge {
    lqcd_lattice_s *lat;
    GaugeSet *g;  // owned by lat; stable address
    size_t bytes;
};

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace lqcd

struct lqcd_server_s {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<lqcd::ServeRequest *> queue;
    std::map<uint64_t, std::unique_ptr<lqcd::ServeRequest>> reqs;
    uint64_t next_ticket = 1;
    std::map<std::vector<int>, lqcd_lattice_s *> lattices;
    std::vector<lqcd::ServeGauge> gauges;
    std::vector<std::thread> threads;
    volatile bool stop = false;
    int pollers = 0;  // lqcd_serve_poll calls in progress (destroy waits for them)
};

namespace lqcd {

static size_t request_bytes(const lqcd_lattice_s *lat, int prec, bool twisted)
{
    return workspace_bytes(lat, 12, prec) + clover_bytes(lat, twisted) + sizeof(double) * lat->dims[3];
}

static void run_request(lqcd_server_s *srv, ServeRequest *r, const ServeGauge &sg, cudaStream_t st)
{
    lqcd_lattice_s *lat = sg.lat;
    GaugeSet &g = *sg.g;
    const int T = lat->dims[3];
    try {
        auto cl = clover_build(lat, g, r->dp, st, true);
        auto ws = workspace_build(lat, 12, r->sp.precision, st, true);
        DevBuf corr;
        corr.set_async(st);
        corr.ensure(sizeof(double) * T);
        r->ts[2] = now_s();
        int failed = solve_on(lat, g, *cl, *ws, r->dp, r->sp, nullptr, nullptr, r->src, 12, r->info,
                              corr.as<double>(), st, &srv->stop);
        r->corr.assign(T, 0.0);
        LQCD_CUDA(cudaMemcpyAsync(r->corr.data(), corr.p, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
        corr.release();
        ws.reset();
        cl.reset();
        LQCD_CUDA(cudaStreamSynchronize(st));
        if (srv->stop) {
            r->status = LQCD_ETIMEOUT;
            r->err = "server stopped";
        } else {
            r->status = failed ? LQCD_ENOCONV : LQCD_OK;
            if (failed) r->err = std::to_string(failed) + " column(s) did not converge";
        }
    } catch (const Error &e) {
        r->status = e.code;
        r->err = e.msg;
        cudaStreamSynchronize(st);
    } catch (const std::bad_alloc &) {
        r->status = LQCD_ENOMEM;
        r->err = "host allocation failed";
    }
}

static void slot_main(lqcd_server_s *srv)
{
    cudaSetDevice(srv->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
        ServeRequest *r = nullptr;
        ServeGauge sg{};
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                return srv->stop || (!srv->queue.empty() && srv->used + srv->queue.front()->bytes <= srv->budget);
            });
            if (srv->stop) break;
            r = srv->queue.front();
            srv->queue.pop_front();
            srv->used += r->bytes;
            r->ts[1] = now_s();
            sg = srv->gauges[r->gauge];
        }
        if (st)
            run_request(srv, r, sg, st);
        else {
            r->status = LQCD_ECUDA;
            r->err = "could not create a CUDA stream";
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->used -= r->bytes;
            r->ts[3] = now_s();
            r->done = true;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_serve_create(int device, size_t hbm_budget_bytes, int max_slots, lqcd_server *out)
{
    if (!out) return fail(LQCD_EINVAL, "null argument");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return fail(LQCD_EINVAL, "max_slots must be in 1..64");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(LQCD_ECUDA, "no such CUDA device");
    try {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return fail(LQCD_ECUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
        auto *srv = new lqcd_server_s();
        srv->device = device;
        srv->budget = hbm_budget_bytes ? hbm_budget_bytes : size_t(0.9 * double(free_b));
        srv->max_slots = max_slots;
        for (int k = 0; k < max_slots; ++k) srv->threads.emplace_back(slot_main, srv);
        *out = srv;
        return LQCD_OK;
    } catch (const std::exception &) {
        return fail(LQCD_ENOMEM, "could not start the server threads");
    }
}

int lqcd_serve_gauge(lqcd_server srv, const int dims[4], const double *U, int *gauge_id)
{
    if (!srv || !dims || !U || !gauge_id) return fail(LQCD_EINVAL, "null argument");
    std::vector<int> key(dims, dims + 4);
    lqcd_lattice_s *lat = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->lattices.find(key);
        if (it != srv->lattices.end()) lat = it->second;
    }
    if (!lat) {
        lqcd_lattice h = nullptr;
        if (int rc = lqcd_lattice_create(dims, srv->device, &h)) return rc;
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->lattices.emplace(key, h);
        lat = h;
    }
    const size_t need = gauge_bytes(lat);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->used + need > srv->budget)
            return fail(LQCD_ENOMEM, "HBM budget too small for the gauge field (" + std::to_string(need) +
                                         " bytes needed, " + std::to_string(srv->budget - srv->used) + " left)");
        srv->used += need;
    }
    int local = -1;
    int rc = lqcd_gauge_upload(lat, U, &local);
    try {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(srv->device);
        lat->staging.release();  // the upload staging buffer is not kept by the server
        cudaSetDevice(prev);
    } catch (...) {
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (rc) {
        srv->used -= need;
        return rc;
    }
    GaugeSet *gs = nullptr;
    {
        std::lock_guard<std::mutex> llk(lat->mu);
        gs = lat->gauges.at(local).get();
    }
    srv->gauges.push_back(ServeGauge{lat, gs, need});
    *gauge_id = int(srv->gauges.size()) - 1;
    return LQCD_OK;
}

int lqcd_serve_submit(lqcd_server srv, int gauge_id, const lqcd_dirac_params *dp, const lqcd_solver_params *sp,
                      const int src[4], uint64_t *ticket)
{
    if (!srv || !dp || !sp || !src || !ticket) return fail(LQCD_EINVAL, "null argument");
    if (!(dp->kappa >= 0.0) || !std::isfinite(dp->csw) || !std::isfinite(dp->mu))
        return fail(LQCD_EINVAL, "bad dirac params");
    // SF requests would need the SF hopping links of the shared gauge field,
    // which the slots do not build concurrently
    if (dp->bc != LQCD_BC_PERIODIC && dp->bc != LQCD_BC_OPEN)
        return fail(LQCD_EINVAL, "served requests take periodic or open boundaries");
    if (dp->bc == LQCD_BC_OPEN && !std::isfinite(dp->cF)) return fail(LQCD_EINVAL, "bad dirac params");
    if (!(sp->tol > 0.0 && sp->tol < 1.0) || sp->maxiter < 1 || sp->precision < LQCD_PREC_FP64 ||
        sp->precision > LQCD_PREC_MIXED_FP16 || sp->inner_tol < 0.0 || sp->inner_tol >= 1.0)
        return fail(LQCD_EINVAL, "bad solver params");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (gauge_id < 0 || gauge_id >= int(srv->gauges.size())) return fail(LQCD_EINVAL, "unknown gauge id");
    const lqcd_lattice_s *lat = srv->gauges[gauge_id].lat;
    for (int m = 0; m < 4; ++m)
        if (src[m] < 0 || src[m] >= lat->dims[m]) return fail(LQCD_EINVAL, "source outside the lattice");
    auto r = std::make_unique<ServeRequest>();
    r->ticket = srv->next_ticket++;
    r->gauge = gauge_id;
    r->dp = *dp;
    r->sp = *sp;
    std::memcpy(r->src, src, sizeof r->src);
    r->bytes = request_bytes(lat, sp->precision, dp->mu != 0.0);
    size_t resident = 0;
    for (const ServeGauge &g : srv->gauges) resident += g.bytes;
    if (resident + r->bytes > srv->budget)
        return fail(LQCD_ENOMEM, "request needs " + std::to_string(r->bytes) + " bytes of HBM; the budget leaves " +
                                     std::to_string(srv->budget - std::min(srv->budget, resident)) +
                                     " beside the resident gauge fields");
    r->ts[0] = now_s();
    *ticket = r->ticket;
    srv->queue.push_back(r.get());
    srv->reqs.emplace(r->ticket, std::move(r));
    srv->cv_work.notify_all();
    return LQCD_OK;
}

int lqcd_serve_poll(lqcd_server srv, uint64_t ticket, double *corr, lqcd_solve_info *info, double timestamps[4],
                    int timeout_ms)
{
    if (!srv) return fail(LQCD_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    // counted while inside, so that lqcd_serve_destroy waits for this call to leave
    struct Inside {
        lqcd_server_s *s;
        Inside(lqcd_server_s *s_) : s(s_) { ++s->pollers; }
        ~Inside()
        {
            --s->pollers;
            s->cv_done.notify_all();
        }
    } inside(srv);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(LQCD_ENOTFOUND, "unknown ticket");
    ServeRequest *r = it->second.get();
    if (!r->done) {
        if (timeout_ms == 0) return LQCD_EBUSY;
        auto pred = [&] { return r->done; };
        if (timeout_ms < 0)
            srv->cv_done.wait(lk, pred);
        else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
            return fail(LQCD_ETIMEOUT, "request still pending after the timeout");
    }
    if (corr) std::copy(r->corr.begin(), r->corr.end(), corr);
    if (info) std::memcpy(info, r->info, sizeof r->info);
    if (timestamps) std::memcpy(timestamps, r->ts, sizeof r->ts);
    const int status = r->status;
    if (status != LQCD_OK) set_error(r->err);
    srv->reqs.erase(it);
    return status;
}

int lqcd_serve_destroy(lqcd_server srv)
{
    if (!srv) return LQCD_OK;
    {
        // queued requests will never run: they finish now, so that a poll
        // waiting on one of them returns instead of waiting forever
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        const double t = now_s();
        for (ServeRequest *r : srv->queue) {
            r->status = LQCD_ETIMEOUT;
            r->err = "server stopped";
            r->ts[1] = r->ts[2] = r->ts[3] = t;
            r->done = true;
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (auto &t : srv->threads) t.join();  // running requests stop at their next poll and finish
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->cv_done.wait(lk, [&] { return srv->pollers == 0; });
    }
    for (auto &kv : srv->lattices) lqcd_lattice_destroy(kv.second);
    delete srv;
    return LQCD_OK;
}

}  // extern "C"
