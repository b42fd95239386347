// serve.cpp -- continuous-batching render server.
//
// Requests (one view of one resident volume, any image size, any storage)
// are queued by gbd_submit.  A scheduler thread admits queued requests into
// waves as request slots and HBM budget free up, and launches each wave as
// multi-request kernels (wave_kernel in march.cu, up to kReqsPerLaunch
// requests per launch) on one of several streams.  Up to `max_waves` waves are on the GPU at once, so a wave formed
// from requests that arrived while earlier ones were running starts filling
// SMs as soon as the earlier wave's tail drains.  Completion is signalled by a
// host-function callback; waiting is always bounded by the caller's timeout
// and no device code ever waits on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

namespace gbd {
namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct ServedReq {
    uint64_t ticket = 0;
    uint64_t seq = 0;
    gbd_volume vid = 0;
    Volume *vol = nullptr;     // pinned while the request is queued or running
    VolDev vdev{};
    ViewDev view{};
    gbd_image_spec spec{};
    int32_t priority = 0;
    uint64_t bytes = 0;        // device bytes its image (and counts) occupy while it runs
    int state = kPending;
    int status = GBD_OK;
    bool cancel_requested = false;
    double t_submit = 0, t_launch = 0, t_done = 0;
    float device_ms = 0.f;
    uint64_t cells = 0;        // n_x n_y n_z M of its volume (for statistics)
};

struct WaveSlot {
    Server *server = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    WaveArgs *args = nullptr;  // launch arguments (about 30 KB), reused per launch
    std::vector<uint64_t> tickets;
    std::atomic<bool> gpu_done{false};
    double t_gpu_done = 0;
    bool busy = false;
};

}  // namespace

struct Server {
    Ctx *ctx = nullptr;
    int device = 0;
    gbd_serve_config cfg{};
    LaunchCfg launch{8, 4, 8, 1, 1, 0, 0, 1};
    uint64_t request_budget = 0;
    std::mutex mu;
    std::condition_variable cv;       // wakes the scheduler
    std::condition_variable done_cv;  // wakes waiters
    std::thread thread;
    bool stop = false;
    std::map<uint64_t, ServedReq> reqs;
    uint64_t next_ticket = 0, next_seq = 0;
    std::vector<WaveSlot *> slots;
    uint64_t in_flight_bytes = 0;
    int in_flight_reqs = 0;
    int pending = 0;
    // statistics since the last reset
    std::vector<double> latencies_ms;
    uint64_t completed = 0, waves = 0, wave_requests = 0;
    int max_waves_seen = 0;
    double t_first_submit = 0, t_last_done = 0;

    void run();
    void retire(WaveSlot &w);
    bool launch_wave_from_queue(WaveSlot &w);
};

namespace {

void CUDART_CB on_wave_done(void *p)
{
    // Runs on a CUDA callback thread: no CUDA calls here.
    WaveSlot *w = static_cast<WaveSlot *>(p);
    Server *s = w->server;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        w->t_gpu_done = now_s();
        w->gpu_done.store(true);
    }
    s->cv.notify_all();
}

bool terminal(int state) { return state == kDone || state == kCancelled || state == kFailed; }

void fill_stats(const ServedReq &r, gbd_stats *st)
{
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->status = r.status;
    st->queue_ms = r.t_launch > 0 ? (r.t_launch - r.t_submit) * 1e3 : 0.0;
    st->latency_ms = terminal(r.state) && r.t_done > 0 ? (r.t_done - r.t_submit) * 1e3 : 0.0;
    st->device_ms = r.device_ms;
}

}  // namespace

void Server::retire(WaveSlot &w)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.ev_start, w.ev_stop);
    for (uint64_t t : w.tickets) {
        auto it = reqs.find(t);
        if (it == reqs.end()) continue;
        ServedReq &r = it->second;
        r.t_done = w.t_gpu_done;
        r.device_ms = ms;
        if (r.cancel_requested) {
            r.state = kCancelled;
            r.status = GBD_ERR_CANCELLED;
        } else {
            r.state = kDone;
            r.status = GBD_OK;
            latencies_ms.push_back((r.t_done - r.t_submit) * 1e3);
            ++completed;
            t_last_done = std::max(t_last_done, r.t_done);
        }
        in_flight_bytes -= r.bytes;
        --in_flight_reqs;
        r.vol->pinned_by_requests.fetch_sub(1);
    }
    w.tickets.clear();
    w.busy = false;
    w.gpu_done.store(false);
    done_cv.notify_all();
}

// Forms one wave from the queue (priority first, then arrival order) within
// the wave size, the request slots and the request memory budget, and
// launches it.  Returns false if nothing could be admitted.
bool Server::launch_wave_from_queue(WaveSlot &w)
{
    std::vector<ServedReq *> cand;
    for (auto &kv : reqs)
        if (kv.second.state == kPending) cand.push_back(&kv.second);
    if (cand.empty()) return false;
    std::sort(cand.begin(), cand.end(), [](const ServedReq *a, const ServedReq *b) {
        return a->priority != b->priority ? a->priority > b->priority : a->seq < b->seq;
    });
    std::vector<ServedReq *> take;
    uint64_t bytes = 0;
    for (ServedReq *r : cand) {
        if (static_cast<int>(take.size()) >= cfg.max_requests_per_wave) break;
        if (in_flight_reqs + static_cast<int>(take.size()) >= cfg.max_requests_in_flight) break;
        if (in_flight_bytes + bytes + r->bytes > request_budget) break;  // keep arrival order under memory pressure
        if (fault_injected("admit")) {
            r->state = kFailed;
            r->status = GBD_ERR_NOMEM;
            r->t_done = now_s();
            r->vol->pinned_by_requests.fetch_sub(1);
            --pending;
            done_cv.notify_all();
            continue;
        }
        take.push_back(r);
        bytes += r->bytes;
    }
    if (take.empty()) return false;

    // Request table; images of host-output requests go to one device buffer
    // allocated in stream order (released after their copy back).
    uint64_t host_img_bytes = 0;
    for (ServedReq *r : take)
        if (r->spec.out_on_host) host_img_bytes += static_cast<uint64_t>(r->spec.width) * r->spec.height * 4;
    char *d_img = nullptr;
    cudaError_t e = cudaSuccess;
    if (host_img_bytes) e = cudaMallocAsync(reinterpret_cast<void **>(&d_img), host_img_bytes, w.stream);
    uint64_t img_off = 0;
    std::vector<uint64_t> host_off(take.size(), 0);
    if (e == cudaSuccess) e = cudaEventRecord(w.ev_start, w.stream);
    for (size_t first = 0; first < take.size() && e == cudaSuccess; first += kReqsPerLaunch) {
        const size_t cnt = std::min<size_t>(kReqsPerLaunch, take.size() - first);
        WaveArgs &a = *w.args;
        std::memset(&a, 0, sizeof(a));
        int cta_begin = 0;
        for (size_t i = 0; i < cnt; ++i) {
            ServedReq &r = *take[first + i];
            ReqDev &d = a.reqs[i];
            d.vol = r.vdev;
            d.view = r.view;
            d.width = r.spec.width;
            d.height = r.spec.height;
            d.tiles_x = (r.spec.width + launch.packet_w - 1) / launch.packet_w;
            d.tiles_y = (r.spec.height + launch.packet_h - 1) / launch.packet_h;
            d.cta_begin = cta_begin;
            cta_begin += (d.tiles_x * d.tiles_y + launch.cta_warps - 1) / launch.cta_warps;
            if (r.spec.out_on_host) {
                d.out = reinterpret_cast<float *>(d_img + img_off);
                host_off[first + i] = img_off;
                img_off += static_cast<uint64_t>(r.spec.width) * r.spec.height * 4;
            } else {
                d.out = r.spec.out;
                d.samples = r.spec.samples;
            }
        }
        a.n_reqs = static_cast<int>(cnt);
        a.packet_w = launch.packet_w;
        a.packet_h = launch.packet_h;
        a.total_ctas = cta_begin;
        a.error_word = ctx->err_word;
        e = launch_wave(a, launch, w.stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(w.ev_stop, w.stream);
    for (size_t i = 0; i < take.size() && e == cudaSuccess; ++i) {
        ServedReq &r = *take[i];
        if (r.spec.out_on_host)
            e = cudaMemcpyAsync(r.spec.out, d_img + host_off[i],
                                static_cast<size_t>(r.spec.width) * r.spec.height * 4, cudaMemcpyDeviceToHost,
                                w.stream);
    }
    if (d_img) cudaFreeAsync(d_img, w.stream);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(w.stream, on_wave_done, &w);
    const double t = now_s();
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (ServedReq *r : take) {
            r->state = kFailed;
            r->status = GBD_ERR_CUDA;
            r->t_done = t;
            r->vol->pinned_by_requests.fetch_sub(1);
            --pending;
        }
        done_cv.notify_all();
        return true;
    }
    w.busy = true;
    w.tickets.clear();
    for (ServedReq *r : take) {
        r->state = kRunning;
        r->t_launch = t;
        w.tickets.push_back(r->ticket);
        in_flight_bytes += r->bytes;
        ++in_flight_reqs;
        --pending;
    }
    ++waves;
    wave_requests += take.size();
    int busy = 0;
    for (WaveSlot *s : slots) busy += s->busy ? 1 : 0;
    max_waves_seen = std::max(max_waves_seen, busy);
    return true;
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        bool any_busy = false;
        for (WaveSlot *w : slots) {
            if (w->busy && w->gpu_done.load()) retire(*w);
            any_busy |= w->busy;
        }
        if (stop && !any_busy && pending == 0) break;
        bool launched = false;
        if (pending > 0) {
            for (WaveSlot *w : slots) {
                if (!w->busy) {
                    launched = launch_wave_from_queue(*w);
                    break;
                }
            }
        }
        if (launched) continue;
        cv.wait_for(lock, std::chrono::milliseconds(2));
    }
}

int serve_start(Ctx &ctx, const gbd_serve_config *c)
{
    if (ctx.server) return GBD_OK;
    auto s = std::make_unique<Server>();
    s->ctx = &ctx;
    s->device = ctx.device;
    gbd_serve_config d{};
    d.max_waves = 3;
    d.max_requests_per_wave = 256;
    d.max_requests_in_flight = 1024;
    d.request_budget_bytes = 0;
    if (c) {
        if (c->max_waves > 0) d.max_waves = c->max_waves;
        if (c->max_requests_per_wave > 0) d.max_requests_per_wave = c->max_requests_per_wave;
        if (c->max_requests_in_flight > 0) d.max_requests_in_flight = c->max_requests_in_flight;
        d.request_budget_bytes = c->request_budget_bytes;
        d.launch = c->launch;
    }
    if (d.max_waves > 8 || d.max_requests_per_wave > 4096)
        return fail(GBD_ERR_INVALID, "serve: at most 8 waves of at most 4096 requests");
    s->cfg = d;
    LaunchCfg lc = resolve_launch(c ? &d.launch : nullptr);
    const gbd_launch &ul = d.launch;
    if (ul.packet_w == 0 && ul.packet_h == 0 && ul.cta_warps == 0 && ul.depth == 0 && ul.regcap == 0) {
        // launch left unset: the shape the tuner picks for batches (small
        // CTAs, two cells ahead, the capped register budget)
        lc.cta_warps = 4;
        lc.depth = 2;
        lc.regcap = 1;
    }
    if (lc.depth > 2) lc.depth = 2;
    lc.persistent = 1;
    lc.region = 0;  // waves march whole rays
    int rc = check_launch(lc);
    if (rc) return rc;
    s->launch = lc;
    const uint64_t free_budget = ctx.budget > ctx.used ? ctx.budget - ctx.used : 0;
    s->request_budget = d.request_budget_bytes ? std::min<uint64_t>(d.request_budget_bytes, free_budget) : free_budget;
    for (int i = 0; i < d.max_waves; ++i) {
        auto *w = new WaveSlot();
        w->server = s.get();
        w->index = i;
        s->slots.push_back(w);
        cudaError_t e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&w->ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&w->ev_stop);
        w->args = new WaveArgs();
        if (e != cudaSuccess) {
            ctx.server = s.release();
            serve_shutdown(ctx);
            return cuda_fail(e, "serve start");
        }
    }
    Server *raw = s.get();
    s->thread = std::thread([raw]() { raw->run(); });
    ctx.server = s.release();
    return GBD_OK;
}

void serve_shutdown(Ctx &ctx)
{
    Server *s = ctx.server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        // queued requests that never started are cancelled; running ones drain
        for (auto &kv : s->reqs) {
            ServedReq &r = kv.second;
            if (r.state == kPending) {
                r.state = kCancelled;
                r.status = GBD_ERR_CANCELLED;
                r.vol->pinned_by_requests.fetch_sub(1);
                --s->pending;
            }
        }
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->thread.joinable()) s->thread.join();
    for (WaveSlot *w : s->slots) {
        if (w->stream) cudaStreamSynchronize(w->stream);
        if (w->ev_start) cudaEventDestroy(w->ev_start);
        if (w->ev_stop) cudaEventDestroy(w->ev_stop);
        delete w->args;
        if (w->stream) cudaStreamDestroy(w->stream);
        delete w;
    }
    s->done_cv.notify_all();
    delete s;
    ctx.server = nullptr;
}

}  // namespace gbd

using namespace gbd;

extern "C" {

int gbd_serve_start(gbd_ctx *ctx, const gbd_serve_config *config)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    return serve_start(*ctx, config);
}

int gbd_serve_stop(gbd_ctx *ctx)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    serve_shutdown(*ctx);
    return GBD_OK;
}

int gbd_submit(gbd_ctx *ctx, const gbd_request *req, uint64_t *ticket)
{
    if (!ctx || !req || !ticket) return fail(GBD_ERR_INVALID, "NULL argument");
    *ticket = 0;
    const gbd_image_spec &sp = req->spec;
    if (sp.width < 1 || sp.height < 1 || sp.width > 16384 || sp.height > 16384)
        return fail(GBD_ERR_INVALID, "image: width/height must be in [1, 16384]");
    if (!sp.out) return fail(GBD_ERR_INVALID, "image: out is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    int rc;
    if (!ctx->server && (rc = serve_start(*ctx, nullptr))) return rc;
    Server &s = *ctx->server;
    Volume *vol = ctx->find(req->volume);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(req->volume));
    if (sp.out_on_host) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, sp.out) != cudaSuccess || attr.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(GBD_ERR_INVALID, "serving needs device output or pinned (page-locked) host output");
        }
    }
    ServedReq r;
    if ((rc = make_view(*vol, req->view, sp.width, sp.height, sp.fov_u, sp.fov_v, r.view))) return rc;
    // A running request's HBM footprint is the image it writes: a device
    // buffer of the library's when the output is host memory, the caller's own
    // buffer (and its sample counts) when it is device memory.
    const uint64_t img_bytes = static_cast<uint64_t>(sp.width) * sp.height * 4;
    r.bytes = img_bytes + (!sp.out_on_host && sp.samples ? img_bytes : 0);
    if (r.bytes > s.request_budget)
        return fail(GBD_ERR_BUDGET, "request needs %llu device bytes, the serving budget is %llu",
                    static_cast<unsigned long long>(r.bytes), static_cast<unsigned long long>(s.request_budget));
    r.vid = req->volume;
    r.vol = vol;
    r.vdev = vol_dev(*vol);
    r.spec = sp;
    if (sp.out_on_host) r.spec.samples = nullptr;
    r.priority = req->priority;
    r.cells = static_cast<uint64_t>(vol->grid.n[0]) * vol->grid.n[1] * vol->grid.n[2] * vol->grid.n_epochs;
    vol->pinned_by_requests.fetch_add(1);
    {
        std::lock_guard<std::mutex> sl(s.mu);
        r.ticket = ++s.next_ticket;
        r.seq = ++s.next_seq;
        r.t_submit = now_s();
        if (s.t_first_submit == 0) s.t_first_submit = r.t_submit;
        *ticket = r.ticket;
        s.reqs[r.ticket] = r;
        ++s.pending;
    }
    s.cv.notify_all();
    return GBD_OK;
}

int gbd_poll(gbd_ctx *ctx, uint64_t ticket, int32_t *done, gbd_stats *st)
{
    if (!ctx || !done) return fail(GBD_ERR_INVALID, "NULL argument");
    *done = 0;
    Server *s = ctx->server;
    if (!s) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    fill_stats(it->second, st);
    if (!terminal(it->second.state)) return GBD_OK;
    *done = 1;
    const int status = it->second.status;
    s->reqs.erase(it);  // a finished request is reported once
    return status == GBD_OK ? GBD_OK : fail(status, "request %llu ended with status %d",
                                            static_cast<unsigned long long>(ticket), status);
}

int gbd_wait(gbd_ctx *ctx, uint64_t ticket, uint32_t timeout_ms, gbd_stats *st)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    Server *s = ctx->server;
    if (!s) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    const bool ok = s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&]() {
        auto j = s->reqs.find(ticket);
        return j == s->reqs.end() || terminal(j->second.state);
    });
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GBD_ERR_NOTFOUND, "request %llu was already reported", static_cast<unsigned long long>(ticket));
    fill_stats(it->second, st);
    if (!ok) return fail(GBD_ERR_TIMEOUT, "request %llu not finished after %u ms", static_cast<unsigned long long>(ticket), timeout_ms);
    const int status = it->second.status;
    s->reqs.erase(it);
    return status == GBD_OK ? GBD_OK : fail(status, "request %llu ended with status %d",
                                            static_cast<unsigned long long>(ticket), status);
}

int gbd_cancel(gbd_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    Server *s = ctx->server;
    if (!s) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(GBD_ERR_NOTFOUND, "no request %llu", static_cast<unsigned long long>(ticket));
        ServedReq &r = it->second;
        if (r.state == kPending) {
            r.state = kCancelled;
            r.status = GBD_ERR_CANCELLED;
            r.t_done = now_s();
            r.vol->pinned_by_requests.fetch_sub(1);
            --s->pending;
        } else if (r.state == kRunning) {
            r.cancel_requested = true;  // its GPU work drains; the result is discarded
        }
    }
    s->done_cv.notify_all();
    return GBD_OK;
}

int gbd_serve_stats(gbd_ctx *ctx, int32_t reset, gbd_serve_summary *out)
{
    if (!ctx || !out) return fail(GBD_ERR_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    Server *s = ctx->server;
    if (!s) return GBD_OK;
    std::lock_guard<std::mutex> lock(s->mu);
    std::vector<double> l = s->latencies_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, static_cast<size_t>(q * (l.size() - 1) + 0.5))]; };
    out->completed = s->completed;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.empty() ? 0.0 : l.back();
    out->waves = s->waves;
    out->mean_requests_per_wave = s->waves ? static_cast<double>(s->wave_requests) / s->waves : 0.0;
    out->max_waves_in_flight = s->max_waves_seen;
    const double span = s->t_last_done - s->t_first_submit;
    out->requests_per_s = span > 0 ? s->completed / span : 0.0;
    out->pending = s->pending;
    out->in_flight = s->in_flight_reqs;
    if (reset) {
        s->latencies_ms.clear();
        s->completed = s->waves = s->wave_requests = 0;
        s->max_waves_seen = 0;
        s->t_first_submit = s->t_last_done = 0;
    }
    return GBD_OK;
}

}  // extern "C"
