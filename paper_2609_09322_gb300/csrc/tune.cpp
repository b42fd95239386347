// tune.cpp -- autotuner of the march launch and of the volume layout.
//
// For one (grid, storage, epochs, image size, batch size, lookback) class the
// tuner times every candidate launch configuration (warp packet shape, warps
// per CTA, cells gathered ahead per lane) with CUDA events and, on request,
// every candidate brick / super-brick layout by re-packing the resident volume
// on the device.  The winner is cached in the context and used by render calls
// that pass no launch configuration; with GBD_TUNE_CACHE=<file> results are
// also appended to, and read back from, a text file.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

namespace gbd {

TuneKey tune_key(const Volume &vol, int width, int height, int n_views, uint32_t flags)
{
    TuneKey k;
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < 3; ++i) k.n[i] = vol.grid.n[i];
    k.M = vol.grid.n_epochs;
    k.store = vol.store;
    k.width = width;
    k.height = height;
    k.n_views = n_views;
    k.lookback = (flags & GBD_LOOKBACK) ? 1 : 0;
    return k;
}

namespace {

std::mutex g_file_mu;

std::string key_text(const TuneKey &k)
{
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d %d %d %d %d %d %d %d %d", k.n[0], k.n[1], k.n[2], k.M, k.store, k.width,
                  k.height, k.n_views, k.lookback);
    return buf;
}

void append_cache_file(const TuneKey &k, const TuneEntry &e)
{
    const char *path = std::getenv("GBD_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lock(g_file_mu);
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s -> %d %d %d %d %d %d %d %d %d %d %.6f\n", key_text(k).c_str(), e.cfg.packet_w,
                 e.cfg.packet_h, e.cfg.cta_warps, e.cfg.depth, e.cfg.persistent, e.cfg.regcap, e.cfg.region,
                 e.cfg.group, e.brick, e.super_brick, e.ms);
    std::fclose(f);
}

// Renders once with the given configuration; returns the elapsed time in ms
// (median of `reps` timed repetitions after one warm-up).
int time_config(Ctx &ctx, const Volume &vol, const std::vector<ViewDev> &hv, const gbd_image_spec &spec,
                const LaunchCfg &cfg, cudaStream_t st, int reps, float &ms_out)
{
    const int n = static_cast<int>(hv.size());
    char *scratch = nullptr;
    int nreg[3];
    const int slots = region_slots(vol, cfg, spec, nreg, n);
    const RegionPlan plan = slots > 0 ? region_plan(vol, cfg, spec, hv) : RegionPlan();
    const size_t qbytes = slots > 0 ? plan.total : (static_cast<size_t>(n) * sizeof(int) + 255) / 256 * 256;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), qbytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "tune scratch");
    if (slots > 0) e = upload_region_tables(plan, scratch, st);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    std::vector<float> times;
    auto args = std::make_unique<MarchArgs>();
    const int chunks = march_chunks(n);
    const std::vector<double> work = view_works(vol, hv, spec.width, spec.height);
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = slots > 0 ? cudaSuccess : cudaMemsetAsync(scratch, 0, qbytes, st);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        int launches = 0;
        if (slots > 0 && e == cudaSuccess)
            e = enqueue_regions(ctx, vol, hv, plan, spec, cfg, spec.out, scratch, st, &launches);
        for (int c = 0; c < chunks && e == cudaSuccess && slots == 0; ++c) {
            fill_args(*args, vol, hv.data(), n, c, spec, spec.out, nullptr, reinterpret_cast<int *>(scratch), cfg,
                      ctx.err_word);
            group_views(*args, cfg.group);
            if (cfg.persistent && launch_units(*args) == 1)
                args->tile_order = tile_order(ctx, spec.width, spec.height, cfg.packet_w, cfg.packet_h);
            e = launch_march(*args, cfg, ctx.num_sms, work.data() + static_cast<size_t>(c) * kViewsPerLaunch, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (r > 0) times.push_back(ms);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "tune launch");
    std::sort(times.begin(), times.end());
    ms_out = times[times.size() / 2];
    return GBD_OK;
}

}  // namespace

// Re-packs a volume into another brick / super-brick layout on the device.
// The handle keeps its identity; cached graphs of the volume are dropped
// because their kernel parameters point at the old records.
int relayout_volume(Ctx &ctx, Volume &vol, gbd_volume vid, int B, int S, int paired, int morton_cells)
{
    paired = paired ? 1 : 0;
    morton_cells = morton_cells ? 1 : 0;
    if (B == vol.brick && S == vol.super_brick && paired == vol.paired && morton_cells == vol.morton_cells)
        return GBD_OK;
    std::vector<int32_t> tab;
    long long cells = 0, stride = 0;
    if (!build_layout(vol.grid.n, B, S, tab, cells, morton_cells) || (paired && 2 * cells >= (1LL << 31)))
        return fail(GBD_ERR_INVALID, "layout too large");
    const size_t rec_bytes = vol.store == GBD_STORE_F32 ? 16 : 8;
    const size_t bytes = volume_bytes(vol.store, cells, vol.grid.n_epochs, paired, &stride);
    const size_t tab_bytes = tab.size() * sizeof(int32_t);
    if (ctx.used + bytes + tab_bytes > ctx.budget)
        return fail(GBD_ERR_BUDGET, "re-layout needs %zu more bytes", bytes + tab_bytes);
    void *rec = nullptr;
    int32_t *off = nullptr;
    cudaError_t e = cudaMalloc(&rec, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "re-layout allocation");
    e = cudaMalloc(reinterpret_cast<void **>(&off), tab_bytes);
    if (e != cudaSuccess) {
        cudaFree(rec);
        return cuda_fail(e, "re-layout table allocation");
    }
    cudaStream_t st = ctx.load_stream;
    // extra emissivity channels move with the records
    float *chan = nullptr;
    const long long cells_new = paired ? stride / 2 : stride;
    if (vol.chan) {
        e = cudaMalloc(reinterpret_cast<void **>(&chan), vol.chan_bytes / static_cast<uint64_t>(vol.chan_stride) *
                                                            static_cast<uint64_t>(cells_new));
        if (e != cudaSuccess) {
            cudaFree(rec);
            cudaFree(off);
            return cuda_fail(e, "re-layout channel allocation");
        }
    }
    e = cudaMemcpyAsync(off, tab.data(), tab_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, bytes, st);
    if (e == cudaSuccess && chan)
        e = cudaMemsetAsync(chan, 0, vol.chan_bytes / static_cast<uint64_t>(vol.chan_stride) * cells_new, st);
    for (int k = 0; k < vol.n_chan * vol.grid.n_epochs && e == cudaSuccess; ++k) {
        RelayoutArgs ra;
        std::memset(&ra, 0, sizeof(ra));
        ra.src = vol.chan + static_cast<size_t>(k) * vol.chan_stride;
        ra.dst = chan + static_cast<size_t>(k) * cells_new;
        ra.src_off = vol.axis_off;
        ra.dst_off = off;
        for (int i = 0; i < 3; ++i) ra.n[i] = vol.grid.n[i];
        ra.record_bytes = 4;
        e = launch_relayout(ra, st);
    }
    for (int m = 0; m < vol.grid.n_epochs && e == cudaSuccess; ++m) {
        RelayoutArgs ra;
        std::memset(&ra, 0, sizeof(ra));
        ra.src = vol.rec;
        ra.dst = rec;
        ra.src_stride = vol.epoch_stride;
        ra.dst_stride = stride;
        ra.src_paired = vol.paired;
        ra.dst_paired = paired;
        ra.m = m;
        ra.src_off = vol.axis_off;
        ra.dst_off = off;
        for (int i = 0; i < 3; ++i) ra.n[i] = vol.grid.n[i];
        ra.record_bytes = static_cast<int>(rec_bytes);
        e = launch_relayout(ra, st);
    }
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        cudaFree(rec);
        cudaFree(off);
        if (chan) cudaFree(chan);
        return cuda_fail(e, "re-layout");
    }
    drop_graphs_for(ctx, vid);
    cudaDeviceSynchronize();  // work on other streams may still read the old records
    cudaFree(vol.rec);
    cudaFree(vol.axis_off);
    ctx.used -= vol.bytes;
    vol.rec = rec;
    vol.axis_off = off;
    if (chan) {
        cudaFree(vol.chan);
        ctx.used -= vol.chan_bytes;
        vol.chan_bytes = vol.chan_bytes / static_cast<uint64_t>(vol.chan_stride) * cells_new;
        ctx.used += vol.chan_bytes;
        vol.chan = chan;
        vol.chan_stride = cells_new;
    }
    vol.epoch_stride = stride;
    vol.brick = B;
    vol.super_brick = S;
    vol.paired = paired;
    vol.morton_cells = morton_cells;
    vol.bytes = bytes + tab_bytes;
    ctx.used += vol.bytes;
    return GBD_OK;
}

bool lookup_tuned(Ctx &ctx, const TuneKey &k, LaunchCfg &cfg)
{
    auto it = ctx.tuned.find(k);
    if (it == ctx.tuned.end()) return false;
    cfg = it->second.cfg;
    return true;
}

void load_tune_file(Ctx &ctx)
{
    const char *path = std::getenv("GBD_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lock(g_file_mu);
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof(line), f)) {
        TuneKey k;
        std::memset(&k, 0, sizeof(k));
        TuneEntry e;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d -> %d %d %d %d %d %d %d %d %d %d %f", &k.n[0], &k.n[1],
                        &k.n[2], &k.M, &k.store, &k.width, &k.height, &k.n_views, &k.lookback, &e.cfg.packet_w,
                        &e.cfg.packet_h, &e.cfg.cta_warps, &e.cfg.depth, &e.cfg.persistent, &e.cfg.regcap,
                        &e.cfg.region, &e.cfg.group, &e.brick, &e.super_brick, &e.ms) == 20 &&
            check_launch(e.cfg) == GBD_OK)
            ctx.tuned[k] = e;  // later lines win
    }
    std::fclose(f);
}

}  // namespace gbd

using namespace gbd;

extern "C" {

int gbd_relayout(gbd_ctx *ctx, gbd_volume vid, int32_t brick, int32_t super_brick, int32_t paired,
                 int32_t morton_cells)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    if (brick != 1 && brick != 2 && brick != 4 && brick != 8) return fail(GBD_ERR_INVALID, "brick must be 1, 2, 4 or 8");
    if (super_brick != 1 && super_brick != 2 && super_brick != 4)
        return fail(GBD_ERR_INVALID, "super_brick must be 1, 2 or 4");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *v = ctx->find(vid);
    if (!v) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (v->pinned_by_requests.load() > 0) return fail(GBD_ERR_BUSY, "volume has queued requests");
    DeviceGuard guard(ctx->device);
    if (paired != 0 && paired != 1) return fail(GBD_ERR_INVALID, "paired must be 0 or 1");
    return relayout_volume(*ctx, *v, vid, brick, super_brick, paired, morton_cells);
}

int gbd_tune(gbd_ctx *ctx, gbd_volume vid, const gbd_view *views, int32_t n, const gbd_image_spec *spec,
             uint32_t what, void *stream, gbd_tune_result *out)
{
    if (!ctx || !views || !spec || !out) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    if (!spec->out || spec->out_on_host) return fail(GBD_ERR_INVALID, "tuning needs a device output buffer");
    if ((what & ~(GBD_TUNE_LAUNCH | GBD_TUNE_LAYOUT)) != 0u || what == 0u)
        return fail(GBD_ERR_INVALID, "what must combine GBD_TUNE_LAUNCH and GBD_TUNE_LAYOUT");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if ((what & GBD_TUNE_LAYOUT) && vol->pinned_by_requests.load() > 0) return fail(GBD_ERR_BUSY, "volume has queued requests");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    int rc;
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[k]))) return rc;

    const bool verbose = std::getenv("GBD_TUNE_VERBOSE") != nullptr;
    auto report = [&](const LaunchCfg &c, float ms, int B, int S) {
        if (verbose)
            std::fprintf(stderr,
                         "gbd_tune: packet %2dx%-2d warps %d depth %d persistent %d regcap %d region %d group %d "
                         "layout %d/%d: %.4f ms\n",
                         c.packet_w, c.packet_h, c.cta_warps, c.depth, c.persistent, c.regcap, c.region, c.group, B, S,
                         ms);
    };
    LaunchCfg best{8, 4, 8, 2, 1, 0, 0, kGroupDefault};
    float best_ms = 0.f;
    int tried = 0;
    if ((rc = time_config(*ctx, *vol, hv, *spec, best, st, 3, best_ms))) return rc;
    report(best, best_ms, vol->brick, vol->super_brick);
    ++tried;
    if (what & GBD_TUNE_LAUNCH) {
        const int packets[3][2] = {{8, 4}, {4, 8}, {16, 2}};
        const int warps[4] = {1, 2, 4, 8};
        const int depths[3] = {1, 2, 4};
        for (int cap = 0; cap < 2; ++cap)
            for (const auto &pk : packets)
                for (int w : warps)
                    for (int d : depths) {
                        LaunchCfg c{pk[0], pk[1], w, d, 1, cap, 0, kGroupDefault};
                        float ms = 0.f;
                        if ((rc = time_config(*ctx, *vol, hv, *spec, c, st, 3, ms))) return rc;
                        report(c, ms, vol->brick, vol->super_brick);
                        ++tried;
                        if (ms < best_ms) {
                            best_ms = ms;
                            best = c;
                        }
                    }
        LaunchCfg flat{8, 4, 8, 2, 0, 0, 0, kGroupDefault};
        float ms = 0.f;
        if ((rc = time_config(*ctx, *vol, hv, *spec, flat, st, 3, ms))) return rc;
        report(flat, ms, vol->brick, vol->super_brick);
        ++tried;
        if (ms < best_ms) {
            best_ms = ms;
            best = flat;
        }
        // region schedule, for batches of many views
        if (n >= 8) {
            const int regions[2] = {32, 64};
            const int rpackets[2][2] = {{8, 4}, {4, 8}};
            const int rwarps[2] = {4, 8};
            int nreg[3];
            for (int reg : regions)
                for (int cap = 0; cap < 2; ++cap)
                    for (const auto &pk : rpackets)
                        for (int w : rwarps)
                            for (int d = 1; d <= 2; ++d) {
                                LaunchCfg c{pk[0], pk[1], w, d, 0, cap, reg, kGroupDefault};
                                if (region_slots(*vol, c, *spec, nreg, n) == 0) continue;
                                // a region schedule whose scratch (partial slots and ray
                                // lists) would not fit in half the free memory is left out
                                size_t free_b = 0, total_b = 0;
                                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess ||
                                    region_plan(*vol, c, *spec, hv).total > free_b / 2)
                                    continue;
                                float rms = 0.f;
                                if ((rc = time_config(*ctx, *vol, hv, *spec, c, st, 3, rms))) return rc;
                                report(c, rms, vol->brick, vol->super_brick);
                                ++tried;
                                if (rms < best_ms) {
                                    best_ms = rms;
                                    best = c;
                                }
                            }
        }
        // time groups: up to kGroupDefault views per ray is the default;
        // none (1), smaller or larger groups are tried against it
        if (best.region == 0) {
            const LaunchCfg base = best;
            for (int gsz : {1, 2, kGroupMax}) {
                LaunchCfg c = base;
                c.group = gsz;
                float gms = 0.f;
                if ((rc = time_config(*ctx, *vol, hv, *spec, c, st, 3, gms))) return rc;
                report(c, gms, vol->brick, vol->super_brick);
                ++tried;
                if (gms < best_ms) {
                    best_ms = gms;
                    best = c;
                }
            }
        }
    }
    if (what & GBD_TUNE_LAYOUT) {
        // brick, super-brick, Morton cells
        const int layouts[9][3] = {{8, 4, 0}, {8, 2, 0}, {8, 1, 0}, {4, 4, 0}, {4, 2, 0}, {1, 1, 0},
                                   {8, 4, 1}, {4, 4, 1}, {4, 2, 1}};
        int bestB = vol->brick, bestS = vol->super_brick, bestP = vol->paired, bestZ = vol->morton_cells;
        for (int pair = 0; pair < 2; ++pair) {
            // the paired form is tried when two copies of it fit the budget
            long long cells = 0, stride = 0;
            std::vector<int32_t> tab;
            build_layout(vol->grid.n, 8, 4, tab, cells, 0);
            if (pair && (vol->grid.n_epochs < 2 ||
                         ctx->used + volume_bytes(vol->store, cells, vol->grid.n_epochs, 1, &stride) > ctx->budget))
                continue;
            for (const auto &ly : layouts) {
                if ((rc = relayout_volume(*ctx, *vol, vid, ly[0], ly[1], pair, ly[2]))) return rc;
                float ms = 0.f;
                if ((rc = time_config(*ctx, *vol, hv, *spec, best, st, 3, ms))) return rc;
                report(best, ms, ly[0], ly[1] + 10 * pair + 100 * ly[2]);
                ++tried;
                if (ms < best_ms) {
                    best_ms = ms;
                    bestB = ly[0];
                    bestS = ly[1];
                    bestP = pair;
                    bestZ = ly[2];
                }
            }
        }
        if ((rc = relayout_volume(*ctx, *vol, vid, bestB, bestS, bestP, bestZ))) return rc;
    }
    TuneEntry e;
    e.cfg = best;
    e.brick = vol->brick;
    e.super_brick = vol->super_brick;
    e.ms = best_ms;
    const TuneKey key = tune_key(*vol, spec->width, spec->height, n, views[0].flags);
    ctx->tuned[key] = e;
    append_cache_file(key, e);
    out->launch.packet_w = best.packet_w;
    out->launch.packet_h = best.packet_h;
    out->launch.cta_warps = best.cta_warps;
    out->launch.depth = best.depth;
    out->launch.persistent = best.persistent;
    out->launch.regcap = best.regcap;
    out->launch.region = best.region;
    out->launch.group = best.group;
    out->brick = vol->brick;
    out->super_brick = vol->super_brick;
    out->paired = vol->paired;
    out->morton_cells = vol->morton_cells;
    out->ms = best_ms;
    out->candidates = tried;
    return GBD_OK;
}

}  // extern "C"
