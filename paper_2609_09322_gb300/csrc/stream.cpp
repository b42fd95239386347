// stream.cpp -- out-of-core rendering of snapshot volumes held in host memory.
//
// The volume is cut into slabs along z.  A slab is uploaded with only the
// snapshots its rays can reach in time (for each view, the retarded time over
// the slab's box spans [t_obs - s_max / c, t_obs - s_min / c]; the snapshots
// whose hat weights are nonzero there are all a ray inside the slab can read),
// packed as a small volume of its own, and marched for every view; the march
// adds each slab's contribution to the images.  The integral along a ray is a
// sum over the cells it crosses, so the slabs' sums add up to the full render
// (up to rounding: each slab restarts the ray's anchor).  Two slab buffers
// alternate, so the upload and packing of slab k + 1 run on the load stream
// while slab k is marched on the caller's stream.  This is the paper's
// partial sub-region rendering and its selective loading of the snapshots
// that overlap in time (Secs. 5.2, 6.2), with the volume never resident whole.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "runtime.h"

namespace gbd {
namespace {

// Snapshots that rays of view v inside the box [lo, hi] (world units) can
// read: [m0, m1], or m0 > m1 if none.
void epoch_span(const gbd_grid &g, const gbd_view &v, const double lo[3], const double hi[3], int *m0, int *m1)
{
    const int M = g.n_epochs;
    *m0 = 1;
    *m1 = 0;
    double u_lo, u_hi;
    const double u_obs = (v.t_obs - g.t0) / g.dt;
    if (!(v.flags & GBD_LOOKBACK)) {
        u_lo = u_hi = std::min(std::max(u_obs, 0.0), static_cast<double>(M - 1));
    } else if (std::isinf(v.c)) {
        u_lo = u_hi = u_obs;
    } else {
        const double nd = std::sqrt(v.dir[0] * v.dir[0] + v.dir[1] * v.dir[1] + v.dir[2] * v.dir[2]);
        double s_min = HUGE_VAL, s_max = -HUGE_VAL;
        // s of a point x is (x - centre) . s_hat: it is extreme at the corners
        for (int c = 0; c < 8; ++c) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) {
                const double x = ((c >> i) & 1) ? hi[i] : lo[i];
                s += (x - v.center[i]) * v.dir[i] / nd;
            }
            s_min = std::min(s_min, s);
            s_max = std::max(s_max, s);
        }
        const double kk = 1.0 / (v.c * g.dt);
        u_lo = u_obs - kk * s_max;
        u_hi = u_obs - kk * s_min;
    }
    // The hat weights of u reach snapshots floor(u) and floor(u) + 1 (Eq. 7).
    // One more snapshot on either side keeps every sample of the slab clear
    // of the kept range's ends, where a sub-range would fade its end
    // snapshots the way the full range fades only its own (and absorbs any
    // rounding between this estimate and the march's fixed-point u).
    const double a = std::floor(u_lo) - 1.0, b = std::floor(u_hi) + 2.0;
    if (b < 0.0 || a > M - 1.0) return;
    *m0 = static_cast<int>(std::max(a, 0.0));
    *m1 = static_cast<int>(std::min(b, static_cast<double>(M - 1)));
}

struct SlabBuffer {
    Volume vol;                  // the slab as a volume of its own (device records and tables)
    char *stage = nullptr;       // raw fields of a slab: j' of every kept snapshot, then beta
    std::vector<int32_t> tab;    // host copy of the layout tables being uploaded
    cudaEvent_t packed = nullptr, rendered = nullptr;
    bool used = false;
};

void release(SlabBuffer &b)
{
    if (b.vol.rec) cudaFree(b.vol.rec);
    if (b.vol.axis_off) cudaFree(b.vol.axis_off);
    if (b.stage) cudaFree(b.stage);
    if (b.packed) cudaEventDestroy(b.packed);
    if (b.rendered) cudaEventDestroy(b.rendered);
    b.vol.rec = nullptr;
    b.vol.axis_off = nullptr;
    b.stage = nullptr;
    b.packed = b.rendered = nullptr;
}

}  // namespace
}  // namespace gbd

using namespace gbd;

extern "C" int gbd_render_streamed(gbd_ctx *ctx, const gbd_grid *grid, const gbd_fields *f, const gbd_view *views,
                                   int32_t n, const gbd_image_spec *spec, const gbd_launch *launch,
                                   gbd_stream_info *info, void *stream)
{
    if (!ctx || !grid || !f || !views || !spec || !info) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    int rc = check_spec(spec);
    if (rc) return rc;
    if (spec->out_on_host) return fail(GBD_ERR_INVALID, "gbd_render_streamed needs device output");
    const gbd_grid &g = *grid;
    if ((rc = check_grid_fields(g, *f))) return rc;
    if (f->on_device) return fail(GBD_ERR_INVALID, "gbd_render_streamed reads its fields from host memory");
    if (info->slab < 0) return fail(GBD_ERR_INVALID, "slab must be >= 0");
    LaunchCfg cfg = resolve_launch(launch);
    if ((rc = check_launch(cfg))) return rc;
    cfg.region = 0;
    const int B = f->brick ? f->brick : 8;
    const int S = f->super_brick ? f->super_brick : 4;
    const int slab = std::min(info->slab > 0 ? info->slab : 64, g.n[2]);
    const int n_slabs = (g.n[2] + slab - 1) / slab;
    const int M = g.n_epochs;

    // flexload: the snapshots each slab needs, over all views
    std::vector<int> m0(n_slabs, M), m1(n_slabs, -1);
    for (int k = 0; k < n_slabs; ++k) {
        const int z0 = k * slab, z1 = std::min(z0 + slab, g.n[2]);
        if (!info->flexload) {
            m0[k] = 0;
            m1[k] = M - 1;
            continue;
        }
        const double lo[3] = {g.origin[0], g.origin[1], g.origin[2] + z0 * g.dx[2]};
        const double hi[3] = {g.origin[0] + g.n[0] * g.dx[0], g.origin[1] + g.n[1] * g.dx[1],
                              g.origin[2] + z1 * g.dx[2]};
        for (int v = 0; v < n; ++v) {
            int a, b;
            epoch_span(g, views[v], lo, hi, &a, &b);
            if (a <= b) {
                m0[k] = std::min(m0[k], a);
                m1[k] = std::max(m1[k], b);
            }
        }
    }
    int max_epochs = 0;
    for (int k = 0; k < n_slabs; ++k) max_epochs = std::max(max_epochs, m1[k] - m0[k] + 1);

    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    const size_t esz = f->dtype_in == GBD_IN_F64 ? 8 : 4;
    const size_t layer = static_cast<size_t>(g.n[0]) * g.n[1];     // cells per z layer
    const int full_n[3] = {g.n[0], g.n[1], slab};
    std::vector<int32_t> tab;
    long long cells = 0;
    if (!build_layout(full_n, B, S, tab, cells, 0)) return fail(GBD_ERR_INVALID, "slab too large");
    long long stride = 0;
    const size_t rec_bytes = volume_bytes(f->store, cells, std::max(max_epochs, 1), 0, &stride);
    const size_t tab_bytes = tab.size() * sizeof(int32_t);
    const size_t stage_bytes = layer * slab * esz * 4 * static_cast<size_t>(std::max(max_epochs, 1));
    const uint64_t need = 2 * (rec_bytes + tab_bytes + stage_bytes);
    if (ctx->used + need > ctx->budget)
        return fail(GBD_ERR_BUDGET, "two slab buffers need %llu bytes; %llu of %llu budget in use",
                    static_cast<unsigned long long>(need), static_cast<unsigned long long>(ctx->used),
                    static_cast<unsigned long long>(ctx->budget));

    cudaStream_t rs = static_cast<cudaStream_t>(stream);
    cudaStream_t cs = ctx->load_stream;
    SlabBuffer buf[2];
    int *bad = nullptr;
    cudaError_t e = cudaSuccess;
    if (!ctx->aux[0]) e = cudaStreamCreateWithFlags(&ctx->aux[0], cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->aux_done[0]) e = cudaEventCreateWithFlags(&ctx->aux_done[0], cudaEventDisableTiming);
    for (auto &b : buf) {
        if (e == cudaSuccess) e = cudaMalloc(&b.vol.rec, rec_bytes);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b.vol.axis_off), tab_bytes);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b.stage), stage_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.packed, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.rendered, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&bad), 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 256, cs);
    const size_t pix = static_cast<size_t>(spec->width) * spec->height * n;
    if (e == cudaSuccess) e = cudaMemsetAsync(spec->out, 0, pix * sizeof(float), rs);
    if (e == cudaSuccess && spec->samples) e = cudaMemsetAsync(spec->samples, 0, pix * sizeof(uint32_t), rs);

    uint64_t uploaded = 0;
    int slabs_done = 0, launches = 0;
    auto args = std::make_unique<MarchArgs>();
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    char *queue = nullptr;
    const size_t qbytes = (static_cast<size_t>(n) * sizeof(int) + 255) / 256 * 256;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&queue), qbytes * 2);
    for (int k = 0; k < n_slabs && e == cudaSuccess && rc == GBD_OK; ++k) {
        if (m0[k] > m1[k]) continue;  // no ray reaches a snapshot inside this slab
        SlabBuffer &b = buf[slabs_done % 2];
        const int z0 = k * slab, nz = std::min(slab, g.n[2] - z0);
        const int ne = m1[k] - m0[k] + 1;
        // the slab's grid: its z range and the snapshots it keeps
        Volume &sv = b.vol;
        sv.grid = g;
        sv.grid.n[2] = nz;
        sv.grid.origin[2] = g.origin[2] + z0 * g.dx[2];
        sv.grid.n_epochs = ne;
        sv.grid.t0 = g.t0 + m0[k] * g.dt;
        sv.store = f->store;
        sv.brick = B;
        sv.super_brick = S;
        sv.paired = 0;
        sv.morton_cells = 0;
        long long scells = 0;
        build_layout(sv.grid.n, B, S, b.tab, scells, 0);
        volume_bytes(f->store, scells, ne, 0, &sv.epoch_stride);
        // the buffer is free once the march of the slab it held last is done
        if (b.used) e = cudaStreamWaitEvent(cs, b.rendered, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sv.axis_off, b.tab.data(), b.tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(sv.rec, 0, static_cast<size_t>(sv.epoch_stride) * ne * (f->store == GBD_STORE_F32 ? 16 : 8),
                                cs);
        const size_t ncell = layer * g.n[2];
        const size_t scount = layer * nz;
        // The slab's part of each kept snapshot is one contiguous run of the
        // host arrays: one copy per run, j' on the load stream and beta on a
        // side stream, so both copy engines work; the packs wait for both.
        // The staging buffer is reused two slabs later, after this slab's
        // packs on the load stream.
        const size_t jrun = scount * esz, vrun = scount * esz * 3;
        char *jst = b.stage, *vst = b.stage + jrun * ne;
        cudaStream_t vs = ctx->aux[0];
        if (b.used && e == cudaSuccess) e = cudaStreamWaitEvent(vs, b.rendered, 0);
        for (int m = m0[k]; m <= m1[k] && e == cudaSuccess; ++m) {
            e = cudaMemcpyAsync(jst + (m - m0[k]) * jrun, static_cast<const char *>(f->j) + (m * ncell + z0 * layer) * esz,
                                jrun, cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(vst + (m - m0[k]) * vrun,
                                    static_cast<const char *>(f->vel) + (m * ncell + z0 * layer) * esz * 3, vrun,
                                    cudaMemcpyHostToDevice, vs);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->aux_done[0], vs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->aux_done[0], 0);
        for (int m = m0[k]; m <= m1[k] && e == cudaSuccess; ++m) {
            PackArgs pa;
            std::memset(&pa, 0, sizeof(pa));
            pa.j = jst + (m - m0[k]) * jrun;
            pa.vel = vst + (m - m0[k]) * vrun;
            pa.dtype_in = f->dtype_in;
            pa.store = f->store;
            for (int i = 0; i < 3; ++i) pa.n[i] = sv.grid.n[i];
            pa.axis_off = sv.axis_off;
            pa.dst = sv.rec;
            pa.stride = sv.epoch_stride;
            pa.m = m - m0[k];
            pa.paired = 0;
            pa.bad = bad;
            if (e == cudaSuccess) e = launch_pack(pa, cs);
            uploaded += scount * esz * 4;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b.packed, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, b.packed, 0);
        for (int v = 0; v < n && rc == GBD_OK; ++v)
            rc = make_view(sv, views[v], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[v]);
        if (rc != GBD_OK) break;
        int *q = reinterpret_cast<int *>(queue + (slabs_done % 2) * qbytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, qbytes, rs);
        const std::vector<double> work = view_works(sv, hv, spec->width, spec->height);
        for (int c = 0; c < march_chunks(n) && e == cudaSuccess; ++c) {
            fill_args(*args, sv, hv.data(), n, c, *spec, spec->out, spec->samples, q, cfg, ctx->err_word);
            args->accumulate = 1;
            e = launch_march(*args, cfg, ctx->num_sms, work.data() + static_cast<size_t>(c) * kViewsPerLaunch, rs);
            ++launches;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b.rendered, rs);
        b.used = true;
        ++slabs_done;
    }
    int h_bad = 0;
    cudaError_t es = cudaStreamSynchronize(ctx->aux[0]);
    if (e == cudaSuccess) e = es;
    es = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = es;
    es = cudaStreamSynchronize(rs);
    if (e == cudaSuccess) e = es;
    if (e == cudaSuccess && bad) e = cudaMemcpy(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    for (auto &b : buf) release(b);
    if (bad) cudaFree(bad);
    if (queue) cudaFree(queue);
    if (rc != GBD_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "streamed render");
    if (h_bad)
        return fail(GBD_ERR_INVALID, "fields: negative or non-finite j', non-finite beta, or |beta| >= 1");
    info->slabs = slabs_done;
    info->bytes_uploaded = uploaded;
    info->bytes_total = static_cast<uint64_t>(layer) * g.n[2] * M * esz * 4;
    set_launch_count(launches);
    return GBD_OK;
}

// ------------------------------------------------------------ labelled mode
// Several resident volumes, each a sub-domain with its own grid (origin, cell
// size, dimensions, snapshot times): a ray's sum over their union is the sum
// of its sums over each.  The sub-domains are marched side by side on the
// context's side streams, each into an image of its own, and the images are
// added in the order given (the same sums as adding them one by one); with
// sample counts they are marched one after another, adding into the images.
extern "C" int gbd_render_labelled(gbd_ctx *ctx, const gbd_volume *vols, int32_t n_vols, const gbd_view *views,
                                   int32_t n, const gbd_image_spec *spec, const gbd_launch *launch, void *stream)
{
    if (!ctx || !vols || !views || !spec) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n_vols < 1 || n_vols > 4096) return fail(GBD_ERR_INVALID, "n_vols must be in [1, 4096]");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    int rc = check_spec(spec);
    if (rc) return rc;
    if (spec->out_on_host) return fail(GBD_ERR_INVALID, "gbd_render_labelled needs device output");
    LaunchCfg cfg = resolve_launch(launch);
    if ((rc = check_launch(cfg))) return rc;
    cfg.region = 0;
    std::lock_guard<std::mutex> lock(ctx->mu);
    std::vector<Volume *> vs(static_cast<size_t>(n_vols));
    for (int k = 0; k < n_vols; ++k) {
        vs[k] = ctx->find(vols[k]);
        if (!vs[k]) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vols[k]));
    }
    // sub-domains must not overlap: their boxes may only touch
    for (int a = 0; a < n_vols; ++a)
        for (int b = a + 1; b < n_vols; ++b) {
            bool overlap = true;
            for (int i = 0; i < 3; ++i) {
                const gbd_grid &ga = vs[a]->grid, &gb = vs[b]->grid;
                const double alo = ga.origin[i], ahi = ga.origin[i] + ga.n[i] * ga.dx[i];
                const double blo = gb.origin[i], bhi = gb.origin[i] + gb.n[i] * gb.dx[i];
                const double tol = 1e-9 * std::max({std::fabs(alo), std::fabs(ahi), std::fabs(blo), std::fabs(bhi), 1.0});
                if (!(std::min(ahi, bhi) - std::max(alo, blo) > tol)) overlap = false;
            }
            if (overlap) return fail(GBD_ERR_INVALID, "sub-domains %d and %d overlap", a, b);
        }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t pix = static_cast<size_t>(spec->width) * spec->height * n;
    cudaError_t e = cudaMemsetAsync(spec->out, 0, pix * sizeof(float), st);
    if (e == cudaSuccess && spec->samples) e = cudaMemsetAsync(spec->samples, 0, pix * sizeof(uint32_t), st);
    char *queue = nullptr;
    const size_t qbytes = (static_cast<size_t>(n) * sizeof(int) + 255) / 256 * 256;
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&queue), qbytes * n_vols, st);
    if (e != cudaSuccess) return cuda_fail(e, "labelled render setup");
    if ((e = cudaMemsetAsync(queue, 0, qbytes * n_vols, st)) != cudaSuccess) {
        cudaFreeAsync(queue, st);
        return cuda_fail(e, "labelled render setup");
    }
    auto args = std::make_unique<MarchArgs>();
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    int launches = 0;
    const bool side_by_side = n_vols > 1 && !spec->samples;
    float *parts = nullptr;
    cudaEvent_t start = nullptr;
    if (side_by_side) {
        for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
            if (!ctx->aux[s]) e = cudaStreamCreateWithFlags(&ctx->aux[s], cudaStreamNonBlocking);
            if (e == cudaSuccess && !ctx->aux_done[s])
                e = cudaEventCreateWithFlags(&ctx->aux_done[s], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&parts), pix * sizeof(float) * n_vols, st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(start, st);
    }
    for (int k = 0; k < n_vols && e == cudaSuccess && rc == GBD_OK; ++k) {
        for (int v = 0; v < n && rc == GBD_OK; ++v)
            rc = make_view(*vs[k], views[v], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[v]);
        if (rc != GBD_OK) break;
        const std::vector<double> work = view_works(*vs[k], hv, spec->width, spec->height);
        int *q = reinterpret_cast<int *>(queue + k * qbytes);
        cudaStream_t ks = side_by_side ? ctx->aux[k % 4] : st;
        if (side_by_side) e = cudaStreamWaitEvent(ks, start, 0);
        for (int c = 0; c < march_chunks(n) && e == cudaSuccess; ++c) {
            if (side_by_side) {
                fill_args(*args, *vs[k], hv.data(), n, c, *spec, parts + pix * k, nullptr, q, cfg, ctx->err_word);
            } else {
                fill_args(*args, *vs[k], hv.data(), n, c, *spec, spec->out, spec->samples, q, cfg, ctx->err_word);
                args->accumulate = 1;
            }
            e = launch_march(*args, cfg, ctx->num_sms, work.data() + static_cast<size_t>(c) * kViewsPerLaunch, ks);
            ++launches;
        }
        // side streams: the caller's stream waits for each sub-domain
        if (side_by_side && e == cudaSuccess) e = cudaEventRecord(ctx->aux_done[k % 4], ks);
        if (side_by_side && e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->aux_done[k % 4], 0);
    }
    if (side_by_side && e == cudaSuccess && rc == GBD_OK) {
        // add the sub-domains' images in order (prefactors already applied)
        auto r = std::make_unique<ReduceArgs>();
        const long long per = static_cast<long long>(spec->width) * spec->height;
        for (int first = 0; first < n && e == cudaSuccess; first += kImagesPerReduce) {
            const int cnt = std::min(kImagesPerReduce, n - first);
            std::memset(r.get(), 0, sizeof(ReduceArgs));
            r->out = spec->out;
            r->partial = parts;
            r->slot_stride = static_cast<long long>(pix);
            r->pix_per_view = per;
            r->n_views = cnt;
            r->n_slots = n_vols;
            for (int v = 0; v < cnt; ++v) {
                r->image[v] = first + v;
                r->prefactor[v] = 1.0f;
            }
            e = launch_reduce(*r, st);
            ++launches;
        }
    }
    if (parts) cudaFreeAsync(parts, st);
    if (start) cudaEventDestroy(start);
    cudaError_t ef = cudaFreeAsync(queue, st);
    if (rc != GBD_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "labelled render");
    if (ef != cudaSuccess) return cuda_fail(ef, "labelled render scratch");
    set_launch_count(launches);
    return GBD_OK;
}
