// noalloc.cu -- batch render that allocates no memory.
//
// gbd_render_batch keeps its per-view tile counters in memory it allocates
// (a cached graph's buffer, or stream-ordered scratch).  Some
// callers cannot let a library allocate device memory while they render:
// applications that hand the whole device to their own allocator or memory
// pool up front (a cudaMalloc inside the library would fail, or break their
// accounting), and latency-critical loops where cudaMalloc / cudaFree, which
// may synchronise the device, are not acceptable.  This entry point serves
// them: its scratch is the fixed-size array below, which every GPU that loads
// the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "runtime.h"

namespace gbd {
namespace {

constexpr int kNoAllocMaxViews = GBD_NOALLOC_MAX_VIEWS;
constexpr size_t kScratchBytes = sizeof(int) * kNoAllocMaxViews;  // one tile counter per view
constexpr int kMaxDevices = 64;

// Device scratch: the tile counters of the persistent grid (the views travel
// in the launch parameters).  In host code this name is only a stand-in for
// the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                          // guards the arrays below
void *g_scratch_addr[kMaxDevices] = {};   // device address of g_scratch, per device
ViewDev g_host_views[kNoAllocMaxViews];   // the views, set up on the host
MarchArgs g_args;                         // launch arguments (about 28 KB: not on the stack)
double g_work[kViewsPerLaunch];           // per-view work estimates of one launch

// Looks up the device address of the scratch array on the current device
// (once per device; the caller holds g_mu and has made `dev` current).  The
// address is kept for the life of the process: a cudaDeviceReset, which
// tears down the context the address belongs to, ends this entry point's use
// on that device.
int scratch_address(int dev, char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(GBD_ERR_INVALID, "device index %d not supported here", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<char *>(g_scratch_addr[dev]);
    return GBD_OK;
}

}  // namespace
}  // namespace gbd

using namespace gbd;

extern "C" int gbd_render_batch_noalloc(gbd_ctx *ctx, gbd_volume vid, const gbd_view *views, int32_t n,
                                        const gbd_image_spec *spec, const gbd_launch *launch, void *stream)
{
    if (!ctx || !views || !spec) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > kNoAllocMaxViews)
        return fail(GBD_ERR_INVALID, "gbd_render_batch_noalloc takes 1 to %d views per call (got %d)",
                    kNoAllocMaxViews, n);
    if (spec->width < 1 || spec->height < 1 || spec->width > 16384 || spec->height > 16384)
        return fail(GBD_ERR_INVALID, "image: width/height must be in [1, 16384]");
    if (!spec->out || spec->out_on_host)
        return fail(GBD_ERR_INVALID, "gbd_render_batch_noalloc needs a device output buffer");
    LaunchCfg cfg = resolve_launch(launch);
    int rc = check_launch(cfg);
    if (rc) return rc;
    // The region schedule needs partial-sum slots that grow with the batch;
    // this entry point has no room for them.
    if (cfg.region != 0)
        return fail(GBD_ERR_INVALID, "gbd_render_batch_noalloc has no region schedule (launch.region must be 0)");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (!launch) {
        // a tuned region schedule is replaced by the whole-ray march (the
        // tuned packet, CTA and group shapes are kept)
        lookup_tuned(*ctx, tune_key(*vol, spec->width, spec->height, n, views[0].flags), cfg);
        cfg.region = 0;
        cfg.persistent = 1;
    }
    DeviceGuard guard(ctx->device);

    std::lock_guard<std::mutex> slock(g_mu);
    char *scratch = nullptr;
    if ((rc = scratch_address(ctx->device, &scratch))) return rc;
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, g_host_views[k])))
            return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *queue = reinterpret_cast<int *>(scratch);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int) * static_cast<size_t>(n), st);  // counters start at zero
    const int chunks = march_chunks(n);
    for (int c = 0; c < chunks && e == cudaSuccess; ++c) {
        fill_args(g_args, *vol, g_host_views, n, c, *spec, spec->out, spec->samples, queue, cfg, ctx->err_word);
        group_views(g_args, cfg.group);
        for (int v = 0; v < g_args.n_views; ++v)
            g_work[v] = view_work(*vol, g_args.views[v], spec->width, spec->height);
        e = launch_march(g_args, cfg, ctx->num_sms, g_work, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc batch launch");
    set_launch_count(chunks);
    return GBD_OK;
}
