// noalloc.cu -- batch render that allocates no memory.
//
// gbd_render_batch keeps its view table and tile counter in memory it
// allocates (a cached graph's buffer, or stream-ordered scratch).  Some
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
constexpr size_t kViewTableBytes = sizeof(ViewDev) * kNoAllocMaxViews;
constexpr size_t kCounterOffset = (kViewTableBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCounterOffset + 256;
constexpr int kMaxDevices = 64;

// Device scratch: the view table, then the tile counter of the persistent
// grid.  In host code this name is only a stand-in for the symbol; its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                          // guards the two arrays below
void *g_scratch_addr[kMaxDevices] = {};   // device address of g_scratch, per device
ViewDev g_host_views[kNoAllocMaxViews];   // host staging of the view table

// Looks up the device address of the scratch array on the current device
// (once per device; the caller holds g_mu and has made `dev` current).
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
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (!launch) lookup_tuned(*ctx, tune_key(*vol, spec->width, spec->height, n, views[0].flags), cfg);
    DeviceGuard guard(ctx->device);

    std::lock_guard<std::mutex> slock(g_mu);
    char *scratch = nullptr;
    if ((rc = scratch_address(ctx->device, &scratch))) return rc;
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, g_host_views[k])))
            return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ViewDev *d_views = reinterpret_cast<ViewDev *>(scratch);
    int *queue = reinterpret_cast<int *>(scratch + kCounterOffset);
    // The host staging array is pageable: the copy has consumed it when the
    // call returns, so the next call may refill it.
    cudaError_t e = cudaMemcpyAsync(d_views, g_host_views, sizeof(ViewDev) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, 256, st);  // the tile counter starts at zero
    MarchArgs a;
    fill_args(a, *vol, d_views, n, *spec, spec->out, spec->samples, queue, cfg, ctx->err_word);
    if (e == cudaSuccess) e = launch_march(a, cfg, ctx->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc batch launch");
    set_launch_count(1);
    return GBD_OK;
}
