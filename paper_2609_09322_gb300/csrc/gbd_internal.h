// gbd_internal.h -- structures shared by the host runtime and the CUDA kernels.
//
// Nothing here is part of the public ABI (include/gbdart.h).
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gbdart.h"

namespace gbd {

// Largest grid edge the kernels accept; the three per-axis offset tables of a
// volume are staged in shared memory, 4 bytes per entry.
constexpr int kMaxAxis = 4096;

// A packed volume as the kernels see it.  The record of cell (ix, iy, iz) at
// epoch m sits at rec + m * epoch_stride + off[ix] + off[nx + iy] + off[nx + ny + iz]:
// every supported layout (linear, bricked, bricked with Morton-ordered
// super-bricks) is a sum of one term per axis, so a single set of tables
// serves all of them and the march can update one term per cell step.
struct VolDev {
    const void *rec;          // record array (16-byte or 8-byte records)
    const int32_t *axis_off;  // n[0] + n[1] + n[2] entries
    const int32_t *mtab;      // march tables, march_table_entries(n) entries (see below)
    long long epoch_stride;   // records per block (padded); paired: a zero record pair
                              // follows the M + 1 blocks, at record (M + 1) * epoch_stride
    int n[3];
    int M;
    int store;                // GBD_STORE_*
    int paired;               // 1: block b holds snapshots b-1 and b side by side
    int plain_boost;          // bfloat16/float16 records whose Gamma^2 = 1 + |u|^2 <= kPlainGamma2:
                              // the march may take D = 1 / (Gamma + u.s_hat) as it stands
};

// Largest Gamma^2 of a bfloat16/float16 volume whose march evaluates the
// Doppler factor in the plain form (Gamma <= 8, beta <= 0.992).
constexpr float kPlainGamma2 = 64.0f;

// March tables.  The march steps every axis towards increasing cell index:
// an axis the view runs down is mirrored (cell k' = n - 1 - k) on the host.
// For each axis the tables hold the forward terms off[0 .. n-1], then two
// sentinels, then the reversed terms off[n-1 .. 0], then two sentinels.  A
// step onto a sentinel is a step out of the box, and the sign bit of the
// sentinel tells the march so; the second sentinel absorbs the read-ahead
// of the next cell's term.
constexpr int32_t kTabSentinel = INT32_MIN;
// Sentinels after the last staged table in shared memory (see stage_tables).
constexpr int kTabPad = 2;
__host__ __device__ inline int march_table_base(const int n[3], int axis)
{
    return axis == 0 ? 0 : (axis == 1 ? 2 * (n[0] + 2) : 2 * (n[0] + 2) + 2 * (n[1] + 2));
}
__host__ __device__ inline int march_table_entries(const int n[3]) { return 2 * (n[0] + n[1] + n[2] + 6); }

// Bits of ViewDev::flags above the public GBD_BEAMING / GBD_LOOKBACK bits:
// axis i is mirrored (the view's direction has s_hat_i < 0).
constexpr uint32_t kFlagMirror0 = 1u << 8;

// Per-view constants, computed on the host in float64 once per view, so that
// the kernels need no float64 arithmetic (the FP64 rate of GB300 is 1/64 of
// FP32).  Lengths along a ray are the parameter s of x = r0 + s s_hat, with s
// measured from the image plane; positions are in grid-index units
// g_i = (x_i - origin_i) / dx_i, so cell faces sit at integers.
//   fixed point: Q24.40 (int64, 2^-40 cells per unit) for positions,
//                Q31.32 (int64, 2^-32 epochs per unit) for epoch coordinates.
// Positions and directions are given in the mirrored frame of each mirrored
// axis (g' = n - g, a' = -a), so every a_i, inv_a_i and w_i is >= 0.
struct ViewDev {
    long long g0[3];   // pixel (0, 0) on the image plane, Q24.40
    long long gu[3];   // change per pixel column, Q24.40
    long long gv[3];   // change per pixel row, Q24.40
    long long u_obs;   // epoch coordinate at s = 0, Q31.32 (fast light: the clamped one)
    long long du[3];   // epochs crossed per face plane of axis i, kk / |a_i|, Q31.32
    float a_hi[3];     // a_i = s_hat_i / dx_i (cells per unit s) as hi + lo floats;
    float a_lo[3];     //   0 for an axis the ray runs parallel to
    float inv_a[3];    // 1 / a_i (face spacing along the ray, Eq. 11), 0 if parallel
    float w_hi[3];     // kk / a_i as hi + lo floats
    float w_lo[3];
    float kk_hi;       // kk = 1 / (c dt): epochs per unit s (0 without lookback)
    float kk_lo;
    float win_lo;      // s range where the retarded time can reach a snapshot
    float win_hi;
    float sh_hi[3];    // s_hat rounded to float ...
    float sh_lo[3];    // ... and the rounding residual (Doppler dot product)
    float expo;        // 2 - alpha
    float prefactor;   // (nu / nu'_0)^alpha
    uint32_t flags;    // GBD_BEAMING | GBD_LOOKBACK | kFlagMirror0 << axis
};

// Views per march launch.  The views travel in the kernel's parameter space
// (up to 32 KB on sm_70 and later with CUDA 12.1+), and each CTA works on one
// view, so every per-view constant is uniform across the CTA and the compiler
// keeps it in uniform registers instead of per-thread ones.  Larger batches
// are split into several launches.
constexpr int kViewsPerLaunch = 128;

// Time groups: views of a batch that differ only in observer time are
// marched together, up to kGroupMax per ray (one sum per member in registers);
// kGroupDefault when the launch does not say.
constexpr int kGroupMax = 8;
constexpr int kGroupDefault = 4;

// One march launch: n_views views of one image geometry.
struct MarchArgs {
    VolDev vol;
    int n_views;              // views in this launch, 1 .. kViewsPerLaunch
    int width, height;
    int packet_w, packet_h;   // packet_w * packet_h == 32
    int tiles_x, tiles_y;     // packets per image row / column
    int cta_begin[kViewsPerLaunch + 1];  // first CTA of each view (or group), then the total (set by plan_march)
    int n_groups;             // 0: every view marched on its own; else time groups of consecutive views
    int group_size;           // time groups: the kernel's member limit (4 or kGroupMax)
    int group_first[kViewsPerLaunch + 1];  // group g: views group_first[g] .. group_first[g + 1] - 1
    int group_ref[kViewsPerLaunch];        // the group's reference view: the largest u_obs
    float group_win[kViewsPerLaunch][2];   // the union of the members' windows
    long long view_delta[kViewsPerLaunch]; // u_obs of the view minus that of its group's reference, Q31.32
    int view_dhi[kViewsPerLaunch];         // view_delta >> 32 (whole epochs, rounded down)
    int persistent;           // CTAs loop over their view's tile counter
    int accumulate;           // add to out (and samples) instead of storing
    float *out;               // n_views * width * height floats
    uint32_t *samples;        // optional, same shape
    int *queue;               // persistent mode: one tile counter per view or group (zeroed before launch)
    const int *tile_order;    // persistent mode: counter value -> tile (centre of the image first), or NULL
    int *error_word;          // checked builds: first bounds violation code
    // vector renders (vector_kernel): extra emissivity channels of the volume
    const float *chan;        // n_chan channels, each M blocks of chan_cell_stride floats
    long long chan_comp_stride;   // floats per channel
    long long chan_cell_stride;   // floats per snapshot (cells of the layout)
    long long img_stride;     // floats between consecutive views' images (0: width * height)
    ViewDev views[kViewsPerLaunch];
};
static_assert(sizeof(MarchArgs) <= 32764, "march launch arguments exceed the kernel parameter limit");

// Region schedule.  A batch of many views over a large volume marches every
// ray region by region: region r (an edge^3 block of cells) is marched for all
// views' rays that cross it while its records sit in L2, and each ray's sum
// over the region goes to partial slot s(r), the sum of r's region coordinates
// in the march frame, which grows by one from region to region along a ray.
// A reduction then adds each ray's slots in order, kImagesPerReduce images
// per launch.
constexpr int kImagesPerReduce = 96;

// Pixel coordinates of a point g of a view's march frame: p = ip . g + p0,
// q = iq . g + q0 (the first two rows of the inverse of [gu gv a]).
struct RegionProj {
    float ip[3], iq[3];
    float p0, q0;
    // and back: pixel (p, q) lies on its ray near g0f + p guf + q gvf (float
    // approximations of the view's fixed-point g0, gu, gv)
    float g0f[3], guf[3], gvf[3];
};

// The views of a region-schedule batch live in device memory (the region
// tables), in march order: all of them go in one launch, so that the rays of
// every view that crosses a region are marched while its records are in L2.
struct RegionArgs {
    VolDev vol;
    int n_views;              // views of the batch
    int width, height;
    int packet_w, packet_h;
    int region;               // region edge in cells
    int nreg[3];              // regions per axis
    float *partial;           // slot s of batch image b at partial + s * slot_stride + b * width * height
    long long slot_stride;    // floats per slot
    long long partial_floats; // floats of all slots (screen_kernel clears them)
    int *error_word;
    const ViewDev *views;     // n_views views in march order (by direction)
    const RegionProj *proj;   // their projections
    const int *image;         // each one's image in the batch
    const int *region_order;  // region r's views in march order: region_order[r * n_views + y]
    // Ray lists (written by screen_kernel, read by region_kernel): the pixels
    // (p | q << 16) of view v whose rays cross region r, longest chord first,
    // at rays + (r * n_views + v) * ctas_per_view * rays_per_cta, and their
    // number at ray_count[r * n_views + v].  Each list has room for every
    // pixel that the region's box can cover in any of the views.
    uint32_t *rays;
    int *ray_count;
    int rays_per_cta;         // 32 * warps per CTA of region_kernel
    int ctas_per_view;        // CTAs of each view in one region (blockIdx.x)
};

// For the launch's views v: out[b][pixel] = prefactor[v] * (sum over slots of
// partial[slot][b][pixel], in slot order), b = image[v] the view's image in the
// batch.
struct ReduceArgs {
    float *out;               // the batch's first image
    const float *partial;     // slot 0 of the batch's first image
    long long slot_stride;    // floats per slot
    long long pix_per_view;
    int n_views;
    int n_slots;
    int image[kImagesPerReduce];
    float prefactor[kImagesPerReduce];
};

// One request of a served wave: its own volume, view, image and outputs.
struct ReqDev {
    VolDev vol;
    ViewDev view;
    int width, height;
    int tiles_x, tiles_y;
    int cta_begin;            // first CTA of this request in the launch
    float *out;               // device image of the request
    uint32_t *samples;        // optional per-pixel cell-sample counts
};

// Requests per wave launch (parameter space, as for views); a larger wave is
// several launches on its stream.
constexpr int kReqsPerLaunch = 96;

// One launch of a served wave: each request gets ceil(tiles / warps per CTA)
// CTAs, one packet per warp.
struct WaveArgs {
    int n_reqs;
    int packet_w, packet_h;
    int total_ctas;
    int *error_word;
    ReqDev reqs[kReqsPerLaunch];  // sorted by cta_begin
};
static_assert(sizeof(WaveArgs) <= 32764, "wave launch arguments exceed the kernel parameter limit");

// Launch configuration after defaults have been applied.
struct LaunchCfg {
    int packet_w, packet_h, cta_warps, depth, persistent, regcap, region, group;
};

// A planned kernel launch.
struct KernelLaunch {
    void *func;
    dim3 grid, block;
    int smem;
};

// Kernel entry points (march.cu, pack.cu).  plan_march picks the kernel and
// grid for a filled MarchArgs and sets its cta_begin; `work` (n_views
// estimates, or NULL for equal shares) splits a persistent grid over the
// views.  launch_march plans and launches.
cudaError_t plan_march(MarchArgs &a, const LaunchCfg &cfg, int num_sms, const double *work, KernelLaunch &k);
cudaError_t launch_march(MarchArgs &a, const LaunchCfg &cfg, int num_sms, const double *work, cudaStream_t stream);
cudaError_t launch_wave(const WaveArgs &a, const LaunchCfg &cfg, cudaStream_t stream);
// Memory analysis: sets bit m * cells + cell of `bits` for every record the
// views' samples read (a non-persistent launch planned like the march).
cudaError_t launch_touch(MarchArgs &a, uint32_t *bits, long long cells, const LaunchCfg &cfg, int num_sms,
                         cudaStream_t stream);
// Vector render: n_chan (1 or 3) extra channels besides j'; image v's
// component c at out + v * img_stride + c * width * height.
cudaError_t launch_vector(MarchArgs &a, int n_chan, const LaunchCfg &cfg, int num_sms, const double *work,
                          cudaStream_t stream);
// Region schedule: the caller has filled everything but the grid, which
// launch_screen (a warp per view and region) and launch_region (ctas_per_view
// x views x regions) derive from the counts.  launch_screen writes the ray
// lists that the following launch_region of the same arguments marches.
cudaError_t launch_screen(const RegionArgs &a, cudaStream_t stream);
cudaError_t launch_region(const RegionArgs &a, const LaunchCfg &cfg, cudaStream_t stream);
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t stream);

struct PackArgs {
    const void *j;            // one epoch, [nz][ny][nx]
    const void *vel;          // one epoch, [nz][ny][nx][3]
    int dtype_in;             // GBD_IN_F64 / GBD_IN_F32
    int store;                // GBD_STORE_*
    int n[3];
    const int32_t *axis_off;  // device tables
    void *dst;                // the whole record array
    long long stride;         // records per block
    int m;                    // epoch being packed
    int paired;               // write into blocks m (second slot) and m + 1 (first slot)
    int *bad;                 // device flag: set to 1 on an invalid value
    unsigned *gamma2_max;     // bfloat16/float16 store: atomic max of the bits of the stored
                              // records' Gamma^2 = 1 + |u|^2 (a non-negative float); may be NULL
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream);

struct ChanPackArgs {
    const void *src;          // one channel, one epoch, [nz][ny][nx]
    int dtype_in;             // GBD_IN_F64 / GBD_IN_F32
    int n[3];
    const int32_t *axis_off;  // device tables
    float *dst;               // that channel's epoch block
    int *bad;                 // device flag: set to 1 on a non-finite value
};
cudaError_t launch_chan_pack(const ChanPackArgs &a, cudaStream_t stream);

struct RelayoutArgs {
    const void *src;          // whole record array in the old layout
    void *dst;                // whole record array in the new layout
    const int32_t *src_off;   // per-axis tables of the old layout
    const int32_t *dst_off;   // per-axis tables of the new layout
    long long src_stride, dst_stride;  // records per block
    int src_paired, dst_paired;
    int m;                    // epoch being copied
    int n[3];
    int record_bytes;         // 16 or 8 (records), 4 (channel values, unpaired)
};
cudaError_t launch_relayout(const RelayoutArgs &a, cudaStream_t stream);

}  // namespace gbd
