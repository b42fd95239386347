// gbd_internal.h -- structures shared by the host runtime and the CUDA kernels.
//
// Nothing here is part of the public ABI (include/gbdart.h).
#pragma once

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
    long long epoch_stride;   // records per block (padded)
    int n[3];
    int M;
    int store;                // GBD_STORE_*
    int paired;               // 1: block b holds snapshots b-1 and b side by side
};

// Per-view constants, computed on the host in float64 once per view, so that
// the kernels need no float64 arithmetic (the FP64 rate of GB300 is 1/64 of
// FP32).  Lengths along a ray are the parameter s of x = r0 + s s_hat, with s
// measured from the image plane; positions are in grid-index units
// g_i = (x_i - origin_i) / dx_i, so cell faces sit at integers.
//   fixed point: Q24.40 (int64, 2^-40 cells per unit) for positions,
//                Q31.32 (int64, 2^-32 epochs per unit) for epoch coordinates.
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
    uint32_t flags;    // GBD_BEAMING | GBD_LOOKBACK
};

// One march launch: n_views views of one image geometry.
struct MarchArgs {
    VolDev vol;
    const ViewDev *views;     // device array, n_views entries
    int n_views;
    int width, height;
    int packet_w, packet_h;   // packet_w * packet_h == 32
    int tiles_x, tiles_y;     // packets per image row / column
    long long total_items;    // n_views * tiles_x * tiles_y
    float *out;               // n_views * width * height floats
    uint32_t *samples;        // optional, same shape
    int *queue;               // persistent mode: tile counter (zeroed before launch)
    int *error_word;          // checked builds: first bounds violation code
    int persistent;
};

// One request of a served wave: its own volume, view, image and outputs.
struct ReqDev {
    VolDev vol;
    ViewDev view;
    int width, height;
    int tiles_x, tiles_y;
    long long tile_begin;     // first tile of this request in the wave's queue
    float *out;               // device image of the request
    uint32_t *samples;        // optional per-pixel cell-sample counts
};

// A served wave: many requests in one persistent launch.
struct WaveArgs {
    const ReqDev *reqs;       // device array, sorted by tile_begin
    int n_reqs;
    int packet_w, packet_h;
    long long total_items;    // tiles of all requests
    int *queue;               // tile counter (zeroed before launch)
    int *error_word;
};

// Launch configuration after defaults have been applied.
struct LaunchCfg {
    int packet_w, packet_h, cta_warps, depth, persistent, regcap;
};

// Kernel entry points (march.cu, pack.cu).
cudaError_t launch_march(const MarchArgs &a, const LaunchCfg &cfg, int num_sms, cudaStream_t stream);
cudaError_t march_occupancy(const LaunchCfg &cfg, int store, int smem_bytes, int *blocks_per_sm);
cudaError_t launch_wave(const WaveArgs &a, const LaunchCfg &cfg, int num_sms, cudaStream_t stream);

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
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream);

struct RelayoutArgs {
    const void *src;          // whole record array in the old layout
    void *dst;                // whole record array in the new layout
    const int32_t *src_off;   // per-axis tables of the old layout
    const int32_t *dst_off;   // per-axis tables of the new layout
    long long src_stride, dst_stride;  // records per block
    int src_paired, dst_paired;
    int m;                    // epoch being copied
    int n[3];
    int record_bytes;         // 16 or 8
};
cudaError_t launch_relayout(const RelayoutArgs &a, cudaStream_t stream);

}  // namespace gbd
