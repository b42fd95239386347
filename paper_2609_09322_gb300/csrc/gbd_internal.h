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
    long long epoch_stride;   // records per epoch (padded)
    int n[3];
    int M;
    double origin[3];
    double dx[3];
    double inv_dx[3];
    double t0, inv_dt;
    int store;                // GBD_STORE_*
};

// Per-view constants, computed on the host in float64 once per view (camera
// basis, pixel pitch, lookback window, power-law prefactor).
struct ViewDev {
    double r00[3];     // centre of pixel (0, 0)
    double du[3];      // h_u e_u: step between pixel columns
    double dv[3];      // h_v e_v: step between pixel rows
    double sh[3];      // s_hat
    double inv_sh[3];  // 1 / s_hat_i, 0 where s_hat_i = 0
    double t_obs;
    double inv_c;      // 1/c, 0 for c = infinity
    double win_lo;     // lookback window of s where t_bar lies in [t_0, t_{M-1}]
    double win_hi;
    float sh_hi[3];    // s_hat rounded to float ...
    float sh_lo[3];    // ... and the rounding residual
    float inv_sh_f[3]; // float 1 / s_hat_i (0 where s_hat_i = 0)
    float u_fast;      // epoch coordinate without lookback, clamped to [0, M-1]
    float expo;        // 2 - alpha
    float prefactor;   // (nu / nu'_0)^alpha
    uint32_t flags;    // GBD_BEAMING | GBD_LOOKBACK
    int32_t pad_;
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

// Launch configuration after defaults have been applied.
struct LaunchCfg {
    int packet_w, packet_h, cta_warps, depth, persistent;
};

// Kernel entry points (march.cu, pack.cu).
cudaError_t launch_march(const MarchArgs &a, const LaunchCfg &cfg, int num_sms, cudaStream_t stream);
cudaError_t march_occupancy(const LaunchCfg &cfg, int store, int smem_bytes, int *blocks_per_sm);

struct PackArgs {
    const void *j;            // one epoch, [nz][ny][nx]
    const void *vel;          // one epoch, [nz][ny][nx][3]
    int dtype_in;             // GBD_IN_F64 / GBD_IN_F32
    int store;                // GBD_STORE_*
    int n[3];
    const int32_t *axis_off;  // device tables
    void *dst;                // records of this epoch
    int *bad;                 // device flag: set to 1 on an invalid value
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream);

struct RelayoutArgs {
    const void *src;          // records of one epoch in the old layout
    void *dst;                // records of the same epoch in the new layout
    const int32_t *src_off;   // per-axis tables of the old layout
    const int32_t *dst_off;   // per-axis tables of the new layout
    int n[3];
    int record_bytes;         // 16 or 8
};
cudaError_t launch_relayout(const RelayoutArgs &a, cudaStream_t stream);

}  // namespace gbd
