/*
 * gbdart.h -- C ABI of the GB300 relativistic ray-marching library.
 *
 * The library renders synthetic observations of optically thin emission from
 * meshed simulation snapshots: for every pixel of an orthographic camera it
 * sums, along the pixel's line of sight, the rest-frame emissivity boosted by
 * the Doppler factor and read at the retarded time of each cell,
 *
 *   I_nu = (nu/nu'_0)^alpha sum_m sum_n W_{n,m} D_{n,m}^{2-alpha} j'_{n,m} ds_n
 *
 * (Whitehead, Elley & Everett, "cuDART", Eq. 19 of Sec. 2.5; the cell chords
 * ds_n of Sec. 2.4; the temporal weights W of Eqs. 6-7, Sec. 2.3; the Doppler
 * factor D of Eq. 14; the retarded time t_bar = t_obs - s/c of Eq. 2).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Every call returns an int status (GBD_OK = 0 or a GBD_ERR_* code) and never
 *    throws, aborts or exits.  gbd_last_error() gives a message for the last
 *    failing call on the calling thread.
 *  - A context is bound to one CUDA device.  It is internally locked: calls from
 *    several host threads are serialised on the host, while the GPU work they
 *    enqueue may overlap when issued on different streams.
 *  - Streams are passed as `void *` holding a cudaStream_t (NULL = the legacy
 *    default stream).  Rendering calls are asynchronous on that stream; the
 *    caller synchronises before reading the image.
 *  - Lengths are in grid units (cells of size dx along each axis), times in the
 *    same unit system; c is the signal speed in those units (cells per unit
 *    time when dx = 1).
 *  - The sign convention for alpha is the paper's: rest-frame emissivity
 *    j' ~ nu'^alpha, so the default synchrotron slope is alpha = -0.6 and the
 *    per-cell boost is D^(2 - alpha) = D^2.6.
 *
 * Geometry of a view (readings of the paper, which does not fix the camera):
 *  - dir is the unit viewing direction s_hat, pointing from the observer into
 *    the scene; the direction to the observer is n_hat = -s_hat, so
 *    D = 1 / (Gamma (1 + beta . s_hat)) = 1 / (Gamma (1 - beta . n_hat)).
 *  - The camera is orthographic.  The image plane passes through `center` and is
 *    normal to s_hat; s is measured from that plane, so t_bar = t_obs - s/c.
 *  - e_v is `up` projected onto the image plane and normalised, e_u = s_hat x e_v.
 *    Pixel (p, q) has its centre at center + (p + 1/2 - W/2) h_u e_u +
 *    (q + 1/2 - H/2) h_v e_v with h_u = fov_u / W, h_v = fov_v / H, and is stored
 *    at out[q * W + p] (row q = 0 is the bottom row).
 *  - The temporal weight of a cell uses t_bar at the midpoint of its chord.
 *    The weights W_{n,m} = 1 - |t_bar - t_m| / dt (for the two snapshots that
 *    bracket t_bar) are summed over the stored snapshots only, so a t_bar
 *    within one cadence outside [t_0, t_{M-1}] keeps a linearly fading weight
 *    on the end snapshot and anything further out contributes nothing.
 *    Without GBD_LOOKBACK every cell is read at t_obs, clamped to
 *    [t_0, t_{M-1}].
 */
#ifndef GBDART_H
#define GBDART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    GBD_OK = 0,
    GBD_ERR_INVALID = 1,   /* bad argument or bad field value                 */
    GBD_ERR_NOMEM = 2,     /* a device or pinned host allocation failed        */
    GBD_ERR_BUDGET = 3,    /* the request can never fit the context's HBM budget */
    GBD_ERR_NOTFOUND = 4,  /* unknown volume handle or ticket                  */
    GBD_ERR_TIMEOUT = 5,   /* a bounded wait ran out                           */
    GBD_ERR_CUDA = 6,      /* a CUDA runtime call failed (message has details) */
    GBD_ERR_CANCELLED = 7, /* the request was cancelled                        */
    GBD_ERR_BUSY = 8       /* the resource is in use (e.g. unload while queued)*/
};

/* Input precision of the snapshot arrays handed to gbd_load_snapshots. */
enum { GBD_IN_F64 = 0, GBD_IN_F32 = 1 };

/* Storage format of the packed volume on the device.
 *  GBD_STORE_F32:      16-byte record {j', beta_x, beta_y, beta_z} in float32.
 *  GBD_STORE_BF16_F16U: 8-byte record {bfloat16 j', float16 u_x, u_y, u_z} with
 *                      u = Gamma beta, the spatial four-velocity.  j' is rounded
 *                      to float32 then to bfloat16 (nearest even); u is computed
 *                      in float64 from the input and rounded once to float16.  The
 *                      four-velocity keeps the Doppler factor well conditioned
 *                      as |beta| -> 1; the arithmetic still accumulates in
 *                      float32. */
enum { GBD_STORE_F32 = 0, GBD_STORE_BF16_F16U = 1 };

/* View flags: routine A of the paper is 0, routine B is GBD_BEAMING, routine C
 * (the default of the paper) is GBD_BEAMING | GBD_LOOKBACK (Sec. 3, Table 1). */
enum { GBD_BEAMING = 1u, GBD_LOOKBACK = 2u };

typedef struct gbd_ctx gbd_ctx;
typedef uint64_t gbd_volume;

/* Uniform Cartesian mesh in the lab frame and its snapshot cadence
 * (Sec. 2.3: t_m = t_0 + m dt; Sec. 2.4: cells need not be cubic). */
typedef struct {
    int32_t n[3];        /* cells along x, y, z (each >= 1, <= 4096)        */
    double origin[3];    /* lower corner of cell (0, 0, 0)                  */
    double dx[3];        /* cell edge along x, y, z (> 0)                   */
    int32_t n_epochs;    /* M >= 1 snapshots                                */
    double t0, dt;       /* epoch m at t0 + m dt; dt > 0                    */
} gbd_grid;

/* The three inputs of the method (Sec. 2.5): rest-frame emissivity j' and
 * velocity beta = v/c per cell and epoch; alpha is given per view.
 *  j   : [M][n_z][n_y][n_x]     C order, x fastest
 *  vel : [M][n_z][n_y][n_x][3]  C order, components (x, y, z)
 * Both are read during the call only; the caller keeps ownership.  When
 * on_device is nonzero both are device pointers on the context's device,
 * otherwise host pointers; device inputs are read after all work already
 * launched on the device has finished (the call waits for it).  j' < 0, non-finite values or |beta| >= 1 reject
 * the whole load with GBD_ERR_INVALID. */
typedef struct {
    const void *j;
    const void *vel;
    int32_t dtype_in;    /* GBD_IN_F64 or GBD_IN_F32                        */
    int32_t store;       /* GBD_STORE_F32 or GBD_STORE_BF16_F16U            */
    int32_t on_device;
    int32_t brick;       /* layout: brick edge 4 or 8; 0 = library default  */
    int32_t super_brick; /* bricks per super-brick edge 1, 2 or 4; 0 = default */
    int32_t paired;      /* 1: keep the records of snapshots m and m + 1 of
                            each cell side by side (M + 1 blocks), so a cell
                            sample under lookback is one contiguous load;
                            costs about 2 (M + 1) / M times the memory      */
    int32_t morton_cells;/* 1: cells inside a brick in Morton order instead
                            of x fastest                                    */
} gbd_fields;

/* One observation (Secs. 2.1-2.2, 2.5). */
typedef struct {
    double dir[3];       /* viewing direction s_hat into the scene (any length > 0) */
    double up[3];        /* image up before projection; not parallel to dir  */
    double center[3];    /* image-plane centre; s = 0 there                  */
    double t_obs;        /* observer time                                    */
    double c;            /* signal speed; may be +infinity (fast-light limit) */
    double alpha;        /* rest-frame spectral slope (paper sign, e.g. -0.6) */
    double nu_ratio;     /* nu / nu'_0 > 0 (Eq. 20)                          */
    uint32_t flags;      /* GBD_BEAMING | GBD_LOOKBACK                       */
} gbd_view;

/* Image geometry and destination.  out holds width*height floats (per view
 * for batch calls, views stored one after another).  out is a device pointer
 * unless out_on_host is nonzero, in which case the library renders into its
 * own device buffer and copies the image to the host pointer on the stream
 * (pinned host memory makes that copy asynchronous).  samples, if not NULL,
 * is a device array receiving per pixel the number of cell-samples (cells
 * with a positive chord and a nonzero temporal weight); it is ignored when
 * out_on_host is set. */
typedef struct {
    int32_t width, height;   /* pixels, each in [1, 16384]                  */
    double fov_u, fov_v;     /* image extent along e_u and e_v (> 0)        */
    float *out;
    uint32_t *samples;
    int32_t out_on_host;
} gbd_image_spec;

/* Launch configuration of the march kernels (chosen by gbd_tune or given).
 * A render called with launch NULL uses the tuned configuration of its class
 * if gbd_tune has run for it, otherwise packet 8x4, 4 warps, depth 2,
 * persistent, capped registers, no region schedule, time groups of up to 4.
 * In a given struct, zero packet/warps/depth/group fields take those
 * defaults. */
typedef struct {
    int32_t packet_w, packet_h;  /* pixels of one warp packet: 8x4, 4x8, 16x2, 32x1 */
    int32_t cta_warps;           /* warps per CTA: 1, 2, 4 or 8                     */
    int32_t depth;               /* cells gathered ahead per lane: 1, 2 or 4       */
    int32_t persistent;          /* 1 = CTAs loop over their view's tile counter;
                                    0 = one packet per warp, one launch wave    */
    int32_t regcap;              /* 1 = kernel built for at most 80 registers/thread */
    int32_t region;              /* batches: 0 = march every ray whole; 16, 32, 64
                                    or 128 = region schedule: march all views' rays
                                    region by region (edge^3 cells, while the region
                                    is in L2), then add each ray's region sums in
                                    order.  Images agree with the whole-ray march to
                                    FP32 rounding (a few 1e-6), not bitwise.  Not
                                    used with sample counts or for batches of more
                                    than 65535 views (their rays march whole);
                                    depth 1 or 2.  Needs
                                    device scratch of 4 B per pixel and partial
                                    slot (the regions along the three axes, less
                                    two) plus 4 B per listed ray; a batch whose
                                    scratch does not fit fails with GBD_ERR_NOMEM,
                                    and the autotuner leaves such schedules out.    */
    int32_t group;               /* batches: time groups.  Consecutive views that
                                    differ only in observer time (same image plane,
                                    direction and grid frame; t_obs, and with it the
                                    window, and nu_ratio free) are marched together,
                                    up to `group` per ray: one traversal, one sum per
                                    view.  0 = the default, 4; 1 = every view on its
                                    own; at most 8.  A grouped view agrees with its
                                    lone render to FP32 rounding, not bitwise.       */
} gbd_launch;

/* Description of a resident volume. */
typedef struct {
    gbd_grid grid;
    int32_t store;
    int32_t brick, super_brick, paired, morton_cells;
    uint64_t bytes;          /* device bytes held by the packed volume       */
    uint64_t record_bytes;   /* 16 (F32) or 8 (BF16_F16U)                    */
    int32_t n_channels;      /* extra emissivity channels (gbd_load_channels) */
    uint64_t channel_bytes;  /* device bytes of those channels               */
} gbd_volume_desc;

/* ------------------------------------------------------------ errors */
/* Static text for a status code. */
const char *gbd_error_string(int status);
/* Message of the last failing call made on this thread ("" if none).  The
 * pointer stays valid until the next call on the same thread. */
const char *gbd_last_error(void);

/* ------------------------------------------------------------ context */
/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold for packed volumes, render buffers and queued
 * requests (0 = 90% of the device's free memory at creation).  *out receives
 * the context, or NULL on failure. */
int gbd_create(gbd_ctx **out, int32_t device, uint64_t hbm_budget_bytes);
/* Waits for the context's outstanding work, frees everything it holds and the
 * context itself.  NULL is accepted. */
int gbd_destroy(gbd_ctx *ctx);

/* ------------------------------------------------------------ volumes */
/* Validates the fields, copies them to the device if needed and packs them
 * into the bricked record layout (device work on an internal stream, finished
 * before the call returns).  *out receives a handle owned by the context until
 * gbd_unload.  GBD_ERR_BUDGET if the packed volume does not fit the budget. */
int gbd_load_snapshots(gbd_ctx *ctx, const gbd_grid *grid, const gbd_fields *fields, gbd_volume *out);
/* Frees a volume.  GBD_ERR_BUSY if queued serving requests still use it. */
int gbd_unload(gbd_ctx *ctx, gbd_volume vol);
int gbd_volume_info(gbd_ctx *ctx, gbd_volume vol, gbd_volume_desc *out);

/* ------------------------------------------------------------ rendering */
/* Renders one view into spec->out (Eq. 19 for every pixel), asynchronously on
 * `stream`.  launch may be NULL (tuned or default configuration). */
int gbd_render(gbd_ctx *ctx, gbd_volume vol, const gbd_view *view, const gbd_image_spec *spec,
               const gbd_launch *launch, void *stream);

/* Renders n views of the same image geometry; view k goes to spec->out +
 * k * width * height (and the sample counts likewise).  Views travel in the
 * kernel launch parameters, up to 128 per launch (larger batches are several
 * launches); the per-view tile counters live in a context-owned device
 * buffer.  The launches are built once into a CUDA graph per (volume, n,
 * geometry, destination, launch) and replayed afterwards, with new views
 * written into the graph's kernel parameters.
 * Concurrent batch calls on one context are serialised on the context's lock,
 * and the GPU work of consecutive calls is ordered on their streams. */
int gbd_render_batch(gbd_ctx *ctx, gbd_volume vol, const gbd_view *views, int32_t n,
                     const gbd_image_spec *spec, const gbd_launch *launch, void *stream);

/* Batch rendering without allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot let the library allocate device
 * memory while they render -- applications that hand the whole device to
 * their own allocator or memory pool up front, and latency-critical loops
 * where cudaMalloc / cudaFree (which may synchronise the device) are not
 * acceptable.  It renders like gbd_render_batch, but keeps the per-view tile
 * counters of the persistent launch in one fixed-size device array of the
 * library (4 KB, held by every GPU that loads the library until the process
 * exits) instead of allocating them, and uses no CUDA graph.
 * Limits and behaviour:
 *  - at most GBD_NOALLOC_MAX_VIEWS views per call, otherwise GBD_ERR_INVALID;
 *  - spec->out (and spec->samples, if set) must be device memory;
 *    out_on_host is rejected with GBD_ERR_INVALID;
 *  - the whole-ray march only: an explicit launch with region != 0 is
 *    rejected with GBD_ERR_INVALID, and a tuned region schedule is replaced
 *    by the persistent whole-ray march with the tuned packet, CTA and group
 *    shapes (its images then agree with gbd_render_batch's to float32
 *    rounding, as any region render does); tiles are taken in counter order,
 *    never from the centre-first order table (which would need an allocation);
 *    otherwise the images equal gbd_render_batch's bit for bit;
 *  - the first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress) and keeps it for the life of the process;
 *    make that first call before any stream capture, and do not use this entry
 *    point on a device after a cudaDeviceReset there;
 *  - every call shares the one array, which keeps the last call's contents
 *    (the tile counters are cleared by each call): calls whose GPU work overlaps,
 *    from any context or stream on the same device, race on it, so the caller
 *    orders them (for example on one stream). */
#define GBD_NOALLOC_MAX_VIEWS 1024
int gbd_render_batch_noalloc(gbd_ctx *ctx, gbd_volume vol, const gbd_view *views, int32_t n,
                             const gbd_image_spec *spec, const gbd_launch *launch, void *stream);

/* Out-of-core rendering (the paper's partial sub-region renders and
 * selective snapshot loading, Secs. 5.2 and 6.2).  Renders n views of a
 * volume that stays in host memory: the volume is cut into slabs of `slab`
 * cells along z (0: 64); each slab is uploaded, with flexload only the
 * snapshots that some view's rays inside the slab can reach in time, packed
 * on the device as a volume of its own and marched for every view, its sums
 * added to the images.  Two slab buffers alternate, so a slab's upload and
 * packing on the context's load stream overlap the previous slab's march on
 * `stream`.
 *  - fields: host arrays (pinned for overlapped copies; on_device must be 0),
 *    laid out as for gbd_load_snapshots; store, brick and super_brick apply to
 *    the slabs;
 *  - spec->out (and samples) must be device memory; they are overwritten;
 *  - the images agree with gbd_render_batch of the whole volume to float32
 *    rounding (each slab restarts the ray's anchor; within 2e-5 relative);
 *  - device memory: two slab buffers (records of the slab's snapshots, its
 *    tables, the slab's raw fields), checked against the budget
 *    (GBD_ERR_BUDGET);
 *  - the call returns when the images are complete; info receives the slabs
 *    marched and the bytes uploaded against the bytes of the whole series. */
typedef struct {
    int32_t slab;              /* in: cells per slab along z (0 = 64)                 */
    int32_t flexload;          /* in: 1 = upload only the snapshots a slab can reach  */
    int32_t slabs;             /* out: slabs marched (slabs no ray reaches are skipped) */
    uint64_t bytes_uploaded;   /* out: raw field bytes copied to the device           */
    uint64_t bytes_total;      /* out: raw field bytes of the whole series            */
} gbd_stream_info;
int gbd_render_streamed(gbd_ctx *ctx, const gbd_grid *grid, const gbd_fields *fields, const gbd_view *views,
                        int32_t n, const gbd_image_spec *spec, const gbd_launch *launch, gbd_stream_info *info,
                        void *stream);

/* Labelled mode (the paper's second input form, Sec. 4): a scene made of
 * several sub-domains of locally homogeneous resolution -- for instance the
 * levels of a mesh-refined simulation -- each loaded as its own volume with
 * its own grid (origin, cell size, dimensions, snapshot times).  A pixel's
 * intensity is the sum over the sub-domains of its ray's sum through each
 * (Eq. 19 over the union of their cells); the sub-domains are marched in the
 * order given and added into spec->out (device memory, overwritten).  The
 * boxes of the sub-domains must not overlap (they may touch), otherwise
 * GBD_ERR_INVALID: where a refined level covers a coarser one, the coarser
 * one is to be cut into boxes around it. */
int gbd_render_labelled(gbd_ctx *ctx, const gbd_volume *vols, int32_t n_vols, const gbd_view *views, int32_t n,
                        const gbd_image_spec *spec, const gbd_launch *launch, void *stream);

/* Vector line-of-sight integration (Sec. 2.1: the traced field f may be a
 * vector; the paper's code integrates a scalar).  gbd_load_channels attaches
 * n_channels (1 or 3) more rest-frame emissivity fields to a volume, laid out
 * [n_channels][M][nz][ny][nx] (C order) like j', sharing the volume's
 * velocity: any finite values (a channel may be a signed component, as for
 * polarisation-ready integrands).  They are stored as float32 in the volume's
 * cell layout (4 bytes per cell, snapshot and channel, charged to the budget)
 * and replace channels loaded before; a re-layout moves them along.
 * gbd_render_vector marches each ray once and sums every channel with the same
 * weights and Doppler factors as j' (Eq. 19 per channel): spec->out receives
 * [n][1 + n_channels][height][width], component 0 being the image of j'.
 * Device output only, no sample counts. */
int gbd_load_channels(gbd_ctx *ctx, gbd_volume vol, const void *channels, int32_t n_channels, int32_t dtype_in,
                      int32_t on_device);
int gbd_render_vector(gbd_ctx *ctx, gbd_volume vol, const gbd_view *views, int32_t n, const gbd_image_spec *spec,
                      const gbd_launch *launch, void *stream);

/* Memory analysis: *records receives the number of distinct (cell, snapshot)
 * records the samples of a batch render of these views read (each counted
 * once however many rays or views read it).  Times the record size, it is
 * the compulsory floor of the render's memory traffic.  The march runs as for
 * gbd_render_batch but marks a bitmap of one bit per cell and snapshot (held
 * during the call) instead of reading records; spec->out is not used. */
int gbd_touched_records(gbd_ctx *ctx, gbd_volume vol, const gbd_view *views, int32_t n,
                        const gbd_image_spec *spec, uint64_t *records);

/* Number of kernels the last successful render call of this thread
 * launched (graph replays count their kernels). */
int32_t gbd_last_launch_count(void);

/* ------------------------------------------------------------ serving
 * Continuous batching of render requests against resident volumes.  Requests
 * of any volume, storage, image size and orientation are queued; a scheduler
 * thread of the context admits them into waves as request slots and device
 * memory free up (a request holds its library-side device bytes -- its image,
 * when the output is host memory -- from launch to completion) and runs each
 * wave as launches over all of its requests' pixel tiles (up to 96 requests
 * per launch, one CTA per warps-per-CTA tiles of a request).  Up to
 * max_waves waves are on the GPU at once on separate streams, so requests that
 * arrive while others run start as soon as the GPU has room.  Every pixel is
 * computed by the same per-ray code as gbd_render, so a request's image is the
 * same whether it is served alone or in a mix.  A volume with queued or
 * running requests cannot be unloaded or re-laid-out (GBD_ERR_BUSY).  Do not
 * call gbd_serve_stop or gbd_destroy while other threads poll or wait. */
typedef struct {
    gbd_volume volume;
    gbd_view view;
    gbd_image_spec spec;     /* out: device memory, or pinned host memory with
                                out_on_host (pageable host memory is rejected) */
    int32_t priority;        /* higher first; arrival order within a priority */
} gbd_request;

typedef struct {
    int32_t status;          /* final status of the request                  */
    double queue_ms;         /* submission to the launch of its wave         */
    double latency_ms;       /* submission to the end of its wave on the GPU */
    double device_ms;        /* GPU time of its wave                         */
} gbd_stats;

typedef struct {
    int32_t max_waves;               /* waves on the GPU at once (default 3, at most 8)  */
    int32_t max_requests_per_wave;   /* default 256, at most 4096                       */
    int32_t max_requests_in_flight;  /* request slots (default 1024)                    */
    uint64_t request_budget_bytes;   /* device bytes for running requests; 0 = what the
                                        volumes leave of the context budget.  Each
                                        request is charged its image (4 B per pixel,
                                        twice with device sample counts): a device
                                        buffer of the library's for host output, the
                                        caller's own buffer for device output      */
    gbd_launch launch;               /* wave kernel configuration (depth 1 or 2); all
                                        zero: packet 8x4, 4 warps, depth 2, capped
                                        registers                                 */
} gbd_serve_config;

typedef struct {
    uint64_t completed;              /* requests finished since the last reset    */
    double p50_ms, p99_ms, max_ms;   /* submission-to-done latency percentiles    */
    double requests_per_s;           /* completed / (last done - first submission) */
    uint64_t waves;                  /* waves launched                            */
    double mean_requests_per_wave;
    int32_t max_waves_in_flight;     /* most waves seen on the GPU at once        */
    int32_t pending, in_flight;      /* requests queued / running now             */
} gbd_serve_summary;

/* Starts the scheduler (config may be NULL for defaults).  gbd_submit starts
 * it with defaults if needed. */
int gbd_serve_start(gbd_ctx *ctx, const gbd_serve_config *config);
/* Cancels queued requests, lets running waves finish, stops the scheduler. */
int gbd_serve_stop(gbd_ctx *ctx);
/* Queues a request; *ticket identifies it.  GBD_ERR_BUDGET if it can never
 * fit the serving budget; GBD_ERR_NOTFOUND for an unknown volume. */
int gbd_submit(gbd_ctx *ctx, const gbd_request *req, uint64_t *ticket);
/* Non-blocking: *done = 1 once the request has ended (its stats then hold the
 * final status, which is also returned); a finished request is reported once. */
int gbd_poll(gbd_ctx *ctx, uint64_t ticket, int32_t *done, gbd_stats *stats);
/* Waits up to timeout_ms for the request; GBD_ERR_TIMEOUT if it is still
 * queued or running (it stays valid and can be waited for again). */
int gbd_wait(gbd_ctx *ctx, uint64_t ticket, uint32_t timeout_ms, gbd_stats *stats);
/* A queued request is removed; a running one drains and ends with
 * GBD_ERR_CANCELLED (its output may have been written). */
int gbd_cancel(gbd_ctx *ctx, uint64_t ticket);
/* Latency percentiles and throughput of completed requests; reset != 0
 * clears the counters after reading. */
int gbd_serve_stats(gbd_ctx *ctx, int32_t reset, gbd_serve_summary *out);

/* ------------------------------------------------------------ autotuning
 * The paper runs one kernel shape; the launch configuration (warp packet
 * shape, warps per CTA, cells gathered ahead per lane) and the volume layout
 * (brick and super-brick edge) are tuned here per class of render: grid
 * dimensions, storage, snapshot count, image size, batch size and lookback.
 */
enum { GBD_TUNE_LAUNCH = 1u, GBD_TUNE_LAYOUT = 2u };

typedef struct {
    gbd_launch launch;       /* best launch configuration found            */
    int32_t brick;           /* layout of the volume after tuning          */
    int32_t super_brick;
    int32_t paired;
    int32_t morton_cells;
    float ms;                /* median time of the best candidate          */
    int32_t candidates;      /* configurations timed                       */
} gbd_tune_result;

/* Times candidate configurations for rendering `views` (as gbd_render_batch
 * would, writing into spec->out, which must be device memory) on `stream`
 * and synchronises it.  With GBD_TUNE_LAYOUT the volume is re-packed on the
 * device into each candidate layout (bricks, and the paired-snapshot form when
 * it fits) and left in the fastest one (the handle stays valid; the re-pack
 * needs room for a second copy within the budget).
 * The best launch configuration is remembered by the context and used by
 * gbd_render and gbd_render_batch calls of the same class that pass
 * launch = NULL.  With the environment variable GBD_TUNE_CACHE naming a file,
 * results are appended to it and read back by later contexts. */
int gbd_tune(gbd_ctx *ctx, gbd_volume vol, const gbd_view *views, int32_t n, const gbd_image_spec *spec,
             uint32_t what, void *stream, gbd_tune_result *out);

/* Re-packs a volume into another layout on the device (brick 1, 2, 4 or 8;
 * super_brick 1, 2 or 4; paired 0 or 1; morton_cells 0 or 1), keeping its
 * handle.  Waits for the device.  Needs room for both copies within the
 * budget while it runs. */
int gbd_relayout(gbd_ctx *ctx, gbd_volume vol, int32_t brick, int32_t super_brick, int32_t paired,
                 int32_t morton_cells);

/* Bounds checking.  In the library built with GBD_CHECKED every gather tests
 * its cell and epoch index against the volume; a violation skips the load and
 * sets bit 0 of a device word instead of faulting.  In every build, the
 * region schedule sets bit 1 if a region's ray list ever ran out of room (its
 * size comes from a bound on the pixels a region can cover, so this does not
 * happen; the rays past the end would go unmarched).  This call waits for the
 * device, stores that word in *out (0 = no violation) and clears it. */
int gbd_bounds_violations(gbd_ctx *ctx, int32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* GBDART_H */
