// runtime.h -- host-side state of a context (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "gbd_internal.h"

namespace gbd {

// A packed, device-resident snapshot series.
struct Volume {
    gbd_grid grid{};
    int store = GBD_STORE_F32;
    int brick = 8, super_brick = 4;
    int paired = 0;                  // blocks of side-by-side snapshot pairs
    int plain_boost = 0;             // bfloat16/float16 records with Gamma^2 <= kPlainGamma2
    int morton_cells = 0;            // Morton order of the cells inside a brick
    void *rec = nullptr;             // records, block after block
    int32_t *axis_off = nullptr;     // per-axis offset tables (n_x + n_y + n_z), then the march tables
    long long epoch_stride = 0;      // records per block (epoch, or epoch pair)
    uint64_t bytes = 0;              // device bytes charged to the budget
    float *chan = nullptr;           // extra emissivity channels (vector renders), unpaired layout
    int n_chan = 0;
    long long chan_stride = 0;       // floats per snapshot of one channel
    uint64_t chan_bytes = 0;         // device bytes of the channels (charged to the budget)
    std::atomic<int> pinned_by_requests{0};  // queued or running serving requests using it
};

struct GraphCache;
struct Server;

// Autotuning class of a render: results are cached per key.
struct TuneKey {
    int n[3];
    int M, store, width, height, n_views, lookback;
    bool operator<(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) < 0; }
};

struct TuneEntry {
    LaunchCfg cfg{8, 4, 8, 2, 1, 0, 0, kGroupDefault};
    int brick = 8, super_brick = 4;
    float ms = 0.f;
};

}  // namespace gbd

struct gbd_ctx {
    int device = 0;
    int num_sms = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::mutex mu;
    std::map<gbd_volume, std::unique_ptr<gbd::Volume>> volumes;
    gbd_volume next_id = 0;
    cudaStream_t load_stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t aux[4] = {};         // side streams of multi-volume renders (created on first use)
    cudaEvent_t aux_done[4] = {};
    // End of the march of the last region-schedule batch enqueued, on any
    // stream: the next one waits for it, so that two batches never march side
    // by side (each relies on its regions' records staying in L2), while a
    // batch's copy to host memory still overlaps the next batch's march.
    cudaEvent_t region_done = nullptr;
    int *err_word = nullptr;          // bounds-check word of checked builds
    gbd::GraphCache *graphs = nullptr;
    gbd::Server *server = nullptr;
    std::map<gbd::TuneKey, gbd::TuneEntry> tuned;
    std::map<std::array<int, 4>, int *> tile_orders;  // device tables of tile_order(), by image and packet shape
    ~gbd_ctx();
    gbd::Volume *find(gbd_volume id);
};

namespace gbd {

using Ctx = ::gbd_ctx;

// Errors: record a message for gbd_last_error() and return the code.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
void set_launch_count(int32_t n);

// Restores the caller's current device on scope exit.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;

  private:
    int prev_ = 0;
};

// Settings read from the environment once (runtime.cpp).
bool graphs_enabled();                 // GBD_GRAPHS=0 disables graph replay of batches
bool fault_injected(const char *site); // GBD_FAULT=alloc:N,admit:N fails the N-th call at a site
void reset_fault_counters();

// View and launch helpers (api.cpp).
int make_view(const Volume &vol, const gbd_view &v, int width, int height, double fov_u, double fov_v, ViewDev &out);
int check_grid_fields(const gbd_grid &g, const gbd_fields &f);
int check_spec(const gbd_image_spec *s);
VolDev vol_dev(const Volume &v);
LaunchCfg resolve_launch(const gbd_launch *l);
int check_launch(const LaunchCfg &c);
// A batch of n views runs as march_chunks(n) launches; fill_args sets up the
// arguments of launch c from the host view array hv.
int march_chunks(int n);
double view_work(const Volume &vol, const ViewDev &V, int width, int height);
// Region schedule (see RegionArgs): slots per ray, 0 when it does not apply.
int region_slots(const Volume &vol, const LaunchCfg &cfg, const gbd_image_spec &spec, int nreg[3], long long n_views);
struct RegionPlan {
    int slots = 0, nreg[3] = {0, 0, 0};
    size_t regions = 0;
    int ctas_per_view = 0;
    size_t rays_off = 0, count_off = 0, views_off = 0, proj_off = 0, image_off = 0, order_off = 0, total = 0;
    std::vector<char> tables;  // host image of the scratch from views_off to total
};
RegionPlan region_plan(const Volume &vol, const LaunchCfg &cfg, const gbd_image_spec &spec,
                       const std::vector<ViewDev> &hv);
cudaError_t upload_region_tables(const RegionPlan &P, char *scratch, cudaStream_t st);
cudaError_t enqueue_regions(Ctx &ctx, const Volume &vol, const std::vector<ViewDev> &hv, const RegionPlan &P,
                            const gbd_image_spec &spec, const LaunchCfg &cfg, float *dev_out, char *scratch,
                            cudaStream_t st, int *launches);
std::vector<double> view_works(const Volume &vol, const std::vector<ViewDev> &hv, int width, int height);
void fill_args(MarchArgs &a, const Volume &vol, const ViewDev *hv, int n, int c, const gbd_image_spec &s,
               float *out, uint32_t *samples, int *queue, const LaunchCfg &cfg, int *err_word);
// Time groups of a filled launch (batched renders; see MarchArgs).
void group_views(MarchArgs &a, int gmax);
// The order in which persistent warps take a view's tiles: by distance of the
// tile from the image centre, nearest first (the longest rays of a centred
// box first, so the launch ends on short ones).  A device table cached in the
// context for up to 64 image geometries; NULL (counter order) beyond them or
// if it cannot be made.  Used by launches of one
// view or time group; with several, warps move on to the other views' tiles
// instead, and counter order keeps neighbouring warps on neighbouring tiles.
const int *tile_order(Ctx &ctx, int width, int height, int packet_w, int packet_h);
// Views, or time groups when grouped, of a filled launch.
int launch_units(const MarchArgs &a);
bool build_layout(const int n[3], int B, int S, std::vector<int32_t> &tab, long long &epoch_stride, int morton_cells);
void destroy_graph_cache(GraphCache *g);

void drop_graphs_for(Ctx &ctx, gbd_volume vol);
int render_direct(Ctx &ctx, const Volume &vol, const std::vector<ViewDev> &hv, const gbd_image_spec &spec,
                  const LaunchCfg &cfg, cudaStream_t st);

// Autotuning (tune.cpp).
TuneKey tune_key(const Volume &vol, int width, int height, int n_views, uint32_t flags);
bool lookup_tuned(Ctx &ctx, const TuneKey &k, LaunchCfg &cfg);
void load_tune_file(Ctx &ctx);
int relayout_volume(Ctx &ctx, Volume &vol, gbd_volume vid, int B, int S, int paired, int morton_cells);
size_t volume_bytes(int store, long long cells_per_epoch, int M, int paired, long long *stride);

// Serving (serve.cpp).
int serve_start(Ctx &ctx, const gbd_serve_config *c);
void serve_shutdown(Ctx &ctx);

}  // namespace gbd
