// api.cpp -- host runtime behind the C ABI of include/gbdart.h.
//
// Owns contexts, the registry of packed volumes, the per-view set-up done in
// float64 on the host (camera basis, pixel pitch, lookback window, power-law
// prefactor), HBM budget accounting, the cached CUDA graphs of batch renders,
// and error reporting.  All device work is issued through the kernels of
// march.cu and pack.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gbd_internal.h"
#include "runtime.h"

namespace gbd {

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string t_last_error;
thread_local int32_t t_last_launches = 0;
}  // namespace

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    if (e == cudaErrorMemoryAllocation) return fail(GBD_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(GBD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void set_launch_count(int32_t n) { t_last_launches = n; }

DeviceGuard::DeviceGuard(int dev)
{
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard()
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != prev_) cudaSetDevice(prev_);
}

// ------------------------------------------------------------------ layout
// Per-axis offset tables of the bricked layout.  With brick edge B and
// super-brick edge S (in bricks), the grid is padded to multiples of B*S; the
// super-bricks are stored in x-fastest order, the S^3 bricks inside a
// super-brick in Morton order, and the B^3 cells inside a brick x-fastest.
// Each of the three contributions is a function of one axis only, so the
// record offset is tab_x[ix] + tab_y[iy] + tab_z[iz].  B = S = 1 gives the
// plain C-ordered layout.
static uint32_t spread3(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

bool build_layout(const int n[3], int B, int S, std::vector<int32_t> &tab, long long &epoch_stride, int morton_cells)
{
    const long long E = static_cast<long long>(B) * S;
    long long P[3], NS[3];
    for (int a = 0; a < 3; ++a) {
        P[a] = (n[a] + E - 1) / E * E;
        NS[a] = P[a] / E;
    }
    const long long super_vol = E * E * E;
    epoch_stride = NS[0] * NS[1] * NS[2] * super_vol;
    if (epoch_stride >= (1LL << 31)) return false;
    const long long B3 = static_cast<long long>(B) * B * B;
    const long long super_stride[3] = {super_vol, NS[0] * super_vol, NS[0] * NS[1] * super_vol};
    const long long cell_stride[3] = {1, B, static_cast<long long>(B) * B};
    tab.resize(static_cast<size_t>(n[0] + n[1] + n[2]));
    size_t w = 0;
    for (int a = 0; a < 3; ++a) {
        for (int i = 0; i < n[a]; ++i) {
            const long long sup = i / E;
            const uint32_t bin = static_cast<uint32_t>((i / B) % S);
            const long long morton = static_cast<long long>(spread3(bin)) << a;
            // cells inside a brick: x fastest, or Morton order (bits of the
            // three local coordinates interleaved, again one term per axis)
            const long long local = morton_cells ? static_cast<long long>(spread3(static_cast<uint32_t>(i % B))) << a
                                                 : (i % B) * cell_stride[a];
            tab[w++] = static_cast<int32_t>(sup * super_stride[a] + morton * B3 + local);
        }
    }
    // the march tables follow the pack tables in the same device array
    tab.resize(w + static_cast<size_t>(march_table_entries(n)));
    size_t src = 0;
    for (int a = 0; a < 3; ++a) {
        int32_t *fwd = tab.data() + w + march_table_base(n, a);
        int32_t *rev = fwd + n[a] + 2;
        for (int i = 0; i < n[a]; ++i) {
            fwd[i] = tab[src + i];
            rev[i] = tab[src + n[a] - 1 - i];
        }
        fwd[n[a]] = fwd[n[a] + 1] = kTabSentinel;
        rev[n[a]] = rev[n[a] + 1] = kTabSentinel;
        src += n[a];
    }
    return true;
}

// Validates a grid and the description of its fields (not their values).
int check_grid_fields(const gbd_grid &g, const gbd_fields &f)
{
    for (int i = 0; i < 3; ++i) {
        if (g.n[i] < 1 || g.n[i] > kMaxAxis) return fail(GBD_ERR_INVALID, "grid: n[%d] must be in [1, %d]", i, kMaxAxis);
        if (!(g.dx[i] > 0.0) || !std::isfinite(g.dx[i]) || !std::isfinite(g.origin[i]))
            return fail(GBD_ERR_INVALID, "grid: dx must be positive and origin finite");
    }
    if (g.n_epochs < 1 || g.n_epochs > 1000000) return fail(GBD_ERR_INVALID, "grid: n_epochs must be >= 1");
    if (!(g.dt > 0.0) || !std::isfinite(g.dt) || !std::isfinite(g.t0))
        return fail(GBD_ERR_INVALID, "grid: dt must be positive and t0 finite");
    if (!f.j || !f.vel) return fail(GBD_ERR_INVALID, "fields: NULL array");
    if (f.dtype_in != GBD_IN_F64 && f.dtype_in != GBD_IN_F32) return fail(GBD_ERR_INVALID, "fields: bad dtype_in");
    if (f.store != GBD_STORE_F32 && f.store != GBD_STORE_BF16_F16U) return fail(GBD_ERR_INVALID, "fields: bad store");
    const int B = f.brick ? f.brick : 8;
    const int S = f.super_brick ? f.super_brick : 4;
    if (B != 1 && B != 2 && B != 4 && B != 8) return fail(GBD_ERR_INVALID, "fields: brick must be 1, 2, 4 or 8");
    if (S != 1 && S != 2 && S != 4) return fail(GBD_ERR_INVALID, "fields: super_brick must be 1, 2 or 4");
    return GBD_OK;
}

// ------------------------------------------------------------------ views
static bool finite3(const double v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int make_view(const Volume &vol, const gbd_view &v, int width, int height, double fov_u, double fov_v, ViewDev &out)
{
    if (!finite3(v.dir) || !finite3(v.up) || !finite3(v.center) || !std::isfinite(v.t_obs) ||
        !std::isfinite(v.alpha) || !(v.nu_ratio > 0.0) || !std::isfinite(v.nu_ratio) || std::isnan(v.c) ||
        !(v.c > 0.0))
        return fail(GBD_ERR_INVALID, "view: non-finite or out-of-range parameter");
    if ((v.flags & ~(GBD_BEAMING | GBD_LOOKBACK)) != 0u) return fail(GBD_ERR_INVALID, "view: unknown flag bits");
    if (width < 1 || height < 1 || width > 16384 || height > 16384)
        return fail(GBD_ERR_INVALID, "image: width/height must be in [1, 16384]");
    if (!(fov_u > 0.0) || !(fov_v > 0.0) || !std::isfinite(fov_u) || !std::isfinite(fov_v))
        return fail(GBD_ERR_INVALID, "image: fov must be positive and finite");
    double sh[3], ev[3], eu[3];
    const double nd = std::sqrt(v.dir[0] * v.dir[0] + v.dir[1] * v.dir[1] + v.dir[2] * v.dir[2]);
    if (!(nd > 0.0)) return fail(GBD_ERR_INVALID, "view: zero direction");
    for (int i = 0; i < 3; ++i) sh[i] = v.dir[i] / nd;
    // Components below 1e-20 are treated as exactly zero (the ray never
    // crosses a face of that axis within any representable grid).
    for (int i = 0; i < 3; ++i)
        if (std::fabs(sh[i]) < 1e-20) sh[i] = 0.0;
    const double us = v.up[0] * sh[0] + v.up[1] * sh[1] + v.up[2] * sh[2];
    for (int i = 0; i < 3; ++i) ev[i] = v.up[i] - us * sh[i];
    const double nv = std::sqrt(ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2]);
    if (!(nv > 1e-12)) return fail(GBD_ERR_INVALID, "view: up is parallel to dir");
    for (int i = 0; i < 3; ++i) ev[i] /= nv;
    eu[0] = sh[1] * ev[2] - sh[2] * ev[1];
    eu[1] = sh[2] * ev[0] - sh[0] * ev[2];
    eu[2] = sh[0] * ev[1] - sh[1] * ev[0];
    const double hu = fov_u / width, hv = fov_v / height;
    const double a0 = (0.5 - 0.5 * width) * hu, b0 = (0.5 - 0.5 * height) * hv;
    std::memset(&out, 0, sizeof(out));
    const gbd_grid &g = vol.grid;
    const int M = g.n_epochs;
    const double t0 = g.t0, dt = g.dt;
    const double two40 = 1099511627776.0, two32 = 4294967296.0;
    // Epoch coordinate u(s) = u_obs - kk s (Eq. 2 with t_m = t0 + m dt).
    const bool lookback = (v.flags & GBD_LOOKBACK) != 0u;
    double u_obs = (v.t_obs - t0) / dt;
    double kk = 0.0;
    double win_lo = -HUGE_VAL, win_hi = HUGE_VAL;
    if (lookback) {
        if (std::isinf(v.c)) {
            if (!(u_obs > -1.0 && u_obs < static_cast<double>(M))) win_lo = HUGE_VAL, win_hi = -HUGE_VAL;
        } else {
            // Retarded times inside (t0 - dt, t0 + M dt) reach a stored snapshot
            // (Eq. 9 over the stored m): s = c (t_obs - t_bar).
            kk = 1.0 / (v.c * dt);
            win_lo = v.c * (v.t_obs - t0 - M * dt);
            win_hi = v.c * (v.t_obs - t0 + dt);
        }
    } else {
        u_obs = std::min(std::max(u_obs, 0.0), static_cast<double>(M - 1));
    }
    double max_a = 0.0, reach = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double r00 = v.center[i] + a0 * eu[i] + b0 * ev[i];
        const double g00 = (r00 - g.origin[i]) / g.dx[i];
        const double gu = hu * eu[i] / g.dx[i], gv = hv * ev[i] / g.dx[i];
        // every pixel position must stay within the fixed-point range
        reach = std::max(reach, std::fabs(g00) + std::fabs(gu) * width + std::fabs(gv) * height + g.n[i]);
        // Components below 1e-9 count as parallel: such a ray moves less than
        // 1e-9 cells per unit length along that axis.
        const bool parallel = std::fabs(sh[i]) < 1e-9;
        // An axis the ray runs down is mirrored, g' = n - g, exactly in fixed
        // point, so that the march always steps up.
        const bool mirror = !parallel && sh[i] < 0.0;
        const long long n40 = static_cast<long long>(g.n[i]) << 40;
        out.g0[i] = mirror ? n40 - std::llround(g00 * two40) : std::llround(g00 * two40);
        out.gu[i] = mirror ? -std::llround(gu * two40) : std::llround(gu * two40);
        out.gv[i] = mirror ? -std::llround(gv * two40) : std::llround(gv * two40);
        if (mirror) out.flags |= kFlagMirror0 << i;
        const double a = parallel ? 0.0 : std::fabs(sh[i]) / g.dx[i];
        out.a_hi[i] = static_cast<float>(a);
        out.a_lo[i] = static_cast<float>(a - static_cast<double>(out.a_hi[i]));
        out.inv_a[i] = a != 0.0 ? static_cast<float>(1.0 / a) : 0.0f;
        const double w = a != 0.0 ? kk / a : 0.0;
        out.w_hi[i] = static_cast<float>(w);
        out.w_lo[i] = static_cast<float>(w - static_cast<double>(out.w_hi[i]));
        out.du[i] = std::llround(std::fabs(w) * two32);
        max_a = std::max(max_a, std::fabs(a));
        out.sh_hi[i] = static_cast<float>(sh[i]);
        out.sh_lo[i] = static_cast<float>(sh[i] - static_cast<double>(out.sh_hi[i]));
    }
    if (!(max_a > 0.0)) return fail(GBD_ERR_INVALID, "view: direction too small");
    if (reach > 4.0e6)
        return fail(GBD_ERR_INVALID, "view: image or grid farther than 4e6 cells from the grid origin");
    // The epoch coordinate along any ray stays within |u_obs| + kk * (path length).
    const double path = reach * std::sqrt(3.0) * std::max(g.dx[0], std::max(g.dx[1], g.dx[2]));
    if (std::fabs(u_obs) + kk * path > 1.0e8)
        return fail(GBD_ERR_INVALID, "view: observer time or c*dt puts the rays more than 1e8 snapshots away");
    out.u_obs = std::llround(u_obs * two32);
    out.kk_hi = static_cast<float>(kk);
    out.kk_lo = static_cast<float>(kk - static_cast<double>(out.kk_hi));
    const float fbig = 3.0e38f;
    out.win_lo = win_lo <= -1e38 ? -fbig : (win_lo >= 1e38 ? fbig : static_cast<float>(win_lo - 1e-6 * (1.0 + std::fabs(win_lo))));
    out.win_hi = win_hi >= 1e38 ? fbig : (win_hi <= -1e38 ? -fbig : static_cast<float>(win_hi + 1e-6 * (1.0 + std::fabs(win_hi))));
    out.flags |= v.flags;
    out.expo = static_cast<float>(2.0 - v.alpha);
    out.prefactor = static_cast<float>(std::pow(v.nu_ratio, v.alpha));
    if (!(out.prefactor > 0.0f) || !std::isfinite(out.prefactor))
        return fail(GBD_ERR_INVALID, "view: nu_ratio^alpha is not a positive float");
    return GBD_OK;
}

// Record bytes of a packed volume; *stride receives the records per block.
size_t volume_bytes(int store, long long cells_per_epoch, int M, int paired, long long *stride)
{
    const size_t rec = store == GBD_STORE_F32 ? 16 : 8;
    *stride = paired ? 2 * cells_per_epoch : cells_per_epoch;
    // paired: M + 1 blocks and one zero record pair after them, which a
    // sample that reads no snapshot loads instead of skipping its load
    return paired ? rec * (static_cast<size_t>(*stride) * static_cast<size_t>(M + 1) + 2)
                  : rec * static_cast<size_t>(*stride) * static_cast<size_t>(M);
}

VolDev vol_dev(const Volume &v)
{
    VolDev d;
    std::memset(&d, 0, sizeof(d));
    d.rec = v.rec;
    d.axis_off = v.axis_off;
    d.mtab = v.axis_off + (v.grid.n[0] + v.grid.n[1] + v.grid.n[2]);
    d.epoch_stride = v.epoch_stride;
    for (int i = 0; i < 3; ++i) d.n[i] = v.grid.n[i];
    d.M = v.grid.n_epochs;
    d.store = v.store;
    d.paired = v.paired;
    d.plain_boost = v.plain_boost;
    return d;
}

LaunchCfg resolve_launch(const gbd_launch *l)
{
    // the default: the shape the autotuner settles on for the workloads here
    // (8x4 packets, 4-warp CTAs, two cells ahead, capped registers, time
    // groups of up to four views)
    LaunchCfg c{8, 4, 4, 2, 1, 1, 0, kGroupDefault};
    if (l) {
        if (l->packet_w > 0) c.packet_w = l->packet_w;
        if (l->packet_h > 0) c.packet_h = l->packet_h;
        if (l->cta_warps > 0) c.cta_warps = l->cta_warps;
        if (l->depth > 0) c.depth = l->depth;
        c.persistent = l->persistent != 0;
        c.regcap = l->regcap != 0;
        c.region = l->region;
        if (l->group > 0) c.group = l->group;
    }
    return c;
}

int check_launch(const LaunchCfg &c)
{
    if (c.packet_w * c.packet_h != 32 || c.packet_w < 1 || c.packet_h < 1)
        return fail(GBD_ERR_INVALID, "launch: packet_w * packet_h must be 32");
    if (c.cta_warps != 1 && c.cta_warps != 2 && c.cta_warps != 4 && c.cta_warps != 8)
        return fail(GBD_ERR_INVALID, "launch: cta_warps must be 1, 2, 4 or 8");
    if (c.depth != 1 && c.depth != 2 && c.depth != 4) return fail(GBD_ERR_INVALID, "launch: depth must be 1, 2 or 4");
    if (c.region != 0 && c.region != 16 && c.region != 32 && c.region != 64 && c.region != 128)
        return fail(GBD_ERR_INVALID, "launch: region must be 0, 16, 32, 64 or 128");
    if (c.region != 0 && c.depth > 2) return fail(GBD_ERR_INVALID, "launch: the region schedule takes depth 1 or 2");
    if (c.group < 1 || c.group > kGroupMax) return fail(GBD_ERR_INVALID, "launch: group must be 0 (default) or 1 .. 8");
    return GBD_OK;
}

int check_spec(const gbd_image_spec *s)
{
    if (!s) return fail(GBD_ERR_INVALID, "image spec is NULL");
    if (s->width < 1 || s->height < 1 || s->width > 16384 || s->height > 16384)
        return fail(GBD_ERR_INVALID, "image: width/height must be in [1, 16384]");
    if (!s->out) return fail(GBD_ERR_INVALID, "image: out is NULL");
    return GBD_OK;
}

int march_chunks(int n) { return (n + kViewsPerLaunch - 1) / kViewsPerLaunch; }

// Estimated cell-samples of one view: the box-and-window chord of a 16 x 16
// subsample of its rays, times the cells crossed per unit length.  It only
// sizes the persistent grid's share per view, so a coarse figure will do.
double view_work(const Volume &vol, const ViewDev &V, int width, int height)
{
    const int sx = std::min(width, 16), sy = std::min(height, 16);
    double rate = 0.0;
    for (int i = 0; i < 3; ++i) rate += static_cast<double>(V.a_hi[i]) + V.a_lo[i];
    double cells = 0.0;
    for (int jy = 0; jy < sy; ++jy) {
        const int q = static_cast<int>((jy + 0.5) * height / sy);
        for (int jx = 0; jx < sx; ++jx) {
            const int p = static_cast<int>((jx + 0.5) * width / sx);
            double lo = V.win_lo, hi = V.win_hi;
            bool hit = true;
            for (int i = 0; i < 3 && hit; ++i) {
                const double g = static_cast<double>(V.g0[i] + p * V.gu[i] + q * V.gv[i]) * 0x1p-40;
                if (V.inv_a[i] != 0.f) {
                    lo = std::max(lo, -g * V.inv_a[i]);
                    hi = std::min(hi, (vol.grid.n[i] - g) * V.inv_a[i]);
                } else if (g < 0.0 || g >= vol.grid.n[i]) {
                    hit = false;
                }
            }
            if (hit && hi > lo) cells += (hi - lo) * rate + 1.0;
        }
    }
    return cells * (static_cast<double>(width) * height) / (static_cast<double>(sx) * sy);
}

std::vector<double> view_works(const Volume &vol, const std::vector<ViewDev> &hv, int width, int height)
{
    std::vector<double> w(hv.size());
    for (size_t k = 0; k < hv.size(); ++k) w[k] = view_work(vol, hv[k], width, height);
    return w;
}

// Launch arguments of chunk c of a batch of n views: views c K .. c K + K - 1
// (K = kViewsPerLaunch), their images and their tile counters.
void fill_args(MarchArgs &a, const Volume &vol, const ViewDev *hv, int n, int c, const gbd_image_spec &s,
               float *out, uint32_t *samples, int *queue, const LaunchCfg &cfg, int *err_word)
{
    std::memset(&a, 0, sizeof(a));
    const int first = c * kViewsPerLaunch;
    const int cnt = std::min(kViewsPerLaunch, n - first);
    const size_t img = static_cast<size_t>(first) * s.width * s.height;
    a.vol = vol_dev(vol);
    a.n_views = cnt;
    a.width = s.width;
    a.height = s.height;
    a.packet_w = cfg.packet_w;
    a.packet_h = cfg.packet_h;
    a.tiles_x = (s.width + cfg.packet_w - 1) / cfg.packet_w;
    a.tiles_y = (s.height + cfg.packet_h - 1) / cfg.packet_h;
    a.persistent = cfg.persistent;
    a.out = out + img;
    a.samples = samples ? samples + img : nullptr;
    a.queue = queue + first;
    a.error_word = err_word;
    std::memcpy(a.views, hv + first, sizeof(ViewDev) * static_cast<size_t>(cnt));
}

// Two views have the same rays when every per-view constant but the epoch
// coordinate at the image plane, the window and the prefactor agrees: the
// same image plane, direction, grid frame, epoch rate per face and boost.
static bool same_rays(const ViewDev &x, const ViewDev &y)
{
    return std::memcmp(x.g0, y.g0, sizeof(x.g0)) == 0 && std::memcmp(x.gu, y.gu, sizeof(x.gu)) == 0 &&
           std::memcmp(x.gv, y.gv, sizeof(x.gv)) == 0 && std::memcmp(x.du, y.du, sizeof(x.du)) == 0 &&
           std::memcmp(x.a_hi, y.a_hi, sizeof(x.a_hi)) == 0 && std::memcmp(x.a_lo, y.a_lo, sizeof(x.a_lo)) == 0 &&
           std::memcmp(x.inv_a, y.inv_a, sizeof(x.inv_a)) == 0 && std::memcmp(x.w_hi, y.w_hi, sizeof(x.w_hi)) == 0 &&
           std::memcmp(x.w_lo, y.w_lo, sizeof(x.w_lo)) == 0 && std::memcmp(&x.kk_hi, &y.kk_hi, sizeof(float)) == 0 &&
           std::memcmp(&x.kk_lo, &y.kk_lo, sizeof(float)) == 0 && std::memcmp(x.sh_hi, y.sh_hi, sizeof(x.sh_hi)) == 0 &&
           std::memcmp(x.sh_lo, y.sh_lo, sizeof(x.sh_lo)) == 0 && std::memcmp(&x.expo, &y.expo, sizeof(float)) == 0 &&
           x.flags == y.flags;
}

// Time groups: each run of consecutive views with the same rays, whose
// neighbours' windows overlap (epoch coordinates at the image plane at most
// M + 1 snapshots apart, else the shared march would cross the gap between
// them), becomes ceil(run / gmax) groups of near-equal size.  n_groups stays 0
// (every view marched on its own) when gmax < 2 or no run holds two views.
void group_views(MarchArgs &a, int gmax)
{
    a.n_groups = 0;
    gmax = std::min(gmax, kGroupMax);
    if (gmax < 2) return;
    const long long reach = static_cast<long long>(a.vol.M + 1) << 32;  // Q31.32
    int ng = 0;
    bool shared = false;
    for (int v = 0; v < a.n_views;) {
        int e = v + 1;
        while (e < a.n_views && same_rays(a.views[v], a.views[e]) &&
               std::llabs(a.views[e].u_obs - a.views[e - 1].u_obs) <= reach)
            ++e;
        const int len = e - v, parts = (len + gmax - 1) / gmax;
        for (int k = 0; k < parts; ++k) a.group_first[ng++] = v + len * k / parts;
        shared = shared || len > 1;
        v = e;
    }
    a.group_first[ng] = a.n_views;
    if (!shared) return;
    a.n_groups = ng;
    int most = 1;
    for (int g = 0; g < ng; ++g) {
        const int v0 = a.group_first[g], v1 = a.group_first[g + 1];
        most = std::max(most, v1 - v0);
        int ref = v0;
        float lo = a.views[v0].win_lo, hi = a.views[v0].win_hi;
        for (int v = v0 + 1; v < v1; ++v) {
            if (a.views[v].u_obs > a.views[ref].u_obs) ref = v;
            lo = std::min(lo, a.views[v].win_lo);
            hi = std::max(hi, a.views[v].win_hi);
        }
        a.group_ref[g] = ref;
        a.group_win[g][0] = lo;
        a.group_win[g][1] = hi;
        for (int v = v0; v < v1; ++v) {
            // both within 1e8 snapshots of zero (make_view), so no overflow
            a.view_delta[v] = a.views[v].u_obs - a.views[ref].u_obs;
            a.view_dhi[v] = static_cast<int>(a.view_delta[v] >> 32);
        }
    }
    a.group_size = most <= 4 ? 4 : kGroupMax;
}

int launch_units(const MarchArgs &a) { return a.n_groups > 0 ? a.n_groups : a.n_views; }

const int *tile_order(Ctx &ctx, int width, int height, int packet_w, int packet_h)
{
    const std::array<int, 4> key{width, height, packet_w, packet_h};
    auto it = ctx.tile_orders.find(key);
    if (it != ctx.tile_orders.end()) return it->second;
    if (ctx.tile_orders.size() >= 64) return nullptr;  // bounded: further geometries keep counter order
    const int tx = (width + packet_w - 1) / packet_w, ty = (height + packet_h - 1) / packet_h;
    std::vector<int> order(static_cast<size_t>(tx) * ty);
    std::vector<double> d2(order.size());
    for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) {
            const double dx = (x + 0.5) * packet_w - 0.5 * width, dy = (y + 0.5) * packet_h - 0.5 * height;
            const int t = y * tx + x;
            order[static_cast<size_t>(t)] = t;
            d2[static_cast<size_t>(t)] = dx * dx + dy * dy;
        }
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return d2[p] < d2[q]; });
    int *dev = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&dev), order.size() * sizeof(int)) != cudaSuccess) return nullptr;
    // on the load stream (not the legacy default stream, which would wait for
    // the caller's streams); the host vector must outlive the copy
    if (cudaMemcpyAsync(dev, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, ctx.load_stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx.load_stream) != cudaSuccess) {
        cudaFree(dev);
        return nullptr;
    }
    ctx.tile_orders[key] = dev;
    return dev;
}

// Bytes of the per-view tile counters of a batch, rounded up to 256.
static size_t queue_bytes(int n) { return (static_cast<size_t>(n) * sizeof(int) + 255) / 256 * 256; }

// ------------------------------------------------------------ region schedule
// Pixel coordinates of the march frame for view V: the first two rows of the
// inverse of the map (p, q, s) -> g0 + p gu + q gv + s a.
RegionProj region_proj(const ViewDev &V)
{
    double m[3][3], g0[3];
    for (int i = 0; i < 3; ++i) {
        m[i][0] = static_cast<double>(V.gu[i]) * 0x1p-40;
        m[i][1] = static_cast<double>(V.gv[i]) * 0x1p-40;
        m[i][2] = static_cast<double>(V.a_hi[i]) + V.a_lo[i];
        g0[i] = static_cast<double>(V.g0[i]) * 0x1p-40;
    }
    const double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    const double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    const double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    const double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    // rows 0 and 1 of the inverse: (adjugate transposed) / det
    const double r0[3] = {c00 / det, (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det,
                          (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det};
    const double r1[3] = {c01 / det, (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det,
                          (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det};
    RegionProj P;
    double p0 = 0.0, q0 = 0.0;
    for (int i = 0; i < 3; ++i) {
        P.ip[i] = static_cast<float>(r0[i]);
        P.iq[i] = static_cast<float>(r1[i]);
        p0 -= r0[i] * g0[i];
        q0 -= r1[i] * g0[i];
    }
    P.p0 = static_cast<float>(p0);
    P.q0 = static_cast<float>(q0);
    for (int i = 0; i < 3; ++i) {
        P.g0f[i] = static_cast<float>(g0[i]);
        P.guf[i] = static_cast<float>(m[i][0]);
        P.gvf[i] = static_cast<float>(m[i][1]);
    }
    return P;
}

// Epoch coordinate (in snapshots) at which view V sees the point x of its
// march frame: x = g0 + p gu + q gv + s a solved for s (Cramer's rule), then
// u = u_obs - kk s.
static double view_epoch_at(const ViewDev &V, const double x[3])
{
    double m[3][3], d[3];
    for (int i = 0; i < 3; ++i) {
        m[i][0] = static_cast<double>(V.gu[i]) * 0x1p-40;
        m[i][1] = static_cast<double>(V.gv[i]) * 0x1p-40;
        m[i][2] = static_cast<double>(V.a_hi[i]) + V.a_lo[i];
        d[i] = x[i] - static_cast<double>(V.g0[i]) * 0x1p-40;
    }
    auto det3 = [](const double c0[3], const double c1[3], const double c2[3]) {
        return c0[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (c0[1] * c2[2] - c0[2] * c2[1]) +
               c2[0] * (c0[1] * c1[2] - c0[2] * c1[1]);
    };
    const double c0[3] = {m[0][0], m[1][0], m[2][0]}, c1[3] = {m[0][1], m[1][1], m[2][1]},
                 c2[3] = {m[0][2], m[1][2], m[2][2]};
    const double det = det3(c0, c1, c2);
    const double s = det != 0.0 ? det3(c0, c1, d) / det : 0.0;
    return static_cast<double>(V.u_obs) * 0x1p-32 - (static_cast<double>(V.kk_hi) + V.kk_lo) * s;
}

// Regions per axis and partial slots of the region schedule for a batch of
// n_views views; 0 if it does not apply (no region edge set, sample counts
// wanted, more than 65535 regions or views: a batch of more views marches its
// rays whole).
int region_slots(const Volume &vol, const LaunchCfg &cfg, const gbd_image_spec &spec, int nreg[3], long long n_views)
{
    if (cfg.region <= 0 || spec.samples || n_views < 1 || n_views > 65535) return 0;
    long long regions = 1;
    int slots = 0;
    for (int i = 0; i < 3; ++i) {
        nreg[i] = (vol.grid.n[i] + cfg.region - 1) / cfg.region;
        regions *= nreg[i];
        slots += nreg[i];
    }
    if (regions > 65535) return 0;
    return slots - 2;
}

// CTAs one view needs per region: room for every pixel whose ray can cross a
// region's box.  The box (edges grown by a cell, far above the screening
// test's own margin and rounding) projects onto the image plane as the
// zonotope spanned by its edge vectors f_i (pixels per cell along axis i
// times the edge), of area A = sum_{i<j} |f_i x f_j| and half-perimeter
// sum_i |f_i|; a convex set holds at most A + P / 2 + 1 points of a unit
// lattice (Nosarzewska's bound), here the pixel centres.
static int region_ctas(const RegionProj &P, int region, const LaunchCfg &cfg)
{
    const double edge = static_cast<double>(region) + 1.0;
    double f[3][2], area = 0.0, half_perim = 0.0;
    for (int i = 0; i < 3; ++i) {
        f[i][0] = static_cast<double>(P.ip[i]) * edge;
        f[i][1] = static_cast<double>(P.iq[i]) * edge;
        half_perim += std::hypot(f[i][0], f[i][1]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) area += std::fabs(f[i][0] * f[j][1] - f[i][1] * f[j][0]);
    const double pixels = area + half_perim + 1.0;
    const int per_cta = 32 * cfg.cta_warps;
    return static_cast<int>(std::min(std::ceil(pixels / per_cta), 2.0e9 / per_cta));
}

// Order in which the region schedule launches a batch's views: by the Morton
// code of the direction s_hat (10 bits per component).  Views of nearby
// directions see a region at nearby depths, hence nearby snapshots, so the CTAs
// that run side by side on a region read the same few snapshots of it.
static std::vector<int> direction_order(const std::vector<ViewDev> &hv)
{
    std::vector<std::pair<uint64_t, int>> key(hv.size());
    for (size_t k = 0; k < hv.size(); ++k) {
        uint64_t code = 0;
        for (int i = 0; i < 3; ++i) {
            const double s = static_cast<double>(hv[k].sh_hi[i]) + hv[k].sh_lo[i];
            const uint64_t c = static_cast<uint64_t>(std::min(1023.0, std::max(0.0, (s + 1.0) * 511.5)));
            for (int bit = 0; bit < 10; ++bit) code |= ((c >> bit) & 1u) << (3 * bit + i);
        }
        key[k] = {code, static_cast<int>(k)};
    }
    std::stable_sort(key.begin(), key.end());
    std::vector<int> order(hv.size());
    for (size_t k = 0; k < hv.size(); ++k) order[k] = key[k].second;
    return order;
}

// Layout of a region-schedule batch's scratch: the partial slots (slots * n *
// W * H floats), the ray lists (room for ctas_per_view CTAs of rays per view
// and region) and their counts, and the region tables: the views in march
// order, their projections and their images in the batch, which the caller
// uploads from `tables` before the batch first runs.
RegionPlan region_plan(const Volume &vol, const LaunchCfg &cfg, const gbd_image_spec &spec,
                       const std::vector<ViewDev> &hv)
{
    RegionPlan P;
    P.slots = region_slots(vol, cfg, spec, P.nreg, static_cast<long long>(hv.size()));
    if (P.slots <= 0) return P;
    const size_t n = hv.size();
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    P.regions = static_cast<size_t>(P.nreg[0]) * P.nreg[1] * P.nreg[2];
    size_t per_view = 1;
    std::vector<RegionProj> proj(n);
    const std::vector<int> order = direction_order(hv);
    for (size_t k = 0; k < n; ++k) {
        proj[k] = region_proj(hv[order[k]]);
        per_view = std::max(per_view, static_cast<size_t>(region_ctas(proj[k], cfg.region, cfg)));
    }
    P.ctas_per_view = static_cast<int>(std::min<size_t>(per_view, 0x7fffffff));
    const size_t pbytes = up(sizeof(float) * static_cast<size_t>(spec.width) * spec.height * n * P.slots);
    const size_t rbytes = up(sizeof(uint32_t) * P.regions * n * per_view * 32 * cfg.cta_warps);
    const size_t cbytes = up(sizeof(int) * P.regions * n);
    P.rays_off = pbytes;
    P.count_off = P.rays_off + rbytes;
    P.views_off = P.count_off + cbytes;
    P.proj_off = P.views_off + up(sizeof(ViewDev) * n);
    P.image_off = P.proj_off + up(sizeof(RegionProj) * n);
    P.order_off = P.image_off + up(sizeof(int) * n);
    P.total = P.order_off + up(sizeof(int) * P.regions * n);
    P.tables.assign(P.total - P.views_off, 0);
    char *t = P.tables.data();
    for (size_t k = 0; k < n; ++k) {
        std::memcpy(t + (P.views_off - P.views_off) + k * sizeof(ViewDev), &hv[order[k]], sizeof(ViewDev));
        std::memcpy(t + (P.proj_off - P.views_off) + k * sizeof(RegionProj), &proj[k], sizeof(RegionProj));
        const int img = order[k];
        std::memcpy(t + (P.image_off - P.views_off) + k * sizeof(int), &img, sizeof(int));
    }
    // Per region, its views by the epoch at which they see the region's centre:
    // the views a region's CTAs march side by side then read the same few
    // snapshots of it.  (Beyond 2^22 view-regions the march order stands.)
    std::vector<std::pair<double, int>> key(n);
    int *region_order = reinterpret_cast<int *>(t + (P.order_off - P.views_off));
    const bool sort_views = P.regions * n <= (size_t(1) << 22);
    for (size_t r = 0; r < P.regions; ++r) {
        if (!sort_views) {
            for (size_t k = 0; k < n; ++k) region_order[r * n + k] = static_cast<int>(k);
            continue;
        }
        const int rr[3] = {static_cast<int>(r % P.nreg[0]), static_cast<int>((r / P.nreg[0]) % P.nreg[1]),
                           static_cast<int>(r / (static_cast<size_t>(P.nreg[0]) * P.nreg[1]))};
        for (size_t k = 0; k < n; ++k) {
            const ViewDev &V = hv[order[k]];
            double x[3];
            for (int i = 0; i < 3; ++i) {
                const int nn = vol.grid.n[i];
                const double c = 0.5 * (rr[i] * cfg.region + std::min((rr[i] + 1) * cfg.region, nn));
                x[i] = (V.flags & (kFlagMirror0 << i)) ? nn - c : c;
            }
            key[k] = {view_epoch_at(V, x), static_cast<int>(k)};
        }
        std::stable_sort(key.begin(), key.end());
        for (size_t k = 0; k < n; ++k) region_order[r * n + k] = key[k].second;
    }
    return P;
}

cudaError_t upload_region_tables(const RegionPlan &P, char *scratch, cudaStream_t st)
{
    return cudaMemcpyAsync(scratch + P.views_off, P.tables.data(), P.tables.size(), cudaMemcpyHostToDevice, st);
}

// Enqueues a region-schedule batch on st (its tables already uploaded): list
// each region's crossing rays of every view by chord length and clear the
// partial slots (one screen_kernel launch), march them region by region (one
// region_kernel launch over all views), then add up each image's slots into
// dev_out (reduce_kernel, kImagesPerReduce images per launch).
cudaError_t enqueue_regions(Ctx &ctx, const Volume &vol, const std::vector<ViewDev> &hv, const RegionPlan &P,
                            const gbd_image_spec &spec, const LaunchCfg &cfg, float *dev_out, char *scratch,
                            cudaStream_t st, int *launches)
{
    const int n = static_cast<int>(hv.size());
    const long long pix = static_cast<long long>(spec.width) * spec.height;
    const long long slot_stride = pix * n;
    float *partial = reinterpret_cast<float *>(scratch);
    *launches = 0;
    if (P.slots <= 0 || n < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    RegionArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vol = vol_dev(vol);
    a.n_views = n;
    a.width = spec.width;
    a.height = spec.height;
    a.packet_w = cfg.packet_w;
    a.packet_h = cfg.packet_h;
    a.region = cfg.region;
    for (int i = 0; i < 3; ++i) a.nreg[i] = P.nreg[i];
    a.partial = partial;
    a.slot_stride = slot_stride;
    a.partial_floats = slot_stride * P.slots;
    a.error_word = ctx.err_word;
    a.views = reinterpret_cast<const ViewDev *>(scratch + P.views_off);
    a.proj = reinterpret_cast<const RegionProj *>(scratch + P.proj_off);
    a.image = reinterpret_cast<const int *>(scratch + P.image_off);
    a.region_order = reinterpret_cast<const int *>(scratch + P.order_off);
    a.rays = reinterpret_cast<uint32_t *>(scratch + P.rays_off);
    a.ray_count = reinterpret_cast<int *>(scratch + P.count_off);
    a.rays_per_cta = 32 * cfg.cta_warps;
    a.ctas_per_view = P.ctas_per_view;
    if (e == cudaSuccess) e = launch_screen(a, st);
    if (e == cudaSuccess) e = launch_region(a, cfg, st);
    *launches += 2;
    auto r = std::make_unique<ReduceArgs>();
    for (int first = 0; first < n && e == cudaSuccess; first += kImagesPerReduce) {
        const int cnt = std::min(kImagesPerReduce, n - first);
        std::memset(r.get(), 0, sizeof(ReduceArgs));
        r->out = dev_out;
        r->partial = partial;
        r->slot_stride = slot_stride;
        r->pix_per_view = pix;
        r->n_views = cnt;
        r->n_slots = P.slots;
        for (int v = 0; v < cnt; ++v) {
            r->image[v] = first + v;
            r->prefactor[v] = hv[first + v].prefactor;
        }
        e = launch_reduce(*r, st);
        ++*launches;
    }
    return e;
}

// Renders n views whose records are already set up on the host, without a
// cached graph: stream-ordered scratch for the tile counters or partial slots
// (and the image when it goes to host memory).
int render_direct(Ctx &ctx, const Volume &vol, const std::vector<ViewDev> &hv, const gbd_image_spec &spec,
                  const LaunchCfg &cfg, cudaStream_t st)
{
    const int n = static_cast<int>(hv.size());
    const size_t pix = static_cast<size_t>(spec.width) * spec.height * n;
    char *scratch = nullptr;
    int nreg[3];
    const int slots = region_slots(vol, cfg, spec, nreg, n);
    if (slots > 0) {
        const RegionPlan plan = region_plan(vol, cfg, spec, hv);
        const size_t pbytes = plan.total;
        const size_t total = pbytes + (spec.out_on_host ? pix * sizeof(float) : 0);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), total, st);
        if (e != cudaSuccess) return cuda_fail(e, "region scratch");
        float *dev_out = spec.out_on_host ? reinterpret_cast<float *>(scratch + pbytes) : spec.out;
        int launches = 0;
        e = upload_region_tables(plan, scratch, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx.region_done, 0);
        if (e == cudaSuccess) e = enqueue_regions(ctx, vol, hv, plan, spec, cfg, dev_out, scratch, st, &launches);
        if (e == cudaSuccess) e = cudaEventRecord(ctx.region_done, st);
        if (e == cudaSuccess && spec.out_on_host)
            e = cudaMemcpyAsync(spec.out, dev_out, pix * sizeof(float), cudaMemcpyDeviceToHost, st);
        cudaError_t ef = cudaFreeAsync(scratch, st);
        if (e != cudaSuccess) return cuda_fail(e, "region render");
        if (ef != cudaSuccess) return cuda_fail(ef, "region scratch free");
        set_launch_count(launches);
        return GBD_OK;
    }
    const size_t img_off = queue_bytes(n);
    const size_t total = img_off + (spec.out_on_host ? pix * sizeof(float) : 0);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), total, st);
    if (e != cudaSuccess) return cuda_fail(e, "render scratch");
    int *queue = reinterpret_cast<int *>(scratch);
    float *dev_out = spec.out_on_host ? reinterpret_cast<float *>(scratch + img_off) : spec.out;
    e = cudaMemsetAsync(queue, 0, img_off, st);
    const int chunks = march_chunks(n);
    auto a = std::make_unique<MarchArgs>();
    const std::vector<double> work = view_works(vol, hv, spec.width, spec.height);
    for (int c = 0; c < chunks && e == cudaSuccess; ++c) {
        fill_args(*a, vol, hv.data(), n, c, spec, dev_out, spec.out_on_host ? nullptr : spec.samples, queue, cfg,
                  ctx.err_word);
        group_views(*a, cfg.group);
        if (cfg.persistent && launch_units(*a) == 1)
            a->tile_order = tile_order(ctx, spec.width, spec.height, cfg.packet_w, cfg.packet_h);
        e = launch_march(*a, cfg, ctx.num_sms, work.data() + static_cast<size_t>(c) * kViewsPerLaunch, st);
    }
    if (e == cudaSuccess && spec.out_on_host)
        e = cudaMemcpyAsync(spec.out, dev_out, pix * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t ef = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "render scratch free");
    set_launch_count(chunks);
    return GBD_OK;
}

// ------------------------------------------------------------------ graphs
struct GraphKey {
    gbd_volume vol;
    int n, width, height;
    const void *out;
    const void *samples;
    int out_on_host;
    LaunchCfg cfg;
    bool operator<(const GraphKey &o) const
    {
        return std::memcmp(this, &o, sizeof(GraphKey)) < 0;
    }
};

// A batch graph: a memset of the tile counters, one kernel node per chunk of
// views (independent, so they may run side by side), and, for host output,
// the copy back.  New views of the same geometry update the kernel nodes'
// parameters in place.  A region-schedule batch is captured from
// enqueue_regions instead (rebuilt for new views), and its copy back to host
// memory is issued after each replay, outside the graph.
struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int region_launches = 0;     // region schedule: kernels per replay (captured; rebuilt for new views)
    std::vector<cudaGraphNode_t> knodes;
    std::vector<void *> kfuncs;  // the kernel of each node
    std::vector<ViewDev> views;  // the views the kernel nodes hold
    char *d_scratch = nullptr;   // tile counters (+ image when out_on_host)
    float *region_img = nullptr; // region schedule with host output: the device image, copied back after each replay
    cudaEvent_t done = nullptr;
    bool launched = false;
    ~GraphEntry()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (done) cudaEventDestroy(done);
        if (d_scratch) cudaFree(d_scratch);
    }
};

// Bounded: the least recently used graph is dropped beyond kMaxGraphs.
constexpr size_t kMaxGraphs = 64;

struct GraphCache {
    std::map<GraphKey, std::unique_ptr<GraphEntry>> entries;
    std::map<GraphKey, uint64_t> last_use;
    uint64_t clock = 0;
};

void destroy_graph_cache(GraphCache *g) { delete g; }

void drop_graphs_for(Ctx &ctx, gbd_volume vol)
{
    if (!ctx.graphs) return;
    auto &m = ctx.graphs->entries;
    for (auto it = m.begin(); it != m.end();) {
        if (it->first.vol == vol) {
            if (it->second->launched) cudaEventSynchronize(it->second->done);
            ctx.graphs->last_use.erase(it->first);
            it = m.erase(it);
        } else {
            ++it;
        }
    }
}

// Kernel node parameters of chunk c of a graph's batch.
static cudaError_t chunk_params(Ctx &ctx, const Volume &vol, const GraphKey &key, const gbd_image_spec &spec,
                                const GraphEntry &g, const ViewDev *hv, int c, MarchArgs &a,
                                cudaKernelNodeParams &kp, void **params)
{
    const size_t img_off = queue_bytes(key.n);
    int *queue = reinterpret_cast<int *>(g.d_scratch);
    float *dev_out = spec.out_on_host ? reinterpret_cast<float *>(g.d_scratch + img_off) : spec.out;
    fill_args(a, vol, hv, key.n, c, spec, dev_out, spec.out_on_host ? nullptr : spec.samples, queue, key.cfg,
              ctx.err_word);
    group_views(a, key.cfg.group);
    if (key.cfg.persistent && launch_units(a) == 1)
        a.tile_order = tile_order(ctx, spec.width, spec.height, key.cfg.packet_w, key.cfg.packet_h);
    double work[kViewsPerLaunch];
    for (int v = 0; v < a.n_views; ++v) work[v] = view_work(vol, a.views[v], spec.width, spec.height);
    KernelLaunch L;
    cudaError_t e = plan_march(a, key.cfg, ctx.num_sms, work, L);
    if (e != cudaSuccess) return e;
    kp = cudaKernelNodeParams{};
    kp.func = L.func;
    kp.gridDim = L.grid;
    kp.blockDim = L.block;
    kp.sharedMemBytes = static_cast<unsigned>(L.smem);
    params[0] = &a;
    kp.kernelParams = params;
    return cudaSuccess;
}

// Whether the views hv would run the same kernel in every node of g (their
// time groups may call for the grouped kernel where g's views did not).
static bool same_kernels(Ctx &ctx, const Volume &vol, const GraphKey &key, const gbd_image_spec &spec,
                         const GraphEntry &g, const std::vector<ViewDev> &hv)
{
    auto a = std::make_unique<MarchArgs>();
    for (size_t c = 0; c < g.knodes.size(); ++c) {
        cudaKernelNodeParams kp;
        void *params[1];
        if (chunk_params(ctx, vol, key, spec, g, hv.data(), static_cast<int>(c), *a, kp, params) != cudaSuccess ||
            kp.func != g.kfuncs[c])
            return false;
    }
    return true;
}

// Region schedule: the batch is captured from enqueue_regions.
static int build_region_graph(Ctx &ctx, const Volume &vol, const GraphKey &key, const gbd_image_spec &spec,
                              const std::vector<ViewDev> &hv, int slots, GraphEntry &g)
{
    const size_t pix = static_cast<size_t>(spec.width) * spec.height * key.n;
    const RegionPlan plan = region_plan(vol, key.cfg, spec, hv);
    const size_t pbytes = plan.total;
    const size_t total = pbytes + (spec.out_on_host ? pix * sizeof(float) : 0);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&g.d_scratch), total);
    if (e != cudaSuccess) return cuda_fail(e, "region batch scratch");
    e = cudaMemcpy(g.d_scratch + plan.views_off, plan.tables.data(), plan.tables.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "region tables");
    e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch event");
    float *dev_out = spec.out_on_host ? reinterpret_cast<float *>(g.d_scratch + pbytes) : spec.out;
    if (spec.out_on_host) g.region_img = dev_out;
    cudaStream_t cap = ctx.capture_stream;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    cudaError_t e2 = enqueue_regions(ctx, vol, hv, plan, spec, key.cfg, dev_out, g.d_scratch, cap, &g.region_launches);
    e = cudaStreamEndCapture(cap, &g.graph);
    if (e2 != cudaSuccess) return cuda_fail(e2, "capture region batch");
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate region batch graph");
    g.views = hv;
    return GBD_OK;
}

static int build_graph(Ctx &ctx, const Volume &vol, const GraphKey &key, const gbd_image_spec &spec,
                       const std::vector<ViewDev> &hv, GraphEntry &g)
{
    int nreg[3];
    const int slots = region_slots(vol, key.cfg, spec, nreg, key.n);
    if (slots > 0) return build_region_graph(ctx, vol, key, spec, hv, slots, g);
    const int n = key.n;
    const size_t img_off = queue_bytes(n);
    const size_t pix = static_cast<size_t>(spec.width) * spec.height * n;
    const size_t total = img_off + (spec.out_on_host ? pix * sizeof(float) : 0);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&g.d_scratch), total);
    if (e != cudaSuccess) return cuda_fail(e, "batch scratch");
    e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch event");
    e = cudaGraphCreate(&g.graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = g.d_scratch;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = img_off / 4;
    mp.height = 1;
    cudaGraphNode_t mnode = nullptr;
    e = cudaGraphAddMemsetNode(&mnode, g.graph, nullptr, 0, &mp);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph memset node");
    auto a = std::make_unique<MarchArgs>();
    const int chunks = march_chunks(n);
    for (int c = 0; c < chunks; ++c) {
        cudaKernelNodeParams kp;
        void *params[1];
        e = chunk_params(ctx, vol, key, spec, g, hv.data(), c, *a, kp, params);
        cudaGraphNode_t kn = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&kn, g.graph, &mnode, 1, &kp);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph kernel node");
        g.knodes.push_back(kn);
        g.kfuncs.push_back(kp.func);
    }
    if (spec.out_on_host) {
        cudaGraphNode_t cn = nullptr;
        e = cudaGraphAddMemcpyNode1D(&cn, g.graph, g.knodes.data(), g.knodes.size(), spec.out,
                                     g.d_scratch + img_off, pix * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph copy node");
    }
    e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate batch graph");
    g.views = hv;
    return GBD_OK;
}

int render_graph(Ctx &ctx, const Volume &vol, gbd_volume vid, const std::vector<ViewDev> &hv,
                 const gbd_image_spec &spec, const LaunchCfg &cfg, cudaStream_t st)
{
    if (!ctx.graphs) ctx.graphs = new GraphCache();
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.vol = vid;
    key.n = static_cast<int>(hv.size());
    key.width = spec.width;
    key.height = spec.height;
    key.out = spec.out;
    key.samples = spec.out_on_host ? nullptr : spec.samples;
    key.out_on_host = spec.out_on_host;
    key.cfg = cfg;
    GraphCache &gc = *ctx.graphs;
    if (gc.entries.find(key) == gc.entries.end() && gc.entries.size() >= kMaxGraphs) {
        auto oldest = std::min_element(gc.last_use.begin(), gc.last_use.end(),
                                       [](const auto &x, const auto &y) { return x.second < y.second; });
        auto victim = gc.entries.find(oldest->first);
        if (victim->second->launched) cudaEventSynchronize(victim->second->done);
        gc.entries.erase(victim);
        gc.last_use.erase(oldest);
    }
    gc.last_use[key] = ++gc.clock;
    auto &slot = gc.entries[key];
    const size_t vbytes = sizeof(ViewDev) * hv.size();
    if (!slot) {
        auto g = std::make_unique<GraphEntry>();
        int rc = build_graph(ctx, vol, key, spec, hv, *g);
        if (rc != GBD_OK) {
            gc.entries.erase(key);
            gc.last_use.erase(key);
            return rc;
        }
        slot = std::move(g);
    } else if (std::memcmp(slot->views.data(), hv.data(), vbytes) != 0 &&
               (slot->region_launches > 0 || !same_kernels(ctx, vol, key, spec, *slot, hv))) {
        // region schedule, or new views that group differently (another
        // kernel): build the batch again for the new views
        if (slot->launched) {
            cudaError_t e = cudaEventSynchronize(slot->done);
            if (e != cudaSuccess) return cuda_fail(e, "wait for previous batch");
        }
        auto g = std::make_unique<GraphEntry>();
        int rc = build_graph(ctx, vol, key, spec, hv, *g);
        if (rc != GBD_OK) {
            gc.entries.erase(key);
            gc.last_use.erase(key);
            return rc;
        }
        slot = std::move(g);
    } else if (std::memcmp(slot->views.data(), hv.data(), vbytes) != 0) {
        // Parameter updates apply to later launches only; a launch in flight
        // keeps the views it started with.
        auto a = std::make_unique<MarchArgs>();
        for (size_t c = 0; c < slot->knodes.size(); ++c) {
            cudaKernelNodeParams kp;
            void *params[1];
            cudaError_t e = chunk_params(ctx, vol, key, spec, *slot, hv.data(), static_cast<int>(c), *a, kp, params);
            if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(slot->exec, slot->knodes[c], &kp);
            if (e != cudaSuccess) return cuda_fail(e, "update batch graph");
        }
        slot->views = hv;
    }
    cudaError_t e = cudaSuccess;
    if (slot->region_launches > 0) {
        // one region batch marches at a time; host output is copied back
        // outside the graph, after the march, so that it overlaps the next
        // batch's march
        e = cudaStreamWaitEvent(st, ctx.region_done, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(slot->exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(ctx.region_done, st);
        if (e == cudaSuccess && slot->region_img)
            e = cudaMemcpyAsync(spec.out, slot->region_img,
                                sizeof(float) * static_cast<size_t>(spec.width) * spec.height * hv.size(),
                                cudaMemcpyDeviceToHost, st);
    } else {
        e = cudaGraphLaunch(slot->exec, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    e = cudaEventRecord(slot->done, st);
    if (e != cudaSuccess) return cuda_fail(e, "graph event");
    slot->launched = true;
    set_launch_count(slot->region_launches > 0 ? slot->region_launches : static_cast<int>(slot->knodes.size()));
    return GBD_OK;
}

}  // namespace gbd

using namespace gbd;

gbd_ctx::~gbd_ctx() = default;

Volume *gbd_ctx::find(gbd_volume id)
{
    auto it = volumes.find(id);
    return it == volumes.end() ? nullptr : it->second.get();
}

// ====================================================================== C ABI
extern "C" {

const char *gbd_error_string(int status)
{
    switch (status) {
    case GBD_OK: return "ok";
    case GBD_ERR_INVALID: return "invalid argument";
    case GBD_ERR_NOMEM: return "out of memory";
    case GBD_ERR_BUDGET: return "exceeds the HBM budget";
    case GBD_ERR_NOTFOUND: return "not found";
    case GBD_ERR_TIMEOUT: return "timed out";
    case GBD_ERR_CUDA: return "CUDA error";
    case GBD_ERR_CANCELLED: return "cancelled";
    case GBD_ERR_BUSY: return "busy";
    default: return "unknown status";
    }
}

const char *gbd_last_error(void) { return t_last_error.c_str(); }

int32_t gbd_last_launch_count(void) { return t_last_launches; }

int gbd_bounds_violations(gbd_ctx *ctx, int32_t *out)
{
    if (!ctx || !out) return fail(GBD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    int word = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&word, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->err_word, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "bounds word");
    *out = word;
    return GBD_OK;
}

int gbd_create(gbd_ctx **out, int32_t device, uint64_t hbm_budget_bytes)
{
    if (!out) return fail(GBD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(GBD_ERR_INVALID, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard guard(device);
    auto ctx = std::make_unique<gbd_ctx>();
    ctx->device = device;
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "multiprocessor count");
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : static_cast<uint64_t>(0.9 * static_cast<double>(free_b));
    e = cudaStreamCreateWithFlags(&ctx->load_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "load stream");
    e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    e = cudaMalloc(reinterpret_cast<void **>(&ctx->err_word), 256);
    if (e != cudaSuccess) return cuda_fail(e, "error word");
    e = cudaMemset(ctx->err_word, 0, 256);
    if (e != cudaSuccess) return cuda_fail(e, "error word clear");
    e = cudaEventCreateWithFlags(&ctx->region_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "region event");
    load_tune_file(*ctx);
    *out = ctx.release();
    return GBD_OK;
}

int gbd_destroy(gbd_ctx *ctx)
{
    if (!ctx) return GBD_OK;
    {
        DeviceGuard guard(ctx->device);
        serve_shutdown(*ctx);
        cudaDeviceSynchronize();
        destroy_graph_cache(ctx->graphs);
        ctx->graphs = nullptr;
        for (auto &kv : ctx->volumes) {
            if (kv.second->rec) cudaFree(kv.second->rec);
            if (kv.second->axis_off) cudaFree(kv.second->axis_off);
            if (kv.second->chan) cudaFree(kv.second->chan);
        }
        ctx->volumes.clear();
        if (ctx->err_word) cudaFree(ctx->err_word);
        if (ctx->region_done) cudaEventDestroy(ctx->region_done);
        for (auto &kv : ctx->tile_orders) cudaFree(kv.second);
        ctx->tile_orders.clear();
        if (ctx->load_stream) cudaStreamDestroy(ctx->load_stream);
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
        for (int k = 0; k < 4; ++k) {
            if (ctx->aux[k]) cudaStreamDestroy(ctx->aux[k]);
            if (ctx->aux_done[k]) cudaEventDestroy(ctx->aux_done[k]);
        }
    }
    delete ctx;
    return GBD_OK;
}

int gbd_load_snapshots(gbd_ctx *ctx, const gbd_grid *grid, const gbd_fields *f, gbd_volume *out)
{
    if (!ctx || !grid || !f || !out) return fail(GBD_ERR_INVALID, "NULL argument");
    *out = 0;
    const gbd_grid &g = *grid;
    int rc = check_grid_fields(g, *f);
    if (rc) return rc;
    const int B = f->brick ? f->brick : 8;
    const int S = f->super_brick ? f->super_brick : 4;

    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard guard(ctx->device);
    auto vol = std::make_unique<Volume>();
    vol->grid = g;
    vol->store = f->store;
    vol->brick = B;
    vol->super_brick = S;
    vol->paired = f->paired ? 1 : 0;
    std::vector<int32_t> tab;
    long long cells = 0;
    vol->morton_cells = f->morton_cells ? 1 : 0;
    if (!build_layout(g.n, B, S, tab, cells, vol->morton_cells) || (vol->paired && 2 * cells >= (1LL << 31)))
        return fail(GBD_ERR_INVALID, "grid too large: one epoch exceeds 2^31 records");
    const size_t bytes = volume_bytes(f->store, cells, g.n_epochs, vol->paired, &vol->epoch_stride);
    const size_t tab_bytes = tab.size() * sizeof(int32_t);
    if (ctx->used + bytes + tab_bytes > ctx->budget)
        return fail(GBD_ERR_BUDGET, "volume needs %zu bytes, %llu of %llu budget in use", bytes + tab_bytes,
                    static_cast<unsigned long long>(ctx->used), static_cast<unsigned long long>(ctx->budget));
    if (fault_injected("alloc")) return fail(GBD_ERR_NOMEM, "injected allocation failure");
    cudaError_t e = cudaMalloc(&vol->rec, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "volume allocation");
    auto cleanup = [&]() {
        cudaFree(vol->rec);
        vol->rec = nullptr;
        if (vol->axis_off) cudaFree(vol->axis_off);
        vol->axis_off = nullptr;
    };
    e = cudaMalloc(reinterpret_cast<void **>(&vol->axis_off), tab_bytes);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "layout table allocation"); }
    cudaStream_t st = ctx->load_stream;
    if (f->on_device) {
        // Device inputs may still be being written by work on any stream of
        // the caller (the call takes no stream): wait for the whole device.
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "wait for device inputs"); }
    }
    e = cudaMemcpyAsync(vol->axis_off, tab.data(), tab_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(vol->rec, 0, bytes, st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "volume init"); }

    const size_t esz = f->dtype_in == GBD_IN_F64 ? 8 : 4;
    const size_t ncell = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
    char *stage = nullptr;
    int *bad = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&bad), 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 256, st);
    if (e == cudaSuccess && !f->on_device) e = cudaMallocAsync(reinterpret_cast<void **>(&stage), ncell * esz * 4, st);
    for (int m = 0; m < g.n_epochs && e == cudaSuccess; ++m) {
        const char *jsrc = static_cast<const char *>(f->j) + m * ncell * esz;
        const char *vsrc = static_cast<const char *>(f->vel) + m * ncell * esz * 3;
        PackArgs pa;
        std::memset(&pa, 0, sizeof(pa));
        if (f->on_device) {
            pa.j = jsrc;
            pa.vel = vsrc;
        } else {
            e = cudaMemcpyAsync(stage, jsrc, ncell * esz, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(stage + ncell * esz, vsrc, ncell * esz * 3, cudaMemcpyHostToDevice, st);
            pa.j = stage;
            pa.vel = stage + ncell * esz;
        }
        pa.dtype_in = f->dtype_in;
        pa.store = f->store;
        for (int i = 0; i < 3; ++i) pa.n[i] = g.n[i];
        pa.axis_off = vol->axis_off;
        pa.dst = vol->rec;
        pa.stride = vol->epoch_stride;
        pa.m = m;
        pa.paired = vol->paired;
        pa.bad = bad;
        pa.gamma2_max = reinterpret_cast<unsigned *>(bad) + 1;
        if (e == cudaSuccess) e = launch_pack(pa, st);
        // The host staging buffer is reused for the next epoch only after
        // this epoch's pack has consumed it.
        if (e == cudaSuccess && !f->on_device) e = cudaStreamSynchronize(st);
    }
    int h_bad[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_bad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (stage) cudaFreeAsync(stage, st);
    if (bad) cudaFreeAsync(bad, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "volume pack"); }
    if (h_bad[0]) {
        cleanup();
        return fail(GBD_ERR_INVALID, "fields: negative or non-finite j', non-finite beta, or |beta| >= 1 "
                                     "(float32 storage needs |beta|^2 <= 1 - 2^-20)");
    }
    if (f->store == GBD_STORE_BF16_F16U) {
        float g2 = 0.f;
        std::memcpy(&g2, &h_bad[1], sizeof(g2));
        vol->plain_boost = g2 <= kPlainGamma2 ? 1 : 0;
    }
    vol->bytes = bytes + tab_bytes;
    ctx->used += vol->bytes;
    const gbd_volume id = ++ctx->next_id;
    ctx->volumes[id] = std::move(vol);
    *out = id;
    return GBD_OK;
}

int gbd_unload(gbd_ctx *ctx, gbd_volume vid)
{
    if (!ctx) return fail(GBD_ERR_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *v = ctx->find(vid);
    if (!v) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (v->pinned_by_requests.load() > 0) return fail(GBD_ERR_BUSY, "volume has %d queued requests", v->pinned_by_requests.load());
    DeviceGuard guard(ctx->device);
    drop_graphs_for(*ctx, vid);
    // Work already enqueued on other streams may still read the volume.
    cudaDeviceSynchronize();
    cudaFree(v->rec);
    cudaFree(v->axis_off);
    if (v->chan) cudaFree(v->chan);
    ctx->used -= v->bytes + v->chan_bytes;
    ctx->volumes.erase(vid);
    return GBD_OK;
}

int gbd_volume_info(gbd_ctx *ctx, gbd_volume vid, gbd_volume_desc *out)
{
    if (!ctx || !out) return fail(GBD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *v = ctx->find(vid);
    if (!v) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    out->grid = v->grid;
    out->store = v->store;
    out->brick = v->brick;
    out->super_brick = v->super_brick;
    out->paired = v->paired;
    out->morton_cells = v->morton_cells;
    out->bytes = v->bytes;
    out->record_bytes = v->store == GBD_STORE_F32 ? 16 : 8;
    out->n_channels = v->n_chan;
    out->channel_bytes = v->chan_bytes;
    return GBD_OK;
}

int gbd_render(gbd_ctx *ctx, gbd_volume vid, const gbd_view *view, const gbd_image_spec *spec,
               const gbd_launch *launch, void *stream)
{
    if (!ctx || !view) return fail(GBD_ERR_INVALID, "NULL argument");
    int rc = check_spec(spec);
    if (rc) return rc;
    LaunchCfg cfg = resolve_launch(launch);
    if ((rc = check_launch(cfg))) return rc;
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (!launch) lookup_tuned(*ctx, tune_key(*vol, spec->width, spec->height, 1, view->flags), cfg);
    DeviceGuard guard(ctx->device);
    std::vector<ViewDev> hv(1);
    if ((rc = make_view(*vol, *view, spec->width, spec->height, spec->fov_u, spec->fov_v, hv[0]))) return rc;
    return render_direct(*ctx, *vol, hv, *spec, cfg, static_cast<cudaStream_t>(stream));
}

int gbd_load_channels(gbd_ctx *ctx, gbd_volume vid, const void *chans, int32_t n_chan, int32_t dtype_in,
                      int32_t on_device)
{
    if (!ctx || !chans) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n_chan != 1 && n_chan != 3) return fail(GBD_ERR_INVALID, "n_channels must be 1 or 3");
    if (dtype_in != GBD_IN_F64 && dtype_in != GBD_IN_F32) return fail(GBD_ERR_INVALID, "bad dtype_in");
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *v = ctx->find(vid);
    if (!v) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (v->pinned_by_requests.load() > 0) return fail(GBD_ERR_BUSY, "volume has queued requests");
    DeviceGuard guard(ctx->device);
    const gbd_grid &g = v->grid;
    std::vector<int32_t> tab;
    long long cells = 0;
    build_layout(g.n, v->brick, v->super_brick, tab, cells, v->morton_cells);
    const uint64_t bytes = sizeof(float) * static_cast<uint64_t>(cells) * g.n_epochs * n_chan;
    const uint64_t freed = v->chan_bytes;
    if (ctx->used - freed + bytes > ctx->budget)
        return fail(GBD_ERR_BUDGET, "channels need %llu bytes", static_cast<unsigned long long>(bytes));
    float *dst = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&dst), bytes);
    if (e != cudaSuccess) return cuda_fail(e, "channel allocation");
    cudaStream_t st = ctx->load_stream;
    const size_t esz = dtype_in == GBD_IN_F64 ? 8 : 4;
    const size_t ncell = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
    char *stage = nullptr;
    int *bad = nullptr;
    if (on_device) {
        // device inputs may still be written by the caller's work on any stream
        e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&bad), 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 256, st);
    if (e == cudaSuccess && !on_device) e = cudaMallocAsync(reinterpret_cast<void **>(&stage), ncell * esz, st);
    for (int c = 0; c < n_chan && e == cudaSuccess; ++c)
        for (int m = 0; m < g.n_epochs && e == cudaSuccess; ++m) {
            const char *src = static_cast<const char *>(chans) + (static_cast<size_t>(c) * g.n_epochs + m) * ncell * esz;
            ChanPackArgs pa;
            std::memset(&pa, 0, sizeof(pa));
            if (on_device) {
                pa.src = src;
            } else {
                e = cudaMemcpyAsync(stage, src, ncell * esz, cudaMemcpyHostToDevice, st);
                pa.src = stage;
            }
            pa.dtype_in = dtype_in;
            for (int i = 0; i < 3; ++i) pa.n[i] = g.n[i];
            pa.axis_off = v->axis_off;
            pa.dst = dst + (static_cast<size_t>(c) * g.n_epochs + m) * cells;
            pa.bad = bad;
            if (e == cudaSuccess) e = launch_chan_pack(pa, st);
            if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);  // the stage takes the next epoch
        }
    int h_bad[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_bad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (stage) cudaFreeAsync(stage, st);
    if (bad) cudaFreeAsync(bad, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess || h_bad[0]) {
        cudaFree(dst);
        if (e != cudaSuccess) return cuda_fail(e, "channel pack");
        return fail(GBD_ERR_INVALID, "channels: non-finite value");
    }
    if (v->chan) cudaFree(v->chan);
    ctx->used = ctx->used - freed + bytes;
    v->chan = dst;
    v->n_chan = n_chan;
    v->chan_stride = cells;
    v->chan_bytes = bytes;
    return GBD_OK;
}

int gbd_touched_records(gbd_ctx *ctx, gbd_volume vid, const gbd_view *views, int32_t n,
                        const gbd_image_spec *spec, uint64_t *records)
{
    if (!ctx || !views || !spec || !records) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    if (spec->width < 1 || spec->height < 1 || spec->width > 16384 || spec->height > 16384)
        return fail(GBD_ERR_INVALID, "image: width/height must be in [1, 16384]");
    *records = 0;
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    DeviceGuard guard(ctx->device);
    int rc;
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[k]))) return rc;
    std::vector<int32_t> tab;
    long long cells = 0;
    build_layout(vol->grid.n, vol->brick, vol->super_brick, tab, cells, vol->morton_cells);
    const size_t words = (static_cast<size_t>(cells) * vol->grid.n_epochs + 31) / 32;
    uint32_t *bits = nullptr;
    cudaStream_t st = ctx->load_stream;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&bits), words * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, words * 4, st);
    LaunchCfg cfg = resolve_launch(nullptr);
    auto a = std::make_unique<MarchArgs>();
    gbd_image_spec s = *spec;
    s.out = nullptr;  // the analysis writes no image
    for (int c = 0; c < march_chunks(n) && e == cudaSuccess; ++c) {
        fill_args(*a, *vol, hv.data(), n, c, s, reinterpret_cast<float *>(bits), nullptr, nullptr, cfg, ctx->err_word);
        e = launch_touch(*a, bits, cells, cfg, ctx->num_sms, st);
    }
    std::vector<uint32_t> host(words);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), bits, words * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bits) cudaFree(bits);
    if (e != cudaSuccess) return cuda_fail(e, "touched records");
    uint64_t count = 0;
    for (uint32_t w : host) count += static_cast<uint64_t>(__builtin_popcount(w));
    *records = count;
    return GBD_OK;
}

int gbd_render_vector(gbd_ctx *ctx, gbd_volume vid, const gbd_view *views, int32_t n, const gbd_image_spec *spec,
                      const gbd_launch *launch, void *stream)
{
    if (!ctx || !views) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    int rc = check_spec(spec);
    if (rc) return rc;
    if (spec->out_on_host || spec->samples)
        return fail(GBD_ERR_INVALID, "gbd_render_vector takes device output and no sample counts");
    LaunchCfg cfg = resolve_launch(launch);
    if ((rc = check_launch(cfg))) return rc;
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (!vol->chan) return fail(GBD_ERR_INVALID, "the volume has no channels (gbd_load_channels)");
    DeviceGuard guard(ctx->device);
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[k]))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t qbytes = (static_cast<size_t>(n) * sizeof(int) + 255) / 256 * 256;
    int *queue = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&queue), qbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, qbytes, st);
    const long long plane = static_cast<long long>(spec->width) * spec->height;
    const long long img_stride = plane * (1 + vol->n_chan);
    const std::vector<double> work = view_works(*vol, hv, spec->width, spec->height);
    auto a = std::make_unique<MarchArgs>();
    int launches = 0;
    for (int c = 0; c < march_chunks(n) && e == cudaSuccess; ++c) {
        fill_args(*a, *vol, hv.data(), n, c, *spec, spec->out, nullptr, queue, cfg, ctx->err_word);
        a->out = spec->out + static_cast<long long>(c) * kViewsPerLaunch * img_stride;
        a->img_stride = img_stride;
        a->chan = vol->chan;
        a->chan_comp_stride = vol->chan_stride * vol->grid.n_epochs;
        a->chan_cell_stride = vol->chan_stride;
        e = launch_vector(*a, vol->n_chan, cfg, ctx->num_sms, work.data() + static_cast<size_t>(c) * kViewsPerLaunch,
                          st);
        ++launches;
    }
    cudaError_t ef = queue ? cudaFreeAsync(queue, st) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "vector render");
    if (ef != cudaSuccess) return cuda_fail(ef, "vector render scratch");
    set_launch_count(launches);
    return GBD_OK;
}

int gbd_render_batch(gbd_ctx *ctx, gbd_volume vid, const gbd_view *views, int32_t n, const gbd_image_spec *spec,
                     const gbd_launch *launch, void *stream)
{
    if (!ctx || !views) return fail(GBD_ERR_INVALID, "NULL argument");
    if (n < 1 || n > (1 << 20)) return fail(GBD_ERR_INVALID, "batch size must be in [1, 2^20]");
    int rc = check_spec(spec);
    if (rc) return rc;
    LaunchCfg cfg = resolve_launch(launch);
    if ((rc = check_launch(cfg))) return rc;
    std::lock_guard<std::mutex> lock(ctx->mu);
    Volume *vol = ctx->find(vid);
    if (!vol) return fail(GBD_ERR_NOTFOUND, "unknown volume %llu", static_cast<unsigned long long>(vid));
    if (!launch) lookup_tuned(*ctx, tune_key(*vol, spec->width, spec->height, n, views[0].flags), cfg);
    DeviceGuard guard(ctx->device);
    std::vector<ViewDev> hv(static_cast<size_t>(n));
    for (int k = 0; k < n; ++k)
        if ((rc = make_view(*vol, views[k], spec->width, spec->height, spec->fov_u, spec->fov_v, hv[k]))) return rc;
    if (graphs_enabled()) return render_graph(*ctx, *vol, vid, hv, *spec, cfg, static_cast<cudaStream_t>(stream));
    return render_direct(*ctx, *vol, hv, *spec, cfg, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
