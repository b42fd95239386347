// march.cu -- sm_103a ray-march kernels for the relativistic line-of-sight sum.
//
// One lane owns one ray (pixel) from entry to exit, so every pixel is summed in
// one fixed order whether it is rendered alone, in a batch or in a served mix.
// A warp owns a packet of 32 neighbouring pixels (8x4 by default), so at each
// step its lanes gather neighbouring cells of the bricked volume.
//
// Per view, on the host in float64: the constants of ViewDev (fixed-point
// pixel positions, face spacings, epoch rates), with every axis the view runs
// down mirrored so that the march always steps to increasing cell index.
// Per ray (Sec. 2.4 traversal, Sec. 5.1 fast-forward, Eqs. 2, 6-9, 14, 19),
// with no float64 on the device:
//   * once: the pixel position in Q24.40 fixed point, an anchor at the later of
//     the box entry and the window start where the retarded time can reach a
//     stored snapshot, the anchor's cell, and the epoch coordinate there in
//     Q31.32 fixed point;
//   * per cell: the nearest next face crossing (each recomputed from its plane
//     count, never accumulated), the chord ds from the previous one, the epoch
//     coordinate at the chord midpoint, the two snapshot records, the Doppler
//     boost of each, their linear interpolation, and a compensated float32
//     accumulation of value * ds.
// Cells are gathered DEPTH at a time: the traversal runs ahead, all loads of
// the group are issued, then the group is evaluated, so each lane keeps up to
// 2 * DEPTH independent loads in flight.
//
// Time groups (batched renders of one direction at several observer times):
// one traversal per ray serves up to 4 or 8 views, each with its own sums
// (march_group, group_kernel).
//
// bfloat16/float16 records (march_ray_bf16, march_group_bf16) take a lighter
// march whose storage error (2^-9 in j', 2^-11 in u) dwarfs its arithmetic:
// the epoch coordinate is a float linear in s instead of the exact fixed
// point, the step runs without branches for every lane (a lane whose ray has
// ended takes no step and reads nothing), the Doppler factor is the plain
// 1 / (Gamma + u.s_hat) where the volume's Gamma allows it, and the sum is
// not compensated.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cfloat>

#include "gbd_internal.h"

namespace gbd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// Per-view float constants held in registers during the march.
struct BoostConsts {
    float shx, shy, shz;  // s_hat rounded to float
    float slx, sly, slz;  // rounding residual of s_hat
    float expo;           // 2 - alpha
    bool beaming;
    bool plain;           // bfloat16/float16 records: D = 1 / (Gamma + u.s_hat) (volume's Gamma <= 8)
};

template <int STORE>
struct Record;

// 16-byte record {j', beta_x, beta_y, beta_z}.
template <>
struct Record<GBD_STORE_F32> {
    using T = float4;
    static __device__ __forceinline__ T load(const void *base, long long off)
    {
        return __ldg(reinterpret_cast<const float4 *>(base) + off);
    }
    static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    // Both snapshots of a paired block: 32 contiguous bytes.
    static __device__ __forceinline__ void load_pair(const void *base, long long off, T &lo, T &hi)
    {
        const float4 *p = reinterpret_cast<const float4 *>(base) + off;
        lo = __ldg(p);
        hi = __ldg(p + 1);
    }
    // D^(2 - alpha) j' with D = sqrt(1 - beta^2) / (1 + beta . s_hat) (Eq. 14).
    // 1 + beta.s_hat and 1 - beta^2 are formed with fused multiply-adds so
    // each is rounded once near its (possibly small) value.
    static __device__ __forceinline__ float emissivity(const T r) { return r.x; }
    // D^(2 - alpha), or 1 without beaming
    static __device__ __forceinline__ float boost(const T r, const BoostConsts &c)
    {
        if (!c.beaming) return 1.0f;
        float den = fmaf(r.y, c.shx, fmaf(r.z, c.shy, fmaf(r.w, c.shz, 1.0f)));
        den += fmaf(r.y, c.slx, fmaf(r.z, c.sly, r.w * c.slz));
        const float inv_g2 = fmaf(-r.y, r.y, fmaf(-r.z, r.z, fmaf(-r.w, r.w, 1.0f)));
        const float log2_d = fmaf(0.5f, lg2_approx(inv_g2), -lg2_approx(den));
        return ex2_approx(c.expo * log2_d);
    }
    static __device__ __forceinline__ float boosted(const T r, const BoostConsts &c)
    {
        return emissivity(r) * boost(r, c);
    }
    // boosted() of two records.  Scalar: pairing the fields of two float4
    // records for the paired float32 instructions costs register moves, and
    // measured slower than the scalar steps.
    static __device__ __forceinline__ float2 boosted2(const T lo, const T hi, const BoostConsts &c)
    {
        return make_float2(boosted(lo, c), boosted(hi, c));
    }
};

// 8-byte record {bf16 j', f16 u_x, f16 u_y, f16 u_z}, u = Gamma beta.
template <>
struct Record<GBD_STORE_BF16_F16U> {
    using T = uint2;
    static __device__ __forceinline__ T load(const void *base, long long off)
    {
        return __ldg(reinterpret_cast<const uint2 *>(base) + off);
    }
    static __device__ __forceinline__ T zero() { return make_uint2(0u, 0u); }
    // Both snapshots of a paired block: one 16-byte load (off is even).
    static __device__ __forceinline__ void load_pair(const void *base, long long off, T &lo, T &hi)
    {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(base) + (off >> 1));
        lo = make_uint2(v.x, v.y);
        hi = make_uint2(v.z, v.w);
    }
    // The same by byte address.
    static __device__ __forceinline__ T load_at(unsigned long long a) { return __ldg(reinterpret_cast<const uint2 *>(a)); }
    static __device__ __forceinline__ void load_pair_at(unsigned long long a, T &lo, T &hi)
    {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a));
        lo = make_uint2(v.x, v.y);
        hi = make_uint2(v.z, v.w);
    }
    // D = 1 / (Gamma + u.s_hat).  When u.s_hat < 0 (motion towards the
    // observer) the denominator cancels, so the same D is evaluated as
    // (Gamma + |u.s_hat|) / (1 + |u|^2 - (u.s_hat)^2), which has no cancellation.
    // s_hat enters rounded to float: its rounding (6e-8) is far below the
    // float16 resolution of u (5e-4 relative), unlike in the float32 record.
    static __device__ __forceinline__ float emissivity(const T r) { return __uint_as_float(r.x << 16); }
    // D^(2 - alpha), or 1 without beaming
    static __device__ __forceinline__ float boost(const T r, const BoostConsts &c)
    {
        if (!c.beaming) return 1.0f;
        // u_x is the high half of r.x, (u_y, u_z) the two halves of r.y
        __half2 hx, hyz;
        memcpy(&hx, &r.x, sizeof(hx));
        memcpy(&hyz, &r.y, sizeof(hyz));
        const float ux = __high2float(hx);
        const float2 uyz = __half22float2(hyz);
        const float uy = uyz.x, uz = uyz.y;
        const float us = fmaf(ux, c.shx, fmaf(uy, c.shy, uz * c.shz));
        const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float gp = sqrt_approx(1.0f + uu) + fabsf(us);
        const float perp = 1.0f + fmaf(-us, us, uu);
        const float log2_d = (us < 0.f) ? (lg2_approx(gp) - lg2_approx(perp)) : -lg2_approx(gp);
        return ex2_approx(c.expo * log2_d);
    }
    static __device__ __forceinline__ float boosted(const T r, const BoostConsts &c)
    {
        return emissivity(r) * boost(r, c);
    }
    // boosted2() in the plain form D = 1 / (Gamma + u.s_hat), log2 D =
    // -log2(Gamma + u.s_hat).  For u.s_hat near -Gamma the sum cancels: its
    // float32 rounding (about 3.3e-7 Gamma absolute) over Gamma + u.s_hat >=
    // 1 / (2 Gamma) bounds the relative error of D by 6.6e-7 Gamma^2, at most
    // 4.3e-5 (1.1e-4 in D^2.6) for Gamma <= 8, the volumes this form is used
    // for (beta <= 0.992); the float16 u itself carries 4.9e-4.
    static __device__ __forceinline__ float2 boosted2_plain(const T lo, const T hi, const BoostConsts &c)
    {
        const float2 j = make_float2(__uint_as_float(lo.x << 16), __uint_as_float(hi.x << 16));
        if (!c.beaming) return j;
        const uint32_t px = __byte_perm(lo.x, hi.x, 0x7632);  // (u_x lo, u_x hi)
        const uint32_t py = __byte_perm(lo.y, hi.y, 0x5410);  // (u_y lo, u_y hi)
        const uint32_t pz = __byte_perm(lo.y, hi.y, 0x7632);  // (u_z lo, u_z hi)
        __half2 hx, hy, hz;
        memcpy(&hx, &px, sizeof(hx));
        memcpy(&hy, &py, sizeof(hy));
        memcpy(&hz, &pz, sizeof(hz));
        const float2 ux = __half22float2(hx), uy = __half22float2(hy), uz = __half22float2(hz);
        const float2 us = __ffma2_rn(ux, f2(c.shx), __ffma2_rn(uy, f2(c.shy), __fmul2_rn(uz, f2(c.shz))));
        const float2 g2 = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __ffma2_rn(uz, uz, f2(1.0f))));  // Gamma^2
        const float2 den = __fadd2_rn(make_float2(sqrt_approx(g2.x), sqrt_approx(g2.y)), us);
        const float2 e = __fmul2_rn(f2(-c.expo), make_float2(lg2_approx(den.x), lg2_approx(den.y)));
        return __fmul2_rn(j, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
    }
    // boosted() of two records at once: their u components are paired by
    // byte permutes, then each lane takes the same correctly rounded steps as
    // boosted() (paired float32 instructions of sm_100 and later).
    static __device__ __forceinline__ float2 boosted2(const T lo, const T hi, const BoostConsts &c)
    {
        const float2 j = make_float2(__uint_as_float(lo.x << 16), __uint_as_float(hi.x << 16));
        if (!c.beaming) return j;
        const uint32_t px = __byte_perm(lo.x, hi.x, 0x7632);  // (u_x lo, u_x hi)
        const uint32_t py = __byte_perm(lo.y, hi.y, 0x5410);  // (u_y lo, u_y hi)
        const uint32_t pz = __byte_perm(lo.y, hi.y, 0x7632);  // (u_z lo, u_z hi)
        __half2 hx, hy, hz;
        memcpy(&hx, &px, sizeof(hx));
        memcpy(&hy, &py, sizeof(hy));
        memcpy(&hz, &pz, sizeof(hz));
        const float2 ux = __half22float2(hx), uy = __half22float2(hy), uz = __half22float2(hz);
        const float2 us = __ffma2_rn(ux, f2(c.shx), __ffma2_rn(uy, f2(c.shy), __fmul2_rn(uz, f2(c.shz))));
        const float2 uu = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __fmul2_rn(uz, uz)));
        const float2 g1 = __fadd2_rn(f2(1.0f), uu);
        const float2 gp = __fadd2_rn(make_float2(sqrt_approx(g1.x), sqrt_approx(g1.y)),
                                     make_float2(fabsf(us.x), fabsf(us.y)));
        const float2 perp = __fadd2_rn(f2(1.0f), __ffma2_rn(neg2(us), us, uu));
        const float2 lgp = make_float2(lg2_approx(gp.x), lg2_approx(gp.y));
        const float2 lpp = make_float2(lg2_approx(perp.x), lg2_approx(perp.y));
        const float2 dif = __fadd2_rn(lgp, neg2(lpp));
        const float2 lg = make_float2(us.x < 0.f ? dif.x : -lgp.x, us.y < 0.f ? dif.y : -lgp.y);
        const float2 e = __fmul2_rn(f2(c.expo), lg);
        return __fmul2_rn(j, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
    }
};

#ifdef GBD_CHECKED
__device__ __forceinline__ bool check_cell(const VolDev &vol, int *err_word, int ix, int iy, int iz, int m)
{
    const bool ok = ix >= 0 && ix < vol.n[0] && iy >= 0 && iy < vol.n[1] && iz >= 0 && iz < vol.n[2] &&
                    m >= 0 && m < vol.M;
    if (!ok && err_word) atomicCAS(err_word, 0, 1);
    return ok;
}
#endif

// The epoch coordinate u = (t_bar - t0) / dt is carried in Q31.32 fixed point
// (int64, 2^-32 epochs per unit): float32 cannot resolve u to better than half
// an ulp of the snapshot count (about 4e-6 at u ~ 64), which a fast-changing
// field amplifies beyond a 1e-5 relative pixel tolerance; integer updates are
// exact and cheap.
constexpr float kTwo32 = 4294967296.0f;        // 2^32
constexpr float kTwo40 = 1099511627776.0f;      // 2^40
constexpr float kInv2p40 = 9.094947017729282e-13f;  // 2^-40

// x (a float) times y = y_hi + y_lo (a double-float), as a fixed-point
// integer of scale `scale`: the product x * y_hi is split exactly into its
// rounded value and rounding error with a fused multiply-add, and each part
// is converted separately, so the result carries about 48 bits of y.
__device__ __forceinline__ long long dd_mul_fix(float x, float y_hi, float y_lo, float scale)
{
    const float p = __fmul_rn(x, y_hi);
    const float e = fmaf(x, y_hi, -p);
    const float r = fmaf(x, y_lo, e);
    return __float2ll_rn(p * scale) + __float2ll_rn(r * scale);
}

__device__ __forceinline__ float fix_to_float(long long v, float inv_scale)
{
    return __ll2float_rn(v) * inv_scale;
}

// One term of the march tables at byte offset `cur` from `base`: shared
// memory in the single-volume kernel, global memory when serving.
template <bool SMEM>
__device__ __forceinline__ int32_t tab_at(const int32_t *base, uint32_t cur)
{
    const int32_t *p = reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(base) + cur);
    if (SMEM) return *p;
    return __ldg(p);
}

// Copies a volume's march tables into shared memory, followed by kTabPad
// sentinels: the branch-free step of a lane whose ray has ended reads up to
// two entries past the sentinel pair it stopped at.
__device__ __forceinline__ void stage_tables(int32_t *s_tab, const int32_t *src, int ntab)
{
    for (int i = threadIdx.x; i < ntab + kTabPad; i += blockDim.x) s_tab[i] = i < ntab ? src[i] : kTabSentinel;
}

// State of one axis of a ray: the next face crossing and what changes there.
struct AxisState {
    float nkf;      // planes from the anchor cell's lower face to the next crossing
    float sn;       // s of the next crossing, relative to the anchor
    float of;       // the anchor's offset inside its cell, times the face spacing
    long long un;   // epoch coordinate at the next crossing, Q31.32
    uint32_t cur;   // byte offset of the current cell's table term
    int32_t o;      // table term of the current cell
    int32_t pn;     // table term of the next cell (read ahead)
};

// Steps a ray into its next cell through the face of axis 0, 1 or 2 (x0, x1,
// else axis 2): that axis's next crossing is recomputed from its plane count
// (never accumulated), its epoch coordinate drops by the exact per-plane
// amount, and the table term of the cell after is read ahead.  Every update is
// a select on the exit axis, so the lanes of a warp never diverge here;
// recomputing an axis's crossing from an unchanged plane count reproduces it
// (an axis the ray runs parallel to has of = -3e38 and inv_a = 0, so its
// crossing stays at 3e38).
template <bool SMEM>
__device__ __forceinline__ void step_exit(AxisState (&ax)[3], bool x0, bool x1, float ia0, float ia1, float ia2,
                                          long long du0, long long du1, long long du2, const int32_t *tab)
{
    const bool x2 = !x0 && !x1;
    const uint32_t ce = x0 ? ax[0].cur : (x1 ? ax[1].cur : ax[2].cur);
    const int32_t tn = tab_at<SMEM>(tab, ce + 8u);
    ax[0].nkf = x0 ? ax[0].nkf + 1.0f : ax[0].nkf;
    ax[1].nkf = x1 ? ax[1].nkf + 1.0f : ax[1].nkf;
    ax[2].nkf = x2 ? ax[2].nkf + 1.0f : ax[2].nkf;
    ax[0].un = x0 ? ax[0].un - du0 : ax[0].un;
    ax[1].un = x1 ? ax[1].un - du1 : ax[1].un;
    ax[2].un = x2 ? ax[2].un - du2 : ax[2].un;
    ax[0].o = x0 ? ax[0].pn : ax[0].o;
    ax[1].o = x1 ? ax[1].pn : ax[1].o;
    ax[2].o = x2 ? ax[2].pn : ax[2].o;
    ax[0].pn = x0 ? tn : ax[0].pn;
    ax[1].pn = x1 ? tn : ax[1].pn;
    ax[2].pn = x2 ? tn : ax[2].pn;
    ax[0].cur = x0 ? ax[0].cur + 4u : ax[0].cur;
    ax[1].cur = x1 ? ax[1].cur + 4u : ax[1].cur;
    ax[2].cur = x2 ? ax[2].cur + 4u : ax[2].cur;
    ax[0].sn = fmaf(ax[0].nkf, ia0, -ax[0].of);
    ax[1].sn = fmaf(ax[1].nkf, ia1, -ax[1].of);
    ax[2].sn = fmaf(ax[2].nkf, ia2, -ax[2].of);
}

// The box a ray is marched through, in the march frame (mirrored axes
// mirrored), and where its table terms start: the whole grid for a direct
// render, one region of it for the region schedule.  Along axis i the cells
// lo[i] .. hi[i] - 1 have their terms at byte offsets cur0[i], cur0[i] + 4, ...
// followed by two sentinels.
struct RayBox {
    int lo[3], hi[3];
    uint32_t cur0[3];
};

// The whole grid as seen by view V, with the volume's own march tables.
__device__ __forceinline__ RayBox grid_box(const VolDev &vol, const ViewDev &V)
{
    RayBox B;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool mirrored = (V.flags & (kFlagMirror0 << i)) != 0u;
        B.lo[i] = 0;
        B.hi[i] = vol.n[i];
        B.cur0[i] = 4u * static_cast<uint32_t>(march_table_base(vol.n, i) + (mirrored ? vol.n[i] + 2 : 0));
    }
    return B;
}

// State of a ray during the march: per axis the next crossing, the current
// cell's chord start (the latest face crossed) and its epoch coordinate.
struct RayState {
    AxisState ax[3];
    float s_cur;       // s of the latest face crossed
    long long u_cur;   // epoch coordinate there, Q31.32
    long long u_a;     // epoch coordinate at the anchor (s = 0), Q31.32
    bool alive;
#ifdef GBD_CHECKED
    int kc[3], kd[3];  // current cell in the volume's own frame, and its step per axis
#endif
};

// Ray set-up, once per ray, no float64: the anchor at the later of the box
// entry and the window start [win_lo, win_hi] (a view's own window, or the
// union of a group's), its cell and crossings, and the leading empty chords
// stepped through, so that the march proper starts on the first cell whose
// chord is positive.
template <bool SMEM>
__device__ __forceinline__ void setup_ray(RayState &R, const VolDev &vol, const ViewDev &V, const RayBox &B, int p,
                                          int q, bool in_image, float win_lo, float win_hi,
                                          const int32_t *__restrict__ tab)
{
    AxisState (&ax)[3] = R.ax;
    bool &alive = R.alive;
    float &s_cur = R.s_cur;
    long long &u_cur = R.u_cur;
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
#endif
    alive = in_image;
    // Pixel position on the image plane in grid-index units (Q24.40, exact
    // integer arithmetic from the per-view constants), in the frame where
    // every axis is marched upwards.
    long long g0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        g0[i] = V.g0[i] + static_cast<long long>(p) * V.gu[i] + static_cast<long long>(q) * V.gv[i];
    // Estimated start of the traversal: the later of the box entry and the
    // window start.  This anchor only has to be a point of the ray no more
    // than a cell past the true start (crossings are measured from it, so it
    // should be close to keep them accurate); it may lie outside the box.
    float s_in_e = -3.0e38f, s_out_e = 3.0e38f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (V.inv_a[i] != 0.f) {
            const float gf = fix_to_float(g0[i], kInv2p40);
            s_in_e = fmaxf(s_in_e, (static_cast<float>(B.lo[i]) - gf) * V.inv_a[i]);
            s_out_e = fminf(s_out_e, (static_cast<float>(B.hi[i]) - gf) * V.inv_a[i]);
        } else if (g0[i] < (static_cast<long long>(B.lo[i]) << 40) ||
                   g0[i] >= (static_cast<long long>(B.hi[i]) << 40)) {
            alive = false;  // parallel to this axis and outside the box along it
        }
    }
    const float s_a = fmaxf(s_in_e, win_lo);
    if (!(fminf(s_out_e, win_hi) > s_a - 1e-3f * (1.f + fabsf(s_a)))) alive = false;
    const float sa = alive ? s_a : 0.f;

    // Anchor: the point s_a of the ray, in exact fixed point; its cell (k,
    // clamped onto the grid), the position o inside that cell, and per axis
    // the face spacing along the ray (inv_a, Eq. 11), so that the crossing of
    // the plane nk cells above the cell's lower face is at nk inv_a - o inv_a.
    const long long u_a = V.u_obs - dd_mul_fix(sa, V.kk_hi, V.kk_lo, kTwo32);
    R.u_a = u_a;
    s_cur = -3.0e38f;  // the latest entry face of the anchor cell
    u_cur = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool moving = V.inv_a[i] != 0.f;
        const long long ga = moving ? g0[i] + dd_mul_fix(sa, V.a_hi[i], V.a_lo[i], kTwo40) : g0[i];
        int k = static_cast<int>(ga >> 40);
        k = min(max(k, B.lo[i]), B.hi[i] - 1);
        const float o = fix_to_float(ga - (static_cast<long long>(k) << 40), kInv2p40);
        AxisState &A = ax[i];
        A.nkf = 1.0f;
        A.of = o * V.inv_a[i];
        if (moving) {
            A.sn = V.inv_a[i] - A.of;
            A.un = u_a - dd_mul_fix(1.0f - o, V.w_hi[i], V.w_lo[i], kTwo32);
            // the anchor cell's entry face along this axis (plane nk = 0)
            if (-A.of > s_cur) {
                s_cur = -A.of;
                u_cur = A.un + V.du[i];
            }
        } else {
            A.of = -3.0e38f;     // with inv_a = 0: the crossing stays at 3e38,
            A.sn = 3.0e38f;      // never the nearest face ...
            A.un = LLONG_MIN / 2;  // ... and ends the ray if it ever were
        }
        A.cur = B.cur0[i] + 4u * static_cast<uint32_t>(k - B.lo[i]);
        A.o = 0;
        A.pn = 0;
        if (alive) {
            A.o = tab_at<SMEM>(tab, A.cur);
            A.pn = tab_at<SMEM>(tab, A.cur + 4u);
        }
#ifdef GBD_CHECKED
        kc[i] = (V.flags & (kFlagMirror0 << i)) ? vol.n[i] - 1 - k : k;
#endif
    }
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const long long du0 = V.du[0], du1 = V.du[1], du2 = V.du[2];
#ifdef GBD_CHECKED
    const int kd0 = (V.flags & kFlagMirror0) ? -1 : 1;
    const int kd1 = (V.flags & (kFlagMirror0 << 1)) ? -1 : 1;
    const int kd2 = (V.flags & (kFlagMirror0 << 2)) ? -1 : 1;
    R.kd[0] = kd0;
    R.kd[1] = kd1;
    R.kd[2] = kd2;
#endif

    // Leading empty chords: when the anchor cell was clamped onto the grid, or
    // the anchor sits on a face, the ray can leave a cell along one axis before
    // it has entered it along another.  Those cells are stepped through until
    // the nearest exit lies past the latest entry; from there on the exits
    // only increase, so every chord of the march proper starts at the end of
    // the one before.  Each step moves one table cursor up, and a sentinel
    // stops the ray at the box face, so the loop is bounded by the grid.
    if (alive) {
        for (int guard = B.hi[0] + B.hi[1] + B.hi[2] + 4; guard > 0; --guard) {
            const bool x0 = ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
            const bool x1 = !x0 && ax[1].sn <= ax[2].sn;
            const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
            if (s_exit > s_cur) break;
            step_exit<SMEM>(ax, x0, x1, ia0, ia1, ia2, du0, du1, du2, tab);
#ifdef GBD_CHECKED
            kc[0] += x0 ? kd0 : 0;
            kc[1] += x1 ? kd1 : 0;
            kc[2] += (!x0 && !x1) ? kd2 : 0;
#endif
            if ((ax[0].o | ax[1].o | ax[2].o) < 0) {
                alive = false;
                break;
            }
        }
    }
}

// The float epoch coordinate of the bfloat16/float16 march: u(s) = c0 -
// kk s along the ray (s from the anchor), so that the chord midpoint's is
// c0 + mkk (s_cur + s_exit) with mkk = -kk / 2; the ray has passed the last
// time that reaches a snapshot (u < -1) beyond s_stop.  c0 is the exact
// coordinate at the anchor rounded to float: the coordinate is off by at most
// a few float ulps of M (2e-6 snapshots at M = 16), against the 2^-9 and
// 2^-11 resolution of the stored j' and u.
struct EpochLine {
    float c0, mkk, s_stop;
};
__device__ __forceinline__ EpochLine epoch_line(const RayState &R, const ViewDev &V)
{
    EpochLine L;
    const float kk = V.kk_hi;
    L.c0 = fix_to_float(R.u_a, 1.0f / kTwo32);
    L.mkk = -0.5f * kk;
    L.s_stop = kk > 0.f ? (L.c0 + 1.0f) / kk : 3.0e38f;
    return L;
}

// One step of the bfloat16/float16 march through the face of axis 0, 1 or 2
// (x0, x1, x2, at most one of them set; none once the ray has ended): the
// plane count and crossing of that axis, and its table terms.  Every lane
// executes it; a lane that takes no step changes nothing, and its read of
// the table stays within the padding after the last sentinel.
template <bool SMEM>
__device__ __forceinline__ void step_lite(AxisState (&ax)[3], bool x0, bool x1, bool x2, float ia0, float ia1,
                                          float ia2, const int32_t *tab)
{
    const uint32_t ce = x0 ? ax[0].cur : (x1 ? ax[1].cur : ax[2].cur);
    const int32_t tn = tab_at<SMEM>(tab, ce + 8u);
    ax[0].nkf = x0 ? ax[0].nkf + 1.0f : ax[0].nkf;
    ax[1].nkf = x1 ? ax[1].nkf + 1.0f : ax[1].nkf;
    ax[2].nkf = x2 ? ax[2].nkf + 1.0f : ax[2].nkf;
    ax[0].o = x0 ? ax[0].pn : ax[0].o;
    ax[1].o = x1 ? ax[1].pn : ax[1].o;
    ax[2].o = x2 ? ax[2].pn : ax[2].o;
    ax[0].pn = x0 ? tn : ax[0].pn;
    ax[1].pn = x1 ? tn : ax[1].pn;
    ax[2].pn = x2 ? tn : ax[2].pn;
    ax[0].cur = x0 ? ax[0].cur + 4u : ax[0].cur;
    ax[1].cur = x1 ? ax[1].cur + 4u : ax[1].cur;
    ax[2].cur = x2 ? ax[2].cur + 4u : ax[2].cur;
    ax[0].sn = fmaf(ax[0].nkf, ia0, -ax[0].of);
    ax[1].sn = fmaf(ax[1].nkf, ia1, -ax[1].of);
    ax[2].sn = fmaf(ax[2].nkf, ia2, -ax[2].of);
}

// The march of march_ray for bfloat16/float16 records (see the file
// header): same cells, chords, midpoints and hat weights (Eqs. 2, 6-9, 19),
// with the epoch coordinate of EpochLine.  PLAIN: the Doppler factor in the
// plain form (volumes whose Gamma <= 8).
template <int DEPTH, bool PAIRED, bool PARTIAL, bool PLAIN>
__device__ __forceinline__ void march_ray_bf16(const VolDev &vol, const ViewDev &V, const RayBox &B, int p, int q,
                                               int width, int height, float *out_img, uint32_t *cnt_img,
                                               int *err_word, const int32_t *__restrict__ tab, bool accumulate)
{
    using Rec = Record<GBD_STORE_BF16_F16U>;
    const bool in_image = (p < width) && (q < height);
    RayState R;
    setup_ray<true>(R, vol, V, B, p, q, in_image, V.win_lo, V.win_hi, tab);
    AxisState (&ax)[3] = R.ax;
    bool alive = R.alive;
    float s_cur = R.s_cur;
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const EpochLine L = epoch_line(R, V);
    const int M = vol.M;
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
    const int kd0 = R.kd[0], kd1 = R.kd[1], kd2 = R.kd[2];
#endif

    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;
    bc.plain = PLAIN;

    // block b starts at byte recb + b es_bytes; a cell's record (paired: its
    // record pair) is kUnit bytes at its layout offset
    constexpr unsigned long long kUnit = PAIRED ? 16ull : 8ull;
    const unsigned long long recb = reinterpret_cast<unsigned long long>(vol.rec);
    const long long es_bytes = vol.epoch_stride * 8LL;

    float acc = 0.f;
    uint32_t count = 0;
    while (__any_sync(kFull, alive)) {
        unsigned long long pa[DEPTH];
        float wgt[DEPTH], dsv[DEPTH];
        bool has_lo[DEPTH], has_hi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            // the nearest face (ties to the lowest axis), the chord, and the
            // epoch coordinate at the chord midpoint: m_bar + w
            const bool x0 = alive && ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
            const bool x1 = alive && !x0 && ax[1].sn <= ax[2].sn;
            const bool x2 = alive && !x0 && !x1;
            const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
            const float ds = s_exit - s_cur;
            const float um = fmaf(L.mkk, s_cur + s_exit, L.c0);
            const float fl = floorf(um);
            const float w = um - fl;
            const int mb = static_cast<int>(fl);
            // -1 <= m_bar <= M - 1; snapshots m_bar (weight 1 - w) and m_bar + 1 (w)
            const bool take = alive && ds > 0.f && static_cast<unsigned>(mb + 1) <= static_cast<unsigned>(M);
            has_lo[d] = take && mb >= 0;
            has_hi[d] = take && mb < M - 1 && w != 0.f;
#ifdef GBD_CHECKED
            if ((has_lo[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb)) ||
                (has_hi[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb + 1)))
                has_lo[d] = has_hi[d] = false;
            kc[0] += x0 ? kd0 : 0;
            kc[1] += x1 ? kd1 : 0;
            kc[2] += x2 ? kd2 : 0;
#endif
            const int sum = ax[0].o + ax[1].o + ax[2].o;
            // unpaired: snapshot m at block m; paired: snapshots mb and mb + 1
            // side by side in block mb + 1
            pa[d] = recb + static_cast<unsigned long long>(static_cast<long long>(PAIRED ? mb + 1 : mb) * es_bytes) +
                    static_cast<unsigned long long>(static_cast<uint32_t>(sum)) * kUnit;
            wgt[d] = take ? w : 0.f;
            dsv[d] = take ? ds : 0.f;
            step_lite<true>(ax, x0, x1, x2, ia0, ia1, ia2, tab);
            s_cur = s_exit;
            // past the last time that reaches a snapshot, or out of the box
            alive = alive && s_exit <= L.s_stop && (ax[0].o | ax[1].o | ax[2].o) >= 0;
        }
        typename Rec::T rlo[DEPTH], rhi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            rlo[d] = Rec::zero();
            rhi[d] = Rec::zero();
            if (PAIRED) {
                if (has_lo[d] || has_hi[d]) Rec::load_pair_at(pa[d], rlo[d], rhi[d]);
            } else {
                if (has_lo[d]) rlo[d] = Rec::load_at(pa[d]);
                if (has_hi[d]) rhi[d] = Rec::load_at(pa[d] + es_bytes);
            }
        }
        // A snapshot a sample does not read is a zero record (boosted value
        // exactly 0), and a sample not taken has weight and chord 0.
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            const float2 vv = PLAIN ? Rec::boosted2_plain(rlo[d], rhi[d], bc) : Rec::boosted2(rlo[d], rhi[d], bc);
            const float v = fmaf(wgt[d], vv.y - vv.x, vv.x);  // Eq. 8
            acc = fmaf(v, dsv[d], acc);
            count += (has_lo[d] || has_hi[d]) ? 1u : 0u;
        }
    }

    if (in_image) {
        const long long pix = static_cast<long long>(q) * width + p;
        if (PARTIAL) {
            if (count > 0u) atomicAdd(out_img + pix, acc);
        } else if (accumulate) {
            out_img[pix] += V.prefactor * acc;
            if (cnt_img) cnt_img[pix] += count;
        } else {
            out_img[pix] = V.prefactor * acc;
            if (cnt_img) cnt_img[pix] = count;
        }
    }
}

// step_lite with the exact epoch coordinate of each axis (float32 march).
template <bool SMEM>
__device__ __forceinline__ void step_nb(AxisState (&ax)[3], bool x0, bool x1, bool x2, float ia0, float ia1,
                                        float ia2, long long du0, long long du1, long long du2, const int32_t *tab)
{
    step_lite<SMEM>(ax, x0, x1, x2, ia0, ia1, ia2, tab);
    ax[0].un = x0 ? ax[0].un - du0 : ax[0].un;
    ax[1].un = x1 ? ax[1].un - du1 : ax[1].un;
    ax[2].un = x2 ? ax[2].un - du2 : ax[2].un;
}

// The march of march_ray for float32 records without branches: the step of
// march_ray_bf16 (every lane executes it; a lane whose ray has ended takes no
// step and reads no record) with the exact Q31.32 epoch coordinate, the
// float32 Doppler factor of Eq. 14 and the compensated sum.  Its arithmetic
// is that of the branching form, value for value.
template <int DEPTH, bool PAIRED, bool PARTIAL>
__device__ __forceinline__ void march_ray_f32(const VolDev &vol, const ViewDev &V, const RayBox &B, int p, int q,
                                              int width, int height, float *out_img, uint32_t *cnt_img,
                                              int *err_word, const int32_t *__restrict__ tab, bool accumulate)
{
    using Rec = Record<GBD_STORE_F32>;
    const bool in_image = (p < width) && (q < height);
    RayState R;
    setup_ray<true>(R, vol, V, B, p, q, in_image, V.win_lo, V.win_hi, tab);
    AxisState (&ax)[3] = R.ax;
    bool alive = R.alive;
    float s_cur = R.s_cur;
    long long u_cur = R.u_cur;
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const long long du0 = V.du[0], du1 = V.du[1], du2 = V.du[2];
    const int Mm1 = vol.M - 1;
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
    const int kd0 = R.kd[0], kd1 = R.kd[1], kd2 = R.kd[2];
#endif
    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;
    bc.plain = false;
    // block b starts at byte recb + b es_bytes; a cell's record (paired: its
    // record pair) is kUnit bytes at its layout offset.  Paired: a sample that
    // reads no snapshot loads the zero record pair after the last block
    // (faster for 32-byte pairs than a predicated load).
    constexpr unsigned long long kUnit = PAIRED ? 32ull : 16ull;
    const unsigned long long recb = reinterpret_cast<unsigned long long>(vol.rec);
    const long long es_bytes = vol.epoch_stride * 16LL;
    const unsigned long long zero_addr = recb + static_cast<unsigned long long>((vol.M + 1) * es_bytes);

    float acc = 0.f, comp = 0.f;
    uint32_t count = 0;
    while (__any_sync(kFull, alive)) {
        unsigned long long pa[DEPTH];
        float wgt[DEPTH], dsv[DEPTH];
        bool has_lo[DEPTH], has_hi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            const bool x0 = alive && ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
            const bool x1 = alive && !x0 && ax[1].sn <= ax[2].sn;
            const bool x2 = alive && !x0 && !x1;
            const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
            const long long u_exit = x0 ? ax[0].un : (x1 ? ax[1].un : ax[2].un);
            const float ds = s_exit - s_cur;
            // epoch coordinate at the chord midpoint: m_bar + w, w in [0, 1)
            const long long um = (u_cur + u_exit) >> 1;
            const int mb = static_cast<int>(um >> 32);
            const uint32_t frac = static_cast<uint32_t>(um);
            const float w = static_cast<float>(frac) * 2.3283064365386963e-10f;
            // -1 <= m_bar <= M - 1 (at u = -1 exactly both weights vanish)
            const bool take = alive && ds > 0.f && static_cast<unsigned>(mb + 1) <= static_cast<unsigned>(Mm1 + 1);
            has_lo[d] = take && mb >= 0;
            has_hi[d] = take && mb < Mm1 && frac != 0u;
#ifdef GBD_CHECKED
            if ((has_lo[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb)) ||
                (has_hi[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb + 1)))
                has_lo[d] = has_hi[d] = false;
            kc[0] += x0 ? kd0 : 0;
            kc[1] += x1 ? kd1 : 0;
            kc[2] += x2 ? kd2 : 0;
#endif
            const int sum = ax[0].o + ax[1].o + ax[2].o;
            const unsigned long long a = recb + static_cast<unsigned long long>(static_cast<long long>(PAIRED ? mb + 1 : mb) * es_bytes) +
                    static_cast<unsigned long long>(static_cast<uint32_t>(sum)) * kUnit;
            pa[d] = PAIRED ? ((has_lo[d] || has_hi[d]) ? a : zero_addr) : a;
            wgt[d] = w;
            dsv[d] = ds;
            step_nb<true>(ax, x0, x1, x2, ia0, ia1, ia2, du0, du1, du2, tab);
            s_cur = s_exit;
            u_cur = u_exit;
            // past the last time that reaches a snapshot (u < -1), or out of the box
            alive = alive && static_cast<int>(u_exit >> 32) >= -1 && (ax[0].o | ax[1].o | ax[2].o) >= 0;
        }
        typename Rec::T rlo[DEPTH], rhi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            if (PAIRED) {
                const float4 *ptr = reinterpret_cast<const float4 *>(pa[d]);
                rlo[d] = __ldg(ptr);
                rhi[d] = __ldg(ptr + 1);
            } else {
                rlo[d] = has_lo[d] ? __ldg(reinterpret_cast<const float4 *>(pa[d])) : Rec::zero();
                rhi[d] = has_hi[d] ? __ldg(reinterpret_cast<const float4 *>(pa[d] + es_bytes)) : Rec::zero();
            }
        }
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            // a snapshot the sample does not read is a zero record (boosted
            // value exactly 0); the compensated sum takes the sample only where
            // it read one
            const float vlo = Rec::boosted(rlo[d], bc);
            const float vhi = Rec::boosted(rhi[d], bc);
            const float v = fmaf(wgt[d], vhi - vlo, vlo);  // Eq. 8
            const float y = fmaf(v, dsv[d], -comp);
            const float t = acc + y;
            const bool take = has_lo[d] || has_hi[d];
            comp = take ? (t - acc) - y : comp;
            acc = take ? t : acc;
            count += take ? 1u : 0u;
        }
    }
    if (in_image) {
        const long long pix = static_cast<long long>(q) * width + p;
        if (PARTIAL) {
            if (count > 0u) atomicAdd(out_img + pix, acc);
        } else if (accumulate) {
            out_img[pix] += V.prefactor * acc;
            if (cnt_img) cnt_img[pix] += count;
        } else {
            out_img[pix] = V.prefactor * acc;
            if (cnt_img) cnt_img[pix] = count;
        }
    }
}

// Marches the ray of pixel (p, q) of one image through box B.  Direct
// (PARTIAL false): stores the pixel value (Eq. 19, with the prefactor) and,
// if cnt_img is set, its cell-sample count, or adds them to what is there
// when `accumulate` is set (one thread owns each pixel, so the adds of
// successive launches land in launch order).  PARTIAL: adds the ray's sum over
// the box, without the prefactor, to out_img[pixel] if the ray sampled at
// least one cell there (one region per slot and ray, so the add lands on
// zero).  tab points at the march tables (shared memory when SMEM).
//
// NCH > 0 (vector renders, Sec. 2.1): the volume carries NCH more emissivity
// channels sharing its velocity; each is summed with the same weights and
// Doppler factors as j' (Eq. 19 per channel) into component c + 1 of the
// pixel, at out_img + (c + 1) * width * height.
//
// TOUCH (memory analysis, not a render): instead of reading the two records
// of a sample, set the bits of (snapshot, cell) in the bitmap `touch`, whose
// bit m * cell_stride + cell stands for that record.
struct ChanPtrs {
    const float *chan;
    long long comp_stride, cell_stride;
    uint32_t *touch;
};

template <int STORE, int DEPTH, bool PAIRED, bool SMEM, bool PARTIAL = false, int NCH = 0, bool TOUCH = false>
__device__ __forceinline__ void march_ray(const VolDev &vol, const ViewDev &V, const RayBox &B, int p, int q,
                                          int width, int height, float *out_img, uint32_t *cnt_img, int *err_word,
                                          const int32_t *__restrict__ tab, bool accumulate = false,
                                          const ChanPtrs ch = ChanPtrs{nullptr, 0, 0, nullptr})
{
    if constexpr (STORE == GBD_STORE_BF16_F16U && NCH == 0 && !TOUCH && SMEM) {
        if (vol.plain_boost)
            march_ray_bf16<DEPTH, PAIRED, PARTIAL, true>(vol, V, B, p, q, width, height, out_img, cnt_img, err_word,
                                                         tab, accumulate);
        else
            march_ray_bf16<DEPTH, PAIRED, PARTIAL, false>(vol, V, B, p, q, width, height, out_img, cnt_img, err_word,
                                                          tab, accumulate);
        return;
    }
    if constexpr (STORE == GBD_STORE_F32 && NCH == 0 && !TOUCH && SMEM) {
        march_ray_f32<DEPTH, PAIRED, PARTIAL>(vol, V, B, p, q, width, height, out_img, cnt_img, err_word, tab,
                                              accumulate);
        return;
    }
    using Rec = Record<STORE>;
    const bool in_image = (p < width) && (q < height);
    RayState R;
    setup_ray<SMEM>(R, vol, V, B, p, q, in_image, V.win_lo, V.win_hi, tab);
    AxisState (&ax)[3] = R.ax;
    bool &alive = R.alive;
    float &s_cur = R.s_cur;
    long long &u_cur = R.u_cur;
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const long long du0 = V.du[0], du1 = V.du[1], du2 = V.du[2];
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
    const int kd0 = R.kd[0], kd1 = R.kd[1], kd2 = R.kd[2];
#endif
    const int Mm1 = vol.M - 1;

    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;

    const long long es = vol.epoch_stride;
    const void *recs = vol.rec;
    // Paired float32 records: a sample that reads no snapshot loads the zero
    // record pair after the last block instead of skipping its loads (faster
    // for the 32-byte pairs; for 16-byte pairs it costs registers and time).
    constexpr bool kZeroPair = PAIRED && NCH == 0 && !TOUCH && STORE == GBD_STORE_F32;
    const long long zero_off = static_cast<long long>(vol.M + 1) * es;

    float acc = 0.f, comp = 0.f;
    uint32_t count = 0;
    float cacc[NCH > 0 ? NCH : 1], ccomp[NCH > 0 ? NCH : 1];
#pragma unroll
    for (int c = 0; c < (NCH > 0 ? NCH : 1); ++c) cacc[c] = ccomp[c] = 0.f;

    // ---------------- the march, float32 per cell ----------------
    // Per cell: the nearest face, the chord from the previous exit, the epoch
    // coordinate at the chord midpoint, and one step of the exit axis.  The
    // ray ends past the last time that reaches a snapshot or at a sentinel.
    while (__any_sync(kFull, alive)) {
        long long off[DEPTH];
        long long coff[DEPTH];  // channel offset (vector renders)
        float wgt[DEPTH], dsv[DEPTH];
        bool has_lo[DEPTH], has_hi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            has_lo[d] = false;
            has_hi[d] = false;
            off[d] = kZeroPair ? zero_off : 0;
            coff[d] = 0;
            wgt[d] = 0.f;
            dsv[d] = 0.f;
            if (alive) {
                // The cell is left through the nearest face; ties go to the
                // lowest axis (the zero-length chord that follows adds nothing).
                const bool x0 = ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
                const bool x1 = !x0 && ax[1].sn <= ax[2].sn;
                const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
                const long long u_exit = x0 ? ax[0].un : (x1 ? ax[1].un : ax[2].un);
                const float ds = s_exit - s_cur;
                // epoch coordinate at the chord midpoint: m_bar + w, w in [0, 1)
                const long long um = (u_cur + u_exit) >> 1;
                const int mb = static_cast<int>(um >> 32);
                const uint32_t frac = static_cast<uint32_t>(um);
                const float w = static_cast<float>(frac) * 2.3283064365386963e-10f;
                // -1 <= m_bar <= M - 1 (at u = -1 exactly both weights vanish below)
                const bool inside = static_cast<unsigned>(mb + 1) <= static_cast<unsigned>(Mm1 + 1);
                if (ds > 0.f && inside) {
                    has_lo[d] = mb >= 0;
                    has_hi[d] = (mb < Mm1) && (frac != 0u);
#ifdef GBD_CHECKED
                    if ((has_lo[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb)) ||
                        (has_hi[d] && !check_cell(vol, err_word, kc[0], kc[1], kc[2], mb + 1))) {
                        has_lo[d] = has_hi[d] = false;
                    }
#endif
                    const int sum = ax[0].o + ax[1].o + ax[2].o;
                    // unpaired: snapshot m at block m; paired: snapshots mb and
                    // mb + 1 side by side in block mb + 1
                    if (!kZeroPair || has_lo[d] || has_hi[d])
                        off[d] = PAIRED ? static_cast<long long>(mb + 1) * es + 2LL * sum
                                        : static_cast<long long>(mb) * es + sum;
                    if constexpr (NCH > 0 || TOUCH) coff[d] = static_cast<long long>(mb) * ch.cell_stride + sum;
                    wgt[d] = w;
                    dsv[d] = ds;
                }
                step_exit<SMEM>(ax, x0, x1, ia0, ia1, ia2, du0, du1, du2, tab);
#ifdef GBD_CHECKED
                kc[0] += x0 ? kd0 : 0;
                kc[1] += x1 ? kd1 : 0;
                kc[2] += (!x0 && !x1) ? kd2 : 0;
#endif
                s_cur = s_exit;
                u_cur = u_exit;
                // Past the last time that reaches a snapshot (u < -1: the high
                // word below -1; at u = -1 exactly one more empty step), or out
                // of the box: nothing further along the ray can contribute.
                alive = static_cast<int>(u_exit >> 32) >= -1 && (ax[0].o | ax[1].o | ax[2].o) >= 0;
            }
        }
        typename Rec::T rlo[DEPTH], rhi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            if constexpr (TOUCH) {
                rlo[d] = Rec::zero();
                rhi[d] = Rec::zero();
                if (has_lo[d]) atomicOr(ch.touch + (coff[d] >> 5), 1u << (coff[d] & 31));
                if (has_hi[d]) {
                    const long long i = coff[d] + ch.cell_stride;
                    atomicOr(ch.touch + (i >> 5), 1u << (i & 31));
                }
            } else if (kZeroPair) {
                Rec::load_pair(recs, off[d], rlo[d], rhi[d]);  // the zero pair when it reads no snapshot
            } else if (PAIRED) {
                rlo[d] = Rec::zero();
                rhi[d] = Rec::zero();
                if (has_lo[d] || has_hi[d]) Rec::load_pair(recs, off[d], rlo[d], rhi[d]);
            } else {
                rlo[d] = has_lo[d] ? Rec::load(recs, off[d]) : Rec::zero();
                rhi[d] = has_hi[d] ? Rec::load(recs, off[d] + es) : Rec::zero();
            }
        }
        float clo[DEPTH][NCH > 0 ? NCH : 1], chi[DEPTH][NCH > 0 ? NCH : 1];
        if constexpr (NCH > 0) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d)
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const float *base = ch.chan + c * ch.comp_stride + coff[d];
                    clo[d][c] = has_lo[d] ? __ldg(base) : 0.f;
                    chi[d][c] = has_hi[d] ? __ldg(base + ch.cell_stride) : 0.f;
                }
        }
        if constexpr (NCH == 0) {
            // A snapshot that a sample does not read is a zero record (not
            // loaded, or the zero record beside the first and the last
            // snapshot of a paired layout), whose boosted value is exactly 0,
            // so both are evaluated without a branch.  The compensated sum
            // takes a sample only where it read a snapshot, so a ray's sum
            // does not depend on how long the other lanes of its warp march.
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                float vlo, vhi;
                if constexpr (STORE == GBD_STORE_F32) {
                    // per record (the lone march measured faster this way)
                    vlo = Rec::boosted(rlo[d], bc);
                    vhi = Rec::boosted(rhi[d], bc);
                } else {
                    const float2 vv = Rec::boosted2(rlo[d], rhi[d], bc);
                    vlo = vv.x;
                    vhi = vv.y;
                }
                const float v = fmaf(wgt[d], vhi - vlo, vlo);       // Eq. 8
                const float y = fmaf(v, dsv[d], -comp);             // compensated sum
                const float t = acc + y;
                const bool take = has_lo[d] || has_hi[d];
                comp = take ? (t - acc) - y : comp;
                acc = take ? t : acc;
                count += take ? 1u : 0u;
            }
        } else {
            // vector renders: the Doppler factor of each snapshot serves every channel
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                if (!(has_lo[d] || has_hi[d])) continue;
                const float blo = has_lo[d] ? Rec::boost(rlo[d], bc) : 0.f;
                const float bhi = has_hi[d] ? Rec::boost(rhi[d], bc) : 0.f;
                const float vlo = has_lo[d] ? Rec::emissivity(rlo[d]) * blo : 0.f;
                const float vhi = has_hi[d] ? Rec::emissivity(rhi[d]) * bhi : 0.f;
                const float v = fmaf(wgt[d], vhi - vlo, vlo);
                const float y = fmaf(v, dsv[d], -comp);
                const float t = acc + y;
                comp = (t - acc) - y;
                acc = t;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const float ulo = clo[d][c] * blo, uhi = chi[d][c] * bhi;
                    const float u = fmaf(wgt[d], uhi - ulo, ulo);
                    const float yc = fmaf(u, dsv[d], -ccomp[c]);
                    const float tc = cacc[c] + yc;
                    ccomp[c] = (tc - cacc[c]) - yc;
                    cacc[c] = tc;
                }
                ++count;
            }
        }
    }

    if (in_image && !TOUCH) {
        const long long pix = static_cast<long long>(q) * width + p;
        if (PARTIAL) {
            if (count > 0u) atomicAdd(out_img + pix, acc);
        } else if (accumulate) {
            out_img[pix] += V.prefactor * acc;
            if (cnt_img) cnt_img[pix] += count;
        } else {
            out_img[pix] = V.prefactor * acc;
            if (cnt_img) cnt_img[pix] = count;
        }
        if constexpr (NCH > 0) {
            const long long plane = static_cast<long long>(width) * height;
#pragma unroll
            for (int c = 0; c < NCH; ++c) out_img[(c + 1) * plane + pix] = V.prefactor * cacc[c];
        }
    }
}

// march_group for bfloat16/float16 records, with the float epoch coordinate
// of the bfloat16/float16 march (EpochLine of the reference member) and the
// step without branches.  Member g's coordinate at a chord midpoint is the
// reference member's plus dlf[g] = Delta_g rounded to float.  GD cells are
// traversed per iteration; then each member gathers its records of all GD
// cells before evaluating them, so a member keeps GD loads in flight.
template <bool PAIRED, int G, bool PLAIN, int GD>
__device__ __forceinline__ void march_group_bf16(const VolDev &vol, const ViewDev &V, float win_lo, float win_hi,
                                                 const ViewDev *GV, const long long *dl, const int *dh, int gcnt,
                                                 const RayBox &B, int p, int q, int width, int height, float *out,
                                                 long long img_stride, uint32_t *cnt_img, int *err_word,
                                                 const int32_t *__restrict__ tab)
{
    using Rec = Record<GBD_STORE_BF16_F16U>;
    const bool in_image = (p < width) && (q < height);
    RayState R;
    setup_ray<true>(R, vol, V, B, p, q, in_image, win_lo, win_hi, tab);
    AxisState (&ax)[3] = R.ax;
    bool alive = R.alive;
    float s_cur = R.s_cur;
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const EpochLine L = epoch_line(R, V);
    const int M = vol.M;
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
    const int kd0 = R.kd[0], kd1 = R.kd[1], kd2 = R.kd[2];
#endif

    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;
    bc.plain = PLAIN;
    constexpr unsigned long long kUnit = PAIRED ? 16ull : 8ull;
    const unsigned long long recb = reinterpret_cast<unsigned long long>(vol.rec);
    const long long es_bytes = vol.epoch_stride * 8LL;

    float dlf[G];
    float acc[G];
    uint32_t count[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        dlf[g] = g < gcnt ? fix_to_float(dl[g], 1.0f / kTwo32) : 0.f;
        acc[g] = 0.f;
        count[g] = 0u;
    }

    while (__any_sync(kFull, alive)) {
        float umv[GD], dsv[GD];  // reference member's epoch coordinate at the chord midpoints, chords
        int smv[GD];             // layout offsets of the cells
        bool posv[GD];           // positive chords
#ifdef GBD_CHECKED
        int kcs[GD][3];
#endif
        int mlo = INT_MAX, mhi = INT_MIN;  // the warp's range of reference snapshot indices
#pragma unroll
        for (int d = 0; d < GD; ++d) {
            const bool x0 = alive && ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
            const bool x1 = alive && !x0 && ax[1].sn <= ax[2].sn;
            const bool x2 = alive && !x0 && !x1;
            const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
            dsv[d] = s_exit - s_cur;
            umv[d] = fmaf(L.mkk, s_cur + s_exit, L.c0);
            posv[d] = alive && dsv[d] > 0.f;
            smv[d] = ax[0].o + ax[1].o + ax[2].o;
            const int mref = static_cast<int>(floorf(umv[d]));
            mlo = posv[d] ? min(mlo, mref) : mlo;
            mhi = posv[d] ? max(mhi, mref) : mhi;
#ifdef GBD_CHECKED
            kcs[d][0] = kc[0];
            kcs[d][1] = kc[1];
            kcs[d][2] = kc[2];
            kc[0] += x0 ? kd0 : 0;
            kc[1] += x1 ? kd1 : 0;
            kc[2] += x2 ? kd2 : 0;
#endif
            step_lite<true>(ax, x0, x1, x2, ia0, ia1, ia2, tab);
            s_cur = s_exit;
            alive = alive && s_exit <= L.s_stop && (ax[0].o | ax[1].o | ax[2].o) >= 0;
        }
        mlo = __reduce_min_sync(kFull, mlo);
        mhi = __reduce_max_sync(kFull, mhi);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            // Member g's snapshot index at a midpoint is mref + dh[g] or one
            // more: skip it when no lane of the warp can reach [-1, M - 1].
            if (g >= gcnt || mlo > mhi || static_cast<long long>(mhi) + dh[g] < -2 ||
                static_cast<long long>(mlo) + dh[g] > M - 1)
                continue;
            typename Rec::T rlo[GD], rhi[GD];
            float wg[GD];
            bool tk[GD];
#pragma unroll
            for (int d = 0; d < GD; ++d) {
                const float ug = umv[d] + dlf[g];
                const float fl = floorf(ug);
                const float w = ug - fl;
                const int mb = static_cast<int>(fl);
                const bool take = posv[d] && static_cast<unsigned>(mb + 1) <= static_cast<unsigned>(M);
                bool has_lo = take && mb >= 0;
                bool has_hi = take && mb < M - 1 && w != 0.f;
#ifdef GBD_CHECKED
                if ((has_lo && !check_cell(vol, err_word, kcs[d][0], kcs[d][1], kcs[d][2], mb)) ||
                    (has_hi && !check_cell(vol, err_word, kcs[d][0], kcs[d][1], kcs[d][2], mb + 1)))
                    has_lo = has_hi = false;
#endif
                const unsigned long long pa =
                    recb + static_cast<unsigned long long>(static_cast<long long>(PAIRED ? mb + 1 : mb) * es_bytes) +
                    static_cast<unsigned long long>(static_cast<uint32_t>(smv[d])) * kUnit;
                rlo[d] = Rec::zero();
                rhi[d] = Rec::zero();
                if (PAIRED) {
                    if (has_lo || has_hi) Rec::load_pair_at(pa, rlo[d], rhi[d]);
                } else {
                    if (has_lo) rlo[d] = Rec::load_at(pa);
                    if (has_hi) rhi[d] = Rec::load_at(pa + es_bytes);
                }
                wg[d] = take ? w : 0.f;
                tk[d] = has_lo || has_hi;
            }
#pragma unroll
            for (int d = 0; d < GD; ++d) {
                const float2 vv = PLAIN ? Rec::boosted2_plain(rlo[d], rhi[d], bc) : Rec::boosted2(rlo[d], rhi[d], bc);
                const float v = fmaf(wg[d], vv.y - vv.x, vv.x);  // Eq. 8
                acc[g] = fmaf(v, posv[d] ? dsv[d] : 0.f, acc[g]);
                count[g] += tk[d] ? 1u : 0u;
            }
        }
    }

    if (in_image) {
        const long long pix = static_cast<long long>(q) * width + p;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= gcnt) break;
            out[g * img_stride + pix] = GV[g].prefactor * acc[g];
            if (cnt_img) cnt_img[g * img_stride + pix] = count[g];
        }
    }
}

// march_group for float32 records without branches (the step of
// march_ray_f32), exact epoch coordinate and compensated sums.  Each member's
// arithmetic is that of the branching form, value for value.
template <bool PAIRED, int G>
__device__ __forceinline__ void march_group_f32(const VolDev &vol, const ViewDev &V, float win_lo, float win_hi,
                                                const ViewDev *GV, const long long *dl, const int *dh, int gcnt,
                                                const RayBox &B, int p, int q, int width, int height, float *out,
                                                long long img_stride, uint32_t *cnt_img, int *err_word,
                                                const int32_t *__restrict__ tab)
{
    using Rec = Record<GBD_STORE_F32>;
    const bool in_image = (p < width) && (q < height);
    RayState R;
    setup_ray<true>(R, vol, V, B, p, q, in_image, win_lo, win_hi, tab);
    AxisState (&ax)[3] = R.ax;
    bool alive = R.alive;
    float s_cur = R.s_cur;
    long long u_cur = R.u_cur;
    const float ia0 = V.inv_a[0], ia1 = V.inv_a[1], ia2 = V.inv_a[2];
    const long long du0 = V.du[0], du1 = V.du[1], du2 = V.du[2];
    const int Mm1 = vol.M - 1;
#ifdef GBD_CHECKED
    int (&kc)[3] = R.kc;
    const int kd0 = R.kd[0], kd1 = R.kd[1], kd2 = R.kd[2];
#endif
    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;
    bc.plain = false;
    constexpr unsigned long long kUnit = PAIRED ? 32ull : 16ull;
    const unsigned long long recb = reinterpret_cast<unsigned long long>(vol.rec);
    const long long es_bytes = vol.epoch_stride * 16LL;
    const unsigned long long zero_addr = recb + static_cast<unsigned long long>((vol.M + 1) * es_bytes);

    float acc[G], comp[G];
    uint32_t count[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc[g] = comp[g] = 0.f;
        count[g] = 0u;
    }

    while (__any_sync(kFull, alive)) {
        const bool x0 = alive && ax[0].sn <= ax[1].sn && ax[0].sn <= ax[2].sn;
        const bool x1 = alive && !x0 && ax[1].sn <= ax[2].sn;
        const bool x2 = alive && !x0 && !x1;
        const float s_exit = x0 ? ax[0].sn : (x1 ? ax[1].sn : ax[2].sn);
        const long long u_exit = x0 ? ax[0].un : (x1 ? ax[1].un : ax[2].un);
        const float ds = s_exit - s_cur;
        const long long um = (u_cur + u_exit) >> 1;  // reference epoch coordinate at the chord midpoint
        const bool pos = alive && ds > 0.f;
        const int sm = ax[0].o + ax[1].o + ax[2].o;
        const int mref = static_cast<int>(um >> 32);
        const int mlo = __reduce_min_sync(kFull, pos ? mref : INT_MAX);
        const int mhi = __reduce_max_sync(kFull, pos ? mref : INT_MIN);
#ifdef GBD_CHECKED
        const int kc0 = kc[0], kc1 = kc[1], kc2 = kc[2];
        kc[0] += x0 ? kd0 : 0;
        kc[1] += x1 ? kd1 : 0;
        kc[2] += x2 ? kd2 : 0;
#endif
        step_nb<true>(ax, x0, x1, x2, ia0, ia1, ia2, du0, du1, du2, tab);
        s_cur = s_exit;
        u_cur = u_exit;
        alive = alive && static_cast<int>(u_exit >> 32) >= -1 && (ax[0].o | ax[1].o | ax[2].o) >= 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            // Member g's snapshot index at a midpoint is mref + dh[g] or one
            // more: skip it when no lane of the warp can reach [-1, M - 1].
            if (g >= gcnt || mlo > mhi || static_cast<long long>(mhi) + dh[g] < -2 ||
                static_cast<long long>(mlo) + dh[g] > Mm1)
                continue;
            const long long ug = um + dl[g];
            const int mb = static_cast<int>(ug >> 32);
            const uint32_t frac = static_cast<uint32_t>(ug);
            const float w = static_cast<float>(frac) * 2.3283064365386963e-10f;
            const bool take = pos && static_cast<unsigned>(mb + 1) <= static_cast<unsigned>(Mm1 + 1);
            bool has_lo = take && mb >= 0;
            bool has_hi = take && mb < Mm1 && frac != 0u;
#ifdef GBD_CHECKED
            if ((has_lo && !check_cell(vol, err_word, kc0, kc1, kc2, mb)) ||
                (has_hi && !check_cell(vol, err_word, kc0, kc1, kc2, mb + 1)))
                has_lo = has_hi = false;
#endif
            const unsigned long long a =
                recb + static_cast<unsigned long long>(static_cast<long long>(PAIRED ? mb + 1 : mb) * es_bytes) +
                static_cast<unsigned long long>(static_cast<uint32_t>(sm)) * kUnit;
            typename Rec::T rlo, rhi;
            if (PAIRED) {
                const float4 *ptr = reinterpret_cast<const float4 *>((has_lo || has_hi) ? a : zero_addr);
                rlo = __ldg(ptr);
                rhi = __ldg(ptr + 1);
            } else {
                rlo = has_lo ? __ldg(reinterpret_cast<const float4 *>(a)) : Rec::zero();
                rhi = has_hi ? __ldg(reinterpret_cast<const float4 *>(a + es_bytes)) : Rec::zero();
            }
            const float vlo = Rec::boosted(rlo, bc), vhi = Rec::boosted(rhi, bc);
            const float v = fmaf(w, vhi - vlo, vlo);     // Eq. 8
            const float y = fmaf(v, ds, -comp[g]);       // compensated sum
            const float t = acc[g] + y;
            const bool tk = has_lo || has_hi;
            comp[g] = tk ? (t - acc[g]) - y : comp[g];
            acc[g] = tk ? t : acc[g];
            count[g] += tk ? 1u : 0u;
        }
    }

    if (in_image) {
        const long long pix = static_cast<long long>(q) * width + p;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= gcnt) break;
            out[g * img_stride + pix] = GV[g].prefactor * acc[g];
            if (cnt_img) cnt_img[g * img_stride + pix] = count[g];
        }
    }
}

// Time groups (batched renders).  Views that differ only in observer time
// (and so in window and prefactor) share their rays; one lane marches its ray
// once for up to kGroupMax such views.  The traversal covers the union of the
// members' windows and carries the epoch coordinate of the reference member,
// the one whose window ends last (largest u_obs); member g's coordinate
// differs from it by the exact constant Delta_g = u_obs,g - u_obs,ref <= 0
// (Q31.32), so at a chord midpoint it is um + Delta_g.  Per cell the
// traversal is done once, and every member whose window some lane of the warp
// reaches gathers, boosts and sums its own two snapshots into its own
// compensated sum (Eq. 19 per view).  A member's pixel is summed over the same
// cells, chords and midpoints as when its view is marched alone; the crossings
// are measured from the group's anchor instead of the view's own, so the two
// agree to float rounding, not bit for bit.  Member g's image is at
// out + g * img_stride.
template <int STORE, int DEPTH, bool PAIRED, int G>
__device__ __forceinline__ void march_group(const VolDev &vol, const ViewDev &V, float win_lo, float win_hi,
                                            const ViewDev *GV, const long long *dl, const int *dh, int gcnt,
                                            const RayBox &B, int p, int q, int width, int height, float *out,
                                            long long img_stride, uint32_t *cnt_img, int *err_word,
                                            const int32_t *__restrict__ tab)
{
    if constexpr (STORE == GBD_STORE_F32) {
        march_group_f32<PAIRED, G>(vol, V, win_lo, win_hi, GV, dl, dh, gcnt, B, p, q, width, height, out, img_stride,
                                   cnt_img, err_word, tab);
        return;
    }
    if constexpr (STORE == GBD_STORE_BF16_F16U) {
        if (vol.plain_boost)
            march_group_bf16<PAIRED, G, true, DEPTH>(vol, V, win_lo, win_hi, GV, dl, dh, gcnt, B, p, q, width, height,
                                                     out, img_stride, cnt_img, err_word, tab);
        else
            march_group_bf16<PAIRED, G, false, DEPTH>(vol, V, win_lo, win_hi, GV, dl, dh, gcnt, B, p, q, width, height,
                                                      out, img_stride, cnt_img, err_word, tab);
        return;
    }
}

// MINB = 1 leaves the register count to the compiler; MINB = 3 asks for
// three 256-thread CTAs per SM (at most 80 registers per thread).
//
// Each CTA works on one view, one packet per warp: its tile directly, or,
// persistent, tiles pulled from the view's counter until none are left (with
// STEAL, then from the other views' counters in turn).  The
// CTAs of view v are cta_begin[v] .. cta_begin[v + 1] - 1 (persistent grids
// give each view a share of the GPU in proportion to its estimated work); a
// binary search over these parameter-space bounds keeps the view index
// uniform across the CTA.
template <int STORE, int DEPTH, int MINB, bool PAIRED, bool STEAL>
__global__ void __launch_bounds__(256, MINB) march_kernel(const __grid_constant__ MarchArgs a)
{
    extern __shared__ int32_t s_tab[];
    const int ntab = march_table_entries(a.vol.n);
    stage_tables(s_tab, a.vol.mtab, ntab);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int b = static_cast<int>(blockIdx.x);
    int home = 0, hi = a.n_views - 1;  // last view whose first CTA is <= b
    while (home < hi) {
        const int mid = (home + hi + 1) >> 1;
        if (a.cta_begin[mid] <= b) home = mid;
        else hi = mid - 1;
    }
    const int cb = b - a.cta_begin[home];
    const int tiles = a.tiles_x * a.tiles_y;
    const long long stride = a.img_stride ? a.img_stride : static_cast<long long>(a.width) * a.height;
    if constexpr (STEAL) {
        // Persistent warps take their home view's tiles first, then, once
        // its counter is spent, the other views' tiles in turn, so that no SM
        // idles while any view of the launch has tiles left.  The view index
        // depends on the CTA and the round only, and the exit test is a warp
        // vote, so the view's constants stay warp-uniform.
        const int rounds = a.persistent ? a.n_views : 1;
        for (int r = 0; r < rounds; ++r) {
            const int vi = home + r < a.n_views ? home + r : home + r - a.n_views;
            const ViewDev &V = a.views[vi];
            const RayBox box = grid_box(a.vol, V);
            float *out = a.out + vi * stride;
            uint32_t *cnt = a.samples ? a.samples + vi * stride : nullptr;
            int tile = cb * wpc + warp;
            for (;;) {
                if (a.persistent) {
                    int it = 0;
                    if (lane == 0) it = atomicAdd(a.queue + vi, 1);
                    tile = __shfl_sync(kFull, it, 0);
                }
                if (__any_sync(kFull, tile >= tiles)) break;
                if (a.persistent && a.tile_order) tile = __ldg(a.tile_order + tile);
                const int tx = tile % a.tiles_x;
                const int ty = tile / a.tiles_x;
                const int p = tx * a.packet_w + lane % a.packet_w;
                const int q = ty * a.packet_h + lane / a.packet_w;
                march_ray<STORE, DEPTH, PAIRED, true>(a.vol, V, box, p, q, a.width, a.height, out, cnt,
                                                      a.error_word, s_tab, a.accumulate != 0);
                if (!a.persistent) break;
            }
        }
    } else {
        // one view (or one packet per warp): the home view's tiles only
        const ViewDev &V = a.views[home];
        const RayBox box = grid_box(a.vol, V);
        float *out = a.out + home * stride;
        uint32_t *cnt = a.samples ? a.samples + home * stride : nullptr;
        int tile = cb * wpc + warp;
        for (;;) {
            if (a.persistent) {
                int it = 0;
                if (lane == 0) it = atomicAdd(a.queue + home, 1);
                tile = __shfl_sync(kFull, it, 0);
            }
            if (tile >= tiles) break;
            if (a.persistent && a.tile_order) tile = __ldg(a.tile_order + tile);
            const int p = (tile % a.tiles_x) * a.packet_w + lane % a.packet_w;
            const int q = (tile / a.tiles_x) * a.packet_h + lane / a.packet_w;
            march_ray<STORE, DEPTH, PAIRED, true>(a.vol, V, box, p, q, a.width, a.height, out, cnt, a.error_word,
                                                  s_tab, a.accumulate != 0);
            if (!a.persistent) break;
        }
    }
}

// Time groups: march_kernel's work split over groups of views instead of
// single views (group g is views group_first[g] .. group_first[g + 1] - 1,
// its CTAs cta_begin[g] .. cta_begin[g + 1] - 1, its tile counter queue[g]).
// DEPTH cells per iteration for bfloat16/float16 records (each member
// gathers all of them before evaluating any), one for float32 records, and at
// most 80 registers: with the compiler's budget (110 - 150) fewer warps fit
// and the grouped march ran slower than the lone one.
template <int STORE, int DEPTH, bool PAIRED, int G>
__global__ void __launch_bounds__(256, 3) group_kernel(const __grid_constant__ MarchArgs a)
{
    extern __shared__ int32_t s_tab[];
    const int ntab = march_table_entries(a.vol.n);
    stage_tables(s_tab, a.vol.mtab, ntab);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int b = static_cast<int>(blockIdx.x);
    int home = 0, hi = a.n_groups - 1;  // last group whose first CTA is <= b
    while (home < hi) {
        const int mid = (home + hi + 1) >> 1;
        if (a.cta_begin[mid] <= b) home = mid;
        else hi = mid - 1;
    }
    const int cb = b - a.cta_begin[home];
    const int tiles = a.tiles_x * a.tiles_y;
    const long long stride = a.img_stride ? a.img_stride : static_cast<long long>(a.width) * a.height;
    // home group first, then the other groups' tiles in turn (as march_kernel)
    const int rounds = a.persistent ? a.n_groups : 1;
    for (int r = 0; r < rounds; ++r) {
        const int gi = home + r < a.n_groups ? home + r : home + r - a.n_groups;
        const int first = a.group_first[gi];
        const int gcnt = a.group_first[gi + 1] - first;
        const ViewDev *GV = a.views + first;
        const ViewDev &V = a.views[a.group_ref[gi]];
        const float win_lo = a.group_win[gi][0], win_hi = a.group_win[gi][1];
        const RayBox box = grid_box(a.vol, V);
        float *out = a.out + first * stride;
        uint32_t *cnt = a.samples ? a.samples + first * stride : nullptr;
        int tile = cb * wpc + warp;
        for (;;) {
            if (a.persistent) {
                int it = 0;
                if (lane == 0) it = atomicAdd(a.queue + gi, 1);
                tile = __shfl_sync(kFull, it, 0);
            }
            if (__any_sync(kFull, tile >= tiles)) break;  // uniform across the warp
            if (a.persistent && a.tile_order) tile = __ldg(a.tile_order + tile);
            const int tx = tile % a.tiles_x;
            const int ty = tile / a.tiles_x;
            const int p = tx * a.packet_w + lane % a.packet_w;
            const int q = ty * a.packet_h + lane / a.packet_w;
            march_group<STORE, DEPTH, PAIRED, G>(a.vol, V, win_lo, win_hi, GV, a.view_delta + first,
                                                 a.view_dhi + first, gcnt, box, p, q, a.width, a.height, out, stride,
                                                 cnt, a.error_word, s_tab);
            if (!a.persistent) break;
        }
    }
}

// Vector renders: march_kernel's work split with NCH extra channels summed
// along every ray (depth 2, the compiler's register budget).
template <int STORE, int NCH, bool PAIRED, int MINB>
__global__ void __launch_bounds__(256, MINB) vector_kernel(const __grid_constant__ MarchArgs a)
{
    extern __shared__ int32_t s_tab[];
    const int ntab = march_table_entries(a.vol.n);
    stage_tables(s_tab, a.vol.mtab, ntab);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int b = static_cast<int>(blockIdx.x);
    int home = 0, hi = a.n_views - 1;
    while (home < hi) {
        const int mid = (home + hi + 1) >> 1;
        if (a.cta_begin[mid] <= b) home = mid;
        else hi = mid - 1;
    }
    const int cb = b - a.cta_begin[home];
    const int tiles = a.tiles_x * a.tiles_y;
    const ChanPtrs ch{a.chan, a.chan_comp_stride, a.chan_cell_stride};
    // home view first, then the other views' tiles in turn (as march_kernel)
    const int rounds = a.persistent ? a.n_views : 1;
    for (int r = 0; r < rounds; ++r) {
        const int vi = home + r < a.n_views ? home + r : home + r - a.n_views;
        const ViewDev &V = a.views[vi];
        const RayBox box = grid_box(a.vol, V);
        float *out = a.out + static_cast<long long>(vi) * a.img_stride;
        int tile = cb * wpc + warp;
        for (;;) {
            if (a.persistent) {
                int it = 0;
                if (lane == 0) it = atomicAdd(a.queue + vi, 1);
                tile = __shfl_sync(kFull, it, 0);
            }
            if (__any_sync(kFull, tile >= tiles)) break;  // uniform across the warp
            const int tx = tile % a.tiles_x;
            const int ty = tile / a.tiles_x;
            const int p = tx * a.packet_w + lane % a.packet_w;
            const int q = ty * a.packet_h + lane / a.packet_w;
            march_ray<STORE, 2, PAIRED, true, false, NCH>(a.vol, V, box, p, q, a.width, a.height, out, nullptr,
                                                           a.error_word, s_tab, false, ch);
            if (!a.persistent) break;
        }
    }
}

// Memory analysis: marks every (snapshot, cell) record the views' samples
// read (one packet per warp, no persistent queue).
template <int STORE, bool PAIRED>
__global__ void __launch_bounds__(256, 1) touch_kernel(const __grid_constant__ MarchArgs a, uint32_t *bits,
                                                        long long cells)
{
    extern __shared__ int32_t s_tab[];
    const int ntab = march_table_entries(a.vol.n);
    stage_tables(s_tab, a.vol.mtab, ntab);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int b = static_cast<int>(blockIdx.x);
    int vi = 0, hi = a.n_views - 1;
    while (vi < hi) {
        const int mid = (vi + hi + 1) >> 1;
        if (a.cta_begin[mid] <= b) vi = mid;
        else hi = mid - 1;
    }
    const ViewDev &V = a.views[vi];
    const RayBox box = grid_box(a.vol, V);
    const int tile = (b - a.cta_begin[vi]) * wpc + warp;
    if (tile >= a.tiles_x * a.tiles_y) return;
    const int p = (tile % a.tiles_x) * a.packet_w + lane % a.packet_w;
    const int q = (tile / a.tiles_x) * a.packet_h + lane / a.packet_w;
    float *out = a.out + static_cast<long long>(vi) * a.width * a.height;
    const ChanPtrs ch{nullptr, 0, cells, bits};
    march_ray<STORE, 1, PAIRED, true, false, 0, true>(a.vol, V, box, p, q, a.width, a.height, out, nullptr,
                                                       a.error_word, s_tab, false, ch);
}

// Serving: one launch over the tiles of many requests, each with its own
// volume (float32 or bfloat16/float16 records), view and image.  A CTA finds
// its request by binary search over the requests' first CTAs (uniform across
// the CTA) and stages that request's march tables in shared memory (sized for
// the largest volume of the launch); every ray runs the same march_ray as the
// single-volume kernel, so a request's pixels are the same whether it is
// served alone or in a mix.
template <int DEPTH, int MINB>
__global__ void __launch_bounds__(256, MINB) wave_kernel(const __grid_constant__ WaveArgs a)
{
    extern __shared__ int32_t s_tab[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int b = static_cast<int>(blockIdx.x);
    int lo = 0, hi = a.n_reqs - 1;  // last request whose first CTA is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.reqs[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const ReqDev &R = a.reqs[lo];
    const int ntab = march_table_entries(R.vol.n);
    stage_tables(s_tab, R.vol.mtab, ntab);
    __syncthreads();
    const int tile = (b - R.cta_begin) * wpc + warp;
    if (tile >= R.tiles_x * R.tiles_y) return;
    const int tx = tile % R.tiles_x;
    const int ty = tile / R.tiles_x;
    const int p = tx * a.packet_w + lane % a.packet_w;
    const int q = ty * a.packet_h + lane / a.packet_w;
    const RayBox box = grid_box(R.vol, R.view);
    if (R.vol.store == GBD_STORE_F32) {
        if (R.vol.paired)
            march_ray<GBD_STORE_F32, DEPTH, true, true>(R.vol, R.view, box, p, q, R.width, R.height, R.out, R.samples,
                                                        a.error_word, s_tab);
        else
            march_ray<GBD_STORE_F32, DEPTH, false, true>(R.vol, R.view, box, p, q, R.width, R.height, R.out, R.samples,
                                                         a.error_word, s_tab);
    } else {
        if (R.vol.paired)
            march_ray<GBD_STORE_BF16_F16U, DEPTH, true, true>(R.vol, R.view, box, p, q, R.width, R.height, R.out,
                                                              R.samples, a.error_word, s_tab);
        else
            march_ray<GBD_STORE_BF16_F16U, DEPTH, false, true>(R.vol, R.view, box, p, q, R.width, R.height, R.out,
                                                               R.samples, a.error_word, s_tab);
    }
}

// Region schedule (RegionArgs): CTA (x, y) marches rays of one view through
// region y.  The region's table terms along each axis (forward or reversed,
// as the view needs), followed by two sentinels, are staged in shared memory.
// The view's pixels whose rays can cross the region lie in the projection of
// the region's box; the CTA takes one packet of that rectangle per warp,
// keeps the rays that cross the box, sorts them by the length of their chord
// through it (8 buckets, longest first) and hands them to its warps 32 at a
// time, so that the rays of a warp end at about the same step.  Each ray adds
// its region sum to its partial slot.
// Region r of view vi: its box in the view's march frame (mirrored axes
// mirrored) with the offsets of its staged march tables, its partial slot, and
// the pixels p_lo .. p_lo + pw - 1, q_lo .. q_lo + qh - 1 of the image that
// hold every pixel whose centre projects into the box, with a pixel of margin
// (pw = qh = 0 if none).
struct RegionFrame {
    RayBox B;
    int slot;
    int p_lo, q_lo, pw, qh;
};

__device__ __forceinline__ RegionFrame region_frame(const RegionArgs &a, int vi, int r)
{
    const ViewDev &V = a.views[vi];
    const RegionProj &P = a.proj[vi];
    const int rr[3] = {r % a.nreg[0], (r / a.nreg[0]) % a.nreg[1], r / (a.nreg[0] * a.nreg[1])};
    RegionFrame F;
    F.slot = 0;
    float pc = P.p0, qc = P.q0, hp = 0.f, hq = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int n = a.vol.n[i];
        const int olo = rr[i] * a.region;
        const int ohi = min(olo + a.region, n);
        const bool mirrored = (V.flags & (kFlagMirror0 << i)) != 0u;
        F.B.lo[i] = mirrored ? n - ohi : olo;
        F.B.hi[i] = mirrored ? n - olo : ohi;
        F.B.cur0[i] = 4u * static_cast<uint32_t>(i * (a.region + 2));
        F.slot += mirrored ? a.nreg[i] - 1 - rr[i] : rr[i];
        const float c = 0.5f * static_cast<float>(F.B.lo[i] + F.B.hi[i]);
        const float h = 0.5f * static_cast<float>(F.B.hi[i] - F.B.lo[i]);
        pc = fmaf(P.ip[i], c, pc);
        qc = fmaf(P.iq[i], c, qc);
        hp = fmaf(fabsf(P.ip[i]), h, hp);
        hq = fmaf(fabsf(P.iq[i]), h, hq);
    }
    const int p_lo = max(static_cast<int>(floorf(pc - hp)) - 1, 0);
    const int p_hi = min(static_cast<int>(floorf(pc + hp)) + 1, a.width - 1);
    const int q_lo = max(static_cast<int>(floorf(qc - hq)) - 1, 0);
    const int q_hi = min(static_cast<int>(floorf(qc + hq)) + 1, a.height - 1);
    const bool any = p_hi >= p_lo && q_hi >= q_lo;
    F.p_lo = p_lo;
    F.q_lo = q_lo;
    F.pw = any ? p_hi - p_lo + 1 : 0;
    F.qh = any ? q_hi - q_lo + 1 : 0;
    return F;
}

// Chord classes of the ray lists: class 0 holds the longest chords.
constexpr int kChordClasses = 64;
// Warps per CTA of screen_kernel, and the candidates a warp classifies per
// pass (a byte each in shared memory).
constexpr int kScreenWarps = 8;
constexpr int kScreenBatch = 2048;

// Ray lists of the region schedule, one warp per view and region (view
// fastest): the pixels of the region's projected bounding box whose rays
// cross its box inside the view's window, in a counting sort by chord
// length, so that each warp of region_kernel gets 32 rays of nearly equal
// length.  The float slab test runs against the box grown by 0.01 cells, far
// above its rounding (the exact set-up of the march still decides), so no ray
// that the march would sample is dropped.  No chord in the box is longer than
// the crossing time smax of any one axis, which scales the classes.
// Candidates (the bounding box in row-major order) are taken kScreenBatch at a
// time: classified and counted, then placed; each batch appends its own
// sorted run.  The 32 candidates of a step lie along a row, where the chord
// length changes smoothly: each run of lanes with one class takes its places
// with one shared atomic.  The list has room for every pixel the box can cover (the
// host's bound); were it ever full, the pixels past its end would be dropped
// and bit 1 of the error word set.  The launch also clears the partial slots
// that the region march then writes: each warp a contiguous share, before its
// own listing, so that the stores overlap the listing's arithmetic.
__global__ void __launch_bounds__(32 * kScreenWarps) screen_kernel(const __grid_constant__ RegionArgs a)
{
    __shared__ int s_off_all[kScreenWarps][kChordClasses];
    __shared__ uint8_t s_cls_all[kScreenWarps][kScreenBatch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int regions = a.nreg[0] * a.nreg[1] * a.nreg[2];
    const long long pair = static_cast<long long>(blockIdx.x) * kScreenWarps + warp;
    {
        const long long warps = static_cast<long long>(gridDim.x) * kScreenWarps;
        const long long n4 = a.partial_floats >> 2;  // the slots start 256-byte aligned
        const long long share = (n4 + warps - 1) / warps;
        const long long lo = min(pair * share, n4), hi = min(lo + share, n4);
        float4 *p4 = reinterpret_cast<float4 *>(a.partial);
        for (long long i = lo + lane; i < hi; i += 32) __stcs(p4 + i, make_float4(0.f, 0.f, 0.f, 0.f));
        if (pair == 0 && lane < (a.partial_floats & 3)) a.partial[(n4 << 2) + lane] = 0.f;
    }
    if (pair >= static_cast<long long>(a.n_views) * regions) return;
    const int vi = static_cast<int>(pair % a.n_views), r = static_cast<int>(pair / a.n_views);
    int *s_off = s_off_all[warp];
    uint8_t *s_cls = s_cls_all[warp];
    const ViewDev &V = a.views[vi];
    const RegionProj &P = a.proj[vi];
    const RegionFrame F = region_frame(a, vi, r);
    const int cap = a.ctas_per_view * a.rays_per_cta;
    const int n_pix = F.pw * F.qh;
    const int nc = (n_pix + 31) & ~31;  // the whole warp takes each step
    const float inv_pw = F.pw > 0 ? 1.0f / static_cast<float>(F.pw) : 0.f;
    float lo[3], hi[3], ia[3], g0[3], gu[3], gv[3];
    float smax = 3.0e38f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = static_cast<float>(F.B.lo[k]) - 0.01f;
        hi[k] = static_cast<float>(F.B.hi[k]) + 0.01f;
        ia[k] = V.inv_a[k];
        g0[k] = P.g0f[k];
        gu[k] = P.guf[k];
        gv[k] = P.gvf[k];
        if (ia[k] != 0.f) smax = fminf(smax, (hi[k] - lo[k]) * ia[k]);
    }
    const float cls_scale = static_cast<float>(kChordClasses) / smax;
    const float win_lo = V.win_lo, win_hi = V.win_hi;
    uint32_t *list = a.rays + (static_cast<long long>(r) * a.n_views + vi) * cap;
    const uint32_t below = (1u << lane) - 1u;
    int done = 0;
    for (int base = 0; base < nc; base += kScreenBatch) {
        const int nb = min(nc - base, kScreenBatch);
        s_off[lane] = 0;
        s_off[lane + 32] = 0;
        __syncwarp();
        // classify and count (one leader lane per class updates its count)
        for (int i = lane; i < nb; i += 32) {
            const int j = base + i;  // row-major index in the bounding box
            int qo = static_cast<int>(static_cast<float>(j) * inv_pw);
            int po = j - qo * F.pw;
            if (po < 0) { po += F.pw; --qo; }
            if (po >= F.pw) { po -= F.pw; ++qo; }
            const float p = static_cast<float>(F.p_lo + po), q = static_cast<float>(F.q_lo + qo);
            bool hit = j < n_pix;
            float s_lo = win_lo, s_hi = win_hi;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float g = fmaf(q, gv[k], fmaf(p, gu[k], g0[k]));
                if (ia[k] != 0.f) {
                    s_lo = fmaxf(s_lo, (lo[k] - g) * ia[k]);
                    s_hi = fminf(s_hi, (hi[k] - g) * ia[k]);
                } else {
                    hit = hit && g >= lo[k] && g < hi[k];
                }
            }
            hit = hit && s_hi > s_lo - 1e-3f * (1.f + fabsf(s_lo));
            const float f = fminf(fmaxf((s_hi - s_lo) * cls_scale, 0.f), static_cast<float>(kChordClasses - 1));
            const int c = hit ? kChordClasses - 1 - static_cast<int>(f) : kChordClasses;
            s_cls[i] = static_cast<uint8_t>(c);
            const int c_prev = __shfl_up_sync(kFull, c, 1);  // every lane takes part
            const bool head = lane == 0 || c != c_prev;
            const uint32_t heads = __ballot_sync(kFull, head);
            if (head && c < kChordClasses) {
                const uint32_t after = heads & ~below & ~(1u << lane);
                atomicAdd(&s_off[c], (after ? __ffs(after) - 1 : 32) - lane);
            }
        }
        __syncwarp();
        // exclusive prefix sum over the classes, two per lane
        const int c0 = s_off[2 * lane], c1 = s_off[2 * lane + 1];
        int incl = c0 + c1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d);
            incl += lane >= d ? v : 0;
        }
        const int excl = done + incl - c0 - c1;
        __syncwarp();
        s_off[2 * lane] = excl;
        s_off[2 * lane + 1] = excl + c0;
        __syncwarp();
        // place
        for (int i = lane; i < nb; i += 32) {
            const int c = s_cls[i];
            const int c_prev = __shfl_up_sync(kFull, c, 1);  // every lane takes part
            const bool head = lane == 0 || c != c_prev;
            const uint32_t heads = __ballot_sync(kFull, head);
            int pos = 0;
            if (head && c < kChordClasses) {
                const uint32_t after = heads & ~below & ~(1u << lane);
                pos = atomicAdd(&s_off[c], (after ? __ffs(after) - 1 : 32) - lane);
            }
            const int lead = 31 - __clz(heads & (below | (1u << lane)));
            pos = __shfl_sync(kFull, pos, lead) + lane - lead;
            if (c < kChordClasses) {
                const int j = base + i;
                int qo = static_cast<int>(static_cast<float>(j) * inv_pw);
                int po = j - qo * F.pw;
                if (po < 0) { po += F.pw; --qo; }
                if (po >= F.pw) { po -= F.pw; ++qo; }
                if (pos < cap)
                    list[pos] = static_cast<uint32_t>(F.p_lo + po) | (static_cast<uint32_t>(F.q_lo + qo) << 16);
                else if (a.error_word)
                    atomicOr(a.error_word, 2);
            }
        }
        done += __shfl_sync(kFull, incl, 31);
        __syncwarp();  // the counts and classes are reused by the next batch
    }
    if (lane == 0) a.ray_count[r * a.n_views + vi] = min(done, cap);
}

// The march of the region schedule: CTA (blockIdx.x) of the region's
// blockIdx.y-th view (region_order) in region blockIdx.z stages the region's
// march tables and gives each warp the next 32 rays of the view's ray list for
// the region, so that warp w of CTA cb marches entries (cb * warps + w) * 32 ..
// + 31.  CTAs past the end of the list return at once.
template <int STORE, int DEPTH, int MINB, bool PAIRED>
__global__ void __launch_bounds__(256, MINB) region_kernel(const __grid_constant__ RegionArgs a)
{
    extern __shared__ int32_t s_tab[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int r = static_cast<int>(blockIdx.z);
    const int vi = __ldg(a.region_order + static_cast<long long>(r) * a.n_views + blockIdx.y);
    const int count = __ldg(a.ray_count + r * a.n_views + vi);
    const int first = static_cast<int>(blockIdx.x) * a.rays_per_cta;
    if (first >= count) return;
    const ViewDev &V = a.views[vi];
    const RegionFrame F = region_frame(a, vi, r);
    for (int i = 0; i < 3; ++i) {
        const bool mirrored = (V.flags & (kFlagMirror0 << i)) != 0u;
        const int len = F.B.hi[i] - F.B.lo[i];
        const int src = march_table_base(a.vol.n, i) + (mirrored ? a.vol.n[i] + 2 : 0) + F.B.lo[i];
        for (int j = threadIdx.x; j < len + 2; j += blockDim.x)
            s_tab[i * (a.region + 2) + j] = j < len ? a.vol.mtab[src + j] : kTabSentinel;
    }
    if (threadIdx.x < kTabPad) s_tab[3 * (a.region + 2) + threadIdx.x] = kTabSentinel;
    const int k = first + warp * 32 + lane;
    const uint32_t *list = a.rays + (static_cast<long long>(r) * a.n_views + vi) * a.ctas_per_view * a.rays_per_cta;
    const uint32_t pq = k < count ? __ldg(list + k) : (static_cast<uint32_t>(a.width) | (static_cast<uint32_t>(a.height) << 16));
    __syncthreads();  // tables staged
    if (__all_sync(kFull, k >= count)) return;
    float *out = a.partial + static_cast<long long>(F.slot) * a.slot_stride +
                 static_cast<long long>(a.image[vi]) * a.width * a.height;
    march_ray<STORE, DEPTH, PAIRED, true, true>(a.vol, V, F.B, static_cast<int>(pq & 0xffffu), static_cast<int>(pq >> 16),
                                                a.width, a.height, out, nullptr, a.error_word, s_tab);
}

// One view per blockIdx.y.
__global__ void __launch_bounds__(256) reduce_kernel(const __grid_constant__ ReduceArgs a)
{
    const int v = static_cast<int>(blockIdx.y);
    const long long img = static_cast<long long>(a.image[v]) * a.pix_per_view;
    const float pre = a.prefactor[v];
    for (long long px = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; px < a.pix_per_view;
         px += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = img + px;
        float acc = 0.f, comp = 0.f;
        for (int s = 0; s < a.n_slots; ++s) {
            const float y = a.partial[static_cast<long long>(s) * a.slot_stride + i] - comp;
            const float t = acc + y;
            comp = (t - acc) - y;
            acc = t;
        }
        a.out[i] = pre * acc;
    }
}

template <int STORE, int DEPTH, int MINB, bool PAIRED>
void *kernel_ptr(bool steal)
{
    return steal ? reinterpret_cast<void *>(&march_kernel<STORE, DEPTH, MINB, PAIRED, true>)
                 : reinterpret_cast<void *>(&march_kernel<STORE, DEPTH, MINB, PAIRED, false>);
}

template <int STORE, int MINB, bool PAIRED>
void *select_depth(int depth, bool steal)
{
    switch (depth) {
    case 1: return kernel_ptr<STORE, 1, MINB, PAIRED>(steal);
    case 2: return kernel_ptr<STORE, 2, MINB, PAIRED>(steal);
    case 4: return kernel_ptr<STORE, 4, MINB, PAIRED>(steal);
    default: return nullptr;
    }
}

template <int STORE, bool PAIRED>
void *select_cap(int depth, int capped, bool steal)
{
    return capped ? select_depth<STORE, 3, PAIRED>(depth, steal) : select_depth<STORE, 1, PAIRED>(depth, steal);
}

template <int STORE, bool PAIRED, int DEPTH>
void *select_group_depth(int size)
{
    if (size == 4) return reinterpret_cast<void *>(&group_kernel<STORE, DEPTH, PAIRED, 4>);
    if (size == kGroupMax) return reinterpret_cast<void *>(&group_kernel<STORE, DEPTH, PAIRED, kGroupMax>);
    return nullptr;
}

template <int STORE, bool PAIRED>
void *select_group_size(int size, int depth)
{
    // float32 groups march one cell per iteration whatever the depth: with two
    // or four, the extra record registers cost more warps than the loads gain
    if constexpr (STORE == GBD_STORE_F32) {
        return (depth == 1 || depth == 2 || depth == 4) ? select_group_depth<STORE, PAIRED, 1>(size) : nullptr;
    } else {
        switch (depth) {
        case 1: return select_group_depth<STORE, PAIRED, 1>(size);
        case 2: return select_group_depth<STORE, PAIRED, 2>(size);
        case 4: return select_group_depth<STORE, PAIRED, 4>(size);
        default: return nullptr;
        }
    }
}

// Time groups: a kernel for groups of up to 4 views and one for up to 8.
void *select_group(int store, int paired, int size, int depth)
{
    if (store == GBD_STORE_F32)
        return paired ? select_group_size<GBD_STORE_F32, true>(size, depth)
                      : select_group_size<GBD_STORE_F32, false>(size, depth);
    if (store == GBD_STORE_BF16_F16U)
        return paired ? select_group_size<GBD_STORE_BF16_F16U, true>(size, depth)
                      : select_group_size<GBD_STORE_BF16_F16U, false>(size, depth);
    return nullptr;
}

// steal: persistent CTAs move on to the other views' tiles once their own
// view's are spent (launches of more than one view).
void *select_kernel(int store, int depth, int capped, int paired, bool steal)
{
    if (store == GBD_STORE_F32)
        return paired ? select_cap<GBD_STORE_F32, true>(depth, capped, steal)
                      : select_cap<GBD_STORE_F32, false>(depth, capped, steal);
    if (store == GBD_STORE_BF16_F16U)
        return paired ? select_cap<GBD_STORE_BF16_F16U, true>(depth, capped, steal)
                      : select_cap<GBD_STORE_BF16_F16U, false>(depth, capped, steal);
    return nullptr;
}

template <int STORE, int MINB, bool PAIRED>
void *select_region_depth(int depth)
{
    switch (depth) {
    case 1: return reinterpret_cast<void *>(&region_kernel<STORE, 1, MINB, PAIRED>);
    case 2: return reinterpret_cast<void *>(&region_kernel<STORE, 2, MINB, PAIRED>);
    default: return nullptr;
    }
}

void *select_region(int store, int depth, int capped, int paired)
{
    if (store == GBD_STORE_F32) {
        if (paired) return capped ? select_region_depth<GBD_STORE_F32, 3, true>(depth)
                                  : select_region_depth<GBD_STORE_F32, 1, true>(depth);
        return capped ? select_region_depth<GBD_STORE_F32, 3, false>(depth)
                      : select_region_depth<GBD_STORE_F32, 1, false>(depth);
    }
    if (store == GBD_STORE_BF16_F16U) {
        if (paired) return capped ? select_region_depth<GBD_STORE_BF16_F16U, 3, true>(depth)
                                  : select_region_depth<GBD_STORE_BF16_F16U, 1, true>(depth);
        return capped ? select_region_depth<GBD_STORE_BF16_F16U, 3, false>(depth)
                      : select_region_depth<GBD_STORE_BF16_F16U, 1, false>(depth);
    }
    return nullptr;
}

template <int NCH, int MINB>
void *select_vector_store(int store, int paired)
{
    if (store == GBD_STORE_F32)
        return paired ? reinterpret_cast<void *>(&vector_kernel<GBD_STORE_F32, NCH, true, MINB>)
                      : reinterpret_cast<void *>(&vector_kernel<GBD_STORE_F32, NCH, false, MINB>);
    if (store == GBD_STORE_BF16_F16U)
        return paired ? reinterpret_cast<void *>(&vector_kernel<GBD_STORE_BF16_F16U, NCH, true, MINB>)
                      : reinterpret_cast<void *>(&vector_kernel<GBD_STORE_BF16_F16U, NCH, false, MINB>);
    return nullptr;
}



void *select_wave(int depth, int capped)
{
    if (depth == 1) return capped ? reinterpret_cast<void *>(&wave_kernel<1, 3>) : reinterpret_cast<void *>(&wave_kernel<1, 1>);
    if (depth == 2) return capped ? reinterpret_cast<void *>(&wave_kernel<2, 3>) : reinterpret_cast<void *>(&wave_kernel<2, 1>);
    return nullptr;
}

}  // namespace

cudaError_t launch_wave(const WaveArgs &a, const LaunchCfg &cfg, cudaStream_t stream)
{
    void *k = select_wave(cfg.depth, cfg.regcap);
    if (!k) return cudaErrorInvalidValue;
    if (a.total_ctas < 1) return cudaSuccess;
    // shared memory for the largest march tables of the launch
    int smem = 0;
    for (int r = 0; r < a.n_reqs; ++r)
        smem = std::max(smem, static_cast<int>(sizeof(int32_t)) * (march_table_entries(a.reqs[r].vol.n) + kTabPad));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    void *params[] = {const_cast<WaveArgs *>(&a)};
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(a.total_ctas)), dim3(32 * cfg.cta_warps), params, smem,
                            stream);
}

cudaError_t launch_vector(MarchArgs &a, int n_chan, const LaunchCfg &cfg, int num_sms, const double *work,
                          cudaStream_t stream)
{
    // the compiler's register budget: capped, the three-channel kernel spills
    // and runs slower than the extra resident warps gain
    void *k = n_chan == 1 ? select_vector_store<1, 1>(a.vol.store, a.vol.paired)
                          : (n_chan == 3 ? select_vector_store<3, 1>(a.vol.store, a.vol.paired) : nullptr);
    if (!k) return cudaErrorInvalidValue;
    // grid as planned for the scalar kernel of the same budget
    LaunchCfg c = cfg;
    c.depth = 2;
    c.regcap = 0;
    KernelLaunch L;
    cudaError_t e = plan_march(a, c, num_sms, work, L);
    if (e != cudaSuccess) return e;
    if (L.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
        if (e != cudaSuccess) return e;
    }
    void *params[] = {&a};
    return cudaLaunchKernel(k, L.grid, L.block, params, L.smem, stream);
}

cudaError_t launch_touch(MarchArgs &a, uint32_t *bits, long long cells, const LaunchCfg &cfg, int num_sms,
                         cudaStream_t stream)
{
    void *k = a.vol.store == GBD_STORE_F32
                  ? (a.vol.paired ? reinterpret_cast<void *>(&touch_kernel<GBD_STORE_F32, true>)
                                  : reinterpret_cast<void *>(&touch_kernel<GBD_STORE_F32, false>))
                  : (a.vol.paired ? reinterpret_cast<void *>(&touch_kernel<GBD_STORE_BF16_F16U, true>)
                                  : reinterpret_cast<void *>(&touch_kernel<GBD_STORE_BF16_F16U, false>));
    // one packet per warp: the grid covers every tile
    a.persistent = 0;
    KernelLaunch L;
    cudaError_t e = plan_march(a, cfg, num_sms, nullptr, L);
    if (e != cudaSuccess) return e;
    if (L.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
        if (e != cudaSuccess) return e;
    }
    void *params[] = {&a, &bits, &cells};
    return cudaLaunchKernel(k, L.grid, L.block, params, L.smem, stream);
}

cudaError_t launch_screen(const RegionArgs &a, cudaStream_t stream)
{
    const long long regions = static_cast<long long>(a.nreg[0]) * a.nreg[1] * a.nreg[2];
    if (a.n_views < 1 || a.n_views > 65535 || !a.rays || !a.ray_count || !a.views || !a.proj || a.rays_per_cta < 32 ||
        a.ctas_per_view < 1 || regions < 1 || regions > 65535 || a.partial_floats < 0 ||
        (a.partial_floats > 0 && !a.partial))
        return cudaErrorInvalidValue;
    const long long ctas = (a.n_views * regions + kScreenWarps - 1) / kScreenWarps;
    void *params[] = {const_cast<RegionArgs *>(&a)};
    return cudaLaunchKernel(reinterpret_cast<void *>(&screen_kernel), dim3(static_cast<unsigned>(ctas)),
                            dim3(32 * kScreenWarps), params, 0, stream);
}

cudaError_t launch_region(const RegionArgs &a, const LaunchCfg &cfg, cudaStream_t stream)
{
    void *k = select_region(a.vol.store, cfg.depth, cfg.regcap, a.vol.paired);
    const long long regions = static_cast<long long>(a.nreg[0]) * a.nreg[1] * a.nreg[2];
    if (!k || a.n_views < 1 || a.n_views > 65535 || regions < 1 || regions > 65535 || a.ctas_per_view < 1 ||
        a.rays_per_cta != 32 * cfg.cta_warps || !a.image || !a.region_order)
        return cudaErrorInvalidValue;
    const int smem = static_cast<int>(sizeof(int32_t)) * (3 * (a.region + 2) + kTabPad);
    void *params[] = {const_cast<RegionArgs *>(&a)};
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(a.ctas_per_view), static_cast<unsigned>(a.n_views),
                                    static_cast<unsigned>(regions)),
                            dim3(32 * cfg.cta_warps), params, smem, stream);
}

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t stream)
{
    if (a.n_views < 1 || a.pix_per_view < 1) return cudaSuccess;
    if (a.n_views > kImagesPerReduce) return cudaErrorInvalidValue;
    const long long per_view = std::max<long long>(1, 152LL * 16 / a.n_views);
    const long long blocks = std::min<long long>((a.pix_per_view + 255) / 256, per_view);
    void *params[] = {const_cast<ReduceArgs *>(&a)};
    return cudaLaunchKernel(reinterpret_cast<void *>(&reduce_kernel),
                            dim3(static_cast<unsigned>(blocks), static_cast<unsigned>(a.n_views)), dim3(256), params,
                            0, stream);
}

cudaError_t plan_march(MarchArgs &a, const LaunchCfg &cfg, int num_sms, const double *work, KernelLaunch &L)
{
    // n_groups > 0: time groups, one unit of CTAs per group; else one per view
    const bool grouped = a.n_groups > 0;
    void *k = grouped ? select_group(a.vol.store, a.vol.paired, a.group_size, cfg.depth)
                      : select_kernel(a.vol.store, cfg.depth, cfg.regcap, a.vol.paired,
                                      a.persistent && a.n_views > 1);
    if (!k || a.n_views < 1 || a.n_views > kViewsPerLaunch) return cudaErrorInvalidValue;
    if (grouped && (a.n_groups > a.n_views || a.group_first[0] != 0 || a.group_first[a.n_groups] != a.n_views))
        return cudaErrorInvalidValue;
    const int units = grouped ? a.n_groups : a.n_views;
    double uwork[kViewsPerLaunch];
    for (int u = 0; u < units; ++u) {
        uwork[u] = 0.0;
        const int v0 = grouped ? a.group_first[u] : u, v1 = grouped ? a.group_first[u + 1] : u + 1;
        if (grouped && (v1 <= v0 || v1 - v0 > a.group_size || a.group_ref[u] < v0 || a.group_ref[u] >= v1))
            return cudaErrorInvalidValue;
        for (int v = v0; v < v1; ++v) uwork[u] += work ? std::max(work[v], 0.0) : 1.0;
    }
    const int threads = 32 * cfg.cta_warps;
    const int smem = static_cast<int>(sizeof(int32_t)) * (march_table_entries(a.vol.n) + kTabPad);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const long long tiles = static_cast<long long>(a.tiles_x) * a.tiles_y;
    const long long needed = (tiles + cfg.cta_warps - 1) / cfg.cta_warps;
    long long total = 0;
    if (a.persistent) {
        // enough CTAs to fill the GPU once, shared out over the views in
        // proportion to their estimated work (at least one CTA each)
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const long long resident = static_cast<long long>(per_sm) * num_sms;
        double sum = 0.0;
        for (int u = 0; u < units; ++u) sum += uwork[u];
        for (int u = 0; u < units; ++u) {
            const double share = sum > 0.0 ? uwork[u] / sum : 1.0 / units;
            const long long c = std::min(needed, std::max(1LL, static_cast<long long>(share * resident + 0.5)));
            a.cta_begin[u] = static_cast<int>(total);
            total += c;
        }
    } else {
        for (int u = 0; u < units; ++u) {
            a.cta_begin[u] = static_cast<int>(total);
            total += needed;
        }
    }
    if (total < 1 || total > 0x7fffffffLL) return cudaErrorInvalidValue;
    a.cta_begin[units] = static_cast<int>(total);
    L.func = k;
    L.grid = dim3(static_cast<unsigned>(total));
    L.block = dim3(threads);
    L.smem = smem;
    return cudaSuccess;
}

cudaError_t launch_march(MarchArgs &a, const LaunchCfg &cfg, int num_sms, const double *work, cudaStream_t stream)
{
    KernelLaunch L;
    cudaError_t e = plan_march(a, cfg, num_sms, work, L);
    if (e != cudaSuccess) return e;
    void *params[] = {&a};
    return cudaLaunchKernel(L.func, L.grid, L.block, params, L.smem, stream);
}

}  // namespace gbd
