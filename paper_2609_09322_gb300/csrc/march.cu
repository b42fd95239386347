// march.cu -- sm_103a ray-march kernels for the relativistic line-of-sight sum.
//
// One lane owns one ray (pixel) from entry to exit, so every pixel is summed in
// one fixed order whether it is rendered alone, in a batch or in a served mix.
// A warp owns a packet of 32 neighbouring pixels (8x4 by default), so at each
// step its lanes gather neighbouring cells of the bricked volume.
//
// Per ray (Sec. 2.4 traversal, Sec. 5.1 fast-forward, Eqs. 2, 6-9, 14, 19):
//   * float64, once: pixel centre, slab entry/exit against the grid box, the
//     s-window where the retarded time can reach a stored snapshot, the entry
//     cell, and the epoch coordinate at the window start;
//   * float32 per cell: the next face crossing of each axis recomputed from the
//     integer cell index (never accumulated), the chord ds between the current
//     and next crossing, the epoch coordinate at the chord midpoint, the two
//     snapshot records, the Doppler boost of each, their linear interpolation,
//     and a compensated float32 accumulation of value * ds.
// Cells are gathered DEPTH at a time: the traversal runs ahead, all loads of
// the group are issued, then the group is evaluated, so each lane keeps up to
// 2 * DEPTH independent loads in flight.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

// Per-view float constants held in registers during the march.
struct BoostConsts {
    float shx, shy, shz;  // s_hat rounded to float
    float slx, sly, slz;  // rounding residual of s_hat
    float expo;           // 2 - alpha
    bool beaming;
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
    // D^(2 - alpha) j' with D = sqrt(1 - beta^2) / (1 + beta . s_hat) (Eq. 14).
    // 1 + beta.s_hat and 1 - beta^2 are formed with fused multiply-adds so
    // each is rounded once near its (possibly small) value.
    static __device__ __forceinline__ float boosted(const T r, const BoostConsts &c)
    {
        if (!c.beaming) return r.x;
        float den = fmaf(r.y, c.shx, fmaf(r.z, c.shy, fmaf(r.w, c.shz, 1.0f)));
        den += fmaf(r.y, c.slx, fmaf(r.z, c.sly, r.w * c.slz));
        const float inv_g2 = fmaf(-r.y, r.y, fmaf(-r.z, r.z, fmaf(-r.w, r.w, 1.0f)));
        const float log2_d = fmaf(0.5f, lg2_approx(inv_g2), -lg2_approx(den));
        return r.x * ex2_approx(c.expo * log2_d);
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
    // D = 1 / (Gamma + u.s_hat).  When u.s_hat < 0 (motion towards the
    // observer) the denominator cancels, so the same D is evaluated as
    // (Gamma + |u.s_hat|) / (1 + |u|^2 - (u.s_hat)^2), which has no cancellation.
    static __device__ __forceinline__ float boosted(const T r, const BoostConsts &c)
    {
        const float j = __uint_as_float(r.x << 16);
        if (!c.beaming) return j;
        const float ux = __half2float(__ushort_as_half(static_cast<unsigned short>(r.x >> 16)));
        const float uy = __half2float(__ushort_as_half(static_cast<unsigned short>(r.y & 0xffffu)));
        const float uz = __half2float(__ushort_as_half(static_cast<unsigned short>(r.y >> 16)));
        float us = fmaf(ux, c.shx, fmaf(uy, c.shy, uz * c.shz));
        us += fmaf(ux, c.slx, fmaf(uy, c.sly, uz * c.slz));
        const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float gp = sqrt_approx(1.0f + uu) + fabsf(us);
        const float perp = 1.0f + fmaf(-us, us, uu);
        const float log2_d = (us < 0.f) ? (lg2_approx(gp) - lg2_approx(perp)) : -lg2_approx(gp);
        return j * ex2_approx(c.expo * log2_d);
    }
};

#ifdef GBD_CHECKED
__device__ __forceinline__ bool check_cell(const MarchArgs &a, int ix, int iy, int iz, int m)
{
    const bool ok = ix >= 0 && ix < a.vol.n[0] && iy >= 0 && iy < a.vol.n[1] && iz >= 0 && iz < a.vol.n[2] &&
                    m >= 0 && m < a.vol.M;
    if (!ok && a.error_word) atomicCAS(a.error_word, 0, 1);
    return ok;
}
#endif

// Double-float (hi + lo) arithmetic for the epoch coordinate.  The
// intrinsics are never contracted into fused multiply-adds, which keeps the
// error-free transformations exact.
struct DD {
    float h, l;
};

__device__ __forceinline__ DD two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DD renorm(float h, float l)
{
    const float s = __fadd_rn(h, l);
    return {s, __fsub_rn(l, __fsub_rn(s, h))};
}

// A - B * k for double-float A, B and a small integer k (exact in float).
__device__ __forceinline__ DD dd_sub_mul(DD A, DD B, float k)
{
    const float p = __fmul_rn(B.h, k);
    const float pe = fmaf(B.h, k, -p);  // B.h * k = p + pe exactly
    const DD s = two_sum(A.h, -p);
    const float l = __fadd_rn(s.l, __fsub_rn(__fsub_rn(A.l, pe), __fmul_rn(B.l, k)));
    return renorm(s.h, l);
}

__device__ __forceinline__ DD dd_mid(DD a, DD b)
{
    const DD s = two_sum(a.h, b.h);
    const DD r = renorm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
    return {0.5f * r.h, 0.5f * r.l};
}

__device__ __forceinline__ DD to_dd(double x)
{
    const float h = static_cast<float>(x);
    return {h, static_cast<float>(x - static_cast<double>(h))};
}

template <int STORE, int DEPTH>
__device__ __forceinline__ void march_ray(const MarchArgs &a, const ViewDev &V, int vi, int p, int q,
                                          const int32_t *__restrict__ offx, const int32_t *__restrict__ offy,
                                          const int32_t *__restrict__ offz)
{
    using Rec = Record<STORE>;
    const VolDev &vol = a.vol;
    const bool in_image = (p < a.width) && (q < a.height);
    bool alive = in_image;

    // ---------------- ray setup, float64, once per ray ----------------
    double r0[3], lo[3], hi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r0[i] = fma(static_cast<double>(q), V.dv[i], fma(static_cast<double>(p), V.du[i], V.r00[i]));
        lo[i] = vol.origin[i];
        hi[i] = fma(static_cast<double>(vol.n[i]), vol.dx[i], vol.origin[i]);
    }
    double s_in = -DBL_MAX, s_out = DBL_MAX;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (V.inv_sh[i] != 0.0) {
            const double t1 = (lo[i] - r0[i]) * V.inv_sh[i];
            const double t2 = (hi[i] - r0[i]) * V.inv_sh[i];
            s_in = fmax(s_in, fmin(t1, t2));
            s_out = fmin(s_out, fmax(t1, t2));
        } else if (r0[i] < lo[i] || r0[i] >= hi[i]) {
            alive = false;
        }
    }
    // Fast-forward: the traversal starts in the cell holding the first point
    // whose retarded time can reach a stored snapshot (Sec. 5.1).
    const double s0 = fmax(s_in, V.win_lo);
    if (!(fmin(s_out, V.win_hi) > s0)) alive = false;

    // Epoch coordinate u = (t_bar - t0) / dt = u0 - kk * s_local (Eq. 2).
    const bool lookback = (V.flags & GBD_LOOKBACK) != 0u;
    const double u0 = lookback ? (V.t_obs - s0 * V.inv_c - vol.t0) * vol.inv_dt : static_cast<double>(V.u_fast);
    const double kk = lookback ? V.inv_c * vol.inv_dt : 0.0;

    // Per axis: entry cell index, local origin o (entry point minus the cell's
    // lower corner), and the epoch coordinate at that axis' face planes,
    // u(k) = A - B k for the plane k cells above the entry cell's lower face,
    // evaluated from float64 constants kept as double-floats.
    int idx[3], step[3], base_idx[3], nk[3];
    float o[3], dxf[3], inv_d[3];
    DD A[3], B[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double xe = fma(s0, V.sh[i], r0[i]);
        int k = __double2int_rd((xe - lo[i]) * vol.inv_dx[i]);
        k = min(max(k, 0), vol.n[i] - 1);
        idx[i] = k;
        base_idx[i] = k;
        const double od = alive ? xe - fma(static_cast<double>(k), vol.dx[i], lo[i]) : 0.0;
        o[i] = static_cast<float>(od);
        dxf[i] = static_cast<float>(vol.dx[i]);
        inv_d[i] = V.inv_sh_f[i];
        step[i] = V.sh[i] > 0.0 ? 1 : (V.sh[i] < 0.0 ? -1 : 0);
        nk[i] = step[i] > 0 ? 1 : 0;  // plane of the next crossing
        A[i] = to_dd(alive ? u0 + kk * od * V.inv_sh[i] : 0.0);
        B[i] = to_dd(kk * vol.dx[i] * V.inv_sh[i]);
    }
    // Face crossing of plane k of axis i in the local frame (s from s0),
    // recomputed from the integer index.
    auto crossing = [&](int i, int k_rel) -> float {
        return (static_cast<float>(k_rel) * dxf[i] - o[i]) * inv_d[i];
    };
    float sn[3];
    float s_cur = -FLT_MAX;
    DD u_cur = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        sn[i] = step[i] == 0 ? FLT_MAX : crossing(i, nk[i]);
        if (step[i] != 0) {
            // the entry cell's own entry face: the latest of its three
            const int ek = step[i] > 0 ? 0 : 1;
            const float se = crossing(i, ek);
            if (se > s_cur) {
                s_cur = se;
                u_cur = dd_sub_mul(A[i], B[i], static_cast<float>(ek));
            }
        }
    }
    const float Mf = static_cast<float>(vol.M);
    const int Mm1 = vol.M - 1;

    BoostConsts bc;
    bc.shx = V.sh_hi[0]; bc.shy = V.sh_hi[1]; bc.shz = V.sh_hi[2];
    bc.slx = V.sh_lo[0]; bc.sly = V.sh_lo[1]; bc.slz = V.sh_lo[2];
    bc.expo = V.expo;
    bc.beaming = (V.flags & GBD_BEAMING) != 0u;

    int32_t ox = alive ? offx[idx[0]] : 0;
    int32_t oy = alive ? offy[idx[1]] : 0;
    int32_t oz = alive ? offz[idx[2]] : 0;
    const long long es = vol.epoch_stride;
    const void *recs = vol.rec;

    float acc = 0.f, comp = 0.f;
    uint32_t count = 0;
    // A ray crosses at most n_x + n_y + n_z cells; the budget bounds the loop
    // whatever the floating-point crossings do.
    int steps_left = vol.n[0] + vol.n[1] + vol.n[2] + 4;

    // ---------------- the march, float32 per cell ----------------
    while (__any_sync(kFull, alive)) {
        long long off[DEPTH];
        float wgt[DEPTH], dsv[DEPTH];
        bool has_lo[DEPTH], has_hi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            has_lo[d] = false;
            has_hi[d] = false;
            off[d] = 0;
            wgt[d] = 0.f;
            dsv[d] = 0.f;
            if (alive) {
                // The cell is left through the nearest face; ties go to the
                // lowest axis (the zero-length chord that follows adds nothing).
                const bool x0 = sn[0] <= sn[1] && sn[0] <= sn[2];
                const bool x1 = !x0 && sn[1] <= sn[2];
                const float s_exit = x0 ? sn[0] : (x1 ? sn[1] : sn[2]);
                const int kx = x0 ? nk[0] : (x1 ? nk[1] : nk[2]);
                const DD Ax = x0 ? A[0] : (x1 ? A[1] : A[2]);
                const DD Bx = x0 ? B[0] : (x1 ? B[1] : B[2]);
                const DD u_exit = dd_sub_mul(Ax, Bx, static_cast<float>(kx));
                const float ds = s_exit - s_cur;
                // epoch coordinate at the chord midpoint: m_bar + w, w in [0, 1)
                const DD um = dd_mid(u_cur, u_exit);
                float fm = floorf(um.h);
                float w = (um.h - fm) + um.l;
                if (w >= 1.f) { fm += 1.f; w -= 1.f; }
                if (w < 0.f) { fm -= 1.f; w += 1.f; }
                const bool inside = (fm > -1.f || (fm == -1.f && w > 0.f)) && fm < Mf;
                if (ds > 0.f && inside) {
                    const int mb = static_cast<int>(fm);
                    has_lo[d] = mb >= 0;
                    has_hi[d] = (mb < Mm1) && (w > 0.f);
#ifdef GBD_CHECKED
                    if ((has_lo[d] && !check_cell(a, idx[0], idx[1], idx[2], mb)) ||
                        (has_hi[d] && !check_cell(a, idx[0], idx[1], idx[2], mb + 1))) {
                        has_lo[d] = has_hi[d] = false;
                    }
#endif
                    off[d] = static_cast<long long>(mb) * es + (ox + oy + oz);
                    wgt[d] = w;
                    dsv[d] = ds;
                }
                // Past the last time that reaches a snapshot: nothing further
                // along the ray can contribute.
                if (u_exit.h + u_exit.l <= -1.00001f || --steps_left <= 0) {
                    alive = false;
                } else if (x0) {
                    const int k = idx[0] + step[0];
                    if (step[0] == 0 || k < 0 || k >= vol.n[0]) {
                        alive = false;
                    } else {
                        idx[0] = k;
                        nk[0] += step[0];
                        sn[0] = crossing(0, nk[0]);
                        ox = offx[k];
                    }
                } else if (x1) {
                    const int k = idx[1] + step[1];
                    if (step[1] == 0 || k < 0 || k >= vol.n[1]) {
                        alive = false;
                    } else {
                        idx[1] = k;
                        nk[1] += step[1];
                        sn[1] = crossing(1, nk[1]);
                        oy = offy[k];
                    }
                } else {
                    const int k = idx[2] + step[2];
                    if (step[2] == 0 || k < 0 || k >= vol.n[2]) {
                        alive = false;
                    } else {
                        idx[2] = k;
                        nk[2] += step[2];
                        sn[2] = crossing(2, nk[2]);
                        oz = offz[k];
                    }
                }
                s_cur = s_exit;
                u_cur = u_exit;
            }
        }
        typename Rec::T rlo[DEPTH], rhi[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            rlo[d] = has_lo[d] ? Rec::load(recs, off[d]) : Rec::zero();
            rhi[d] = has_hi[d] ? Rec::load(recs, off[d] + es) : Rec::zero();
        }
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            if (has_lo[d] || has_hi[d]) {
                const float vlo = has_lo[d] ? Rec::boosted(rlo[d], bc) : 0.f;
                const float vhi = has_hi[d] ? Rec::boosted(rhi[d], bc) : 0.f;
                const float v = fmaf(wgt[d], vhi - vlo, vlo);       // Eq. 8
                const float y = fmaf(v, dsv[d], -comp);             // compensated sum
                const float t = acc + y;
                comp = (t - acc) - y;
                acc = t;
                ++count;
            }
        }
    }

    if (in_image) {
        const long long pix = static_cast<long long>(vi) * a.width * a.height + static_cast<long long>(q) * a.width + p;
        a.out[pix] = V.prefactor * acc;
        if (a.samples) a.samples[pix] = count;
    }
}

template <int STORE, int DEPTH>
__global__ void __launch_bounds__(256) march_kernel(const MarchArgs a)
{
    extern __shared__ int32_t s_off[];
    const int nx = a.vol.n[0], ny = a.vol.n[1], nz = a.vol.n[2];
    const int ntab = nx + ny + nz;
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) s_off[i] = a.vol.axis_off[i];
    __syncthreads();
    const int32_t *offx = s_off;
    const int32_t *offy = s_off + nx;
    const int32_t *offz = s_off + nx + ny;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const long long tiles_per_view = static_cast<long long>(a.tiles_x) * a.tiles_y;
    long long item = static_cast<long long>(blockIdx.x) * wpc + warp;
    for (;;) {
        if (a.persistent) {
            int it = 0;
            if (lane == 0) it = atomicAdd(a.queue, 1);
            item = __shfl_sync(kFull, it, 0);
        }
        if (item >= a.total_items) break;
        const int vi = static_cast<int>(item / tiles_per_view);
        const int tile = static_cast<int>(item - static_cast<long long>(vi) * tiles_per_view);
        const int tx = tile % a.tiles_x;
        const int ty = tile / a.tiles_x;
        const int p = tx * a.packet_w + lane % a.packet_w;
        const int q = ty * a.packet_h + lane / a.packet_w;
        march_ray<STORE, DEPTH>(a, a.views[vi], vi, p, q, offx, offy, offz);
        if (!a.persistent) break;
    }
}

template <int STORE, int DEPTH>
void *kernel_ptr()
{
    return reinterpret_cast<void *>(&march_kernel<STORE, DEPTH>);
}

void *select_kernel(int store, int depth)
{
    if (store == GBD_STORE_F32) {
        switch (depth) {
        case 1: return kernel_ptr<GBD_STORE_F32, 1>();
        case 2: return kernel_ptr<GBD_STORE_F32, 2>();
        case 4: return kernel_ptr<GBD_STORE_F32, 4>();
        default: return nullptr;
        }
    }
    if (store == GBD_STORE_BF16_F16U) {
        switch (depth) {
        case 1: return kernel_ptr<GBD_STORE_BF16_F16U, 1>();
        case 2: return kernel_ptr<GBD_STORE_BF16_F16U, 2>();
        case 4: return kernel_ptr<GBD_STORE_BF16_F16U, 4>();
        default: return nullptr;
        }
    }
    return nullptr;
}

}  // namespace

cudaError_t march_occupancy(const LaunchCfg &cfg, int store, int smem_bytes, int *blocks_per_sm)
{
    void *k = select_kernel(store, cfg.depth);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * cfg.cta_warps, smem_bytes);
}

cudaError_t launch_march(const MarchArgs &a, const LaunchCfg &cfg, int num_sms, cudaStream_t stream)
{
    void *k = select_kernel(a.vol.store, cfg.depth);
    if (!k) return cudaErrorInvalidValue;
    const int threads = 32 * cfg.cta_warps;
    const int smem = static_cast<int>(sizeof(int32_t)) * (a.vol.n[0] + a.vol.n[1] + a.vol.n[2]);
    long long blocks;
    if (a.persistent) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        blocks = static_cast<long long>(per_sm) * num_sms;
        const long long needed = (a.total_items + cfg.cta_warps - 1) / cfg.cta_warps;
        if (blocks > needed) blocks = needed;
    } else {
        blocks = (a.total_items + cfg.cta_warps - 1) / cfg.cta_warps;
    }
    if (blocks < 1) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    MarchArgs args = a;
    void *params[] = {&args};
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(blocks)), dim3(threads), params, smem, stream);
}

}  // namespace gbd
