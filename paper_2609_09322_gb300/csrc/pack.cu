// pack.cu -- converts one snapshot epoch from C-ordered input arrays into the
// packed record layout of the march kernels, validating every value.
//
// The method's inputs are the rest-frame emissivity j' and the velocity beta
// of every cell (Sec. 2.5).  Records are written at the per-axis offset sum
// described in gbd_internal.h; padding cells are left as the caller cleared
// them.
//
// GBD_STORE_F32 keeps {j', beta} as float32 (rounded to nearest).
// GBD_STORE_BF16_F16U keeps j' rounded to float32 then to bfloat16, and the
// four-velocity u = Gamma beta computed in float64 with explicitly rounded
// operations (b2 = (bx*bx + by*by) + bz*bz, Gamma = 1/sqrt(1 - b2),
// u_i = beta_i * Gamma) and rounded once to float16, so that the stored value
// is a fixed function of the input.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gbd_internal.h"

namespace gbd {
namespace {

template <typename T>
__device__ __forceinline__ double ld(const T *p, long long i)
{
    return static_cast<double>(p[i]);
}

template <typename TIN>
__global__ void pack_kernel(const PackArgs a)
{
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = static_cast<long long>(nx) * ny * nz;
    const TIN *jin = static_cast<const TIN *>(a.j);
    const TIN *vin = static_cast<const TIN *>(a.vel);
    const int32_t *offx = a.axis_off;
    const int32_t *offy = a.axis_off + nx;
    const int32_t *offz = a.axis_off + nx + ny;
    float g2max = 0.f;  // largest Gamma^2 of this thread's stored bfloat16/float16 records
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < ncell;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ix = static_cast<int>(i % nx);
        const long long r = i / nx;
        const int iy = static_cast<int>(r % ny);
        const int iz = static_cast<int>(r / ny);
        const long long cell = static_cast<long long>(offx[ix]) + offy[iy] + offz[iz];
        // paired blocks: snapshot m is the second record of block m and the
        // first record of block m + 1
        const long long off = a.paired ? static_cast<long long>(a.m) * a.stride + 2 * cell + 1
                                       : static_cast<long long>(a.m) * a.stride + cell;
        const long long off2 = off + a.stride - 1;
        const double j = ld(jin, i);
        const double bx = ld(vin, 3 * i), by = ld(vin, 3 * i + 1), bz = ld(vin, 3 * i + 2);
        bool ok = isfinite(j) && j >= 0.0 && isfinite(bx) && isfinite(by) && isfinite(bz);
        if (a.store == GBD_STORE_F32) {
            const float jf = __double2float_rn(j);
            const float fx = __double2float_rn(bx), fy = __double2float_rn(by), fz = __double2float_rn(bz);
            // |beta| as stored must stay below 1 with room for float32
            // rounding of 1 - beta^2.
            const double b2 = static_cast<double>(fx) * fx + static_cast<double>(fy) * fy + static_cast<double>(fz) * fz;
            ok = ok && isfinite(jf) && b2 <= 1.0 - 1.0 / 1048576.0;
            const float4 rec = ok ? make_float4(jf, fx, fy, fz) : make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4 *>(a.dst)[off] = rec;
            if (a.paired) reinterpret_cast<float4 *>(a.dst)[off2] = rec;
        } else {
            const double b2 = __dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz));
            ok = ok && b2 < 1.0;
            const double g = ok ? __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, -b2))) : 1.0;
            const __half ux = __double2half(__dmul_rn(bx, g));
            const __half uy = __double2half(__dmul_rn(by, g));
            const __half uz = __double2half(__dmul_rn(bz, g));
            const __nv_bfloat16 jb = __float2bfloat16_rn(__double2float_rn(j));
            ok = ok && isfinite(__bfloat162float(jb)) && __hisinf(ux) == 0 && __hisinf(uy) == 0 && __hisinf(uz) == 0;
            uint2 rec;
            rec.x = static_cast<uint32_t>(__bfloat16_as_ushort(jb)) | (static_cast<uint32_t>(__half_as_ushort(ux)) << 16);
            rec.y = static_cast<uint32_t>(__half_as_ushort(uy)) | (static_cast<uint32_t>(__half_as_ushort(uz)) << 16);
            if (!ok) rec = make_uint2(0u, 0u);
            // Gamma^2 of the stored u, as the march computes it from the
            // float16 values
            const float fx = __half2float(ux), fy = __half2float(uy), fz = __half2float(uz);
            if (ok) g2max = fmaxf(g2max, fmaf(fx, fx, fmaf(fy, fy, fmaf(fz, fz, 1.0f))));
            reinterpret_cast<uint2 *>(a.dst)[off] = rec;
            if (a.paired) reinterpret_cast<uint2 *>(a.dst)[off2] = rec;
        }
        if (!ok) atomicExch(a.bad, 1);
    }
    if (a.gamma2_max) {
        // one atomic per warp (non-negative floats order as their bits)
        for (int o = 16; o > 0; o >>= 1) g2max = fmaxf(g2max, __shfl_xor_sync(0xffffffffu, g2max, o));
        if ((threadIdx.x & 31) == 0 && g2max > 0.f) atomicMax(a.gamma2_max, __float_as_uint(g2max));
    }
}

// One epoch of one extra emissivity channel (vector renders): a float per
// cell at the cell's layout offset; any finite value (a channel may be a
// signed component).
template <typename TIN>
__global__ void chan_pack_kernel(const ChanPackArgs a)
{
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = static_cast<long long>(nx) * ny * nz;
    const TIN *in = static_cast<const TIN *>(a.src);
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < ncell;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ix = static_cast<int>(i % nx);
        const long long r = i / nx;
        const int iy = static_cast<int>(r % ny);
        const int iz = static_cast<int>(r / ny);
        const long long cell = static_cast<long long>(a.axis_off[ix]) + a.axis_off[nx + iy] + a.axis_off[nx + ny + iz];
        const float v = __double2float_rn(static_cast<double>(in[i]));
        const bool ok = isfinite(v);
        a.dst[cell] = ok ? v : 0.f;
        if (!ok) atomicExch(a.bad, 1);
    }
}

// Copies every record of one epoch from one layout to another (the tables of
// both layouts have the same n_x + n_y + n_z entries).
template <typename R>
__global__ void relayout_kernel(const RelayoutArgs a)
{
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = static_cast<long long>(nx) * ny * nz;
    const R *src = static_cast<const R *>(a.src);
    R *dst = static_cast<R *>(a.dst);
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < ncell;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ix = static_cast<int>(i % nx);
        const long long r = i / nx;
        const int iy = static_cast<int>(r % ny);
        const int iz = static_cast<int>(r / ny);
        const long long cs = static_cast<long long>(a.src_off[ix]) + a.src_off[nx + iy] + a.src_off[nx + ny + iz];
        const long long cd = static_cast<long long>(a.dst_off[ix]) + a.dst_off[nx + iy] + a.dst_off[nx + ny + iz];
        const long long from = a.src_paired ? static_cast<long long>(a.m) * a.src_stride + 2 * cs + 1
                                            : static_cast<long long>(a.m) * a.src_stride + cs;
        const R v = src[from];
        if (a.dst_paired) {
            dst[static_cast<long long>(a.m) * a.dst_stride + 2 * cd + 1] = v;
            dst[static_cast<long long>(a.m + 1) * a.dst_stride + 2 * cd] = v;
        } else {
            dst[static_cast<long long>(a.m) * a.dst_stride + cd] = v;
        }
    }
}

}  // namespace

cudaError_t launch_relayout(const RelayoutArgs &a, cudaStream_t stream)
{
    const long long ncell = static_cast<long long>(a.n[0]) * a.n[1] * a.n[2];
    long long blocks = (ncell + 255) / 256;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (blocks < 1) return cudaSuccess;
    RelayoutArgs args = a;
    void *params[] = {&args};
    void *k = a.record_bytes == 16 ? reinterpret_cast<void *>(&relayout_kernel<uint4>)
                                   : (a.record_bytes == 8 ? reinterpret_cast<void *>(&relayout_kernel<uint2>)
                                                          : reinterpret_cast<void *>(&relayout_kernel<float>));
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(blocks)), dim3(256), params, 0, stream);
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream)
{
    const long long ncell = static_cast<long long>(a.n[0]) * a.n[1] * a.n[2];
    long long blocks = (ncell + 255) / 256;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (blocks < 1) return cudaSuccess;
    PackArgs args = a;
    void *params[] = {&args};
    void *k = a.dtype_in == GBD_IN_F64 ? reinterpret_cast<void *>(&pack_kernel<double>)
                                       : reinterpret_cast<void *>(&pack_kernel<float>);
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(blocks)), dim3(256), params, 0, stream);
}

cudaError_t launch_chan_pack(const ChanPackArgs &a, cudaStream_t stream)
{
    const long long ncell = static_cast<long long>(a.n[0]) * a.n[1] * a.n[2];
    long long blocks = (ncell + 255) / 256;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (blocks < 1) return cudaSuccess;
    ChanPackArgs args = a;
    void *params[] = {&args};
    void *k = a.dtype_in == GBD_IN_F64 ? reinterpret_cast<void *>(&chan_pack_kernel<double>)
                                       : reinterpret_cast<void *>(&chan_pack_kernel<float>);
    return cudaLaunchKernel(k, dim3(static_cast<unsigned>(blocks)), dim3(256), params, 0, stream);
}

}  // namespace gbd
