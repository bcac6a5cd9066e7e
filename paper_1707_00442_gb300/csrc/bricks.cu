// bricks.cu -- float32 cube -> 32^3 bricks of bfloat16 / binary16 with a 1-voxel
// replicated apron (34^3 stored per brick), rounding to nearest even; batch plans that
// pack their own bricks also take 16^3 bricks (18^3 stored).
//
// The apron holds copies of the neighbouring bricks' border voxels (clamped at
// the cube's faces), so that all 8 corners of any interpolation cell are in one
// brick at fixed offsets, and the marcher needs no edge clamping of corners.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace shw {

template <typename T>
__device__ __forceinline__ unsigned short round_store(float v);
template <>
__device__ __forceinline__ unsigned short round_store<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <>
__device__ __forceinline__ unsigned short round_store<__half>(float v)
{
    return __half_as_ushort(__float2half_rn(v));
}

// One thread per stored element; consecutive threads walk lx, so reads of a
// brick row are contiguous in x and writes are contiguous.  E: the brick edge.
template <typename T, int E>
__global__ void __launch_bounds__(256) pack_kernel(const float *__restrict__ in, unsigned short *__restrict__ out,
                                                   int nx, int ny, int nz, int nbx, int nby, long long total)
{
    constexpr int S = E + 2 * SHW_BRICK_APRON;
    constexpr int kElems = S * S * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long brick = i / kElems;
        const int e = (int)(i - brick * kElems);
        const int lz = e / (S * S), ly = (e / S) % S, lx = e % S;
        const int bx = (int)(brick % nbx), by = (int)((brick / nbx) % nby), bz = (int)(brick / ((long long)nbx * nby));
        const int x = min(max(bx * E + lx - 1, 0), nx - 1);
        const int y = min(max(by * E + ly - 1, 0), ny - 1);
        const int z = min(max(bz * E + lz - 1, 0), nz - 1);
        out[i] = round_store<T>(__ldg(in + ((size_t)z * ny + y) * nx + x));
    }
}

// The pair storages: both cubes of a line ratio rounded into one 32-bit element (low half
// the first cube).  in: the float32 pair buffer.
template <typename T>
__global__ void __launch_bounds__(256) pack_pair_kernel(const float2 *__restrict__ in, unsigned *__restrict__ out,
                                                        int nx, int ny, int nz, int nbx, int nby, long long total)
{
    constexpr int S = kBrickStored;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long brick = i / kBrickElems;
        const int e = (int)(i - brick * kBrickElems);
        const int lz = e / (S * S), ly = (e / S) % S, lx = e % S;
        const int bx = (int)(brick % nbx), by = (int)((brick / nbx) % nby), bz = (int)(brick / ((long long)nbx * nby));
        const int x = min(max(bx * kBrick + lx - 1, 0), nx - 1);
        const int y = min(max(by * kBrick + ly - 1, 0), ny - 1);
        const int z = min(max(bz * kBrick + lz - 1, 0), nz - 1);
        const float2 v = __ldg(in + ((size_t)z * ny + y) * nx + x);
        out[i] = (unsigned)round_store<T>(v.x) | ((unsigned)round_store<T>(v.y) << 16);
    }
}

// Linear 16-bit storages: element v = voxel v, rounded; four voxels per thread and step
// (16-byte loads, 8-byte stores) where the count allows, then the remainder.
template <typename T>
__global__ void __launch_bounds__(256) convert_kernel(const float *__restrict__ in, unsigned short *__restrict__ out,
                                                      long long n, bool vec)
{
    const long long n4 = vec ? n / 4 : 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long i = i0; i < n4; i += stride) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(in) + i);
        ushort4 o;
        o.x = round_store<T>(v.x);
        o.y = round_store<T>(v.y);
        o.z = round_store<T>(v.z);
        o.w = round_store<T>(v.w);
        reinterpret_cast<ushort4 *>(out)[i] = o;
    }
    for (long long i = 4 * n4 + i0; i < n; i += stride) out[i] = round_store<T>(__ldg(in + i));
}

template <typename T>
__global__ void __launch_bounds__(256) convert_pair_kernel(const float2 *__restrict__ in, unsigned *__restrict__ out,
                                                           long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = __ldg(in + i);
        out[i] = (unsigned)round_store<T>(v.x) | ((unsigned)round_store<T>(v.y) << 16);
    }
}

// Bytes of one cube as 16-bit bricks of edge E (16 or 32); 0 for another edge.
size_t bricked_bytes_edge(int nx, int ny, int nz, int edge)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || (edge != 16 && edge != 32)) return 0;
    const size_t s = (size_t)edge + 2 * SHW_BRICK_APRON;
    return (size_t)ceil_div(nx, edge) * ceil_div(ny, edge) * ceil_div(nz, edge) * s * s * s * 2;
}

// Enqueue the rounding of a float32 cube into 16-bit bricks of edge 16 or 32 (storage
// SHW_BF16_BRICK or SHW_F16_BRICK; the layout of shw_pack_bricks with 32 replaced by the
// edge).  out: device, 2-byte aligned, bricked_bytes_edge bytes.  The batch plans' own
// bricks; arguments are checked by the caller.
shw_status pack_bricks_edge(const float *in, int nx, int ny, int nz, int storage, int edge, void *out,
                            cudaStream_t st)
{
    const long long total = (long long)(bricked_bytes_edge(nx, ny, nz, edge) / 2);
    if (total <= 0 || (storage != SHW_BF16_BRICK && storage != SHW_F16_BRICK)) return SHW_EINVAL;
    const int nbx = ceil_div(nx, edge), nby = ceil_div(ny, edge);
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;  // grid-stride beyond 64 CTAs per SM
    auto *o = static_cast<unsigned short *>(out);
    const unsigned g = (unsigned)blocks;
    if (storage == SHW_BF16_BRICK) {
        if (edge == 16)
            pack_kernel<__nv_bfloat16, 16><<<g, 256, 0, st>>>(in, o, nx, ny, nz, nbx, nby, total);
        else
            pack_kernel<__nv_bfloat16, 32><<<g, 256, 0, st>>>(in, o, nx, ny, nz, nbx, nby, total);
    } else {
        if (edge == 16)
            pack_kernel<__half, 16><<<g, 256, 0, st>>>(in, o, nx, ny, nz, nbx, nby, total);
        else
            pack_kernel<__half, 32><<<g, 256, 0, st>>>(in, o, nx, ny, nz, nbx, nby, total);
    }
    return after_launch();
}

}  // namespace shw

using namespace shw;

extern "C" {

size_t shw_bricked_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t storage)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
    const size_t nvox = (size_t)nx * ny * nz;
    if (storage == SHW_BF16 || storage == SHW_F16) return 2 * nvox;
    if (storage == SHW_BF16_PAIR || storage == SHW_F16_PAIR) return 4 * nvox;
    const bool pair = storage == SHW_BF16_PAIR_BRICK || storage == SHW_F16_PAIR_BRICK;
    if (storage != SHW_BF16_BRICK && storage != SHW_F16_BRICK && !pair) return 0;
    const size_t nb = (size_t)ceil_div(nx, kBrick) * ceil_div(ny, kBrick) * ceil_div(nz, kBrick);
    return nb * kBrickElems * (pair ? 4 : 2);
}

shw_status shw_pack_bricks(const float *in, int32_t nx, int32_t ny, int32_t nz, int32_t storage, void *out,
                           size_t out_bytes, void *stream)
{
    NvtxRange nvtx_range("shw_pack_bricks");
    if (!in || !out || nx <= 0 || ny <= 0 || nz <= 0 || !aligned(in, 4) || !aligned(out, 2)) return SHW_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (storage >= SHW_BF16 && storage <= SHW_F16_PAIR) {
        // linear 16-bit storages: a plain element-wise rounding
        const bool lpair = storage >= SHW_BF16_PAIR;
        if (lpair && (!aligned(in, 8) || !aligned(out, 4))) return SHW_EINVAL;
        if (out_bytes < shw_bricked_bytes(nx, ny, nz, storage)) return SHW_ENOMEM;
        const long long n = (long long)nx * ny * nz;
        const bool vec = !lpair && aligned(in, 16) && aligned(out, 8);
        long long blocks = ((vec ? n / 4 + 3 : n) + 255) / 256;
        if (blocks > 152LL * 64) blocks = 152LL * 64;
        if (blocks < 1) blocks = 1;
        if (lpair) {
            const float2 *ip = reinterpret_cast<const float2 *>(in);
            auto *op = static_cast<unsigned *>(out);
            if (storage == SHW_BF16_PAIR)
                convert_pair_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(ip, op, n);
            else
                convert_pair_kernel<__half><<<(unsigned)blocks, 256, 0, st>>>(ip, op, n);
        } else {
            auto *o = static_cast<unsigned short *>(out);
            if (storage == SHW_BF16)
                convert_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(in, o, n, vec);
            else
                convert_kernel<__half><<<(unsigned)blocks, 256, 0, st>>>(in, o, n, vec);
        }
        return after_launch();
    }
    const bool pair = storage == SHW_BF16_PAIR_BRICK || storage == SHW_F16_PAIR_BRICK;
    if (storage != SHW_BF16_BRICK && storage != SHW_F16_BRICK && !pair) return SHW_EINVAL;
    if (pair && (!aligned(in, 8) || !aligned(out, 4))) return SHW_EINVAL;
    const size_t need = shw_bricked_bytes(nx, ny, nz, storage);
    if (out_bytes < need) return SHW_ENOMEM;
    const long long total = (long long)(need / (pair ? 4 : 2));
    const int nbx = ceil_div(nx, kBrick), nby = ceil_div(ny, kBrick);
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;  // grid-stride beyond 64 CTAs per SM
    if (pair) {
        const float2 *ip = reinterpret_cast<const float2 *>(in);
        auto *op = static_cast<unsigned *>(out);
        if (storage == SHW_BF16_PAIR_BRICK)
            pack_pair_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(ip, op, nx, ny, nz, nbx, nby, total);
        else
            pack_pair_kernel<__half><<<(unsigned)blocks, 256, 0, st>>>(ip, op, nx, ny, nz, nbx, nby, total);
        return after_launch();
    }
    return pack_bricks_edge(in, nx, ny, nz, storage, kBrick, out, st);
}

}  // extern "C"
