// smooth.cu -- separable 3-D Gaussian smoothing (Section 4.2, Eqs. 5-6) in one pass
// over HBM.
//
// The paper convolves per axis in successive 1-D passes; here the three passes
// are fused so the cube is read once and written once (no intermediate cube,
// no scratch memory).  A CTA owns a 32 x 32 column block of (x, y) and a chunk of
// z planes and streams through z:
//   1. load the (32+2r) x (32+2r) input tile of plane z' into shared memory
//      (clamp-to-edge addressing),
//   2. x-pass into a (32+2r) x 32 shared tile,
//   3. y-pass: each thread produces YB consecutive rows of its column and pushes
//      them into a register ring holding the last 2r+1 planes,
//   4. z-pass from the ring once it is full, written straight to HBM.
// Neighbouring CTAs sweep z in lockstep, so their halo reads hit L2.
#include <cmath>

#include "common.cuh"

namespace shw {

struct SmoothWeights {
    float w[2 * SHW_MAX_SMOOTH_RADIUS + 1];
};

__device__ __forceinline__ int clampi_s(int v, int lo, int hi) { return min(max(v, lo), hi); }

template <int R, int YB>
__global__ void __launch_bounds__(32 * (32 / YB)) smooth_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                                int nx, int ny, int nz, int zchunk, SmoothWeights W)
{
    constexpr int TX = 32, TY = 32, TR = TY / YB, K = 2 * R + 1;
    constexpr int IW = TX + 2 * R, IH = TY + 2 * R;
    __shared__ float s_in[IH][IW];
    __shared__ float s_xp[IH][TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const size_t plane = (size_t)nx * ny;

    float ring[YB][K];
#pragma unroll
    for (int j = 0; j < YB; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) ring[j][k] = 0.0f;

    for (int zz = zb - R; zz < ze + R; ++zz) {
        const float *src = in + (size_t)clampi_s(zz, 0, nz - 1) * plane;
        for (int i = tid; i < IH * IW; i += TR * 32) {
            const int yy = i / IW, xx = i - yy * IW;
            const int gy = clampi_s(y0 - R + yy, 0, ny - 1), gx = clampi_s(x0 - R + xx, 0, nx - 1);
            s_in[yy][xx] = __ldg(src + (size_t)gy * nx + gx);
        }
        __syncthreads();
        for (int yy = ty; yy < IH; yy += TR) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __fmaf_rn(W.w[k], s_in[yy][tx + k], acc);
            s_xp[yy][tx] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < YB; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __fmaf_rn(W.w[k], s_xp[ty * YB + j + k][tx], acc);
#pragma unroll
            for (int k = 0; k < K - 1; ++k) ring[j][k] = ring[j][k + 1];
            ring[j][K - 1] = acc;
        }
        if (zz >= zb + R) {  // the ring holds planes zz-2R .. zz: emit plane zz-R
            const int zo = zz - R, gx = x0 + tx;
#pragma unroll
            for (int j = 0; j < YB; ++j) {
                const int gy = y0 + ty * YB + j;
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < K; ++k) acc = __fmaf_rn(W.w[k], ring[j][k], acc);
                if (gx < nx && gy < ny) out[(size_t)zo * plane + (size_t)gy * nx + gx] = acc;
            }
        }
    }
}

template <int R>
static void launch_smooth_r(const float *in, float *out, int nx, int ny, int nz, const SmoothWeights &w,
                            cudaStream_t st)
{
    constexpr int YB = (R <= 8) ? 4 : 2;
    const int tiles = ceil_div(nx, 32) * ceil_div(ny, 32);
    int zc = nz < 128 ? nz : 128;
    const int zmin = (2 * R > 16) ? 2 * R : 16;
    while ((long long)tiles * ceil_div(nz, zc) < 1216 && zc / 2 >= zmin) zc /= 2;
    const dim3 grid((unsigned)ceil_div(nx, 32), (unsigned)ceil_div(ny, 32), (unsigned)ceil_div(nz, zc));
    const dim3 block(32, 32 / YB);
    smooth_kernel<R, YB><<<grid, block, 0, st>>>(in, out, nx, ny, nz, zc, w);
}

static shw_status smooth_dispatch(const float *in, float *out, int nx, int ny, int nz, const SmoothWeights &w,
                                  int r, cudaStream_t st)
{
    switch (r) {
#define SHW_R(n) \
    case n: launch_smooth_r<n>(in, out, nx, ny, nz, w, st); break;
        SHW_R(0) SHW_R(1) SHW_R(2) SHW_R(3) SHW_R(4) SHW_R(5) SHW_R(6) SHW_R(7) SHW_R(8)
        SHW_R(9) SHW_R(10) SHW_R(11) SHW_R(12) SHW_R(13) SHW_R(14) SHW_R(15) SHW_R(16)
#undef SHW_R
    default: return SHW_EUNSUPPORTED;
    }
    return after_launch();
}

static shw_status smooth_check(const float *in, float *out, int nx, int ny, int nz, int r)
{
    if (!in || !out || nx <= 0 || ny <= 0 || nz <= 0 || r < 0) return SHW_EINVAL;
    if (!aligned(in, 4) || !aligned(out, 4)) return SHW_EINVAL;
    if (r > SHW_MAX_SMOOTH_RADIUS) return SHW_EUNSUPPORTED;
    const size_t bytes = (size_t)nx * ny * nz * 4;
    const char *a = reinterpret_cast<const char *>(in), *b = reinterpret_cast<const char *>(out);
    if (a < b + bytes && b < a + bytes) return SHW_EINVAL;  // in-place or overlapping
    return SHW_OK;
}

}  // namespace shw

using namespace shw;

extern "C" {

shw_status shw_smooth(const float *in, float *out, int32_t nx, int32_t ny, int32_t nz, float sigma, int32_t radius,
                      void *stream)
{
    shw_status s = smooth_check(in, out, nx, ny, nz, radius);
    if (s != SHW_OK) return s;
    if (!std::isfinite(sigma) || !(sigma > 0.0f)) return SHW_EINVAL;
    // Eq. 5 sampled at the integer taps, normalised to unit sum (host, double)
    double w[2 * SHW_MAX_SMOOTH_RADIUS + 1], sum = 0.0;
    for (int k = -radius; k <= radius; ++k) {
        w[k + radius] = std::exp(-(double)k * k / (2.0 * (double)sigma * sigma));
        sum += w[k + radius];
    }
    SmoothWeights W{};
    for (int k = 0; k <= 2 * radius; ++k) W.w[k] = (float)(w[k] / sum);
    return smooth_dispatch(in, out, nx, ny, nz, W, radius, as_stream(stream));
}

shw_status shw_smooth_weights(const float *in, float *out, int32_t nx, int32_t ny, int32_t nz, const float *w_host,
                              int32_t radius, void *stream)
{
    shw_status s = smooth_check(in, out, nx, ny, nz, radius);
    if (s != SHW_OK) return s;
    if (!w_host) return SHW_EINVAL;
    SmoothWeights W{};
    for (int k = 0; k <= 2 * radius; ++k) {
        if (!std::isfinite(w_host[k])) return SHW_EINVAL;
        W.w[k] = w_host[k];
    }
    return smooth_dispatch(in, out, nx, ny, nz, W, radius, as_stream(stream));
}

}  // extern "C"
