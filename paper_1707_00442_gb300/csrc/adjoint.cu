// adjoint.cu -- reverse-mode gradient of the compositing render (Algorithm 3 in
// premultiplied form) with respect to the voxels, the 256-entry colour map and the
// opacity scale.
//
// Forward recurrence per ray (k = 0..K-1, K = samples processed):
//   a_k = clamp(s * A_lut(v_hat_k), 0, 1),  C += T_k a_k c_k,  T_{k+1} = T_k (1 - a_k),
//   outputs (C, 1 - T_K).
// Reverse, with gT = dL/dT_{k+1} carried from the end (gT = -dL/dalpha at k = K):
//   dL/da_k   = sum_c gC_c T_k c_k,c  - gT T_k
//   dL/dc_k   = gC T_k a_k
//   dL/dT_k   = gT (1 - a_k) + sum_c gC_c a_k c_k,c
// The transmittance T_k is not stored per sample: the forward kept it every
// `ckpt_interval` samples, and each segment is recomputed from its checkpoint
// into a per-thread array before being walked backwards (memory O(K / interval)
// per ray instead of O(K)).  Clamp kinks pass the gradient on the closed interval.
#include "common.cuh"
#include "ray.cuh"
#include "render_impl.cuh"
#include "sampler.cuh"

namespace shw {

constexpr int kMaxCkptInterval = 64;
constexpr int kBwdThreads = 256, kBwdTile = 16;  // 16 x 16 pixels per CTA, 8 x 4 per warp

__device__ __forceinline__ void bwd_pixel(int &px, int &py)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = blockIdx.x * kBwdTile + (warp & 1) * 8 + (lane & 7);
    py = blockIdx.y * kBwdTile + (warp >> 1) * 4 + (lane >> 3);
}

struct BackwardArgs {
    const float4 *grad_rgba;  // [H][W]
    const int *ckpt_K;        // [H][W]
    const float *ckpt_T;      // [nckpt][H][W]
    float *grad_vol;          // [nz][ny][nx] or null
    float *grad_lut;          // [256][4] or null
    float *grad_scale;        // [1] or null
    const float4 *lut;
    int width, height, nckpt, ckpt_interval, nmax;
    float step, lo, inv_range, opacity_scale;
};

// Scatter g * (trilinear weight) onto the 8 corners (clamped indices accumulate on the edge voxel).
__device__ __forceinline__ void scatter_trilinear(float *gv, int nx, int ny, int nz, long long X, long long Y,
                                                  long long Z, float g)
{
    const int ix = clampi(fx_cell(X), -1, nx - 1), iy = clampi(fx_cell(Y), -1, ny - 1),
              iz = clampi(fx_cell(Z), -1, nz - 1);
    const float fx = fx_frac(X), fy = fx_frac(Y), fz = fx_frac(Z);
    const int x0 = max(ix, 0), x1 = min(ix + 1, nx - 1);
    const int y0 = max(iy, 0), y1 = min(iy + 1, ny - 1);
    const int z0 = max(iz, 0), z1 = min(iz + 1, nz - 1);
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
    const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
        atomicAdd(gv + ((size_t)zs[d] * sz + (size_t)ys[b] * sy + xs[a]), g * wx[a] * wy[b] * wz[d]);
    }
}

template <int INTERP>
__global__ void __launch_bounds__(kBwdThreads) backward_kernel(SamplerF32<long long> s, shw_camera cam,
                                                                   BackwardArgs a)
{
    __shared__ float4 lut_s[kLut];
    __shared__ float glut_s[kLut * 4];
    __shared__ float gs_s;
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) lut_s[i] = a.lut[i];
    for (int i = threadIdx.x; i < kLut * 4; i += blockDim.x) glut_s[i] = 0.0f;
    if (threadIdx.x == 0) gs_s = 0.0f;
    __syncthreads();

    float gs = 0.0f;
    int px, py;
    bwd_pixel(px, py);
    if (px < a.width && py < a.height) {
        const long long pix = (long long)py * a.width + px;
        const long long npix = (long long)a.width * a.height;
        RayFx r;
        const bool hit = setup_ray(cam, px, py, s.nx, s.ny, s.nz, a.step, r);
        const int K = hit ? min(min(a.ckpt_K[pix], r.N), a.nmax) : 0;
        const float4 g = a.grad_rgba[pix];
        float gT = -g.w;  // alpha_out = 1 - T_K
        const int I = a.ckpt_interval;
        float vseg[kMaxCkptInterval], Tseg[kMaxCkptInterval];
        for (int m = (K - 1) / I; K > 0 && m >= 0; --m) {
            const int k0 = m * I, k1 = min(k0 + I, K);
            // recompute the segment forward from its checkpoint
            float T = (m < a.nckpt) ? a.ckpt_T[(long long)m * npix + pix] : 0.0f;
            for (int j = 0; j < k1 - k0; ++j) {
                const long long X = r.P[0] + (long long)(k0 + j) * r.D[0];
                const long long Y = r.P[1] + (long long)(k0 + j) * r.D[1];
                const long long Z = r.P[2] + (long long)(k0 + j) * r.D[2];
                const float v = fetch<INTERP>(s, X, Y, Z);
                vseg[j] = v;
                Tseg[j] = T;
                const float vv = isnan(v) ? a.lo : v;
                const float4 c = lut_eval(lut_s, normalise(vv, a.lo, a.inv_range));
                const float al = __saturatef(a.opacity_scale * c.w);
                T = T * (1.0f - al);
            }
            // walk it backwards
            for (int j = k1 - k0 - 1; j >= 0; --j) {
                const float v = vseg[j];
                const bool nan = isnan(v);
                const float vv = nan ? a.lo : v;
                const float x = (vv - a.lo) * a.inv_range;
                const float vh = __saturatef(x);
                const float u = vh * 255.0f;
                const int i0 = min(__float2int_rd(u), 254);
                const float f = u - (float)i0;
                const float4 L0 = lut_s[i0], L1 = lut_s[i0 + 1];
                const float4 c = make_float4(lerp(L0.x, L1.x, f), lerp(L0.y, L1.y, f), lerp(L0.z, L1.z, f),
                                             lerp(L0.w, L1.w, f));
                const float alpha = a.opacity_scale * c.w;
                const float al = __saturatef(alpha);
                const float Tk = Tseg[j];
                const float ga = (g.x * c.x + g.y * c.y + g.z * c.z) * Tk - gT * Tk;
                const float wc = Tk * al;
                const float gcr = g.x * wc, gcg = g.y * wc, gcb = g.z * wc;
                gT = gT * (1.0f - al) + al * (g.x * c.x + g.y * c.y + g.z * c.z);
                const float galpha = (alpha >= 0.0f && alpha <= 1.0f) ? ga : 0.0f;
                gs = __fmaf_rn(galpha, c.w, gs);
                const float gca = galpha * a.opacity_scale;
                if (a.grad_lut != nullptr) {
                    const float w0 = 1.0f - f;
                    float *q0 = glut_s + 4 * i0, *q1 = glut_s + 4 * (i0 + 1);
                    atomicAdd(q0 + 0, w0 * gcr);
                    atomicAdd(q0 + 1, w0 * gcg);
                    atomicAdd(q0 + 2, w0 * gcb);
                    atomicAdd(q0 + 3, w0 * gca);
                    atomicAdd(q1 + 0, f * gcr);
                    atomicAdd(q1 + 1, f * gcg);
                    atomicAdd(q1 + 2, f * gcb);
                    atomicAdd(q1 + 3, f * gca);
                }
                if (a.grad_vol != nullptr && !nan) {
                    const float gvh = 255.0f * (gcr * (L1.x - L0.x) + gcg * (L1.y - L0.y) + gcb * (L1.z - L0.z) +
                                                gca * (L1.w - L0.w));
                    const float gv = (x >= 0.0f && x <= 1.0f) ? gvh * a.inv_range : 0.0f;
                    if (gv != 0.0f) {
                        const long long X = r.P[0] + (long long)(k0 + j) * r.D[0];
                        const long long Y = r.P[1] + (long long)(k0 + j) * r.D[1];
                        const long long Z = r.P[2] + (long long)(k0 + j) * r.D[2];
                        if constexpr (INTERP == SHW_NEAREST) {
                            const int xi = clampi(fx_round(X), 0, s.nx - 1), yi = clampi(fx_round(Y), 0, s.ny - 1),
                                      zi = clampi(fx_round(Z), 0, s.nz - 1);
                            atomicAdd(a.grad_vol + ((size_t)zi * s.nx * s.ny + (size_t)yi * s.nx + xi), gv);
                        } else {
                            scatter_trilinear(a.grad_vol, s.nx, s.ny, s.nz, X, Y, Z, gv);
                        }
                    }
                }
            }
        }
    }
    // block reduction of the colour-map and scale gradients: warp shuffles, then one
    // shared atomic per warp, then one global atomic per entry per CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&gs_s, gs);
    __syncthreads();
    if (a.grad_lut != nullptr)
        for (int i = threadIdx.x; i < kLut * 4; i += blockDim.x)
            if (glut_s[i] != 0.0f) atomicAdd(a.grad_lut + i, glut_s[i]);
    if (threadIdx.x == 0 && a.grad_scale != nullptr) atomicAdd(a.grad_scale, gs_s);
}

// from api.cu
bool valid_volume(const shw_volume *v);
bool valid_camera(const shw_camera *c);
bool valid_params(const shw_render_params *p, const shw_volume *v);
long long max_samples(const shw_volume *v, float step);
long long ckpt_count(const shw_volume *v, const shw_render_params *p);

}  // namespace shw

using namespace shw;

extern "C" shw_status shw_render_backward(const shw_volume *vol, const shw_camera *cam, const shw_render_params *p,
                                          const float *grad_rgba, const void *ckpt, size_t ckpt_bytes,
                                          float *grad_vol, float *grad_lut, float *grad_scale, void *stream)
{
    NvtxRange nvtx_range("shw_render_backward");
    if (!valid_volume(vol) || !valid_camera(cam) || !valid_params(p, vol)) return SHW_EINVAL;
    if (p->mode != SHW_COMPOSITE || !grad_rgba || !ckpt || !aligned(grad_rgba, 16) || !aligned(ckpt, 4))
        return SHW_EINVAL;
    if (p->ckpt_interval <= 0) return SHW_EINVAL;
    if (p->ckpt_interval > kMaxCkptInterval) return SHW_EUNSUPPORTED;
    if (vol->storage != SHW_F32) return SHW_EUNSUPPORTED;
    if (p->filter != SHW_FILTER_NONE || p->smooth != SHW_SMOOTH_NONE)
        return SHW_EUNSUPPORTED;  // the adjoint has no filter and no smoothing
    if ((grad_vol && !aligned(grad_vol, 4)) || (grad_lut && !aligned(grad_lut, 4)) ||
        (grad_scale && !aligned(grad_scale, 4)))
        return SHW_EINVAL;
    if (ckpt_bytes < shw_ckpt_bytes(vol, cam, p)) return SHW_ENOMEM;
    const long long npix = (long long)cam->width * cam->height;
    BackwardArgs a{};
    a.grad_rgba = reinterpret_cast<const float4 *>(grad_rgba);
    a.ckpt_K = static_cast<const int *>(ckpt);
    a.ckpt_T = reinterpret_cast<const float *>(static_cast<const char *>(ckpt) + npix * 4);
    a.grad_vol = grad_vol;
    a.grad_lut = grad_lut;
    a.grad_scale = grad_scale;
    a.lut = reinterpret_cast<const float4 *>(p->lut);
    a.width = cam->width;
    a.height = cam->height;
    a.nckpt = (int)ckpt_count(vol, p);
    a.ckpt_interval = p->ckpt_interval;
    a.nmax = (int)max_samples(vol, p->step);
    a.step = p->step;
    a.lo = p->lo;
    a.inv_range = 1.0f / (p->hi - p->lo);
    a.opacity_scale = p->opacity_scale;
    SamplerF32<long long> s{static_cast<const float *>(vol->data), vol->nx, vol->ny, vol->nz, (long long)vol->nx,
                            (long long)vol->nx * vol->ny};
    const dim3 grid((unsigned)ceil_div(cam->width, kBwdTile), (unsigned)ceil_div(cam->height, kBwdTile));
    cudaStream_t st = as_stream(stream);
    if (p->interp == SHW_NEAREST)
        backward_kernel<SHW_NEAREST><<<grid, kBwdThreads, 0, st>>>(s, *cam, a);
    else
        backward_kernel<SHW_TRILINEAR><<<grid, kBwdThreads, 0, st>>>(s, *cam, a);
    return after_launch();
}
