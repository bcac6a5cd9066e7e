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
#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace shw {

struct SmoothWeights {
    float w[2 * SHW_MAX_SMOOTH_RADIUS + 1];
    float2 w2[2 * SHW_MAX_SMOOTH_RADIUS + 1];  // (w_k, w_k): the packed FMAs' weight operand
};


__device__ __forceinline__ int clampi_s(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ZIP: out is the interleaved pair buffer, (first[v], smoothed[v]) per voxel.
template <int R, int YB, bool ZIP>
__global__ void __launch_bounds__(32 * (32 / YB)) smooth_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                                int nx, int ny, int nz, int zchunk, SmoothWeights W,
                                                                const float *__restrict__ first)
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
                if (gx < nx && gy < ny) {
                    const size_t o = (size_t)zo * plane + (size_t)gy * nx + gx;
                    if constexpr (ZIP) {
                        out[2 * o] = __ldg(first + o);
                        out[2 * o + 1] = acc;
                    } else {
                        out[o] = acc;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// TMA pipeline (radius 1..8, nx a multiple of 4, 16-byte aligned cube).
//
// Per CTA: a 32 x 32 (x, y) output block and a chunk of z planes.  One thread
// issues cp.async.bulk.tensor loads of the 52 x (32+2r) input box of each plane
// into a 3-stage shared ring, signalled through mbarriers; the box's x start
// (x0 - 8) keeps the TMA coordinate 16-byte aligned.  Out-of-range elements arrive
// as zeros and, in blocks touching the cube's faces, are replaced by the edge values
// (clamp-to-edge).  Then:
//   x-pass: 4(32+2r) threads each make 8 consecutive outputs of a row from at most
//           six float4 reads, as four packed FP32x2 accumulators (__ffma2_rn rounds
//           each lane exactly as a scalar FMA, in the same tap order);
//   y-pass: each thread makes 2 rows x 2 adjacent columns with packed FMAs;
//   z-pass: from a ring of the last 2r+1 y-pass results held in registers, written
//           straight to HBM as float2.  The ring slot of a plane is picked by one
//           switch, so every ring index is a compile-time constant.
// The stage rows are 52 floats apart and the x-pass rows 36: the 16-byte shared
// accesses of eight consecutive threads (two rows) then fall on distinct banks.
constexpr int kSmTX = 32, kSmTY = 32, kSmXP = 8, kSmBW = 52, kSmXPitch = 36, kSmStages = 3, kSmThreads = 256;

// Call f(std::integral_constant<int, v>) for the runtime value v in [0, N) through one
// switch: the callee sees v as a compile-time constant.
template <int N, class F>
__device__ __forceinline__ void static_slot(int v, F &&f)
{
    static_assert(N <= 2 * SHW_MAX_SMOOTH_RADIUS + 1 && N <= 17, "one case per ring slot");
    switch (v) {
#define SHW_SLOT(n)                                                  \
    case n:                                                          \
        if constexpr (n < N) f(std::integral_constant<int, n>{});    \
        break;
        SHW_SLOT(0) SHW_SLOT(1) SHW_SLOT(2) SHW_SLOT(3) SHW_SLOT(4) SHW_SLOT(5) SHW_SLOT(6) SHW_SLOT(7)
        SHW_SLOT(8) SHW_SLOT(9) SHW_SLOT(10) SHW_SLOT(11) SHW_SLOT(12) SHW_SLOT(13) SHW_SLOT(14)
        SHW_SLOT(15) SHW_SLOT(16)
#undef SHW_SLOT
    default:
        break;
    }
}


// Replace the zero-filled out-of-range border of a staged tile by the edge values
// (clamp-to-edge): first the columns outside [c_lo, c_hi], then whole rows outside
// [r_lo, r_hi].  Only the out-of-range elements are touched.
template <int IH>
__device__ __forceinline__ void clamp_tile_edges(float *tile, int c_lo, int c_hi, int r_lo, int r_hi, int tid)
{
    const int nl = c_lo, nr = kSmBW - 1 - c_hi, ncol = nl + nr;
    if (ncol > 0) {
        for (int e = tid; e < IH * ncol; e += kSmThreads) {
            const int r = e / ncol, j = e - r * ncol;
            const int c = j < nl ? j : c_hi + 1 + (j - nl);
            tile[r * kSmBW + c] = tile[r * kSmBW + (j < nl ? c_lo : c_hi)];
        }
        __syncthreads();
    }
    const int nt = r_lo, nb = IH - 1 - r_hi, nrow = nt + nb;
    if (nrow > 0) {
        for (int e = tid; e < nrow * kSmBW; e += kSmThreads) {
            const int j = e / kSmBW, c = e - j * kSmBW;
            const int r = j < nt ? j : r_hi + 1 + (j - nt);
            tile[r * kSmBW + c] = tile[(j < nt ? r_lo : r_hi) * kSmBW + c];
        }
        __syncthreads();
    }
}

// x-pass of eight consecutive outputs: row points at the staged row, (8 q) floats in;
// output 2p + e takes the taps at row[kSmXP - R + 2p + e + k], k = 0..2R, accumulated in
// tap order from +0 (the scalar pass's rounding, two outputs per packed FMA).
template <int R>
__device__ __forceinline__ void xpass8(const float *row, float *dst, const SmoothWeights &W)
{
    constexpr int F0 = (kSmXP - R) / 4, F1 = (kSmXP + 7 + R) / 4, NF = F1 - F0 + 1;
    constexpr int B = kSmXP - R - 4 * F0;  // v index of output 0's first tap
    static_assert(B + 7 + 2 * R < 4 * NF, "the float4 reads cover every tap");
    float v[4 * NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const float4 q = reinterpret_cast<const float4 *>(row)[F0 + f];
        v[4 * f] = q.x;
        v[4 * f + 1] = q.y;
        v[4 * f + 2] = q.z;
        v[4 * f + 3] = q.w;
    }
    float2 acc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[p] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k)
#pragma unroll
        for (int p = 0; p < 4; ++p)
            acc[p] = __ffma2_rn(W.w2[k], make_float2(v[B + 2 * p + k], v[B + 2 * p + k + 1]), acc[p]);
    reinterpret_cast<float4 *>(dst)[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
    reinterpret_cast<float4 *>(dst)[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
}

// resident CTAs per SM each form is compiled for (register budget 65536 / (256 x blocks)):
// the zip form holds the first cube's values of a plane in registers too, and radii above
// 6 hold a longer z ring
template <int R, bool ZIP>
constexpr int smooth_min_blocks()
{
    return (ZIP || R > 6) ? 2 : 3;
}

// floats from one ring stage to the next: the box, rounded up to 128 bytes (TMA destinations)
template <int R>
constexpr int smooth_stage_floats()
{
    return ((kSmTY + 2 * R) * kSmBW + 31) & ~31;
}

template <int R, bool ZIP>
__global__ void __launch_bounds__(kSmThreads, smooth_min_blocks<R, ZIP>())
    smooth_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ out, int nx, int ny, int nz,
                      int zchunk, SmoothWeights W, unsigned *err, const float *__restrict__ first, int skip_plane,
                      int polls)
{
    constexpr int IH = kSmTY + 2 * R, K = 2 * R + 1;
    constexpr int STAGE_FLOATS = smooth_stage_floats<R>();
    constexpr uint32_t STAGE_BYTES = IH * kSmBW * 4;  // what one copy lands
    static_assert(4 * IH <= kSmThreads, "one x-pass unit per thread");
    extern __shared__ __align__(128) float smem[];
    float *s_in = smem;                             // [stages][IH][BW] (stage stride STAGE_FLOATS)
    float *s_xp = smem + kSmStages * STAGE_FLOATS;  // [2][IH][XPitch]
    __shared__ __align__(8) uint64_t bars[kSmStages];

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kSmTX, y0 = blockIdx.y * kSmTY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const int zfirst = zb - R, nplanes = (ze + R) - zfirst;
    const size_t plane = (size_t)nx * ny;

    __shared__ int s_bad;
    if (tid == 0) {
        s_bad = 0;
        for (int s = 0; s < kSmStages; ++s) s_bad |= !tma_dst_ok(s_in + s * STAGE_FLOATS, err);
        for (int s = 0; s < kSmStages; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (s_bad) return;  // reported in the error word; nothing was issued
    if (tid == 0) {
        for (int s = 0; s < kSmStages && s < nplanes; ++s) {
            if (s == skip_plane) continue;  // fault injection: this plane's copy is never issued
            mbar_arrive_expect_tx(&bars[s], STAGE_BYTES);
            tma_load_3d(s_in + s * STAGE_FLOATS, &tmap, x0 - kSmXP, y0 - R, min(max(zfirst + s, 0), nz - 1),
                        &bars[s]);
        }
    }
    // clamp-to-edge bounds inside the tile (columns / rows that hold real data)
    const int c_lo = max(0, kSmXP - x0), c_hi = min(kSmBW - 1, nx - 1 - (x0 - kSmXP));
    const int r_lo = max(0, R - y0), r_hi = min(IH - 1, ny - 1 - (y0 - R));
    const bool edge = c_lo > 0 || c_hi < kSmBW - 1 || r_lo > 0 || r_hi < IH - 1;

    // x-pass unit of this thread: row xr, outputs 8 xq .. 8 xq + 7
    const bool xunit = tid < 4 * IH;
    const int xsrc = (tid >> 2) * kSmBW + 8 * (tid & 3), xdst = (tid >> 2) * kSmXPitch + 8 * (tid & 3);

    // y/z passes: each thread owns columns 2cp, 2cp+1 of rows 2rg, 2rg+1, kept as
    // float2 pairs so that packed FP32x2 FMAs need no operand shuffling
    const int lane = tid & 31, cp = lane & 15, rg = (lane >> 4) + 2 * (tid >> 5);
    const int gx = x0 + 2 * cp, gy = y0 + 2 * rg;
    const bool st0 = gx < nx && gy < ny, st1 = gx < nx && gy + 1 < ny;
    // outputs of plane zb at rows gy, gy + 1 (pair units for the zip form); advanced by a
    // plane per plane written.  ZIP: the first cube's values of the same voxels.
    constexpr int OE = ZIP ? 2 : 1;
    float *op = out + ((size_t)zb * plane + (size_t)gy * nx + gx) * OE;
    const float *fp = ZIP ? first + (size_t)zb * plane + (size_t)gy * nx + gx : nullptr;
    const size_t orow = (size_t)nx * OE;
    float2 ring[2][K];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) ring[j][k] = make_float2(0.0f, 0.0f);

    bool failed = false;
    int fail_i = 0;  // the plane whose wait gave up
    int stage = 0, slot = 0;
    uint32_t phase = 0;
    for (int i = 0; i < nplanes; ++i) {
        // ZIP: this plane's output pairs take the first cube's values; load them now, so
        // the latency hides behind the passes (a lane outside the cube loads nothing)
        float2 fpre[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
        if constexpr (ZIP) {
            if (i >= 2 * R) {
                if (st0) fpre[0] = __ldg(reinterpret_cast<const float2 *>(fp));
                if (st1) fpre[1] = __ldg(reinterpret_cast<const float2 *>(fp + nx));
            }
        }
        const bool ok = mbar_wait(&bars[stage], phase, err, polls);
        float *tile = s_in + stage * STAGE_FLOATS;
        if (edge) clamp_tile_edges<IH>(tile, c_lo, c_hi, r_lo, r_hi, tid);
        float *xp = s_xp + (i & 1) * IH * kSmXPitch;
        if (xunit) xpass8<R>(tile + xsrc, xp + xdst, W);
        if (edge) fence_proxy_async();  // the edge clamp wrote the stage that a tensor copy refills next
        // one barrier per plane: it orders the x pass before the refill and the y pass, and
        // reports a wait that gave up (the x pass then read a stage whose copy may not have
        // landed; nothing of this plane reaches memory outside the CTA)
        if (__syncthreads_or(!ok)) {
            failed = true;
            fail_i = i;
            break;
        }
        // the stage is consumed: refill it with plane i + stages
        if (tid == 0 && i + kSmStages < nplanes) {
            mbar_arrive_expect_tx(&bars[stage], STAGE_BYTES);
            tma_load_3d(tile, &tmap, x0 - kSmXP, y0 - R, min(max(zfirst + i + kSmStages, 0), nz - 1), &bars[stage]);
        }
        if (++stage == kSmStages) {
            stage = 0;
            phase ^= 1u;
        }
        // y-pass of this plane
        const float2 *xp2 = reinterpret_cast<const float2 *>(xp) + rg * kSmXPitch + cp;  // row 2 rg
        float2 col[2 + 2 * R];
#pragma unroll
        for (int m = 0; m < 2 + 2 * R; ++m) col[m] = xp2[m * (kSmXPitch / 2)];
        float2 yv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __ffma2_rn(W.w2[k], col[j + k], acc);
            yv[j] = acc;
        }
        // into the register ring at slot i mod K, then the z-pass: the ring holds planes
        // i-2R .. i (oldest in slot (slot+1) mod K).  Only this part is instanced per slot,
        // so the ring is indexed at compile time.
        const bool emit = i >= 2 * R;
        if constexpr (kChecked)
            if (emit) SHW_CHECK(zfirst + i - R >= zb && zfirst + i - R < ze);  // the plane written
        static_slot<K>(slot, [&](auto sc) {
            constexpr int sl = decltype(sc)::value;
            ring[0][sl] = yv[0];
            ring[1][sl] = yv[1];
            if (emit) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc = __ffma2_rn(W.w2[k], ring[j][(sl + 1 + k) % K], acc);
                    if (j == 0 ? st0 : st1) {
                        float *o = op + j * orow;
                        if constexpr (ZIP) {
                            // (first, smoothed) for the voxels gx and gx + 1: one 16-byte store
                            const float2 f = fpre[j];
                            *reinterpret_cast<float4 *>(o) = make_float4(f.x, acc.x, f.y, acc.y);
                        } else {
                            *reinterpret_cast<float2 *>(o) = acc;
                        }
                    }
                }
            }
        });
        if (++slot == K) slot = 0;
        if (emit) {
            op += plane * OE;
            if constexpr (ZIP) fp += plane;
        }
    }
    if (failed && tid == 0) {
        // drain: wait (bounded) for this CTA's copies still in flight before leaving --
        // planes fail_i .. fail_i + stages - 1 were issued and not consumed
        for (int j = fail_i; j < min(nplanes, fail_i + kSmStages); ++j)
            mbar_wait(&bars[j % kSmStages], (uint32_t)((j / kSmStages) & 1), nullptr,
                      j == skip_plane ? polls : kWaitPolls);  // (a copy that was issued lands well within a second)
    }
}

template <int R>
static size_t smooth_tma_smem()
{
    return (size_t)(kSmStages * smooth_stage_floats<R>() + 2 * (kSmTY + 2 * R) * kSmXPitch) * 4;
}

constexpr int kSmoothMaxChunk = 128;  // largest z chunk of one CTA (planes), without a wave count
static int smooth_zchunk(int nx, int ny, int nz, int r)
{
    const long long tiles = (long long)ceil_div(nx, 32) * ceil_div(ny, 32);
    int zc = nz < kSmoothMaxChunk ? nz : kSmoothMaxChunk;
    const int zmin = (4 * r > 16) ? 4 * r : 16;
    while (tiles * ceil_div(nz, zc) < 608 && zc / 2 >= zmin) zc /= 2;
    return zc;
}

// The TMA kernel's z chunk: each chunk re-reads 2r halo planes, and CTAs run in waves of
// `resident` (CTAs per SM x SMs), so pick the number of chunks that minimises
// waves x (planes per chunk + 2r).  resident <= 0: the plain rule above.
static int smooth_zchunk_waves(int nx, int ny, int nz, int r, long long resident)
{
    if (resident <= 0) return smooth_zchunk(nx, ny, nz, r);
    const long long tiles = (long long)ceil_div(nx, 32) * ceil_div(ny, 32);
    const int zmin = (4 * r > 16) ? 4 * r : 16;
    long long best = -1;
    int best_zc = nz;
    for (int nch = 1; nch <= nz; ++nch) {
        const int zc = ceil_div(nz, nch);
        if (zc < zmin && nch > 1) break;
        const long long ctas = tiles * ceil_div(nz, zc);
        const long long waves = (ctas + resident - 1) / resident;
        const long long cost = waves * (zc + 2LL * r);
        if (best < 0 || cost < best) {
            best = cost;
            best_zc = zc;
        }
    }
    return best_zc;
}

template <int R, bool ZIP>
static bool launch_smooth_tma(const float *in, float *out, int nx, int ny, int nz, const SmoothWeights &w,
                              const float *first, cudaStream_t st)
{
    CUtensorMap map;
    if (!encode_tmap_3d_f32(&map, in, nx, ny, nz, kSmBW, kSmTY + 2 * R)) return false;
    unsigned *err = device_error_word();
    const size_t smem = smooth_tma_smem<R>();
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(smooth_tma_kernel<R, ZIP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static int per_sm = -1;  // resident CTAs per SM of this instance, queried once
    if (per_sm < 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, smooth_tma_kernel<R, ZIP>, kSmThreads, smem) !=
            cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        per_sm = n;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 0;
    }
    const int zc = smooth_zchunk_waves(nx, ny, nz, R, (long long)per_sm * nsm);
    const dim3 grid((unsigned)ceil_div(nx, kSmTX), (unsigned)ceil_div(ny, kSmTY), (unsigned)ceil_div(nz, zc));
    // SHW_DEBUG_FAULT_TIMEOUT: plane 1 of every chunk is never copied, and waits end after about
    // a millisecond (instead of a second), so every CTA's wait runs out quickly
    const bool fault = debug(SHW_DEBUG_FAULT_TIMEOUT);
    smooth_tma_kernel<R, ZIP><<<grid, kSmThreads, smem, st>>>(map, out, nx, ny, nz, zc, w, err, first, fault ? 1 : -1,
                                                              fault ? kFaultWaitPolls : kWaitPolls);
    return true;
}

template <int R, bool ZIP>
static void launch_smooth_r(const float *in, float *out, int nx, int ny, int nz, const SmoothWeights &w,
                            const float *first, cudaStream_t st)
{
    constexpr int YB = (R <= 8) ? 4 : 2;
    const int tiles = ceil_div(nx, 32) * ceil_div(ny, 32);
    int zc = nz < 128 ? nz : 128;
    const int zmin = (2 * R > 16) ? 2 * R : 16;
    while ((long long)tiles * ceil_div(nz, zc) < 1216 && zc / 2 >= zmin) zc /= 2;
    const dim3 grid((unsigned)ceil_div(nx, 32), (unsigned)ceil_div(ny, 32), (unsigned)ceil_div(nz, zc));
    const dim3 block(32, 32 / YB);
    smooth_kernel<R, YB, ZIP><<<grid, block, 0, st>>>(in, out, nx, ny, nz, zc, w, first);
}

template <bool ZIP>
static shw_status smooth_dispatch(const float *in, float *out, int nx, int ny, int nz, const SmoothWeights &w,
                                  int r, const float *first, cudaStream_t st)
{
    // TMA pipeline where its alignment rules hold, the staged kernel otherwise
    const bool zip_ok = !ZIP || (aligned(first, 8) && aligned(out, 16));
    if (r >= 1 && r <= 8 && nx % 4 == 0 && aligned(in, 16) && zip_ok && !debug(SHW_DEBUG_SMOOTH_PLAIN)) {
        bool ok = false;
        switch (r) {
#define SHW_T(n) \
    case n: ok = launch_smooth_tma<n, ZIP>(in, out, nx, ny, nz, w, first, st); break;
            SHW_T(1) SHW_T(2) SHW_T(3) SHW_T(4) SHW_T(5) SHW_T(6) SHW_T(7) SHW_T(8)
#undef SHW_T
        }
        if (ok) return after_launch();
    }
    switch (r) {
#define SHW_R(n) \
    case n: launch_smooth_r<n, ZIP>(in, out, nx, ny, nz, w, first, st); break;
        SHW_R(0) SHW_R(1) SHW_R(2) SHW_R(3) SHW_R(4) SHW_R(5) SHW_R(6) SHW_R(7) SHW_R(8)
        SHW_R(9) SHW_R(10) SHW_R(11) SHW_R(12) SHW_R(13) SHW_R(14) SHW_R(15) SHW_R(16)
#undef SHW_R
    default: return SHW_EUNSUPPORTED;
    }
    return after_launch();
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *p = static_cast<const char *>(a), *q = static_cast<const char *>(b);
    return p < q + nb && q < p + na;
}

// Eq. 5 sampled at the integer taps k = -radius..radius, normalised to unit sum (host, double)
static bool gauss_weights(float sigma, int radius, SmoothWeights &W)
{
    if (!std::isfinite(sigma) || !(sigma > 0.0f)) return false;
    double w[2 * SHW_MAX_SMOOTH_RADIUS + 1], sum = 0.0;
    for (int k = -radius; k <= radius; ++k) {
        w[k + radius] = std::exp(-(double)k * k / (2.0 * (double)sigma * sigma));
        sum += w[k + radius];
    }
    for (int k = 0; k <= 2 * radius; ++k) {
        W.w[k] = (float)(w[k] / sum);
        W.w2[k] = make_float2(W.w[k], W.w[k]);
    }
    return true;
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
    NvtxRange nvtx_range("shw_smooth");
    shw_status s = smooth_check(in, out, nx, ny, nz, radius);
    if (s != SHW_OK) return s;
    SmoothWeights W{};
    if (!gauss_weights(sigma, radius, W)) return SHW_EINVAL;
    return smooth_dispatch<false>(in, out, nx, ny, nz, W, radius, nullptr, as_stream(stream));
}

shw_status shw_smooth_zip(const float *in, const float *first, float *out_pair, int32_t nx, int32_t ny, int32_t nz,
                          float sigma, int32_t radius, void *stream)
{
    NvtxRange nvtx_range("shw_smooth_zip");
    if (!in || !first || !out_pair || nx <= 0 || ny <= 0 || nz <= 0 || radius < 0) return SHW_EINVAL;
    if (!aligned(in, 4) || !aligned(first, 4) || !aligned(out_pair, 8)) return SHW_EINVAL;
    if (radius > SHW_MAX_SMOOTH_RADIUS) return SHW_EUNSUPPORTED;
    const size_t bytes = (size_t)nx * ny * nz * 4;
    if (overlaps(in, bytes, out_pair, 2 * bytes) || overlaps(first, bytes, out_pair, 2 * bytes)) return SHW_EINVAL;
    SmoothWeights W{};
    if (!gauss_weights(sigma, radius, W)) return SHW_EINVAL;
    return smooth_dispatch<true>(in, out_pair, nx, ny, nz, W, radius, first, as_stream(stream));
}

shw_status shw_smooth_weights(const float *in, float *out, int32_t nx, int32_t ny, int32_t nz, const float *w_host,
                              int32_t radius, void *stream)
{
    NvtxRange nvtx_range("shw_smooth_weights");
    shw_status s = smooth_check(in, out, nx, ny, nz, radius);
    if (s != SHW_OK) return s;
    if (!w_host) return SHW_EINVAL;
    SmoothWeights W{};
    for (int k = 0; k <= 2 * radius; ++k) {
        if (!std::isfinite(w_host[k])) return SHW_EINVAL;
        W.w[k] = w_host[k];
        W.w2[k] = make_float2(w_host[k], w_host[k]);
    }
    return smooth_dispatch<false>(in, out, nx, ny, nz, W, radius, nullptr, as_stream(stream));
}

}  // extern "C"
