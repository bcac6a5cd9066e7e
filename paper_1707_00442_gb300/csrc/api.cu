// api.cu -- the C ABI: argument validation, dispatch and status reporting.
// Every check here runs on the host before anything is enqueued, so an invalid
// call returns an error without touching the GPU.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "render_impl.cuh"
#include "tma.cuh"

namespace shw {

// The bounds-checked build's per-unit violation words (see SHW_CHECK): readers registered
// while the library loads, polled by shw_sync_status.
static std::mutex &check_mu()
{
    static std::mutex m;
    return m;
}
static std::vector<CheckReader> &check_readers()
{
    static std::vector<CheckReader> v;
    return v;
}
void register_check_reader(CheckReader r)
{
    std::lock_guard<std::mutex> g(check_mu());
    check_readers().push_back(r);
}
unsigned read_check_words()
{
    std::lock_guard<std::mutex> g(check_mu());
    unsigned v = 0;
    for (CheckReader r : check_readers()) v |= r();
    return v;
}

static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<uint32_t> g_debug_flags{0};
uint32_t debug_flags() { return g_debug_flags.load(std::memory_order_relaxed); }

// The device error word: kernels OR in a bit when a bounded wait gives up.
static __device__ unsigned g_device_error;
static std::mutex g_err_mu;
static unsigned *g_err_ptr[64] = {};

unsigned *device_error_word()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_err_mu);
    if (!g_err_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_err_ptr[dev] = static_cast<unsigned *>(p);
    }
    return g_err_ptr[dev];
}

// Work counters of persistent launches: a ring of slots per device, each zeroed on the
// launch's stream just before the launch that takes it.  A slot is reused only after
// kWorkSlots later launches, far more than can be in flight at once.
constexpr int kWorkSlots = 1024;
static __device__ unsigned g_work_ctr[kWorkSlots];
static unsigned *g_work_ptr[64] = {};
static std::atomic<unsigned> g_work_next{0};

unsigned *work_counter(cudaStream_t st)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned *base;
    {
        std::lock_guard<std::mutex> lk(g_err_mu);
        if (!g_work_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_work_ctr) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            g_work_ptr[dev] = static_cast<unsigned *>(p);
        }
        base = g_work_ptr[dev];
    }
    unsigned *slot = base + (g_work_next.fetch_add(1, std::memory_order_relaxed) % kWorkSlots);
    if (cudaMemsetAsync(slot, 0, sizeof(unsigned), st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return slot;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    });
    return fn;
}

bool encode_tmap_3d(CUtensorMap *map, const void *base, int elem_bytes, int nx, int ny, int nz, int bx, int by,
                    int bz)
{
    const auto fn = tmap_encoder();
    if (!fn) return false;
    CUtensorMapDataType dt;
    switch (elem_bytes) {
    case 2: dt = CU_TENSOR_MAP_DATA_TYPE_UINT16; break;
    case 4: dt = CU_TENSOR_MAP_DATA_TYPE_UINT32; break;
    case 8: dt = CU_TENSOR_MAP_DATA_TYPE_UINT64; break;
    default: return false;
    }
    const cuuint64_t eb = (cuuint64_t)elem_bytes;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * eb, (cuuint64_t)nx * ny * eb};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_tmap_3d_f32(CUtensorMap *map, const float *base, int nx, int ny, int nz, int bx, int by)
{
    const auto fn = tmap_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static bool finite3(const float v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool valid_volume(const shw_volume *v)
{
    if (!v || !v->data || v->nx <= 0 || v->ny <= 0 || v->nz <= 0) return false;
    if (v->storage < SHW_F32 || v->storage > SHW_F16_PAIR) return false;
    if (v->storage == SHW_F32 && !aligned(v->data, 4)) return false;
    if (v->storage == SHW_F32_PAIR && !aligned(v->data, 8)) return false;
    if ((v->storage == SHW_BF16_PAIR_BRICK || v->storage == SHW_F16_PAIR_BRICK || v->storage == SHW_BF16_PAIR ||
         v->storage == SHW_F16_PAIR) &&
        !aligned(v->data, 4))
        return false;
    if (!aligned(v->data, 2)) return false;
    return true;
}

bool valid_camera(const shw_camera *c)
{
    if (!c || c->width <= 0 || c->height <= 0) return false;
    if ((long long)c->width * c->height > (1LL << 31) - 1) return false;
    if (c->width > (1 << 19) || c->height > (1 << 19)) return false;  // grid.y <= 65535 tiles
    if (!finite3(c->eye) || !finite3(c->right) || !finite3(c->up) || !finite3(c->fwd)) return false;
    const double nf = (double)c->fwd[0] * c->fwd[0] + (double)c->fwd[1] * c->fwd[1] + (double)c->fwd[2] * c->fwd[2];
    if (!(nf > 0.0)) return false;
    if (c->ortho) return std::isfinite(c->ortho_half_h) && c->ortho_half_h > 0.0f;
    return std::isfinite(c->tan_half_fovy) && c->tan_half_fovy > 0.0f;
}

// Upper bound of N over all rays: a chord is at most the box diagonal.
long long max_samples(const shw_volume *v, float step)
{
    const double diag = std::sqrt((double)v->nx * v->nx + (double)v->ny * v->ny + (double)v->nz * v->nz);
    return (long long)std::floor(diag / (double)step) + 1;
}

bool valid_params(const shw_render_params *p, const shw_volume *v)
{
    if (!p || !p->lut || !aligned(p->lut, 16)) return false;
    if (p->mode < SHW_MIP || p->mode > SHW_RATIO_MIP) return false;
    if (p->interp != SHW_NEAREST && p->interp != SHW_TRILINEAR) return false;
    if (!std::isfinite(p->step) || !(p->step > 0.0f)) return false;
    if (!std::isfinite(p->lo) || !std::isfinite(p->hi) || !(p->hi > p->lo)) return false;
    if (!std::isfinite(1.0f / (p->hi - p->lo))) return false;
    if (!std::isfinite(p->opacity_scale) || !std::isfinite(p->term_alpha) || !std::isfinite(p->ratio_floor))
        return false;
    if (max_samples(v, p->step) > (1LL << 30)) return false;
    if (p->filter < SHW_FILTER_NONE || p->filter > SHW_FILTER_SCALE) return false;
    if (p->alpha_threshold != 0 && p->alpha_threshold != 1) return false;
    if (p->filter != SHW_FILTER_NONE || p->alpha_threshold) {
        if (!std::isfinite(p->min_threshold) || !std::isfinite(p->max_threshold)) return false;
    }
    if (p->filter == SHW_FILTER_CLIP && !(p->min_threshold <= p->max_threshold)) return false;
    if (p->filter == SHW_FILTER_SCALE &&
        (!(p->min_threshold < p->max_threshold) || !std::isfinite(1.0f / (p->max_threshold - p->min_threshold))))
        return false;
    if (p->smooth < SHW_SMOOTH_NONE || p->smooth > SHW_SMOOTH_TAPS) return false;
    if (p->smooth == SHW_SMOOTH_BOX && (p->smooth_arm < 0 || p->smooth_arm > SHW_MAX_SMOOTH_ARM)) return false;
    if (p->smooth == SHW_SMOOTH_TAPS) {
        if (p->smooth_ntaps < 0 || p->smooth_ntaps > SHW_MAX_SMOOTH_TAPS || !std::isfinite(p->smooth_c0))
            return false;
        for (int j = 0; j < p->smooth_ntaps; ++j)
            if (!std::isfinite(p->smooth_weight[j]) || !std::isfinite(p->smooth_offset[j]) ||
                std::fabs(p->smooth_offset[j]) > 64.0f)
                return false;
    }
    return true;
}

long long ckpt_count(const shw_volume *v, const shw_render_params *p)
{
    const long long nmax = max_samples(v, p->step);
    return (nmax + p->ckpt_interval - 1) / p->ckpt_interval;
}

}  // namespace shw

using namespace shw;

extern "C" {

int32_t shw_abi_version(void) { return SHW_ABI_VERSION; }

const char *shw_status_string(int32_t s)
{
    switch (s) {
    case SHW_OK: return "ok";
    case SHW_EINVAL: return "invalid argument";
    case SHW_EUNSUPPORTED: return "unsupported request";
    case SHW_ECUDA: return "CUDA runtime error";
    case SHW_ENOMEM: return "buffer too small or out of memory";
    case SHW_ETIMEOUT: return "timed out";
    case SHW_EDEVICE: return "no usable CUDA device";
    case SHW_EBOUNDS: return "an index outside its array (bounds-checked build)";
    default: return "unknown status";
    }
}

size_t shw_struct_size(int32_t which)
{
    switch (which) {
    case 0: return sizeof(shw_volume);
    case 1: return sizeof(shw_camera);
    case 2: return sizeof(shw_render_params);
    case 3: return sizeof(shw_batch_item);
    case 4: return sizeof(shw_batch_info);
    default: return 0;
    }
}

uint64_t shw_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint32_t shw_set_debug_flags(uint32_t flags) { return g_debug_flags.exchange(flags, std::memory_order_relaxed); }

shw_status shw_sync_status(void *stream)
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return SHW_EDEVICE;
    }
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return SHW_ECUDA;
    if (cudaGetLastError() != cudaSuccess) return SHW_ECUDA;
    unsigned *w = device_error_word();
    unsigned v = 0;
    if (w) {
        if (cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return SHW_ECUDA;
        if (v != 0) {
            const unsigned zero = 0;
            cudaMemcpy(w, &zero, sizeof zero, cudaMemcpyHostToDevice);
        }
    }
    if (read_check_words() != 0) return SHW_EBOUNDS;  // (always 0 unless built with SHW_CHECKED)
    return v != 0 ? SHW_ETIMEOUT : SHW_OK;
}

size_t shw_ckpt_bytes(const shw_volume *vol, const shw_camera *cam, const shw_render_params *p)
{
    if (!valid_volume(vol) || !valid_camera(cam) || !p || !(p->step > 0.0f) || p->ckpt_interval <= 0) return 0;
    const long long npix = (long long)cam->width * cam->height;
    return (size_t)(npix * 4 + ckpt_count(vol, p) * npix * 4);
}

shw_status shw_render(const shw_volume *vol, const shw_volume *vol2, const shw_camera *cam,
                      const shw_render_params *p, float *out_rgba, float *out_scalar, int32_t *out_index,
                      int32_t *out_nsamples, void *ckpt, size_t ckpt_bytes, void *stream)
{
    NvtxRange nvtx_range("shw_render");
    if (!valid_volume(vol) || !valid_camera(cam) || !valid_params(p, vol)) return SHW_EINVAL;
    if (!out_rgba || !aligned(out_rgba, 16)) return SHW_EINVAL;
    if ((out_scalar && !aligned(out_scalar, 4)) || (out_index && !aligned(out_index, 4)) ||
        (out_nsamples && !aligned(out_nsamples, 4)))
        return SHW_EINVAL;
    const int sto = vol->storage;
    const bool pair = sto == SHW_F32_PAIR || sto == SHW_BF16_PAIR_BRICK || sto == SHW_F16_PAIR_BRICK ||
                      sto == SHW_BF16_PAIR || sto == SHW_F16_PAIR;  // both cubes in one volume
    const bool lin16 = sto >= SHW_BF16 && sto <= SHW_F16_PAIR;  // read by the staged marcher only
    if (pair) {
        // both cubes in one volume: the line ratios only, no second volume, no in-ray smoothing
        if (vol2) return SHW_EINVAL;
        if ((p->mode != SHW_RATIO && p->mode != SHW_RATIO_MIP) || p->smooth != SHW_SMOOTH_NONE)
            return SHW_EUNSUPPORTED;
    } else if (p->mode == SHW_RATIO || p->mode == SHW_RATIO_MIP) {
        if (!valid_volume(vol2) || vol2->nx != vol->nx || vol2->ny != vol->ny || vol2->nz != vol->nz ||
            vol2->storage != vol->storage)
            return SHW_EINVAL;
    }
    const long long npix = (long long)cam->width * cam->height;
    RenderArgs a{};
    a.rgba = reinterpret_cast<float4 *>(out_rgba);
    a.scalar = out_scalar;
    a.index = out_index;
    a.nsamples = out_nsamples;
    a.lut = reinterpret_cast<const float4 *>(p->lut);
    a.width = cam->width;
    a.height = cam->height;
    a.step = p->step;
    a.lo = p->lo;
    a.inv_range = 1.0f / (p->hi - p->lo);
    a.opacity_scale = p->opacity_scale;
    a.term_alpha = p->term_alpha;
    a.ratio_floor = p->ratio_floor;
    a.filter = p->filter;
    a.alpha_thr = p->alpha_threshold;
    a.tmin = p->min_threshold;
    a.tmax = p->max_threshold;
    a.tinv = p->filter == SHW_FILTER_SCALE ? (float)(1.0 / ((double)p->max_threshold - (double)p->min_threshold)) : 0.0f;
    a.nx = vol->nx;
    a.ny = vol->ny;
    a.nz = vol->nz;
    a.smooth = p->smooth;
    if (p->smooth == SHW_SMOOTH_BOX) {
        a.smooth_n = p->smooth_arm;
        a.smooth_c0 = (float)(1.0 / (2.0 * p->smooth_arm + 1.0));
        // a step of exactly 1/2 voxel puts the box's neighbours on the ray's own samples
        const bool single = p->mode != SHW_RATIO && p->mode != SHW_RATIO_MIP;
        if (p->smooth_arm > 0 && p->step == 0.5f && single && !debug(SHW_DEBUG_BOX_DIRECT)) a.box_lattice = 2;
    } else if (p->smooth == SHW_SMOOTH_TAPS) {
        a.smooth_n = p->smooth_ntaps;
        a.smooth_c0 = p->smooth_c0;
        for (int j = 0; j < p->smooth_ntaps; ++j) {
            // the offset in 32.32 fixed point (exact for any float of magnitude <= 64 and >= 2^-9)
            a.smooth_off[j] = std::llrint((double)p->smooth_offset[j] * 4294967296.0);
            a.smooth_w[j] = p->smooth_weight[j];
        }
    }
    a.nmax = (int)max_samples(vol, p->step);
    a.warp_shift = warp_shift_for(*cam);
    a.ckpt_interval = p->ckpt_interval > 0 ? p->ckpt_interval : 64;
    if (ckpt) {
        if (p->mode != SHW_COMPOSITE || p->ckpt_interval <= 0 || !aligned(ckpt, 4)) return SHW_EINVAL;
        if (ckpt_bytes < shw_ckpt_bytes(vol, cam, p)) return SHW_ENOMEM;
        a.ckpt_K = static_cast<int *>(ckpt);
        a.ckpt_T = reinterpret_cast<float *>(static_cast<char *>(ckpt) + npix * 4);
        a.nckpt = (int)ckpt_count(vol, p);
    }
    const shw_volume *v2 = (!pair && (p->mode == SHW_RATIO || p->mode == SHW_RATIO_MIP)) ? vol2 : nullptr;
    cudaStream_t st = as_stream(stream);
    // a captured launch would keep the work counter it was given while later calls reuse it
    const int cs = capture_state(st);
    if (cs != 0) return cs > 0 ? SHW_EUNSUPPORTED : SHW_ECUDA;
    if (lin16) return render_slab(p->mode, p->interp, *vol, *cam, a, st);
    if (pair) {
        const shw_status ss = render_slab(p->mode, p->interp, *vol, *cam, a, st);
        if (ss != SHW_EUNSUPPORTED || debug(SHW_DEBUG_REQUIRE_STAGING)) return ss;
        return render_pair(p->mode, p->interp, *vol, *cam, a, st);
    }
    if (a.box_lattice == 2)
        return vol->storage == SHW_F32 ? render_smooth_lat_f32(p->mode, p->interp, *vol, *cam, a, st)
                                       : render_smooth_lat_b16(p->mode, p->interp, *vol, *cam, a, st);
    if (p->smooth != SHW_SMOOTH_NONE)
        return vol->storage == SHW_F32 ? render_smooth_f32(p->mode, p->interp, *vol, v2, *cam, a, st)
                                       : render_smooth_b16(p->mode, p->interp, *vol, v2, *cam, a, st);
    // orthographic views down the spectral axis: the plane sweep, when it applies
    const shw_status sa = render_axis(p->mode, p->interp, *vol, *cam, a, st);
    if (sa != SHW_EUNSUPPORTED) return sa;
    // other views of a float32 cube: the staged marcher, when it applies
    if (sto == SHW_F32) {
        const shw_status ss = render_slab(p->mode, p->interp, *vol, *cam, a, st);
        if (ss != SHW_EUNSUPPORTED || debug(SHW_DEBUG_REQUIRE_STAGING)) return ss;
    }
    switch (vol->storage) {
    case SHW_F32: return render_f32(p->mode, p->interp, *vol, v2, *cam, a, st);
    case SHW_BF16_BRICK: return render_bf16(p->mode, p->interp, *vol, v2, *cam, a, st);
    case SHW_F16_BRICK: return render_f16(p->mode, p->interp, *vol, v2, *cam, a, st);
    default: return SHW_EINVAL;
    }
}

}  // extern "C"
