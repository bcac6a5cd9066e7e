// common.cuh -- shared host/device helpers of libshw (status handling, launch accounting).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "shw.h"

namespace shw {

// An NVTX range named after the ABI call it spans (host side, enqueue only): profilers and
// timeline tools show each library call; without a tool attached it costs a null check.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Counts every kernel launch made by this library (reported by shw_launch_count).
void note_launch();

// The test and diagnosis switches of shw_set_debug_flags (SHW_DEBUG_*).
uint32_t debug_flags();
inline bool debug(uint32_t flag) { return (debug_flags() & flag) != 0u; }

// Whether `st` is being captured into a CUDA graph: 1 yes, 0 no, -1 the runtime cannot say.
inline int capture_state(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return cs != cudaStreamCaptureStatusNone ? 1 : 0;
}

inline shw_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SHW_OK : SHW_ECUDA; }

// Bounds-checked builds (-DSHW_CHECKED).  Device code cannot share one variable across
// translation units without relocatable device code, so every unit has its own violation
// word; each registers, at load, a host reader that returns and clears it, and
// shw_sync_status polls them all.  SHW_CHECK(ok) records a violation; the caller then clamps
// the index so that the access stays inside its array.  In normal builds it compiles away.
using CheckReader = unsigned (*)();
void register_check_reader(CheckReader r);  // (host; called during library load)
unsigned read_check_words();                // (host) OR of every unit's word, all cleared
#ifdef SHW_CHECKED
static __device__ unsigned g_check_word;
namespace {
inline unsigned read_this_unit_check_word()
{
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v != 0) {
        const unsigned zero = 0;
        cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);
    }
    return v;
}
struct CheckRegistration {
    CheckRegistration() { register_check_reader(&read_this_unit_check_word); }
};
CheckRegistration g_check_registration;
}  // namespace
#define SHW_CHECK(ok)                                            \
    do {                                                         \
        if (!(ok)) atomicOr(&::shw::g_check_word, 1u);           \
    } while (0)
constexpr bool kChecked = true;
#else
#define SHW_CHECK(ok) \
    do {              \
    } while (0)
constexpr bool kChecked = false;
#endif

// Status after a launch: a launch-configuration error is reported now.
inline shw_status after_launch()
{
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SHW_OK : SHW_ECUDA;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

constexpr int kLut = SHW_LUT_SIZE;
constexpr int kBrick = SHW_BRICK;
constexpr int kBrickStored = SHW_BRICK + 2 * SHW_BRICK_APRON;  // 34
constexpr int kBrickElems = kBrickStored * kBrickStored * kBrickStored;

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace shw
