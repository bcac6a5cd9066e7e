// common.cuh -- shared host/device helpers of libshw (status handling, launch accounting).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "shw.h"

namespace shw {

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
