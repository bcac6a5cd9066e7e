// batch_b32.cu -- the batch kernel for items that are 32^3 bricks (packed by the caller
// or by the plan); a translation unit of its own so that it compiles beside batch.cu.
#include "batch_kernel.cuh"

namespace shw {

BatchKernel batch_kernel_b32(int tile, int interp)
{
    if (tile == 8)
        return interp == SHW_NEAREST ? batch_kernel<8, SHW_NEAREST, 32> : batch_kernel<8, SHW_TRILINEAR, 32>;
    return interp == SHW_NEAREST ? batch_kernel<16, SHW_NEAREST, 32> : batch_kernel<16, SHW_TRILINEAR, 32>;
}

}  // namespace shw
