// batch_b16.cu -- the batch kernel for items that are 16^3 bricks a plan packed itself;
// a translation unit of its own so that it compiles beside batch.cu.
#include "batch_kernel.cuh"

namespace shw {

BatchKernel batch_kernel_b16(int tile, int interp)
{
    if (tile == 8)
        return interp == SHW_NEAREST ? batch_kernel<8, SHW_NEAREST, 16> : batch_kernel<8, SHW_TRILINEAR, 16>;
    return interp == SHW_NEAREST ? batch_kernel<16, SHW_NEAREST, 16> : batch_kernel<16, SHW_TRILINEAR, 16>;
}

}  // namespace shw
