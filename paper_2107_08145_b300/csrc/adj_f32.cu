// adj_f32.cu -- instantiations of the reverse (adjoint) sweep kernel for float
// (see adjoint.cuh); looked up by configuration through kernels.h.
#include "adjoint.cuh"
#include "kernels.h"

namespace rts {

SweepFn<float> adj_kernel_f32(int tq, int maxr)
{
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B) return sweep_adj_kernel<float, A, B>;
    RTS_CFG(4, 72) RTS_CFG(2, 56) RTS_CFG(1, 56) RTS_CFG(4, 64) RTS_CFG(2, 64) RTS_CFG(1, 64)
#undef RTS_CFG
    return nullptr;
}

}  // namespace rts
