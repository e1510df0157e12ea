// sweep_f32.cu -- instantiations of the forward sweep kernel for float
// (see sweep.cuh); looked up by configuration through kernels.h.
#include "kernels.h"

namespace rts {

SweepFn<float> fwd_kernel_f32(int tq, int maxr, bool ckpt)
{
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B) return ckpt ? nullptr : sweep_kernel<float, A, B, false>;
    RTS_CFG(16, 168) RTS_CFG(12, 168) RTS_CFG(8, 112) RTS_CFG(7, 112) RTS_CFG(6, 104)
#undef RTS_CFG
    // the small tiles also exist with the adjoint's checkpoint
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B) return ckpt ? sweep_kernel<float, A, B, true> : sweep_kernel<float, A, B, false>;
    RTS_CFG(4, 72) RTS_CFG(2, 56) RTS_CFG(1, 56) RTS_CFG(4, 64) RTS_CFG(2, 64) RTS_CFG(1, 64)
#undef RTS_CFG
    return nullptr;
}

}  // namespace rts
