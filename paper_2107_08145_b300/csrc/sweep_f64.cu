// sweep_f64.cu -- instantiations of the forward sweep kernel for double
// (see sweep.cuh); looked up by configuration through kernels.h.
#include "kernels.h"

namespace rts {

SweepFn<double> fwd_kernel_f64(int tq, int maxr, bool ckpt)
{
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B) return ckpt ? nullptr : sweep_kernel<double, A, B, false>;
    RTS_CFG(16, 168) RTS_CFG(12, 168) RTS_CFG(8, 112) RTS_CFG(7, 112) RTS_CFG(6, 104)
#undef RTS_CFG
    // the small tiles also exist with the adjoint's checkpoint
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B) return ckpt ? sweep_kernel<double, A, B, true> : sweep_kernel<double, A, B, false>;
    RTS_CFG(4, 72) RTS_CFG(2, 56) RTS_CFG(1, 56) RTS_CFG(4, 64) RTS_CFG(2, 64) RTS_CFG(1, 64)
#undef RTS_CFG
    return nullptr;
}

}  // namespace rts
