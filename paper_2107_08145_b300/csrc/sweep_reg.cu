// sweep_reg.cu -- instantiations of the register-resident FP32 forward sweep
// (sweep_reg.cuh); looked up by configuration through kernels.h.
#include "kernels.h"
#include "sweep_reg.cuh"

namespace rts {

SweepFn<float> reg_kernel_f32(int tq, int maxr, bool seeded, bool checkpoint)
{
#define RTS_CFG(A, B)                                                                                              \
    if (tq == A && maxr == B)                                                                                      \
        return checkpoint ? sweep_reg_kernel<A, B, false, true>                                                   \
                          : (seeded ? sweep_reg_kernel<A, B, true> : sweep_reg_kernel<A, B, false>);
    RTS_CFG(8, 255) RTS_CFG(4, 168) RTS_CFG(4, 128) RTS_CFG(2, 96)
#undef RTS_CFG
    return nullptr;
}

}  // namespace rts
