// kernels.h -- lookup of the sweep kernel instantiations, which are compiled
// in translation units of their own (sweep_f32.cu, sweep_f64.cu, adj_f32.cu,
// adj_f64.cu) so that the library builds in parallel. Each function returns
// the kernel for a (rows per tile, register cap) configuration, or null if
// that configuration is not instantiated.
#pragma once
#include "sweep.cuh"

namespace rts {

template <typename T>
using SweepFn = void (*)(SweepArgs<T>);

// forward sweep (ckpt: the instantiation that keeps the adjoint's checkpoint)
SweepFn<float> fwd_kernel_f32(int tq, int maxr, bool ckpt);
SweepFn<double> fwd_kernel_f64(int tq, int maxr, bool ckpt);
// register-resident FP32 forward sweep (sweep_reg.cuh)
// seeded: the warm-start instantiation; checkpoint: the adjoint's checkpoint sweep (stores D)
SweepFn<float> reg_kernel_f32(int tq, int maxr, bool seeded = false, bool checkpoint = false);
// reverse (adjoint) sweep
SweepFn<float> adj_kernel_f32(int tq, int maxr);
SweepFn<double> adj_kernel_f64(int tq, int maxr);

}  // namespace rts
