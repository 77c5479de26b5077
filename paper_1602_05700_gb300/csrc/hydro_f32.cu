// FP32 instance of the hydrodynamics' stage kernel (hydro_kernels.cuh), compiled with multiply-add contraction and
// using the approximate division and square root: the compact-arithmetic production path, checked against the FP64
// oracle within tolerance.  The FP64 instance, bit-exact with the oracle, is in hydro.cu.
#include "hydro_kernels.cuh"

namespace hg {
cudaError_t hydro_stage_f32(const HydroStageLaunch& L) { return launch_hydro_stage<float>(L); }
}  // namespace hg
