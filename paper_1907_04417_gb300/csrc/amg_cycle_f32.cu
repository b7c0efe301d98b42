// V-cycle kernels instantiated for the float32 cycle (float64 outer CG).
#include "amg_launch.cuh"

namespace amg {
AMG_DEFINE_LAUNCHERS(float)
}  // namespace amg
