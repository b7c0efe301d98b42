// V-cycle kernels instantiated for the float64 cycle.
#include "amg_launch.cuh"

namespace amg {
AMG_DEFINE_LAUNCHERS(double)
}  // namespace amg
