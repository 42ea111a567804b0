// inst_w1.cu -- kernels and launchers for 64-bit determinant keys.
#include "launch.cuh"

namespace hande {
Ops ops_w1(int kind) { return ops_for<1>(kind); }
}  // namespace hande
