// inst_w2.cu -- kernels and launchers for 128-bit determinant keys.
#include "launch.cuh"

namespace hande {
Ops ops_w2(int kind) { return ops_for<2>(kind); }
}  // namespace hande
