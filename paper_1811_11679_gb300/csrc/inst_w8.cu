// inst_w8.cu -- kernels and launchers for 512-bit determinant keys.
#include "launch.cuh"

namespace hande {
Ops ops_w8(int kind) { return ops_for<8>(kind); }
}  // namespace hande
