// Kernel instantiations for D2Q37 (FP64 and FP32-deviation storage).
#include "ops.cuh"

namespace lbm {
OpsTable ops_q37_f64() { return Ops<D2Q37, double, false>::table(); }
OpsTable ops_q37_f32() { return Ops<D2Q37, float, true>::table(); }
}  // namespace lbm
