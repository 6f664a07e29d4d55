// Kernel instantiations for D2Q9 (FP64 and FP32-deviation storage).
#include "ops.cuh"

namespace lbm {
OpsTable ops_q9_f64() { return Ops<D2Q9, double, false>::table(); }
OpsTable ops_q9_f32() { return Ops<D2Q9, float, true>::table(); }
}  // namespace lbm
