// Kernel instantiations for D2Q17 (FP64 and FP32-deviation storage).
#include "ops.cuh"

namespace lbm {
OpsTable ops_q17_f64() { return Ops<D2Q17, double, false>::table(); }
OpsTable ops_q17_f32() { return Ops<D2Q17, float, true>::table(); }
}  // namespace lbm
