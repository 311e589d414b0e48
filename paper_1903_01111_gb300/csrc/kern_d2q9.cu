// D2Q9 instantiations of the step kernels and of their adjoints (FP64 and
// FP32 shifted storage).
#include "adjoint.cuh"
#include "kernels.cuh"

namespace lbm {
KernelOps ops_d2q9_f64() { return Launch<D2Q9, F64>::ops(); }
KernelOps ops_d2q9_f32s() { return Launch<D2Q9, F32S>::ops(); }
AdjointOps adj_d2q9_f64() { return AdjointLaunch<D2Q9, F64>::ops(); }
AdjointOps adj_d2q9_f32s() { return AdjointLaunch<D2Q9, F32S>::ops(); }
}  // namespace lbm
