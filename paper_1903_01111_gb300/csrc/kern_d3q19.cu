// D3Q19 instantiations of the step kernels and of their adjoints (FP64 and
// FP32 shifted storage).
#include "adjoint.cuh"
#include "kernels.cuh"

namespace lbm {
KernelOps ops_d3q19_f64() { return Launch<D3Q19, F64>::ops(); }
KernelOps ops_d3q19_f32s() { return Launch<D3Q19, F32S>::ops(); }
AdjointOps adj_d3q19_f64() { return AdjointLaunch<D3Q19, F64>::ops(); }
AdjointOps adj_d3q19_f32s() { return AdjointLaunch<D3Q19, F32S>::ops(); }
}  // namespace lbm
