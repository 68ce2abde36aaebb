// Ops<double>: kernels and launchers for the f64 storage format.
#include "lb_ops_impl.cuh"

namespace trt {
template struct Ops<double>;
}  // namespace trt
