// Kernel instantiations: iterate double, weights double.
#include "fw_batch.cuh"
#include "fw_ops.cuh"

namespace fw {
Ops* make_ops_f64(int kmax) { return make_ops_t<double, double>(kmax); }
BatchKern* make_batch_kern_f64(int kmax) { return make_batch_kern_t<double, double>(kmax); }
}  // namespace fw
