// Kernel instantiations: iterate float, weights float.
#include "fw_batch.cuh"
#include "fw_ops.cuh"

namespace fw {
Ops* make_ops_f32(int kmax) { return make_ops_t<float, float>(kmax); }
BatchKern* make_batch_kern_f32(int kmax) { return make_batch_kern_t<float, float>(kmax); }
}  // namespace fw
