// Kernel instantiations: iterate float, weights __nv_bfloat16.
#include "fw_batch.cuh"
#include "fw_ops.cuh"

namespace fw {
Ops* make_ops_bf16(int kmax) { return make_ops_t<float, __nv_bfloat16>(kmax); }
BatchKern* make_batch_kern_bf16(int kmax) { return make_batch_kern_t<float, __nv_bfloat16>(kmax); }
}  // namespace fw
