// Batched USBS kernel, bulk type float, Lanczos basis J = 64.
#define USBS_PLAIN_LOADS 1
#include "batch_kernel.cuh"

namespace usbs {
int batch_launch_f32_j64(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err, int bucket) {
  return launch_batch<float, float, 64>(cs, st, tol, err, bucket);
}
}  // namespace usbs
