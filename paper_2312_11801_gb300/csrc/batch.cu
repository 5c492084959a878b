// Batched USBS: which contexts the persistent kernel takes, and the launch per
// (precision, basis) group.  The kernel itself is in batch_kernel.cuh; each of its
// instantiations is compiled in its own translation unit so they build in parallel.
#include <string>
#include <vector>

#include "common.cuh"

namespace usbs {

int batch_launch_f32_j32(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err, int bucket);
int batch_launch_f32_j64(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err, int bucket);
int batch_launch_f64_j32(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err, int bucket);

// Eligible for the batched kernel: a basis the kernel is instantiated for (J = 32 in
// both precisions, J = 64 in mixed precision) and no per-step host work (debug checks,
// event profiling).
bool batch_eligible(const Ctx* c) {
  // the per-step path alone carries certification, the objective-relative gate and the
  // App. B.1 model-value IPM
  if (c->debug || c->prof || c->prm.certify_restarts > 0 || c->prm.obj_gap_tol > 0.0 ||
      c->prm.model_value_ipm)
    return false;
  if (c->fp64) return c->J == 32;
  return c->J == 32 || c->J == 64;
}

int batch_bucket(int64_t n) { return n < 256 ? 0 : n < 512 ? 1 : n < 1024 ? 2 : n < 2048 ? 3 : 4; }

int batch_run(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err) {
  if (cs.empty()) return USBS_OK;
  const bool fp64 = cs[0]->fp64;
  const int J = cs[0]->J;
  for (const Ctx* c : cs)
    if (c->fp64 != fp64 || c->J != J || !batch_eligible(c)) {
      err = "a batch must share precision and an instantiated Lanczos basis";
      return USBS_EINVAL;
    }
  const int bucket = batch_bucket(cs[0]->n);
  if (fp64) return batch_launch_f64_j32(cs, st, tol, err, bucket);
  if (J == 32) return batch_launch_f32_j32(cs, st, tol, err, bucket);
  return batch_launch_f32_j64(cs, st, tol, err, bucket);
}

}  // namespace usbs
