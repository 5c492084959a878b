// k-sized work of a USBS iteration, one CTA each, FP64 unless stated:
//  - Cholesky factor of the 8 x 8 Gram matrix of a new Lanczos block (with deflation),
//  - Rayleigh-Ritz on the J x J projected matrix (parallel cyclic Jacobi),
//  - the primal-dual interior point method of App. B.2 for eq. compressed_subprob_2,
//  - the model value (App. B.1 in closed form), descent test and gates.
#include <cfloat>
#include <mutex>

#include "common.cuh"
#include "dev_small.cuh"

namespace usbs {

namespace {

__global__ void k_chol_block(DevLanczos* lz, const double* __restrict__ red, int j, int nb,
                             int write_T, int is_resid, int defl_pass, double rel_thr) {
  k_chol_block_dev(lz, red, j, nb, write_T, is_resid, defl_pass, rel_thr);
}

// spec = 1: the cycle's blocks ran without their masked passes.  If one of them found a
// deficient column (defl_seen) the basis is not orthonormal: the step is skipped, T, Y and
// the Ritz values keep their values from the cycle's start, and redo tells the host to run
// the cycle again with the masked passes.
template <typename S, int J>
__global__ void __launch_bounds__(J >= 64 ? 512 : 256, 1) k_ritz(DevLanczos* lz, int kc, double tol, int max_sweeps,
                                              double jac_eps, int spec) {
  const int seen = lz->defl_seen;
  __syncthreads();
  if (threadIdx.x == 0) {
    lz->defl_seen = 0;
    lz->redo = (spec && seen) ? 1 : 0;
  }
  if (spec && seen) return;
  k_ritz_dev<S, J>(lz, kc, tol, max_sweeps, jac_eps);
}

__global__ void __launch_bounds__(256, 1) k_ipm(DevScalars* sc, const double* __restrict__ red, int kc,
                                             double alpha, double rho, double mu_tol, int max_iter,
                                             int first_pass, int b1) {
  k_ipm_dev(sc, red, kc, alpha, rho, mu_tol, max_iter, first_pass, b1);
}

__global__ void k_finish(DevScalars* sc, const DevLanczos* lz, const double* __restrict__ red, int kc,
                         double alpha, double beta, double bnorm, int use_ipm) {
  k_finish_dev(sc, lz, red, kc, alpha, beta, bnorm, use_ipm);
}

__global__ void k_certify(DevScalars* sc, const DevLanczos* lz, const double* __restrict__ red,
                          double alpha) {
  k_certify_dev(sc, lz, red, alpha);
}

__global__ void k_kp_split(DevScalars* sc, const double* __restrict__ red, int kdim, int kp) {
  k_kp_split_dev(sc, red, kdim, kp);
}

__global__ void k_cold(DevScalars* sc, const DevLanczos* lz, double alpha) {
  k_cold_dev(sc, lz, alpha);
}

__global__ void k_begin_step(DevScalars* sc) {
  k_begin_step_dev(sc);
}

__global__ void k_commit(int m, const DevScalars* __restrict__ sc, const double* __restrict__ ycand,
                         double* __restrict__ y) {
  k_commit_dev(blockIdx.x, gridDim.x, m, sc, ycand, y);
}

__global__ void k_lanczos_reset(DevLanczos* lz) {
  k_lanczos_reset_dev(lz);
}

}  // namespace

// dynamic shared memory of k_ritz: A, V, T, Y (J x (J+1)) and T Y_keep (J x J/2), type S
static size_t ritz_smem(size_t es, int J) { return es * (4 * J * (J + 1) + J * J / 2); }

template <typename S, int J>
static void ritz_attr() {
  cudaFuncSetAttribute(k_ritz<S, J>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ritz_smem(sizeof(S), J));
}

void small_init_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    ritz_attr<double, 16>(); ritz_attr<double, 32>(); ritz_attr<double, 64>();
    ritz_attr<float, 16>(); ritz_attr<float, 32>(); ritz_attr<float, 64>();
  });
}

void launch_chol_block(Ctx* c, int j, int nb, int write_T, int is_resid, int defl_pass) {
  USBS_LAUNCH(c, USBS_KIND_SMALL);
  // a column keeps about eps / (norm after / norm before) of orthogonality to the basis:
  // replace it when that ratio drops below 1e-3 (FP32) or 1e-8 (FP64)
  const double thr = c->fp64 ? 1e-16 : 1e-6;
  k_chol_block<<<1, 64, 0, c->stream>>>(c->lz, c->red, j, nb, write_T, is_resid, defl_pass, thr);
}

template <typename S>
static void launch_ritz_t(Ctx* c, int J, int max_sweeps, double eps, int spec) {
  const size_t sm = ritz_smem(sizeof(S), J);
  const int threads = J >= 64 ? 512 : 256;
  if (J == 16)
    k_ritz<S, 16><<<1, threads, sm, c->stream>>>(c->lz, c->kconv, c->prm.lanczos_tol, max_sweeps, eps, spec);
  else if (J == 32)
    k_ritz<S, 32><<<1, threads, sm, c->stream>>>(c->lz, c->kconv, c->prm.lanczos_tol, max_sweeps, eps, spec);
  else
    k_ritz<S, 64><<<1, threads, sm, c->stream>>>(c->lz, c->kconv, c->prm.lanczos_tol, max_sweeps, eps, spec);
}

void launch_ritz(Ctx* c, int J, int keep, int spec) {
  USBS_LAUNCH(c, USBS_KIND_RITZ);
  (void)keep;   // keep = J / 2, fixed by the specialisation
  small_init_attributes();
  if (c->fp64) {
    launch_ritz_t<double>(c, J, 30, 1e-14, spec);
  } else {
    // FP32 rotations reach an off-diagonal floor near J * 2^-24 of ||T||: stop at 1e-5.
    // The restart uses the exact projection Y_keep^T T Y_keep, so loose rotations only
    // cost convergence speed, not accuracy.
    launch_ritz_t<float>(c, J, 12, 1e-5, spec);
  }
}

void launch_ipm(Ctx* c, int first_pass) {
  USBS_LAUNCH(c, USBS_KIND_SMALL);
  k_ipm<<<1, 256, 0, c->stream>>>(c->sc, c->red, c->kdim, c->alpha, c->prm.rho, c->prm.ipm_mu_tol,
                                  c->prm.ipm_max_iter, first_pass, 0);
}

void launch_ipm_b1(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL);
  k_ipm<<<1, 256, 0, c->stream>>>(c->sc, c->red, c->kdim, c->alpha, c->prm.rho, c->prm.ipm_mu_tol,
                                  c->prm.ipm_max_iter, 0, 1);
}

void launch_finish(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL);
  k_finish<<<1, 32, 0, c->stream>>>(c->sc, c->lz, c->red, c->kdim, c->alpha, c->prm.beta, c->bnorm,
                                    c->prm.model_value_ipm);
}

void launch_certify(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL); k_certify<<<1, 32, 0, c->stream>>>(c->sc, c->lz, c->red, c->alpha); }

void launch_kp_split(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL); k_kp_split<<<1, 32, 0, c->stream>>>(c->sc, c->red, c->kdim, c->kp); }

void launch_cold(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL); k_cold<<<1, 32, 0, c->stream>>>(c->sc, c->lz, c->alpha); }

void launch_begin_step(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL); k_begin_step<<<1, 32, 0, c->stream>>>(c->sc); }

void launch_commit(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL);
  int g = (int)((c->m + 255) / 256);
  if (g > c->num_sms * 8) g = c->num_sms * 8;
  k_commit<<<g, 256, 0, c->stream>>>((int)c->m, c->sc, c->ycand, c->y);
}

void launch_lanczos_reset(Ctx* c) {
  USBS_LAUNCH(c, USBS_KIND_SMALL); k_lanczos_reset<<<1, 256, 0, c->stream>>>(c->lz); }

}  // namespace usbs
