// Bulk kernels of one USBS iteration: everything whose size grows with n, nnz or m.
// T is the bulk type: float (mixed precision) or double (plain FP64).  Reductions
// accumulate in T inside a CTA and in FP64 across CTAs, in a fixed order.
//
// Row kernels use one warp per 4 rows: lane L works on row (L >> 3) and on column
// a = L & 7 of an n x 8 row-major block, so the 8 lanes of a row read one 32-byte
// (float) or 64-byte (double) row segment together.
#include <mutex>

#include "common.cuh"
#include "dev_bulk.cuh"

namespace usbs {

namespace {

template <typename T>
__global__ void k_setup_diag(int n, const double* __restrict__ diagC, const int* __restrict__ dptr,
                             const int* __restrict__ dcon, const double* __restrict__ dval,
                             const double* __restrict__ y, T* __restrict__ dM) {
  k_setup_diag_dev<T>(blockIdx.x, gridDim.x, n, diagC, dptr, dcon, dval, y, dM);
}

template <typename T>
__global__ void k_setup_off(int nnz, const double* __restrict__ valC, const int* __restrict__ sptr,
                            const int* __restrict__ scon, const double* __restrict__ sval,
                            const double* __restrict__ y, T* __restrict__ valM) {
  k_setup_off_dev<T>(blockIdx.x, gridDim.x, nnz, valC, sptr, scon, sval, y, valM);
}

template <typename T>
__global__ void __launch_bounds__(256) k_spmm(int n, const int* __restrict__ rowptr,
                                              const int* __restrict__ col,
                                              const T* __restrict__ val, const T* __restrict__ d,
                                              const T* __restrict__ X, T* __restrict__ Y) {
  k_spmm_dev<T>(blockIdx.x, gridDim.x, n, rowptr, col, val, d, X, Y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gstats(int m, const int* __restrict__ con_ptr,
                                                const int* __restrict__ ent_i,
                                                const int* __restrict__ ent_j,
                                                const T* __restrict__ ent_v, const T* __restrict__ V,
                                                const double* __restrict__ ax,
                                                const double* __restrict__ y,
                                                const double* __restrict__ b, double inv_rho,
                                                double* __restrict__ partials) {
  k_gstats_dev<T>(blockIdx.x, gridDim.x, m, con_ptr, ent_i, ent_j, ent_v, V, ax, y, b, inv_rho, partials);
}

template <typename T>
__global__ void __launch_bounds__(256) k_xupdate(int m, const int* __restrict__ con_ptr,
                                                 const int* __restrict__ ent_i,
                                                 const int* __restrict__ ent_j,
                                                 const T* __restrict__ ent_v, const T* __restrict__ V,
                                                 const DevScalars* __restrict__ sc,
                                                 const double* __restrict__ ax,
                                                 const double* __restrict__ y,
                                                 const double* __restrict__ b,
                                                 const uint8_t* __restrict__ ineq, double inv_rho,
                                                 double* __restrict__ axnew,
                                                 double* __restrict__ ycand,
                                                 double* __restrict__ partials) {
  k_xupdate_dev<T>(blockIdx.x, gridDim.x, m, con_ptr, ent_i, ent_j, ent_v, V, sc, ax, y, b, ineq, inv_rho, axnew, ycand, partials);
}

template <typename T>
__global__ void __launch_bounds__(256) k_alt(int m, const int* __restrict__ con_ptr,
                                             const int* __restrict__ ent_i,
                                             const int* __restrict__ ent_j,
                                             const T* __restrict__ ent_v, const T* __restrict__ V,
                                             const DevScalars* __restrict__ sc,
                                             const double* __restrict__ ax,
                                             const double* __restrict__ y,
                                             const double* __restrict__ b,
                                             const uint8_t* __restrict__ ineq, double rho,
                                             double alpha, double* __restrict__ nu,
                                             double* __restrict__ partials) {
  k_alt_dev<T>(blockIdx.x, gridDim.x, m, con_ptr, ent_i, ent_j, ent_v, V, sc, ax, y, b, ineq, rho, alpha, nu, partials);
}

template <typename T>
__global__ void k_constraint_eval(int m, const int* __restrict__ con_ptr, const int* __restrict__ ent_i,
                                  const int* __restrict__ ent_j, const T* __restrict__ ent_v,
                                  const T* __restrict__ V, const double* __restrict__ S,
                                  double* __restrict__ z) {
  k_constraint_eval_dev<T>(blockIdx.x, gridDim.x, m, con_ptr, ent_i, ent_j, ent_v, V, S, z);
}

template <typename T>
__global__ void __launch_bounds__(256) k_vt_psi(int n, int r, const T* __restrict__ V,
                                                const float* __restrict__ Psi,
                                                double* __restrict__ partials) {
  k_vt_psi_dev<T>(blockIdx.x, gridDim.x, n, r, V, Psi, partials);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sketch_update(int n, int r, const T* __restrict__ V,
                                                       const double* __restrict__ S,
                                                       const double* __restrict__ Bsk,
                                                       float* __restrict__ P,
                                                       const double* __restrict__ eta_dev,
                                                       double eta_host) {
  k_sketch_update_dev<T>(blockIdx.x, gridDim.x, n, r, V, S, Bsk, P, eta_dev, eta_host);
}

__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nparts,
                                                int nvals, double* __restrict__ out,
                                                const int* __restrict__ mask) {
  k_reduce_dev(blockIdx.x, gridDim.x, partials, nparts, nvals, out, mask);
}

template <typename T>
__global__ void __launch_bounds__(256) k_constraint_axpy(int m, const int* __restrict__ con_ptr,
                                                         const int* __restrict__ ent_i, const int* __restrict__ ent_j,
                                                         const T* __restrict__ ent_v, const T* __restrict__ V,
                                                         const double* __restrict__ S, const double* __restrict__ eta,
                                                         const double* __restrict__ ax, double* __restrict__ out) {
  k_constraint_axpy_dev<T>(blockIdx.x, gridDim.x, m, con_ptr, ent_i, ent_j, ent_v, V, S, eta, ax, out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_vnext(int n, const T* __restrict__ V, const double* __restrict__ Qp,
                                               const T* __restrict__ U, int kp, int kc, T* __restrict__ W) {
  k_vnext_dev<T>(blockIdx.x, gridDim.x, n, V, Qp, U, kp, kc, W);
}

// per-CTA partial sums of <a, b> (m FP64 entries), fixed order within the CTA
__global__ void __launch_bounds__(256) k_dot(int64_t m, const double* __restrict__ a,
                                             const double* __restrict__ b, double* __restrict__ partials) {
  __shared__ double ws[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    partials[(size_t)blockIdx.x * PART_STRIDE] = t;
  }
}

__global__ void k_reduce_max(const double* __restrict__ partials, int nparts, int slot,
                             double* __restrict__ out) {
  k_reduce_max_dev(blockIdx.x, gridDim.x, partials, nparts, slot, out);
}

}  // namespace

// =========================================================================================
int red_grid(Ctx* c, int64_t rows, int rows_per_cta) {
  int64_t g = (rows + rows_per_cta - 1) / rows_per_cta;
  if (g < 1) g = 1;
  if (g > c->max_parts) g = c->max_parts;
  return (int)g;
}

void reduce_partials(Ctx* c, int nparts, int nvals, double* out, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REDUCE, mask ? 0.0 : 8.0 * nvals * (nparts + 1));
  k_reduce<<<(nvals + 31) / 32, 256, 0, c->stream>>>(c->partials, nparts, nvals, out, mask);
}

void launch_dot(Ctx* c, const double* a, const double* b, int64_t m, double* out) {
  const int g = red_grid(c, m, 256);
  {
    USBS_LAUNCH_B(c, USBS_KIND_REDUCE, 16.0 * m);
    k_dot<<<g, 256, 0, c->stream>>>(m, a, b, c->partials);
  }
  reduce_partials(c, g, 1, out);
}

// algorithmic bytes of a per-constraint kernel: each entry (i, j, value) and con_ptr once,
// V once, and `per_row` bytes of FP64 m-vectors per constraint
static double constr_bytes(Ctx* c, double es, double per_row) {
  return c->nnzA * (8.0 + es) + 4.0 * (c->m + 1) + 8.0 * es * c->n + per_row * c->m;
}

static int row_grid(Ctx* c, int64_t n) {
  int64_t g = (n + 255) / 256;
  int64_t cap = (int64_t)c->num_sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
void Bulk<T>::setup_operator(Ctx* c, const double* y) {
  {
  USBS_LAUNCH(c, USBS_KIND_SETUP);
  k_setup_diag<T><<<row_grid(c, c->n), 256, 0, c->stream>>>((int)c->n, c->diagC64, c->diag_ptr,
                                                              c->diag_con, c->diag_val, y,
                                                              (T*)c->dM);
  }
  if (c->has_offdiag_A && c->nnz_off > 0) {
    USBS_LAUNCH(c, USBS_KIND_SETUP);
    k_setup_off<T><<<row_grid(c, c->nnz_off), 256, 0, c->stream>>>(
        c->nnz_off, c->valC64, c->slot_ptr, c->slot_con, c->slot_val, y, (T*)c->valM);
  }
}

template <typename T>
void Bulk<T>::spmm(Ctx* c, const void* valM, const void* dM, const void* X, void* Y) {
  const double es = sizeof(T);
  USBS_LAUNCH_B(c, USBS_KIND_SPMM, c->nnz_off * (4.0 + es) + 4.0 * (c->n + 1) + es * c->n + 16.0 * es * c->n);
  k_spmm<T><<<row_grid(c, c->n), 256, 0, c->stream>>>((int)c->n, c->rowptr, c->col,
                                                        (const T*)valM, (const T*)dM,
                                                        (const T*)X, (T*)Y);
}

template <typename T>
void Bulk<T>::gstats(Ctx* c, const void* V, const double* ax, const double* y, int nparts) {
  USBS_LAUNCH_B(c, USBS_KIND_CONSTR, constr_bytes(c, sizeof(T), 24.0));
  size_t smem = sizeof(T) * GS_ROWS * AUG + sizeof(double) * 4 * 880;
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_gstats<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_gstats<T><<<nparts, 256, smem, c->stream>>>((int)c->m, c->con_ptr, c->ent_i, c->ent_j,
                                                  (const T*)c->ent_v, (const T*)V, ax, y, c->b,
                                                  1.0 / c->prm.rho, c->partials);
}

template <typename T>
void Bulk<T>::alt_pass(Ctx* c, const void* V, int nparts) {
  USBS_LAUNCH_B(c, USBS_KIND_CONSTR, constr_bytes(c, sizeof(T), 41.0));
  k_alt<T><<<nparts, 256, 0, c->stream>>>((int)c->m, c->con_ptr, c->ent_i, c->ent_j,
                                            (const T*)c->ent_v, (const T*)V, c->sc, c->ax, c->y,
                                            c->b, c->ineq, c->prm.rho, c->alpha, c->nu,
                                            c->partials);
}

template <typename T>
void Bulk<T>::xupdate(Ctx* c, const void* V, int nparts) {
  USBS_LAUNCH_B(c, USBS_KIND_CONSTR, constr_bytes(c, sizeof(T), 41.0));
  k_xupdate<T><<<nparts, 256, 0, c->stream>>>((int)c->m, c->con_ptr, c->ent_i, c->ent_j,
                                                (const T*)c->ent_v, (const T*)V, c->sc, c->ax,
                                                c->y, c->b, c->ineq, 1.0 / c->prm.rho, c->axnew,
                                                c->ycand, c->partials);
}

template <typename T>
void Bulk<T>::vt_psi(Ctx* c, const void* V, int nparts) {
  USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 8.0 * sizeof(T) * c->n + 4.0 * c->n * c->r);
  k_vt_psi<T><<<nparts, 256, 0, c->stream>>>((int)c->n, c->r, (const T*)V, c->Psi, c->partials);
}

template <typename T>
void Bulk<T>::sketch_update(Ctx* c, const void* V, const double* S, const double* Bsk, float* P,
                            const float* Psi, const double* eta_dev, double eta_host) {
  USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 8.0 * sizeof(T) * c->n + 8.0 * c->n * c->r);
  (void)Psi;
  int64_t total = c->n * c->r;
  k_sketch_update<T><<<row_grid(c, total), 256, 0, c->stream>>>((int)c->n, c->r, (const T*)V, S,
                                                                  Bsk, P, eta_dev, eta_host);
}

template <typename T>
void Bulk<T>::constraint_eval(Ctx* c, const void* V, const double* S, double* z) {
  USBS_LAUNCH_B(c, USBS_KIND_CONSTR, constr_bytes(c, sizeof(T), 8.0));
  k_constraint_eval<T><<<row_grid(c, c->m), 256, 0, c->stream>>>(
      (int)c->m, c->con_ptr, c->ent_i, c->ent_j, (const T*)c->ent_v, (const T*)V, S, z);
}

template <typename T>
void Bulk<T>::constraint_axpy(Ctx* c, const void* V, const double* S, const double* eta_dev,
                              const double* ax, double* out) {
  USBS_LAUNCH_B(c, USBS_KIND_CONSTR, constr_bytes(c, sizeof(T), 16.0));
  k_constraint_axpy<T><<<row_grid(c, c->m), 256, 0, c->stream>>>(
      (int)c->m, c->con_ptr, c->ent_i, c->ent_j, (const T*)c->ent_v, (const T*)V, S, eta_dev, ax, out);
}

template <typename T>
void Bulk<T>::vnext(Ctx* c, const void* V, const double* Qp, const void* U, void* W) {
  USBS_LAUNCH_B(c, USBS_KIND_RESTART, 24.0 * sizeof(T) * c->n);
  k_vnext<T><<<row_grid(c, c->n), 256, 0, c->stream>>>((int)c->n, (const T*)V, Qp, (const T*)U, c->kp,
                                                        c->kc, (T*)W);
}

void reduce_max_slot(Ctx* c, int nparts, int slot, double* out) {
  USBS_LAUNCH(c, USBS_KIND_REDUCE);
  k_reduce_max<<<1, 32, 0, c->stream>>>(c->partials, nparts, slot, out);
}

template struct Bulk<float>;
template struct Bulk<double>;

}  // namespace usbs
