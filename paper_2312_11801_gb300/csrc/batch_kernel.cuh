// Batched USBS: many small instances solved by one persistent kernel launch.
//
// One CTA owns one instance at a time and runs its whole solve (cold start, then
// Algorithm 1 iterations until both gates pass or max_iters) without returning to the
// host: the same steps, in the same order, as usbs_solve on that context, built from the
// same device bodies as the per-step kernels, each called with (cta, ncta) = (0, 1) so
// that it covers every row of the instance and writes its final sums straight into the
// context's reduction buffer.  Control flow that the per-step path takes on the host
// (Lanczos restarts, deflation passes, the alternating maximisation, the gates) runs on
// the device from the same flags.  CTAs take instances from an atomic counter, so a
// launch of min(count, resident CTAs) CTAs drains any number of instances.
//
// Every loop is bounded by the instance's parameters (max_iters, lanczos_restarts,
// max_alt, ipm_max_iter, the Jacobi sweep cap), and no CTA waits on another.
//
// Each instantiation (bulk type, basis size) is compiled in its own translation unit
// (batch_*.cu), which must define USBS_PLAIN_LOADS before including this header: a
// buffer written earlier in the launch must not be read through the read-only path.
#pragma once
#ifndef USBS_PLAIN_LOADS
#error "define USBS_PLAIN_LOADS before including batch_kernel.cuh"
#endif

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "dev_bulk.cuh"
#include "dev_orth.cuh"
#include "dev_small.cuh"

namespace usbs {

// Device view of one context, filled from Ctx on the host; the kernel writes the
// outputs at the end.
struct BatchDesc {
  // sizes and parameters
  int n, m, nnz_off, kc, kp, kdim, r, J, keep, has_offdiag_A, any_ineq;
  int restarts, max_alt, ipm_max_iter, max_iters;
  double alpha, rho, beta, bnorm, tol, lanczos_tol, ipm_mu_tol, alt_tol;
  uint64_t seed, rng_counter;
  // operator and constraints
  const int* rowptr; const int* col; const double* valC64; void* valM; const void* valC;
  const double* diagC64; void* dM; const void* dC;
  const int* diag_ptr; const int* diag_con; const double* diag_val;
  const int* slot_ptr; const int* slot_con; const double* slot_val;
  const int* con_ptr; const int* ent_i; const int* ent_j; const void* ent_v;
  const double* b; const uint8_t* ineq;
  // iterate and work buffers
  double* y; double* ycand; double* ax; double* axnew; double* nu;
  void* V; void* Vnew; void* W; void* Q; void* Q2; float* P; const float* Psi;
  DevScalars* sc; DevLanczos* lz; double* red;
  // outputs
  int iters, converged, descent_steps, status;
  int v_swapped, ax_swapped, last_n_alt, last_matvecs;
  long long matvecs;
};

namespace {

constexpr int BT = 256;   // threads per CTA: the bodies are written for 8 warps

template <typename T>
struct BatchCtx {
  BatchDesc* d;
  T* Q;
  T* Q2;
  uint64_t rng;
  long long matvecs;
};

template <typename T>
__device__ void b_orth_block(BatchCtx<T>& b, T* Q, int nb, T* W, T* out, int j, int write_T,
                             int is_resid) {
  const BatchDesc* d = b.d;
  const size_t bs = (size_t)d->n * 8;
  double* red = d->red;
  const double thr = sizeof(T) == 8 ? 1e-16 : 1e-6;
  if (nb > 0) {
    k_tproj_dev<T>(0, 1, d->n, Q, bs, nb, W, red + RED_H, nullptr, &d->lz->status);
    __syncthreads();
  }
  k_tupdate_dev<T>(0, 1, d->n, Q, bs, nb, W, red + RED_H, red + RED_H2, nullptr, &d->lz->status);
  __syncthreads();
  k_chol_block_dev(d->lz, red, j, nb, write_T, is_resid, 0, thr);
  __syncthreads();
  k_tfinalize_dev<T>(0, 1, d->n, Q, bs, nb, W, red + RED_H2, d->lz, out, nullptr,
                     d->seed + 0x1000003ull * (b.rng++), &d->lz->status);
  __syncthreads();
  const int* defl = &d->lz->defl;
  const int* defl2 = &d->lz->defl2;
  for (int pass = 1; pass <= 2; ++pass) {
    const int* mask = pass == 1 ? defl : defl2;
    if (nb > 0) {
      k_tproj_dev<T>(0, 1, d->n, Q, bs, nb, out, red + RED_H, mask, &d->lz->status);
      __syncthreads();
    }
    k_tupdate_dev<T>(0, 1, d->n, Q, bs, nb, out, red + RED_H, red + RED_H2, mask, &d->lz->status);
    __syncthreads();
    k_chol_block_dev(d->lz, red, j, nb, 0, is_resid, pass, thr);
    __syncthreads();
    k_tfinalize_dev<T>(0, 1, d->n, Q, bs, nb, out, red + RED_H2, d->lz, out, mask,
                       d->seed + 0x2000011ull * (b.rng++), &d->lz->status);
    __syncthreads();
  }
}

// Top eigenpairs of C - A*(y): the device twin of the host Lanczos driver, converging
// the top kconv Ritz pairs.  Returns 0 or USBS_ENUMERIC.  start may be null (zero start
// block, replaced by random columns).
template <typename T, typename S, int J>
__device__ int b_lanczos(BatchCtx<T>& b, const double* y, const T* start, T* out_vecs, int kconv) {
  const BatchDesc* d = b.d;
  const int n = d->n;
  const size_t bs = (size_t)n * 8;
  k_setup_diag_dev<T>(0, 1, n, d->diagC64, d->diag_ptr, d->diag_con, d->diag_val, y, (T*)d->dM);
  if (d->has_offdiag_A && d->nnz_off > 0)
    k_setup_off_dev<T>(0, 1, d->nnz_off, d->valC64, d->slot_ptr, d->slot_con, d->slot_val, y,
                       (T*)d->valM);
  k_lanczos_reset_dev(d->lz);
  T* W = (T*)d->W;
  for (size_t t = threadIdx.x; t < bs; t += blockDim.x) W[t] = start ? start[t] : (T)0;
  __syncthreads();
  const T* valM = (const T*)(d->has_offdiag_A ? d->valM : d->valC);
  T* Q = b.Q;
  T* Q2 = b.Q2;
  b_orth_block<T>(b, Q, 0, W, Q, -1, 0, 0);
  constexpr int nblk = J / 8, keep = J / 2;
  const double jac_eps = sizeof(S) == 8 ? 1e-14 : 1e-5;
  const int sweeps = sizeof(S) == 8 ? 30 : 12;
  int nb0 = 0;
  int rc = 0;
  for (int cycle = 0; cycle < d->restarts; ++cycle) {
    for (int j = nb0; j < nblk; ++j) {
      k_spmm_dev<T>(0, 1, n, d->rowptr, d->col, valM, (const T*)d->dM, Q + j * bs, W);
      __syncthreads();
      b.matvecs += 8;
      b_orth_block<T>(b, Q, j + 1, W, Q + (j + 1) * bs, j, 1, j == nblk - 1);
    }
    k_ritz_dev<S, J>(d->lz, kconv, d->lanczos_tol, sweeps, jac_eps);
    __syncthreads();
    if (d->lz->status != 0) { rc = d->lz->status == USBS_ETIMEOUT ? USBS_ETIMEOUT : USBS_ENUMERIC; break; }
    if (d->lz->converged || cycle == d->restarts - 1) break;
    k_trestart_dev<T>(0, 1, n, Q, bs, nblk, keep / 8, d->lz->Y, Q2, bs, Q + nblk * bs, keep / 8, &d->lz->status);
    __syncthreads();
    T* t = Q; Q = Q2; Q2 = t;
    nb0 = keep / 8;
  }
  b.Q = Q;
  b.Q2 = Q2;
  if (rc == 0) {
    k_trestart_dev<T>(0, 1, n, Q, bs, nblk, 1, d->lz->Y, out_vecs, bs, nullptr, 0, &d->lz->status);
    __syncthreads();
  }
  return rc;
}

// One USBS iteration (Algorithm 1), the device twin of the host step.
template <typename T, typename S, int J>
__device__ int b_step(BatchCtx<T>& b, T*& V, T*& Vnew, double*& ax, double*& axnew, int& n_alt_out) {
  BatchDesc* d = b.d;
  const int n = d->n, m = d->m;
  DevScalars* sc = d->sc;
  double* red = d->red;
  k_begin_step_dev(sc);
  // V^T C V
  k_spmm_dev<T>(0, 1, n, d->rowptr, d->col, (const T*)d->valC, (const T*)d->dC, V, (T*)d->W);
  __syncthreads();
  k_tproj_dev<T>(0, 1, n, V, (size_t)n * 8, 1, (const T*)d->W, red + RED_VC, nullptr, &d->lz->status);
  __syncthreads();
  // [G | A Xbar | y - b/rho]^T [G | A Xbar | y - b/rho]
  k_gstats_dev<T>(0, 1, m, d->con_ptr, d->ent_i, d->ent_j, (const T*)d->ent_v, V, ax, d->y, d->b,
                  1.0 / d->rho, red + RED_AUG);
  __syncthreads();
  if (d->r) {
    k_vt_psi_dev<T>(0, 1, n, d->r, V, d->Psi, red + RED_SK);
    __syncthreads();
  }
  for (int c = threadIdx.x; c < m; c += blockDim.x) d->nu[c] = 0.0;
  __syncthreads();
  int n_alt;
  for (n_alt = 1; n_alt <= d->max_alt; ++n_alt) {
    k_ipm_dev(sc, red, d->kdim, d->alpha, d->rho, d->ipm_mu_tol, d->ipm_max_iter, n_alt == 1);
    __syncthreads();
    if (!d->any_ineq) break;
    k_alt_dev<T>(0, 1, m, d->con_ptr, d->ent_i, d->ent_j, (const T*)d->ent_v, V, sc, ax, d->y,
                 d->b, d->ineq, d->rho, d->alpha, d->nu, red + RED_VEC);
    __syncthreads();
    const double dn2 = red[RED_VEC + 37];
    if (sqrt(fmax(dn2, 0.0)) <= d->alt_tol * (1.0 + d->bnorm)) break;
  }
  n_alt_out = min(n_alt, d->max_alt);
  // candidate y~ and A X_{t+1}; the single CTA writes the max |d| to slot 39 itself
  k_xupdate_dev<T>(0, 1, m, d->con_ptr, d->ent_i, d->ent_j, (const T*)d->ent_v, V, sc, ax, d->y,
                   d->b, d->ineq, 1.0 / d->rho, axnew, d->ycand, red + RED_VEC);
  __syncthreads();
  const long long mv0 = b.matvecs;
  const int rc = b_lanczos<T, S, J>(b, d->ycand, V, Vnew, d->kc);
  d->last_matvecs = (int)(b.matvecs - mv0);
  if (rc) return rc;
  if (threadIdx.x < 32) k_finish_dev(sc, d->lz, red, d->kdim, d->alpha, d->beta, d->bnorm);
  __syncthreads();
  k_commit_dev(0, 1, m, sc, d->ycand, d->y);
  if (d->kp == 0) {
    // model update with k_p = 0: Xbar_{t+1} = X_{t+1}, V_{t+1} = the top k_c Ritz vectors
    if (d->r)
      k_sketch_update_dev<T>(0, 1, n, d->r, V, sc->S, red + RED_SK, d->P, &sc->eta, 0.0);
    __syncthreads();
  } else {
    // past information (Sec. 3), as on the per-step path: S = S_p + S_c, Xbar_{t+1} =
    // eta Xbar_t + V S_c V^T, V_{t+1} = an orthonormal basis of [V Q_p, v_1..v_kc]
    __syncthreads();
    k_kp_split_dev(sc, red, d->kdim, d->kp);
    __syncthreads();
    if (d->r)
      k_sketch_update_dev<T>(0, 1, n, d->r, V, sc->Sc, red + RED_SK, d->P, &sc->eta, 0.0);
    k_constraint_axpy_dev<T>(0, 1, m, d->con_ptr, d->ent_i, d->ent_j, (const T*)d->ent_v, V, sc->Sc, &sc->eta,
                             ax, axnew);
    __syncthreads();
    k_vnext_dev<T>(0, 1, n, V, sc->Qp, Vnew, d->kp, d->kc, (T*)d->W);
    __syncthreads();
    b_orth_block<T>(b, b.Q, 0, (T*)d->W, Vnew, -1, 0, 0);
  }
  T* t = V; V = Vnew; Vnew = t;
  double* u = ax; ax = axnew; axnew = u;
  if (threadIdx.x == 0) sc->n_alt = n_alt_out;
  __syncthreads();
  return sc->status != 0 ? USBS_ENUMERIC : 0;
}

template <typename T, typename S, int J>
__global__ void __launch_bounds__(BT) k_batch_solve(BatchDesc* descs, int count, int* next) {
  __shared__ int slot;
  for (;;) {
    if (threadIdx.x == 0) slot = atomicAdd(next, 1);
    __syncthreads();
    const int i = slot;
    __syncthreads();
    if (i >= count) return;
    BatchDesc* d = descs + i;
    BatchCtx<T> b{d, (T*)d->Q, (T*)d->Q2, d->rng_counter, 0};
    T* V = (T*)d->V;
    T* Vnew = (T*)d->Vnew;
    double* ax = d->ax;
    double* axnew = d->axnew;
    const int n = d->n, m = d->m;
    // cold start: y = 0, A Xbar = 0, P = 0, V = 0, then V from an eigen solve at y = 0
    for (int c = threadIdx.x; c < m; c += blockDim.x) { d->y[c] = 0.0; ax[c] = 0.0; }
    for (size_t t = threadIdx.x; t < (size_t)n * d->r; t += blockDim.x) d->P[t] = 0.f;
    for (size_t t = threadIdx.x; t < (size_t)n * 8; t += blockDim.x) V[t] = (T)0;
    __syncthreads();
    int rc = b_lanczos<T, S, J>(b, d->y, V, Vnew, d->kdim);
    int iters = 0, conv = 0, desc = 0, n_alt = 0;
    if (rc == 0) {
      T* t = V; V = Vnew; Vnew = t;
      k_cold_dev(d->sc, d->lz, d->alpha);
      __syncthreads();
      for (int it = 0; it < d->max_iters; ++it) {
        rc = b_step<T, S, J>(b, V, Vnew, ax, axnew, n_alt);
        if (rc) break;
        ++iters;
        desc += d->sc->descent;
        if (d->sc->relgap <= d->tol && d->sc->relinf <= d->tol) { conv = 1; break; }
      }
    }
    if (threadIdx.x == 0) {
      d->iters = iters;
      d->converged = conv;
      d->descent_steps = desc;
      d->status = rc;
      d->v_swapped = (V != (T*)d->V) ? 1 : 0;
      d->ax_swapped = (ax != d->ax) ? 1 : 0;
      d->last_n_alt = n_alt;
      d->matvecs = b.matvecs;
      d->rng_counter = b.rng;
      // the Lanczos buffers may have traded places: report which is which
      d->Q = b.Q;
      d->Q2 = b.Q2;
    }
    __syncthreads();
  }
}

// dynamic shared memory of one batched CTA: the largest of the bodies' needs
template <typename T>
size_t batch_smem(int J) {
  constexpr int TR = sizeof(T) == 8 ? 64 : 128;
  const int nbmax = J / 8;   // projections run against at most J/8 blocks
  size_t m = 0;
  m = std::max(m, sizeof(T) * (2 * (size_t)(nbmax + 1) * BlockStride<T>::value + 8 * 64 + 64));  // tiles
  m = std::max(m, sizeof(double) * 8 * 576);                                      // epilogues
  m = std::max(m, tc_red_bytes(5));                                               // FP32 update
  m = std::max(m, sizeof(T) * (2 * (size_t)nbmax * BlockStride<T>::value) + 8 * (size_t)J * (J / 2));  // restart
  m = std::max(m, sizeof(T) * (4 * (size_t)J * (J + 1) + (size_t)J * J / 2));       // Ritz
  m = std::max(m, sizeof(T) * 128 * AUG + sizeof(double) * 4 * 880);              // gstats
  return m;
}

// Per (instantiation, size bucket) launch plan: pinned and device descriptor arrays, the
// work counter, and a CUDA graph of [descriptors up, counter reset, persistent kernel,
// descriptors down] captured once and replayed while the bucket's instance count and grid
// stay the same (the graph's copies read and write the plan's fixed buffers, so a replay
// only needs the descriptors refreshed in the pinned array).
struct BatchPlan {
  std::mutex mu;
  int count = 0, grid = 0;
  BatchDesc* h = nullptr;     // pinned
  BatchDesc* dd = nullptr;
  int* dnext = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (h) cudaFreeHost(h);
    if (dd) cudaFree(dd);
    if (dnext) cudaFree(dnext);
    exec = nullptr; graph = nullptr; h = nullptr; dd = nullptr; dnext = nullptr;
    count = 0; grid = 0;
  }
};

inline void fill_desc(BatchDesc& d, const Ctx* c, double tol, int max_iters) {
  std::memset(&d, 0, sizeof(d));
  d.n = (int)c->n; d.m = (int)c->m; d.nnz_off = c->nnz_off; d.kc = c->kc; d.kp = c->kp; d.kdim = c->kdim;
  d.r = c->r;
  d.J = c->J; d.keep = c->keep; d.has_offdiag_A = c->has_offdiag_A; d.any_ineq = c->any_ineq;
  d.restarts = c->prm.lanczos_restarts; d.max_alt = c->prm.max_alt;
  d.ipm_max_iter = c->prm.ipm_max_iter; d.max_iters = max_iters;
  d.tol = tol;
  d.alpha = c->alpha; d.rho = c->prm.rho; d.beta = c->prm.beta; d.bnorm = c->bnorm;
  d.lanczos_tol = c->prm.lanczos_tol; d.ipm_mu_tol = c->prm.ipm_mu_tol; d.alt_tol = c->prm.alt_tol;
  d.seed = c->seed; d.rng_counter = c->rng_counter;
  d.rowptr = c->rowptr; d.col = c->col; d.valC64 = c->valC64; d.valM = c->valM; d.valC = c->valC;
  d.diagC64 = c->diagC64; d.dM = c->dM; d.dC = c->dC;
  d.diag_ptr = c->diag_ptr; d.diag_con = c->diag_con; d.diag_val = c->diag_val;
  d.slot_ptr = c->slot_ptr; d.slot_con = c->slot_con; d.slot_val = c->slot_val;
  d.con_ptr = c->con_ptr; d.ent_i = c->ent_i; d.ent_j = c->ent_j; d.ent_v = c->ent_v;
  d.b = c->b; d.ineq = c->ineq;
  d.y = c->y; d.ycand = c->ycand; d.ax = c->ax; d.axnew = c->axnew; d.nu = c->nu;
  d.V = c->V; d.Vnew = c->Vnew; d.W = c->W; d.Q = c->Q; d.Q2 = c->Q2; d.P = c->P; d.Psi = c->Psi;
  d.sc = c->sc; d.lz = c->lz; d.red = c->red;
}

// Cold-start solves of cs (one size bucket of one instantiation) on stream st.  The
// instances go to the CTAs largest first (the atomic counter hands them out in order), and
// the grid (resident CTAs per SM, 1, 2 or the occupancy maximum) is chosen per bucket by a
// timed probe on the first call: each candidate runs the bucket's cold starts and three
// iterations, the fastest wins and is kept for the process.  A probe changes no context:
// its results are not copied back, and the real solve starts cold.
template <typename T, typename S, int J>
int launch_batch(const std::vector<Ctx*>& cs_in, cudaStream_t st, double tol, std::string& err, int bucket) {
  std::vector<Ctx*> cs(cs_in);
  std::stable_sort(cs.begin(), cs.end(), [](const Ctx* a, const Ctx* b) {
    return a->n * (int64_t)(a->nnz_off + a->n) > b->n * (int64_t)(b->nnz_off + b->n);
  });
  const int count = (int)cs.size();
  static std::mutex plans_mu;
  static BatchPlan plans[8];
  static int tuned_per_sm[8] = {};
  const int bk = std::max(0, std::min(bucket, 7));
  BatchPlan& P = plans[bk];
  std::lock_guard<std::mutex> plan_lock(P.mu);
  cudaError_t e;
  auto fail = [&](cudaError_t ee, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(ee);
    cudaGetLastError();
    P.release();
    return USBS_ECUDA;
  };
  const size_t smem = batch_smem<T>(J);
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_batch_solve<T, S, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  int max_per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_per_sm, k_batch_solve<T, S, J>, BT, smem)))
    return fail(e, "occupancy");
  max_per_sm = std::max(max_per_sm, 1);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (P.count != count) {
    P.release();
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&P.h), sizeof(BatchDesc) * count))) return fail(e, "cudaMallocHost");
    if ((e = cudaMalloc(&P.dd, sizeof(BatchDesc) * count))) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&P.dnext, sizeof(int)))) return fail(e, "cudaMalloc");
    P.count = count;
  }
  // autotune the grid of this bucket once
  int per_sm;
  {
    std::lock_guard<std::mutex> lk(plans_mu);
    per_sm = tuned_per_sm[bk];
  }
  if (per_sm == 0) {
    const int cands[3] = {1, std::min(2, max_per_sm), max_per_sm};
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ci = 0; ci < 3; ++ci) {
      if (ci > 0 && cands[ci] == cands[ci - 1]) continue;
      const int grid = std::max(1, std::min(count, cands[ci] * sms));
      for (int i = 0; i < count; ++i) fill_desc(P.h[i], cs[i], tol, std::min(3, cs[i]->prm.max_iters));
      if ((e = cudaMemcpyAsync(P.dd, P.h, sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st))) return fail(e, "probe upload");
      if ((e = cudaMemsetAsync(P.dnext, 0, sizeof(int), st))) return fail(e, "probe reset");
      cudaEventRecord(e0, st);
      k_batch_solve<T, S, J><<<grid, BT, smem, st>>>(P.dd, count, P.dnext);
      cudaEventRecord(e1, st);
      if ((e = cudaStreamSynchronize(st))) return fail(e, "probe");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (per_sm == 0 || ms < best_ms) { best_ms = ms; per_sm = cands[ci]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(plans_mu);
    tuned_per_sm[bk] = per_sm;
  }
  const int grid = std::max(1, std::min(count, per_sm * sms));
  if (!P.exec || P.grid != grid) {
    if (P.exec) { cudaGraphExecDestroy(P.exec); P.exec = nullptr; }
    if (P.graph) { cudaGraphDestroy(P.graph); P.graph = nullptr; }
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal))) return fail(e, "capture");
    cudaMemcpyAsync(P.dd, P.h, sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(P.dnext, 0, sizeof(int), st);
    k_batch_solve<T, S, J><<<grid, BT, smem, st>>>(P.dd, count, P.dnext);
    cudaMemcpyAsync(P.h, P.dd, sizeof(BatchDesc) * count, cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamEndCapture(st, &P.graph))) return fail(e, "capture end");
    if ((e = cudaGraphInstantiate(&P.exec, P.graph, 0))) return fail(e, "graph instantiate");
    P.grid = grid;
  }
  for (int i = 0; i < count; ++i) fill_desc(P.h[i], cs[i], tol, cs[i]->prm.max_iters);
  if ((e = cudaGraphLaunch(P.exec, st))) return fail(e, "graph launch");
  if ((e = cudaStreamSynchronize(st))) return fail(e, "k_batch_solve");
  const BatchDesc* h = P.h;
  for (int i = 0; i < count; ++i) {
    Ctx* c = cs[i];
    const BatchDesc& d = h[i];
    if (d.v_swapped) std::swap(c->V, c->Vnew);
    if (d.ax_swapped) std::swap(c->ax, c->axnew);
    c->Q = d.Q;
    c->Q2 = d.Q2;
    c->rng_counter = d.rng_counter;
    c->total_matvecs += d.matvecs;
    c->started = d.status == USBS_OK;
    // results are read back by the caller from each context
    c->batch_iters = d.iters;
    c->batch_converged = d.converged;
    c->batch_descent = d.descent_steps;
    c->batch_status = d.status;
    c->batch_matvecs = d.matvecs;
    c->batch_last_matvecs = d.last_matvecs;
    c->batch_n_alt = d.last_n_alt;
  }
  return USBS_OK;
}

}  // namespace

}  // namespace usbs
