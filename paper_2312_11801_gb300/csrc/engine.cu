// Host side of libusbs: problem preprocessing (App. E scaling, the A*(y) scatter lists),
// the block Lanczos driver, one USBS iteration (Algorithm 1), the solve loop and the
// extern "C" entry points declared in include/usbs.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <utility>

#include "common.cuh"

namespace usbs {

static thread_local std::string g_create_err;

void prof_resolve(Ctx* c) {
  if (c->prof_pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& pe : c->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      c->prof_ms[pe.kind] += ms;
      c->prof_n[pe.kind] += 1;
    }
    c->ev_pool.push_back(pe.a);
    c->ev_pool.push_back(pe.b);
  }
  c->prof_pending.clear();
  cudaGetLastError();
}

int check_launch(Ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return USBS_ECUDA;
  }
  return USBS_OK;
}

template <typename X>
static int dalloc(Ctx* c, X** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(X));
  if (e != cudaSuccess) {
    c->err = std::string("cudaMalloc(") + std::to_string(count * sizeof(X)) + "): " +
             cudaGetErrorString(e);
    cudaGetLastError();
    return USBS_ENOMEM;
  }
  return USBS_OK;
}

static int dalloc_bytes(Ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    c->err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
    cudaGetLastError();
    return USBS_ENOMEM;
  }
  return USBS_OK;
}

template <typename X>
static int upload(Ctx* c, X** p, const X* host, size_t count) {
  USBS_TRY(dalloc(c, p, count));
  if (count)
    USBS_CUDA_TRY(c, cudaMemcpyAsync(*p, host, count * sizeof(X), cudaMemcpyHostToDevice, c->stream));
  return USBS_OK;
}

static void free_ctx(Ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->rowptr, c->col, c->valC64, c->valM, c->valC, c->diagC64, c->dM, c->dC,
                  c->diag_ptr, c->diag_con, c->diag_val, c->slot_ptr, c->slot_con, c->slot_val,
                  c->con_ptr, c->ent_i, c->ent_j, c->ent_v, c->b, c->ineq, c->y, c->ycand, c->ax,
                  c->axnew, c->nu, c->ytmp, c->V, c->Vnew, c->W, c->Q, c->Q2, c->P, c->Psi,
                  c->sc, c->lz, c->partials, c->red};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& pe : c->prof_pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  if (c->h_lz) cudaFreeHost(c->h_lz);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// ---------------------------------------------------------------------------------------
// Preprocessing: merged operator pattern, scaling, scatter lists, constraint-major entries
// ---------------------------------------------------------------------------------------
struct HostProblem {
  std::vector<int> rowptr, col;
  std::vector<double> offval, diag;
  std::vector<int> diag_ptr, diag_con;
  std::vector<double> diag_val;
  std::vector<int> slot_ptr, slot_con;
  std::vector<double> slot_val;
  std::vector<int> con_ptr, ent_i, ent_j;
  std::vector<double> ent_v;
  std::vector<double> b;
  std::vector<uint8_t> ineq;
  double c_scale = 1.0, tau = 1.0, bnorm = 0.0;
  bool has_offdiag_A = false, any_ineq = false;
};

static int preprocess(Ctx* c, int64_t n, const int64_t* C_rowptr, const int32_t* C_col,
                      const double* C_val, int64_t m, int64_t nnzA, const int32_t* A_con,
                      const int32_t* A_i, const int32_t* A_j, const double* A_val,
                      const double* b, const uint8_t* is_ineq, double trace_hint, HostProblem& hp) {
  if (n < 32 || n > 0x7fffffff - 1) { c->err = "n must be in [32, 2^31-1)"; return USBS_EINVAL; }
  if (m < 1 || m > 0x7fffffff - 1) { c->err = "m must be in [1, 2^31-1)"; return USBS_EINVAL; }
  if (nnzA < 1 || nnzA > 0x7fffffff - 1) { c->err = "nnzA must be in [1, 2^31-1)"; return USBS_EINVAL; }
  if (!C_rowptr || !b || !A_con || !A_i || !A_j || !A_val || !is_ineq) {
    c->err = "NULL array argument";
    return USBS_EINVAL;
  }
  if (C_rowptr[0] != 0) { c->err = "C_rowptr[0] must be 0"; return USBS_EINVAL; }
  const int64_t nnzC = C_rowptr[n];
  if (nnzC < 0 || nnzC > 0x7fffffff - 1) { c->err = "nnz(C) out of range"; return USBS_EINVAL; }
  if (nnzC > 0 && (!C_col || !C_val)) { c->err = "C_col / C_val NULL"; return USBS_EINVAL; }
  hp.diag.assign(n, 0.0);
  // off-diagonal entries of C, checking whether rows are already strictly sorted
  std::vector<int64_t> cnt(n + 1, 0);
  bool sorted = true;
  for (int64_t i = 0; i < n; ++i) {
    if (C_rowptr[i + 1] < C_rowptr[i]) { c->err = "C_rowptr not monotone"; return USBS_EINVAL; }
    int last = -1;
    for (int64_t s = C_rowptr[i]; s < C_rowptr[i + 1]; ++s) {
      const int j = C_col[s];
      if (j < 0 || j >= n) { c->err = "C_col out of range"; return USBS_EINVAL; }
      if (!std::isfinite(C_val[s])) { c->err = "C_val not finite"; return USBS_EINVAL; }
      if (j == i) { hp.diag[i] += C_val[s]; continue; }
      if (j <= last) sorted = false;
      last = j;
      cnt[i + 1]++;
    }
  }
  // A entries: validate, swap to i <= j, collect off-diagonal pattern keys
  std::vector<int> ai(nnzA), aj(nnzA);
  int64_t n_off_a = 0;
  for (int64_t e = 0; e < nnzA; ++e) {
    const int cc = A_con[e];
    int i = A_i[e], j = A_j[e];
    if (cc < 0 || cc >= m || i < 0 || i >= n || j < 0 || j >= n) {
      c->err = "A index out of range at entry " + std::to_string(e);
      return USBS_EINVAL;
    }
    if (!std::isfinite(A_val[e])) { c->err = "A_val not finite"; return USBS_EINVAL; }
    if (i > j) std::swap(i, j);
    ai[e] = i;
    aj[e] = j;
    if (i != j) ++n_off_a;
  }
  hp.has_offdiag_A = n_off_a > 0;
  for (int64_t cidx = 0; cidx < m; ++cidx) {
    if (!std::isfinite(b[cidx])) { c->err = "b not finite"; return USBS_EINVAL; }
    if (is_ineq[cidx]) hp.any_ineq = true;
  }
  // merged off-diagonal pattern (C's entries plus both orientations of A's)
  hp.rowptr.assign(n + 1, 0);
  if (!hp.has_offdiag_A && sorted) {
    for (int64_t i = 0; i < n; ++i) hp.rowptr[i + 1] = hp.rowptr[i] + (int)cnt[i + 1];
    hp.col.resize(hp.rowptr[n]);
    hp.offval.resize(hp.rowptr[n]);
    for (int64_t i = 0; i < n; ++i) {
      int p = hp.rowptr[i];
      for (int64_t s = C_rowptr[i]; s < C_rowptr[i + 1]; ++s) {
        if (C_col[s] == i) continue;
        hp.col[p] = C_col[s];
        hp.offval[p] = C_val[s];
        ++p;
      }
    }
  } else {
    std::vector<std::pair<int64_t, double>> ents;
    ents.reserve((size_t)(nnzC + 2 * n_off_a));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t s = C_rowptr[i]; s < C_rowptr[i + 1]; ++s)
        if (C_col[s] != i) ents.emplace_back(i * n + C_col[s], C_val[s]);
    for (int64_t e = 0; e < nnzA; ++e)
      if (ai[e] != aj[e]) {
        ents.emplace_back((int64_t)ai[e] * n + aj[e], 0.0);
        ents.emplace_back((int64_t)aj[e] * n + ai[e], 0.0);
      }
    std::sort(ents.begin(), ents.end(),
              [](const std::pair<int64_t, double>& x, const std::pair<int64_t, double>& y) {
                return x.first < y.first;
              });
    for (size_t u = 0; u < ents.size();) {
      size_t v = u;
      double s = 0.0;
      while (v < ents.size() && ents[v].first == ents[u].first) s += ents[v++].second;
      const int64_t row = ents[u].first / n;
      hp.col.push_back((int)(ents[u].first % n));
      hp.offval.push_back(s);
      hp.rowptr[row + 1]++;
      u = v;
    }
    for (int64_t i = 0; i < n; ++i) hp.rowptr[i + 1] += hp.rowptr[i];
  }
  // scaling (App. E): ||C||_F = 1, tr(X*) = 1
  double fro = 0.0;
  for (double v : hp.offval) fro += v * v;
  for (double v : hp.diag) fro += v * v;
  hp.c_scale = fro > 0.0 ? std::sqrt(fro) : 1.0;
  double tau = trace_hint;
  if (!(tau > 0.0)) {
    // derive tr(X*) from equality rows that each fix one diagonal entry
    std::vector<int> count(m, 0);
    for (int64_t e = 0; e < nnzA; ++e) count[A_con[e]]++;
    std::vector<char> fixed(n, 0);
    tau = 0.0;
    for (int64_t e = 0; e < nnzA; ++e) {
      const int cc = A_con[e];
      if (count[cc] == 1 && ai[e] == aj[e] && !is_ineq[cc] && A_val[e] != 0.0 && !fixed[ai[e]]) {
        fixed[ai[e]] = 1;
        tau += b[cc] / A_val[e];
      }
    }
    for (int64_t i = 0; i < n; ++i)
      if (!fixed[i]) {
        c->err = "trace_hint is 0 and diag(X) is not fixed by equality rows; give tr(X*)";
        return USBS_EINVAL;
      }
    if (!(tau > 0.0)) { c->err = "derived tr(X*) is not positive"; return USBS_EINVAL; }
  }
  hp.tau = tau;
  for (double& v : hp.offval) v /= hp.c_scale;
  for (double& v : hp.diag) v /= hp.c_scale;
  hp.b.resize(m);
  hp.ineq.resize(m);
  double bn = 0.0;
  for (int64_t cidx = 0; cidx < m; ++cidx) {
    hp.b[cidx] = b[cidx] / tau;
    hp.ineq[cidx] = is_ineq[cidx] ? 1 : 0;
    bn += hp.b[cidx] * hp.b[cidx];
  }
  hp.bnorm = std::sqrt(bn);
  // A*(y) scatter lists: diagonal entries by row, off-diagonal entries by merged slot
  hp.diag_ptr.assign(n + 1, 0);
  for (int64_t e = 0; e < nnzA; ++e)
    if (ai[e] == aj[e]) hp.diag_ptr[ai[e] + 1]++;
  for (int64_t i = 0; i < n; ++i) hp.diag_ptr[i + 1] += hp.diag_ptr[i];
  hp.diag_con.resize(hp.diag_ptr[n]);
  hp.diag_val.resize(hp.diag_ptr[n]);
  {
    std::vector<int> fill(hp.diag_ptr.begin(), hp.diag_ptr.end() - 1);
    for (int64_t e = 0; e < nnzA; ++e)
      if (ai[e] == aj[e]) {
        const int p = fill[ai[e]]++;
        hp.diag_con[p] = A_con[e];
        hp.diag_val[p] = A_val[e];
      }
  }
  const int nnz_off = hp.rowptr[n];
  hp.slot_ptr.assign(nnz_off + 1, 0);
  if (hp.has_offdiag_A) {
    auto find_slot = [&](int i, int j) -> int {
      const int* b0 = hp.col.data() + hp.rowptr[i];
      const int* b1 = hp.col.data() + hp.rowptr[i + 1];
      const int* it = std::lower_bound(b0, b1, j);
      return (int)(it - hp.col.data());
    };
    std::vector<int> s1(nnzA, -1), s2(nnzA, -1);
    for (int64_t e = 0; e < nnzA; ++e)
      if (ai[e] != aj[e]) {
        s1[e] = find_slot(ai[e], aj[e]);
        s2[e] = find_slot(aj[e], ai[e]);
        hp.slot_ptr[s1[e] + 1]++;
        hp.slot_ptr[s2[e] + 1]++;
      }
    for (int s = 0; s < nnz_off; ++s) hp.slot_ptr[s + 1] += hp.slot_ptr[s];
    hp.slot_con.resize(hp.slot_ptr[nnz_off]);
    hp.slot_val.resize(hp.slot_ptr[nnz_off]);
    std::vector<int> fill(hp.slot_ptr.begin(), hp.slot_ptr.end() - 1);
    for (int64_t e = 0; e < nnzA; ++e)
      if (ai[e] != aj[e]) {
        for (int s : {s1[e], s2[e]}) {
          const int p = fill[s]++;
          hp.slot_con[p] = A_con[e];
          hp.slot_val[p] = 0.5 * A_val[e];
        }
      }
  }
  // constraint-major entries
  hp.con_ptr.assign(m + 1, 0);
  for (int64_t e = 0; e < nnzA; ++e) hp.con_ptr[A_con[e] + 1]++;
  for (int64_t cidx = 0; cidx < m; ++cidx) hp.con_ptr[cidx + 1] += hp.con_ptr[cidx];
  hp.ent_i.resize(nnzA);
  hp.ent_j.resize(nnzA);
  hp.ent_v.resize(nnzA);
  {
    std::vector<int> fill(hp.con_ptr.begin(), hp.con_ptr.end() - 1);
    for (int64_t e = 0; e < nnzA; ++e) {
      const int p = fill[A_con[e]]++;
      hp.ent_i[p] = ai[e];
      hp.ent_j[p] = aj[e];
      hp.ent_v[p] = A_val[e];
    }
  }
  return USBS_OK;
}

template <typename T>
static int upload_typed(Ctx* c, void** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  T* p = nullptr;
  USBS_TRY(upload(c, &p, tmp.data(), tmp.size()));
  // the temporary must outlive the async copy
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *dst = p;
  return USBS_OK;
}

static int upload_bulk(Ctx* c, void** dst, const std::vector<double>& src) {
  return c->fp64 ? upload_typed<double>(c, dst, src) : upload_typed<float>(c, dst, src);
}

static int build_ctx(Ctx* c, const HostProblem& hp, const float* Psi) {
  const size_t es = c->fp64 ? sizeof(double) : sizeof(float);
  const int64_t n = c->n, m = c->m;
  c->nnz_off = hp.rowptr[n];
  c->c_scale = hp.c_scale;
  c->tau = hp.tau;
  c->bnorm = hp.bnorm;
  c->has_offdiag_A = hp.has_offdiag_A;
  c->any_ineq = hp.any_ineq;
  USBS_TRY(upload(c, &c->rowptr, hp.rowptr.data(), hp.rowptr.size()));
  USBS_TRY(upload(c, &c->col, hp.col.data(), hp.col.size()));
  USBS_TRY(upload(c, &c->valC64, hp.offval.data(), hp.offval.size()));
  USBS_TRY(upload(c, &c->diagC64, hp.diag.data(), hp.diag.size()));
  USBS_TRY(upload_bulk(c, &c->valC, hp.offval));
  USBS_TRY(upload_bulk(c, &c->dC, hp.diag));
  if (c->has_offdiag_A) {
    USBS_TRY(upload_bulk(c, &c->valM, hp.offval));
  } else {
    c->valM = nullptr;
  }
  USBS_TRY(dalloc_bytes(c, &c->dM, es * n));
  USBS_TRY(upload(c, &c->diag_ptr, hp.diag_ptr.data(), hp.diag_ptr.size()));
  USBS_TRY(upload(c, &c->diag_con, hp.diag_con.data(), hp.diag_con.size()));
  USBS_TRY(upload(c, &c->diag_val, hp.diag_val.data(), hp.diag_val.size()));
  USBS_TRY(upload(c, &c->slot_ptr, hp.slot_ptr.data(), hp.slot_ptr.size()));
  USBS_TRY(upload(c, &c->slot_con, hp.slot_con.data(), hp.slot_con.size()));
  USBS_TRY(upload(c, &c->slot_val, hp.slot_val.data(), hp.slot_val.size()));
  USBS_TRY(upload(c, &c->con_ptr, hp.con_ptr.data(), hp.con_ptr.size()));
  USBS_TRY(upload(c, &c->ent_i, hp.ent_i.data(), hp.ent_i.size()));
  USBS_TRY(upload(c, &c->ent_j, hp.ent_j.data(), hp.ent_j.size()));
  USBS_TRY(upload_bulk(c, &c->ent_v, hp.ent_v));
  USBS_TRY(upload(c, &c->b, hp.b.data(), hp.b.size()));
  USBS_TRY(upload(c, &c->ineq, hp.ineq.data(), hp.ineq.size()));
  for (double** p : {&c->y, &c->ycand, &c->ax, &c->axnew, &c->nu, &c->ytmp}) {
    USBS_TRY(dalloc(c, p, (size_t)m));
    USBS_CUDA_TRY(c, cudaMemsetAsync(*p, 0, sizeof(double) * m, c->stream));
  }
  for (void** p : {&c->V, &c->Vnew, &c->W}) {
    USBS_TRY(dalloc_bytes(c, p, es * 8 * n));
    USBS_CUDA_TRY(c, cudaMemsetAsync(*p, 0, es * 8 * n, c->stream));
  }
  USBS_TRY(dalloc_bytes(c, &c->Q, es * 8 * n * NBMAX));
  USBS_TRY(dalloc_bytes(c, &c->Q2, es * 8 * n * NBMAX));
  if (c->r > 0) {
    USBS_TRY(dalloc(c, &c->P, (size_t)n * c->r));
    USBS_CUDA_TRY(c, cudaMemsetAsync(c->P, 0, sizeof(float) * n * c->r, c->stream));
    USBS_TRY(upload(c, &c->Psi, Psi, (size_t)n * c->r));
  }
  USBS_TRY(dalloc(c, &c->sc, 1));
  USBS_TRY(dalloc(c, &c->lz, 1));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), c->stream));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->lz, 0, sizeof(DevLanczos), c->stream));
  c->max_parts = (int)parts_needed(n, m);
  USBS_TRY(dalloc(c, &c->partials, (size_t)c->max_parts * PART_STRIDE));
  USBS_TRY(dalloc(c, &c->red, (size_t)RED_TOTAL));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->partials, 0, sizeof(double) * c->max_parts * PART_STRIDE, c->stream));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->red, 0, sizeof(double) * RED_TOTAL, c->stream));
  USBS_CUDA_TRY(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_sc), sizeof(DevScalars)));
  USBS_CUDA_TRY(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_lz), sizeof(DevLanczos)));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  tc_register(c);
  return USBS_OK;
}

static void fill_defaults(usbs_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->alpha = 0.0;
  p->rho = 0.01;
  p->beta = 0.25;
  p->k_c = 8;
  p->k_p = 0;
  p->r = 0;
  p->precision = USBS_PRECISION_MIXED;
  p->lanczos_basis = 64;
  p->lanczos_restarts = 10;
  p->lanczos_tol = 0.0;   // 0 = by precision
  p->ipm_mu_tol = 1e-7;
  p->ipm_max_iter = 100;
  p->max_alt = 50;
  p->alt_tol = 1e-8;
  p->trace_hint = 0.0;
  p->max_iters = 1000;
  p->seed = 0;
  p->stream = nullptr;
  p->device = -1;
  p->certify_restarts = 0;
  p->certify_tol = 0.0;   // 0 = by precision
  p->obj_gap_tol = 0.0;
  p->model_value_ipm = 0;
}

static int init_ctx(Ctx* c, int64_t n, int64_t m, int64_t nnzA, const usbs_params* p,
                    const float* Psi) {
  if (p) c->prm = *p; else fill_defaults(&c->prm);
  usbs_params& q = c->prm;
  if (q.k_c < 1 || q.k_c > KB) { c->err = "k_c must be in 1..8"; return USBS_EINVAL; }
  if (q.k_p < 0 || q.k_c + q.k_p > KB) { c->err = "k_p must be >= 0 with k_c + k_p <= 8"; return USBS_EINVAL; }
  if (q.r < 0 || q.r > RMAX) { c->err = "r must be in 0..32"; return USBS_EINVAL; }
  if (q.r > 0 && !Psi) { c->err = "r > 0 needs Psi"; return USBS_EINVAL; }
  if (!(q.rho > 0.0) || !(q.beta > 0.0 && q.beta < 1.0)) { c->err = "rho > 0 and 0 < beta < 1"; return USBS_EINVAL; }
  if (q.precision != USBS_PRECISION_FP64 && q.precision != USBS_PRECISION_MIXED) {
    c->err = "unknown precision";
    return USBS_EINVAL;
  }
  c->n = n;
  c->m = m;
  c->nnzA = nnzA;
  c->kc = q.k_c;
  c->kp = q.k_p;
  c->kdim = q.k_c + q.k_p;
  c->kconv = q.k_c;
  c->r = q.r;
  c->fp64 = q.precision == USBS_PRECISION_FP64;
  c->alpha = q.alpha > 0.0 ? q.alpha : 2.0;
  if (!(q.lanczos_tol > 0.0)) q.lanczos_tol = c->fp64 ? 1e-10 : 1e-6;
  if (q.certify_restarts < 0 || q.obj_gap_tol < 0.0) {
    c->err = "certify_restarts and obj_gap_tol must be >= 0";
    return USBS_EINVAL;
  }
  if (!(q.certify_tol > 0.0)) q.certify_tol = c->fp64 ? 1e-10 : 1e-7;
  if (q.lanczos_restarts < 1) q.lanczos_restarts = 10;
  if (q.ipm_max_iter < 1) q.ipm_max_iter = 100;
  if (q.max_alt < 1) q.max_alt = 50;
  if (q.max_iters < 1) q.max_iters = 1000;
  int J = q.lanczos_basis > 0 ? q.lanczos_basis : 64;
  J = std::min(J, JMAX);
  J = (J / 16) * 16;
  // the basis plus the residual block must leave at least one block of room in R^n,
  // so that random replacement columns always have an orthogonal complement to live in
  const int cap = (int)std::min<int64_t>(JMAX, 16 * ((n - 16) / 16));
  J = std::min(J, cap);
  if (J == 48) J = 32;   // the Ritz kernel is specialised for J in {16, 32, 64}
  if (J < 16) { c->err = "n too small: need n >= 32 (Lanczos basis of 16 plus two blocks)"; return USBS_EINVAL; }
  c->J = J;
  c->keep = J / 2;
  c->seed = q.seed;
  return USBS_OK;
}

// CUDA-side set-up of a validated context: device, SM count, stream.
static int init_cuda(Ctx* c) {
  const usbs_params& q = c->prm;
  if (q.device >= 0) USBS_CUDA_TRY(c, cudaSetDevice(q.device));
  USBS_CUDA_TRY(c, cudaGetDevice(&c->device));
  USBS_CUDA_TRY(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  const char* dbg = std::getenv("USBS_DEBUG");
  c->debug = dbg && dbg[0] == '1';
  const char* nospec = std::getenv("USBS_NO_SPECULATE");
  c->speculate = !(nospec && nospec[0] == '1');
  const char* tcv = std::getenv("USBS_TCGEN05");
  c->use_tc = tcv && tcv[0] == '1';
  if (q.stream) {
    c->stream = (cudaStream_t)q.stream;
    c->own_stream = false;
  } else {
    USBS_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  return USBS_OK;
}

// ---------------------------------------------------------------------------------------
// Block Lanczos with CGS2 reorthogonalisation and thick restart
// ---------------------------------------------------------------------------------------
// masked = false leaves out the second and third passes (a speculative cycle, rerun with
// them when the first pass found a deficient column); the random seeds they would have
// drawn are skipped all the same, so a rerun draws what an unspeculated run draws.
template <typename T>
static void orth_block(Ctx* c, T* Q, int nb, T* W, T* out, int j, int write_T, int is_resid,
                       bool masked = true) {
  const int* defl = DEV_FIELD(c->lz, DevLanczos, defl, int);
  if (nb > 0) {
    const int np = Orth<T>::proj(c, Q, nb, W, nullptr);
    reduce_partials(c, np, nb * 64, c->red + RED_H);
  }
  {
    const int np = Orth<T>::update(c, Q, nb, W, nullptr);
    reduce_partials(c, np, 576, c->red + RED_H2);
  }
  launch_chol_block(c, j, nb, write_T, is_resid, 0);
  Orth<T>::finalize(c, Q, nb, W, out, nullptr, c->seed + 0x1000003ull * (c->rng_counter++));
  // masked second and third passes: only run when a column was replaced by a random
  // vector (the third zeroes what is still dependent after it)
  if (!masked) {
    c->rng_counter += 2;
    return;
  }
  const int* defl2 = DEV_FIELD(c->lz, DevLanczos, defl2, int);
  for (int pass = 1; pass <= 2; ++pass) {
    const int* mask = pass == 1 ? defl : defl2;
    if (nb > 0) {
      const int np = Orth<T>::proj(c, Q, nb, out, mask);
      reduce_partials(c, np, nb * 64, c->red + RED_H, mask);
    }
    const int np = Orth<T>::update(c, Q, nb, out, mask);
    reduce_partials(c, np, 576, c->red + RED_H2, mask);
    launch_chol_block(c, j, nb, 0, is_resid, pass);
    Orth<T>::finalize(c, Q, nb, out, out, mask, c->seed + 0x2000011ull * (c->rng_counter++));
  }
}

// USBS_DEBUG=1: after every block step, synchronise and check the projected matrix,
// the reduced projections and the new block's R factor; print the first non-finite one.
static void debug_block(Ctx* c, int cycle, int j) {
  cudaStreamSynchronize(c->stream);
  std::vector<double> red(RED_TOTAL);
  cudaMemcpy(red.data(), c->red, sizeof(double) * RED_TOTAL, cudaMemcpyDeviceToHost);
  cudaMemcpy(c->h_lz, c->lz, sizeof(DevLanczos), cudaMemcpyDeviceToHost);
  auto bad = [](const double* p, int k) {
    for (int i = 0; i < k; ++i)
      if (!std::isfinite(p[i])) return i;
    return -1;
  };
  int bT = bad(c->h_lz->T, JMAX * JMAX), bH = bad(red.data() + RED_H, 512),
      bH2 = bad(red.data() + RED_H2, 576), bR = bad(c->h_lz->Rinv, 64);
  double gmin = 1e300, gmax = 0.0;
  for (int a = 0; a < 8; ++a) {
    gmin = std::min(gmin, red[RED_GRAM + a * 9]);
    gmax = std::max(gmax, red[RED_GRAM + a * 9]);
  }
  std::fprintf(stderr, "usbs debug: cycle %d block %d defl %d dcol %d%d%d%d%d%d%d%d gram diag [%.3e, %.3e] "
               "badT %d badH %d badH2 %d badRinv %d\n", cycle, j, c->h_lz->defl, c->h_lz->dcol[0],
               c->h_lz->dcol[1], c->h_lz->dcol[2], c->h_lz->dcol[3], c->h_lz->dcol[4], c->h_lz->dcol[5],
               c->h_lz->dcol[6], c->h_lz->dcol[7], gmin, gmax, bT, bH, bH2, bR);
}

struct LanczosOut {
  int cycles = 0, matvecs = 0, converged = 0;
  double max_res = 0.0;
};

// Top eigenpairs of C - A*(y) (y scaled, device).  start: n x 8 device block (T) or
// nullptr.  Writes the top 8 Ritz vectors to out_vecs and Ritz values to lz->theta.
template <typename T>
static int lanczos(Ctx* c, const double* y_dev, const void* start, void* out_vecs, LanczosOut* lo) {
  Bulk<T>::setup_operator(c, y_dev);
  launch_lanczos_reset(c);
  const size_t bs = (size_t)c->n * 8;
  T* Q = (T*)c->Q;
  T* Q2 = (T*)c->Q2;
  T* W = (T*)c->W;
  const void* valM = c->has_offdiag_A ? c->valM : c->valC;
  if (start)
    USBS_CUDA_TRY(c, cudaMemcpyAsync(W, start, bs * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
  else
    USBS_CUDA_TRY(c, cudaMemsetAsync(W, 0, bs * sizeof(T), c->stream));
  orth_block<T>(c, Q, 0, W, Q, -1, 0, 0);
  const int J = c->J, keep = c->keep, nblk = J / 8;
  int nb0 = 0;
  int matvecs = 0;
  int cycle = 0;
  for (cycle = 0; cycle < c->prm.lanczos_restarts; ++cycle) {
    // A cycle first runs speculatively, without the masked passes of its blocks: they are
    // no-ops unless a first pass finds a deficient column.  If one did, its Rayleigh-Ritz
    // step left T, Y and the Ritz values untouched and the cycle runs again from the same
    // state (its kept blocks, T's kept part, the random-seed counter) with the passes.
    const uint64_t rng0 = c->rng_counter;
    const int matvecs0 = matvecs;
    for (int attempt = 0;; ++attempt) {
      const bool spec = c->speculate && attempt == 0;
      for (int j = nb0; j < nblk; ++j) {
        Bulk<T>::spmm(c, valM, c->dM, Q + j * bs, W);
        matvecs += 8;
        orth_block<T>(c, Q, j + 1, W, Q + (j + 1) * bs, j, 1, j == nblk - 1, !spec);
        if (c->debug) debug_block(c, cycle, j);
      }
      launch_ritz(c, J, keep, spec ? 1 : 0);
      USBS_TRY(check_launch(c, "lanczos cycle"));
      USBS_CUDA_TRY(c, cudaMemcpyAsync(c->h_lz, c->lz, sizeof(DevLanczos), cudaMemcpyDeviceToHost,
                                       c->stream));
      USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      if (!spec || !c->h_lz->redo) break;
      c->rng_counter = rng0;
      matvecs = matvecs0;
      c->spec_redos += 1;
    }
    if (c->h_lz->status == USBS_ETIMEOUT) {
      c->err = "a staged tile copy did not complete within its wait limit";
      return USBS_ETIMEOUT;
    }
    if (c->h_lz->status != 0) {
      c->err = "non-finite Lanczos projection";
      return USBS_ENUMERIC;
    }
    if (c->h_lz->converged || cycle == c->prm.lanczos_restarts - 1) break;
    Orth<T>::restart(c, Q, J, keep / 8, DEV_FIELD(c->lz, DevLanczos, Y, double), Q2,
                     Q + nblk * bs, keep / 8);
    std::swap(Q, Q2);
    nb0 = keep / 8;
  }
  c->Q = Q;
  c->Q2 = Q2;
  Orth<T>::restart(c, Q, J, 1, DEV_FIELD(c->lz, DevLanczos, Y, double), out_vecs, nullptr, 0);
  USBS_TRY(check_launch(c, "lanczos output"));
  if (lo) {
    lo->cycles = c->h_lz->cycles;
    lo->matvecs = matvecs;
    lo->converged = c->h_lz->converged;
    double mr = 0.0;
    for (int i = 0; i < c->kconv; ++i) mr = std::max(mr, c->h_lz->res[i]);
    lo->max_res = mr;
  }
  c->total_matvecs += matvecs;
  return USBS_OK;
}

// ---------------------------------------------------------------------------------------
// One USBS iteration (Algorithm 1)
// ---------------------------------------------------------------------------------------
template <typename T>
static int cold_start(Ctx* c) {
  const size_t es = sizeof(T);
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->y, 0, sizeof(double) * c->m, c->stream));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->ax, 0, sizeof(double) * c->m, c->stream));
  if (c->r) USBS_CUDA_TRY(c, cudaMemsetAsync(c->P, 0, sizeof(float) * c->n * c->r, c->stream));
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->V, 0, es * 8 * c->n, c->stream));
  // V_0: the top k_c + k_p eigenvectors of C (all of them converged)
  LanczosOut lo;
  c->kconv = c->kdim;
  const int rc = lanczos<T>(c, c->y, c->V, c->Vnew, &lo);
  c->kconv = c->kc;
  USBS_TRY(rc);
  std::swap(c->V, c->Vnew);
  launch_cold(c);
  c->started = true;
  return check_launch(c, "cold start");
}

static void fill_info(Ctx* c, const DevScalars& s, int matvecs, usbs_step_info* info) {
  if (!info) return;
  info->t = s.t;
  info->descent = s.descent;
  info->n_alt = s.n_alt;
  info->ipm_iters = s.ipm_iters;
  info->matvecs = matvecs;
  info->f_y = s.f_y;
  info->f_cand = s.f_cand;
  info->f_hat = s.f_hat;
  info->lambda_max = s.lam_max;
  info->cx = s.cx_it;
  info->trx = s.tr_it;
  info->eta = s.eta;
  info->relgap = s.relgap;
  info->relinf = s.relinf;
  info->relinf_max = s.relinf_max;
  info->objective = s.cx_it * c->c_scale * c->tau;
  info->dual_bound = s.f_y * c->c_scale * c->tau;
  info->f_hat_closed = s.f_hat_closed;
  info->ipm_iters_b1 = s.ipm_iters_b1;
}

template <typename T>
static int step_impl(Ctx* c, usbs_step_info* info) {
  if (!c->started) USBS_TRY(cold_start<T>(c));
  launch_begin_step(c);
  const int np = red_grid(c, c->n, 128);
  const int npm = red_grid(c, c->m, 256);
  const int npg = red_grid(c, c->m, 128);
  // V^T C V
  Bulk<T>::spmm(c, c->valC, c->dC, c->V, c->W);
  reduce_partials(c, Orth<T>::gram_xy(c, c->V, c->W), 64, c->red + RED_VC);
  // [G | A Xbar | y - b/rho]^T [G | A Xbar | y - b/rho]
  Bulk<T>::gstats(c, c->V, c->ax, c->y, npg);
  reduce_partials(c, npg, 880, c->red + RED_AUG);
  // V^T Psi with the current V, for the sketch update
  if (c->r) {
    Bulk<T>::vt_psi(c, c->V, np);
    reduce_partials(c, np, 8 * c->r, c->red + RED_SK);
  }
  // alternating maximisation (eqs. small_quad_sdp and dual_slack_update)
  USBS_CUDA_TRY(c, cudaMemsetAsync(c->nu, 0, sizeof(double) * c->m, c->stream));
  int n_alt = 0;
  for (n_alt = 1; n_alt <= c->prm.max_alt; ++n_alt) {
    launch_ipm(c, n_alt == 1);
    if (!c->any_ineq) break;
    Bulk<T>::alt_pass(c, c->V, npm);
    reduce_partials(c, npm, 38, c->red + RED_VEC);
    double dn2 = 0.0;
    USBS_CUDA_TRY(c, cudaMemcpyAsync(&c->h_sc->dnu, c->red + RED_VEC + 37, sizeof(double),
                                     cudaMemcpyDeviceToHost, c->stream));
    USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dn2 = c->h_sc->dnu;
    if (std::sqrt(std::max(dn2, 0.0)) <= c->prm.alt_tol * (1.0 + c->bnorm)) break;
  }
  n_alt = std::min(n_alt, c->prm.max_alt);
  // candidate y~ and A X_{t+1}
  Bulk<T>::xupdate(c, c->V, npm);
  reduce_partials(c, npm, 39, c->red + RED_VEC);
  reduce_max_slot(c, npm, 39, c->red + RED_VEC + 39);
  // eigen solve at the candidate
  LanczosOut lo;
  USBS_TRY(lanczos<T>(c, c->ycand, c->V, c->Vnew, &lo));
  if (c->prm.model_value_ipm) launch_ipm_b1(c);
  launch_finish(c);
  launch_commit(c);
  if (c->kp == 0) {
    // model update with k_p = 0: Xbar_{t+1} = X_{t+1}, V_{t+1} = the top k_c Ritz vectors
    if (c->r)
      Bulk<T>::sketch_update(c, c->V, DEV_FIELD(c->sc, DevScalars, S, double), c->red + RED_SK, c->P,
                             c->Psi, DEV_FIELD(c->sc, DevScalars, eta, double), 0.0);
  } else {
    // past information (Sec. 3): S = S_p + S_c; Xbar_{t+1} = eta Xbar_t + V S_c V^T
    // (eq. x_bar_def) through <C, Xbar>, tr Xbar, A Xbar and the sketch; V_{t+1} = an
    // orthonormal basis of [V Q_p, v_1..v_kc] (eq. v_next_def) by Cholesky QR
    launch_kp_split(c);
    if (c->r)
      Bulk<T>::sketch_update(c, c->V, DEV_FIELD(c->sc, DevScalars, Sc, double), c->red + RED_SK, c->P,
                             c->Psi, DEV_FIELD(c->sc, DevScalars, eta, double), 0.0);
    Bulk<T>::constraint_axpy(c, c->V, DEV_FIELD(c->sc, DevScalars, Sc, double),
                             DEV_FIELD(c->sc, DevScalars, eta, double), c->ax, c->axnew);
    Bulk<T>::vnext(c, c->V, DEV_FIELD(c->sc, DevScalars, Qp, double), c->Vnew, c->W);
    orth_block<T>(c, (T*)c->Q, 0, (T*)c->W, (T*)c->Vnew, -1, 0, 0);
  }
  std::swap(c->V, c->Vnew);
  std::swap(c->ax, c->axnew);
  USBS_TRY(check_launch(c, "usbs_step"));
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                   c->stream));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->h_sc->n_alt = n_alt;
  fill_info(c, *c->h_sc, lo.matvecs, info);
  if (info) info->n_alt = n_alt;
  if (c->h_sc->status != 0) {
    c->err = "non-finite value in the subproblem, the model value or the gates";
    return USBS_ENUMERIC;
  }
  return USBS_OK;
}

static int step_dispatch(Ctx* c, usbs_step_info* info) {
  return c->fp64 ? step_impl<double>(c, info) : step_impl<float>(c, info);
}

// Certification of f at the centre y_t: an eigen solve with a 64-column basis (at most
// n - 16), certify_restarts cycles and tolerance certify_tol, started from V; then
// f = alpha lambda_+ + <b, y_t> on the device, the larger of the two values of f(y_t)
// kept and the relative gap re-evaluated (k_certify).  V is left unchanged.
template <typename T>
static int certify_impl(Ctx* c, double* residual, int* matvecs) {
  const int J0 = c->J, keep0 = c->keep, R0 = c->prm.lanczos_restarts;
  const double tol0 = c->prm.lanczos_tol;
  int J = (int)std::min<int64_t>(JMAX, 16 * ((c->n - 16) / 16));
  if (J == 48) J = 32;
  c->J = J;
  c->keep = J / 2;
  c->prm.lanczos_restarts = c->prm.certify_restarts;
  c->prm.lanczos_tol = c->prm.certify_tol;
  c->kconv = 1;     // f(y) needs lambda_max alone
  LanczosOut lo;
  const int rc = lanczos<T>(c, c->y, c->V, c->Vnew, &lo);
  c->kconv = c->kc;
  c->J = J0;
  c->keep = keep0;
  c->prm.lanczos_restarts = R0;
  c->prm.lanczos_tol = tol0;
  USBS_TRY(rc);
  launch_dot(c, c->b, c->y, c->m, c->red + RED_CERT);
  launch_certify(c);
  USBS_TRY(check_launch(c, "certification"));
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                   c->stream));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *residual = lo.max_res;
  *matvecs = lo.matvecs;
  if (c->h_sc->status != 0) {
    c->err = "non-finite value in the certification of f(y)";
    return USBS_ENUMERIC;
  }
  return USBS_OK;
}

// gap relative to the objective itself (scaled units; the ratio is unit-free)
static double obj_gap_of(double f, double cx) {
  return std::fabs(f - cx) / std::max(std::fabs(cx), 1e-300);
}

static bool gates_pass(const Ctx* c, const usbs_step_info& info, double tol) {
  if (!(info.relgap <= tol && info.relinf <= tol)) return false;
  return !(c->prm.obj_gap_tol > 0.0) || obj_gap_of(info.f_y, info.cx) <= c->prm.obj_gap_tol;
}

}  // namespace usbs

// =======================================================================================
// extern "C" entry points
// =======================================================================================
using namespace usbs;

extern "C" {

void usbs_params_default(usbs_params* p) {
  if (p) fill_defaults(p);
}

int usbs_abi_version(void) { return USBS_ABI_VERSION; }

const char* usbs_last_error(const usbs_ctx* ctx) {
  if (!ctx) return g_create_err.c_str();
  return reinterpret_cast<const Ctx*>(ctx)->err.c_str();
}

static int create_common(usbs_ctx** out, int64_t n, const int64_t* C_rowptr, const int32_t* C_col,
                         const double* C_val, int64_t m, int64_t nnzA, const int32_t* A_con,
                         const int32_t* A_i, const int32_t* A_j, const double* A_val,
                         const double* b, const uint8_t* is_ineq, const float* Psi,
                         const usbs_params* p, Ctx** made) {
  if (!out) {
    g_create_err = "out is NULL";
    return USBS_EINVAL;
  }
  *out = nullptr;
  Ctx* c = new Ctx();
  int rc = init_ctx(c, n, m, nnzA, p, Psi);
  HostProblem hp;
  if (rc == USBS_OK)
    rc = preprocess(c, n, C_rowptr, C_col, C_val, m, nnzA, A_con, A_i, A_j, A_val, b, is_ineq,
                    c->prm.trace_hint, hp);
  if (rc == USBS_OK) rc = init_cuda(c);
  if (rc == USBS_OK) rc = build_ctx(c, hp, Psi);
  if (rc != USBS_OK) {
    g_create_err = c->err;
    free_ctx(c);
    return rc;
  }
  *out = reinterpret_cast<usbs_ctx*>(c);
  if (made) *made = c;
  return USBS_OK;
}

int usbs_create(usbs_ctx** out, int64_t n, const int64_t* C_rowptr, const int32_t* C_col,
                const double* C_val, int64_t m, int64_t nnzA, const int32_t* A_con,
                const int32_t* A_i, const int32_t* A_j, const double* A_val, const double* b,
                const uint8_t* is_ineq, const float* Psi, const usbs_params* p) {
  return create_common(out, n, C_rowptr, C_col, C_val, m, nnzA, A_con, A_i, A_j, A_val, b,
                       is_ineq, Psi, p, nullptr);
}

int usbs_destroy(usbs_ctx* ctx) {
  free_ctx(reinterpret_cast<Ctx*>(ctx));
  return USBS_OK;
}

int usbs_extreme_eigs(usbs_ctx* ctx, const double* y, int kc, double* evals, double* evecs,
                      usbs_eig_info* info) {
  if (!ctx) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (kc < 1 || kc > c->kc || !evals) {
    c->err = "kc must be in 1..k_c and evals non-NULL";
    return USBS_EINVAL;
  }
  const double* ydev = c->y;
  if (y) {
    std::vector<double> ys(c->m);
    for (int64_t i = 0; i < c->m; ++i) ys[i] = y[i] / c->c_scale;
    USBS_CUDA_TRY(c, cudaMemcpyAsync(c->ytmp, ys.data(), sizeof(double) * c->m,
                                     cudaMemcpyHostToDevice, c->stream));
    USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ydev = c->ytmp;
  }
  LanczosOut lo;
  int rc = c->fp64 ? lanczos<double>(c, ydev, c->started ? c->V : nullptr, c->Vnew, &lo)
                   : lanczos<float>(c, ydev, c->started ? c->V : nullptr, c->Vnew, &lo);
  if (rc != USBS_OK) return rc;
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->h_lz, c->lz, sizeof(DevLanczos), cudaMemcpyDeviceToHost,
                                   c->stream));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < kc; ++i) evals[i] = c->h_lz->theta[i];
  if (evecs) {
    const size_t es = c->fp64 ? sizeof(double) : sizeof(float);
    std::vector<unsigned char> buf(es * 8 * c->n);
    USBS_CUDA_TRY(c, cudaMemcpy(buf.data(), c->Vnew, buf.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < c->n; ++i)
      for (int a = 0; a < kc; ++a)
        evecs[i * kc + a] = c->fp64 ? reinterpret_cast<double*>(buf.data())[i * 8 + a]
                                    : (double)reinterpret_cast<float*>(buf.data())[i * 8 + a];
  }
  if (info) {
    info->cycles = lo.cycles;
    info->matvecs = lo.matvecs;
    info->converged = lo.converged;
    info->max_residual = lo.max_res;
    info->jacobi_sweeps = c->h_lz->sweeps;
    info->reruns = (int)c->spec_redos;
  }
  return USBS_OK;
}

int usbs_step(usbs_ctx* ctx, usbs_step_info* info) {
  if (!ctx) return USBS_EINVAL;
  return step_dispatch(reinterpret_cast<Ctx*>(ctx), info);
}

int usbs_solve(usbs_ctx* ctx, int warm_start, double tol, usbs_result* out) {
  if (!ctx) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!(tol > 0.0)) { c->err = "tol must be > 0"; return USBS_EINVAL; }
  if (!warm_start) c->started = false;
  usbs_result res;
  std::memset(&res, 0, sizeof(res));
  const long long mv0 = c->total_matvecs;
  int rc = USBS_OK;
  for (int it = 0; it < c->prm.max_iters; ++it) {
    usbs_step_info info;
    rc = step_dispatch(c, &info);
    if (rc != USBS_OK) break;
    res.iters++;
    res.descent_steps += info.descent;
    res.last = info;
    if (!gates_pass(c, info, tol)) continue;
    if (c->prm.certify_restarts > 0) {
      double resid = 0.0;
      int mv = 0;
      rc = c->fp64 ? certify_impl<double>(c, &resid, &mv) : certify_impl<float>(c, &resid, &mv);
      if (rc != USBS_OK) break;
      res.certifications++;
      res.cert_residual = resid;
      info.f_y = c->h_sc->f_y;
      info.relgap = c->h_sc->relgap;
      info.dual_bound = c->h_sc->f_y * c->c_scale * c->tau;
      res.last = info;
      if (!gates_pass(c, info, tol)) continue;
    }
    res.converged = 1;
    break;
  }
  res.obj_gap = obj_gap_of(res.last.f_y, res.last.cx);
  res.matvecs = c->total_matvecs - mv0;
  if (out) *out = res;
  if (rc != USBS_OK) return rc;
  return res.converged ? USBS_OK : USBS_ENOTCONV;
}

}  // extern "C"

namespace usbs {
int batch_result(Ctx* c, usbs_result* out) {
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                   c->stream));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  usbs_result res;
  std::memset(&res, 0, sizeof(res));
  res.iters = c->batch_iters;
  res.converged = c->batch_converged;
  res.descent_steps = c->batch_descent;
  res.matvecs = c->batch_matvecs;
  if (c->batch_iters > 0) {
    c->h_sc->n_alt = c->batch_n_alt;
    fill_info(c, *c->h_sc, c->batch_last_matvecs, &res.last);
    res.obj_gap = obj_gap_of(res.last.f_y, res.last.cx);
  }
  if (out) *out = res;
  if (c->batch_status != USBS_OK) {
    c->err = "non-finite value in the batched solve";
    return c->batch_status;
  }
  return res.converged ? USBS_OK : USBS_ENOTCONV;
}
}  // namespace usbs

extern "C" {

int usbs_get_sketch(usbs_ctx* ctx, float* P, float* Psi, double* scalars) {
  if (!ctx) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const size_t cnt = (size_t)c->n * c->r;
  if (P && c->r) {
    USBS_CUDA_TRY(c, cudaMemcpy(P, c->P, cnt * sizeof(float), cudaMemcpyDeviceToHost));
    const float s = (float)c->tau;
    for (size_t u = 0; u < cnt; ++u) P[u] *= s;
  }
  if (Psi && c->r) USBS_CUDA_TRY(c, cudaMemcpy(Psi, c->Psi, cnt * sizeof(float), cudaMemcpyDeviceToHost));
  if (scalars) {
    USBS_CUDA_TRY(c, cudaMemcpy(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    scalars[0] = c->h_sc->cx * c->c_scale * c->tau;
    scalars[1] = c->h_sc->tr * c->tau;
  }
  return USBS_OK;
}

int usbs_get_dual(usbs_ctx* ctx, double* y) {
  if (!ctx || !y) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  USBS_CUDA_TRY(c, cudaMemcpy(y, c->y, sizeof(double) * c->m, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < c->m; ++i) y[i] *= c->c_scale;
  return USBS_OK;
}

int usbs_get_primal_constraints(usbs_ctx* ctx, double* ax) {
  if (!ctx || !ax) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  USBS_CUDA_TRY(c, cudaMemcpy(ax, c->ax, sizeof(double) * c->m, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < c->m; ++i) ax[i] *= c->tau;
  return USBS_OK;
}

int64_t usbs_state_size(const usbs_ctx* ctx) {
  if (!ctx) return -1;
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  return 2 * c->m + 3 + c->n * c->kdim + c->n * c->r;
}

int usbs_get_state(usbs_ctx* ctx, double* st) {
  if (!ctx || !st) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int64_t m = c->m, n = c->n;
  USBS_CUDA_TRY(c, cudaMemcpy(st, c->y, sizeof(double) * m, cudaMemcpyDeviceToHost));
  USBS_CUDA_TRY(c, cudaMemcpy(st + m, c->ax, sizeof(double) * m, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < m; ++i) {
    st[i] *= c->c_scale;
    st[m + i] *= c->tau;
  }
  USBS_CUDA_TRY(c, cudaMemcpy(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
  st[2 * m] = c->h_sc->cx * c->c_scale * c->tau;
  st[2 * m + 1] = c->h_sc->tr * c->tau;
  st[2 * m + 2] = c->h_sc->f_y * c->c_scale * c->tau;
  double* Vo = st + 2 * m + 3;
  const size_t es = c->fp64 ? sizeof(double) : sizeof(float);
  std::vector<unsigned char> buf(es * 8 * n);
  USBS_CUDA_TRY(c, cudaMemcpy(buf.data(), c->V, buf.size(), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < c->kdim; ++a)
      Vo[i * c->kdim + a] = c->fp64 ? reinterpret_cast<double*>(buf.data())[i * 8 + a]
                                    : (double)reinterpret_cast<float*>(buf.data())[i * 8 + a];
  if (c->r) {
    std::vector<float> P((size_t)n * c->r);
    USBS_CUDA_TRY(c, cudaMemcpy(P.data(), c->P, P.size() * sizeof(float), cudaMemcpyDeviceToHost));
    double* Po = Vo + n * c->kdim;
    for (size_t u = 0; u < P.size(); ++u) Po[u] = (double)P[u] * c->tau;
  }
  return USBS_OK;
}

int usbs_set_state(usbs_ctx* ctx, const double* st) {
  if (!ctx || !st) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  const int64_t m = c->m, n = c->n;
  // writes go on the context's stream (a pageable cudaMemcpy may return before its DMA
  // lands, and the stream is non-blocking), with one synchronisation at the end
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<double> y(m), ax(m);
  for (int64_t i = 0; i < m; ++i) {
    y[i] = st[i] / c->c_scale;
    ax[i] = st[m + i] / c->tau;
  }
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->y, y.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->ax, ax.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
  USBS_CUDA_TRY(c, cudaMemcpy(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
  c->h_sc->cx = st[2 * m] / (c->c_scale * c->tau);
  c->h_sc->tr = st[2 * m + 1] / c->tau;
  c->h_sc->f_y = st[2 * m + 2] / (c->c_scale * c->tau);
  c->h_sc->cx_it = c->h_sc->cx;
  c->h_sc->tr_it = c->h_sc->tr;
  c->h_sc->status = 0;
  USBS_CUDA_TRY(c, cudaMemcpyAsync(c->sc, c->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
  const double* Vi = st + 2 * m + 3;
  if (c->fp64) {
    std::vector<double> Vb((size_t)8 * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < c->kdim; ++a) Vb[i * 8 + a] = Vi[i * c->kdim + a];
    USBS_CUDA_TRY(c, cudaMemcpyAsync(c->V, Vb.data(), Vb.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  } else {
    std::vector<float> Vb((size_t)8 * n, 0.f);
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < c->kdim; ++a) Vb[i * 8 + a] = (float)Vi[i * c->kdim + a];
    USBS_CUDA_TRY(c, cudaMemcpyAsync(c->V, Vb.data(), Vb.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  }
  if (c->r) {
    std::vector<float> P((size_t)n * c->r);
    const double* Pi = Vi + n * c->kdim;
    for (size_t u = 0; u < P.size(); ++u) P[u] = (float)(Pi[u] / c->tau);
    USBS_CUDA_TRY(c, cudaMemcpyAsync(c->P, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  }
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->started = true;
  return USBS_OK;
}

int usbs_grow(usbs_ctx* ctx_old, usbs_ctx** out, int64_t n, const int64_t* C_rowptr,
              const int32_t* C_col, const double* C_val, int64_t m, int64_t nnzA,
              const int32_t* A_con, const int32_t* A_i, const int32_t* A_j, const double* A_val,
              const double* b, const uint8_t* is_ineq, const float* Psi_new) {
  if (!ctx_old || !out) {
    g_create_err = "ctx_old and out must be non-NULL";
    return USBS_EINVAL;
  }
  Ctx* o = reinterpret_cast<Ctx*>(ctx_old);
  if (n < o->n || m < o->m) {
    o->err = "the grown problem must keep the old vertices and constraints";
    return USBS_EINVAL;
  }
  usbs_params prm = o->prm;
  prm.stream = o->own_stream ? nullptr : o->prm.stream;
  prm.trace_hint = 0.0;
  Ctx* c = nullptr;
  int rc = create_common(out, n, C_rowptr, C_col, C_val, m, nnzA, A_con, A_i, A_j, A_val, b,
                         is_ineq, Psi_new, &prm, &c);
  if (rc != USBS_OK) return rc;
  const int64_t n0 = o->n, m0 = o->m;
  // old state in problem units
  std::vector<double> st0(usbs_state_size(ctx_old));
  rc = usbs_get_state(ctx_old, st0.data());
  if (rc != USBS_OK) { usbs_destroy(*out); *out = nullptr; return rc; }
  const double* y0 = st0.data();
  const double* ax0 = y0 + m0;
  const double cx0 = st0[2 * m0], tr0 = st0[2 * m0 + 1];
  const double* V0 = st0.data() + 2 * m0 + 3;
  const double* P0 = V0 + n0 * o->kdim;
  // old C (problem units): merged pattern and diagonal
  std::vector<int> orow(n0 + 1), ocol(o->nnz_off);
  std::vector<double> oval(o->nnz_off), odiag(n0);
  bool ok_primal = tr0 > 0.0;
  auto fail = [&](cudaError_t e) {
    o->err = cudaGetErrorString(e);
    usbs_destroy(*out);
    *out = nullptr;
    return USBS_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMemcpy(orow.data(), o->rowptr, sizeof(int) * (n0 + 1), cudaMemcpyDeviceToHost))) return fail(e);
  if (o->nnz_off &&
      ((e = cudaMemcpy(ocol.data(), o->col, sizeof(int) * o->nnz_off, cudaMemcpyDeviceToHost)) ||
       (e = cudaMemcpy(oval.data(), o->valC64, sizeof(double) * o->nnz_off, cudaMemcpyDeviceToHost))))
    return fail(e);
  if ((e = cudaMemcpy(odiag.data(), o->diagC64, sizeof(double) * n0, cudaMemcpyDeviceToHost))) return fail(e);
  // change of C on old x old entries: off-diagonal changes end the primal warm start,
  // diagonal changes are paid through X_ii fixed by one-entry rows of the old problem
  std::vector<double> ddiag(n0, 0.0);
  for (int64_t i = 0; i < n0 && ok_primal; ++i) {
    ddiag[i] = -odiag[i] * o->c_scale;
    std::vector<std::pair<int, double>> rowc;
    for (int64_t s2 = C_rowptr[i]; s2 < C_rowptr[i + 1]; ++s2) {
      const int j = C_col[s2];
      if (j == i) ddiag[i] += C_val[s2];
      else if (j < n0) rowc.emplace_back(j, C_val[s2]);
    }
    std::sort(rowc.begin(), rowc.end());
    std::vector<std::pair<int, double>> merged;
    for (auto& pr : rowc) {
      if (!merged.empty() && merged.back().first == pr.first) merged.back().second += pr.second;
      else merged.push_back(pr);
    }
    size_t u = 0;
    for (int s2 = orow[i]; s2 < orow[i + 1]; ++s2) {
      const double ov = oval[s2] * o->c_scale;
      double nv = 0.0;
      while (u < merged.size() && merged[u].first < ocol[s2]) {
        if (merged[u].second != 0.0) ok_primal = false;
        ++u;
      }
      if (u < merged.size() && merged[u].first == ocol[s2]) nv = merged[u++].second;
      if (nv != ov) ok_primal = false;
    }
    for (; u < merged.size(); ++u)
      if (merged[u].second != 0.0) ok_primal = false;
  }
  double corr = 0.0;
  if (ok_primal) {
    std::vector<int> cnt(m0, 0), fixc(n0, -1);
    std::vector<double> fixv(n0, 0.0);
    for (int64_t e2 = 0; e2 < nnzA; ++e2)
      if (A_con[e2] < m0) cnt[A_con[e2]]++;
    for (int64_t e2 = 0; e2 < nnzA; ++e2) {
      const int cc = A_con[e2];
      if (cc < m0 && cnt[cc] == 1 && A_i[e2] == A_j[e2] && A_i[e2] < n0 && A_val[e2] != 0.0) {
        fixc[A_i[e2]] = cc;
        fixv[A_i[e2]] = A_val[e2];
      }
      // rows added by the growth may only involve new vertices
      if (cc >= m0 && A_i[e2] < n0 && A_j[e2] < n0) ok_primal = false;
    }
    for (int64_t i = 0; i < n0 && ok_primal; ++i) {
      if (ddiag[i] == 0.0) continue;
      if (fixc[i] < 0) { ok_primal = false; break; }
      corr += ddiag[i] * ax0[fixc[i]] / fixv[i];
    }
  }
  std::vector<double> st(usbs_state_size(*out), 0.0);
  double* y = st.data();
  double* ax = y + m;
  for (int64_t i = 0; i < m0; ++i) y[i] = y0[i];
  if (ok_primal) {
    for (int64_t i = 0; i < m0; ++i) ax[i] = ax0[i];
    st[2 * m] = cx0 + corr;
    st[2 * m + 1] = tr0;
  }
  double* V = st.data() + 2 * m + 3;
  for (int64_t i = 0; i < n0; ++i)
    for (int a = 0; a < c->kdim; ++a) V[i * c->kdim + a] = V0[i * o->kdim + a];
  if (c->r && ok_primal) {
    double* P = V + n * c->kdim;
    for (int64_t i = 0; i < n0; ++i)
      for (int a = 0; a < c->r; ++a) P[i * c->r + a] = P0[i * o->r + a];
  }
  rc = usbs_set_state(*out, st.data());
  if (rc != USBS_OK) { usbs_destroy(*out); *out = nullptr; return rc; }
  // V and f(y) from an eigen solve at the new y, started from the padded V
  LanczosOut lo;
  rc = c->fp64 ? lanczos<double>(c, c->y, c->V, c->Vnew, &lo) : lanczos<float>(c, c->y, c->V, c->Vnew, &lo);
  if (rc != USBS_OK) { usbs_destroy(*out); *out = nullptr; return rc; }
  std::swap(c->V, c->Vnew);
  double by = 0.0;
  for (int64_t i = 0; i < m; ++i) by += (b[i] / c->tau) * (y[i] / c->c_scale);
  cudaStreamSynchronize(c->stream);
  c->h_sc->f_y = c->alpha * std::max(c->h_lz->theta[0], 0.0) + by;
  c->h_sc->lam_max = c->h_lz->theta[0];
  if ((e = cudaMemcpyAsync(c->sc, c->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaStreamSynchronize(c->stream)))
    return fail(e);
  return USBS_OK;
}

int usbs_profile(usbs_ctx* ctx, int on) {
  if (!ctx) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  prof_resolve(c);
  for (int k = 0; k < USBS_NUM_KINDS; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
    c->prof_bytes[k] = 0.0;
  }
  c->prof = on != 0;
  return USBS_OK;
}

int usbs_kernel_stats(usbs_ctx* ctx, int kind, double* total_ms, long long* launches,
                      double* bytes) {
  if (!ctx || kind < 0 || kind >= USBS_NUM_KINDS) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  prof_resolve(c);
  if (total_ms) *total_ms = c->prof_ms[kind];
  if (launches) *launches = c->prof_n[kind];
  if (bytes) *bytes = c->prof_bytes[kind];
  return USBS_OK;
}

long long usbs_launch_count(const usbs_ctx* ctx) {
  if (!ctx) return -1;
  return reinterpret_cast<const Ctx*>(ctx)->launches;
}

int usbs_scaling(const usbs_ctx* ctx, double* c_scale, double* tau) {
  if (!ctx) return USBS_EINVAL;
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (c_scale) *c_scale = c->c_scale;
  if (tau) *tau = c->tau;
  return USBS_OK;
}

int usbs_dims(const usbs_ctx* ctx, int64_t* n, int64_t* m, int* k_c, int* r, int* precision,
              int* basis) {
  if (!ctx) return USBS_EINVAL;
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (n) *n = c->n;
  if (m) *m = c->m;
  if (k_c) *k_c = c->kc;
  if (r) *r = c->r;
  if (precision) *precision = c->fp64 ? USBS_PRECISION_FP64 : USBS_PRECISION_MIXED;
  if (basis) *basis = c->J;
  return USBS_OK;
}

int usbs_op_matmul(usbs_ctx* ctx, const double* y_scaled_dev, const void* X_dev, void* Y_dev) {
  if (!ctx || !y_scaled_dev || !X_dev || !Y_dev) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  const void* valM = c->has_offdiag_A ? c->valM : c->valC;
  if (c->fp64) {
    Bulk<double>::setup_operator(c, y_scaled_dev);
    Bulk<double>::spmm(c, valM, c->dM, X_dev, Y_dev);
  } else {
    Bulk<float>::setup_operator(c, y_scaled_dev);
    Bulk<float>::spmm(c, valM, c->dM, X_dev, Y_dev);
  }
  return check_launch(c, "usbs_op_matmul");
}

int usbs_op_constraint_eval(usbs_ctx* ctx, const void* V_dev, const double* S_dev, double* z_dev) {
  if (!ctx || !V_dev || !S_dev || !z_dev) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (c->fp64) Bulk<double>::constraint_eval(c, V_dev, S_dev, z_dev);
  else Bulk<float>::constraint_eval(c, V_dev, S_dev, z_dev);
  return check_launch(c, "usbs_op_constraint_eval");
}

int usbs_op_sketch_update(usbs_ctx* ctx, const void* V_dev, const double* S_dev,
                          const float* Psi_dev, float* P_dev, double eta) {
  if (!ctx || !V_dev || !S_dev || !Psi_dev || !P_dev) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (c->r < 1) { c->err = "context has r = 0"; return USBS_EINVAL; }
  const int np = red_grid(c, c->n, 128);
  float* saved = c->Psi;
  c->Psi = const_cast<float*>(Psi_dev);
  if (c->fp64) {
    Bulk<double>::vt_psi(c, V_dev, np);
    reduce_partials(c, np, 8 * c->r, c->red + RED_SK);
    Bulk<double>::sketch_update(c, V_dev, S_dev, c->red + RED_SK, P_dev, Psi_dev, nullptr, eta);
  } else {
    Bulk<float>::vt_psi(c, V_dev, np);
    reduce_partials(c, np, 8 * c->r, c->red + RED_SK);
    Bulk<float>::sketch_update(c, V_dev, S_dev, c->red + RED_SK, P_dev, Psi_dev, nullptr, eta);
  }
  c->Psi = saved;
  return check_launch(c, "usbs_op_sketch_update");
}

}  // extern "C"
