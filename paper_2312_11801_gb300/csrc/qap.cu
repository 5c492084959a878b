// QAP rounding of a solve's sketch (App. E, QAP: Rounding), on the device.
//
// The primal of the QAP relaxation (eq. qap_sdp) is indexed by [1; vec(Pi)] (vec stacking
// the columns of the nq x nq assignment matrix).  From the rank-r reconstruction
// X_hat = U diag(lam) U^T of the sketch (usbs_nystrom_round), every column u_k of U gives a
// candidate: orient u_k so that its first entry (paired with X_00 = 1) is non-negative,
// drop that entry, reshape the rest column by column into M_k (nq x nq), and take the
// permutation Pi_k maximising <M_k, Pi_k> (the Hungarian method); its cost is
// tr(W Pi_k D Pi_k^T).  The cheapest candidate is the rounded solution.
//
// One warp per column: the Hungarian method with row and column potentials (the O(nq^3)
// shortest augmenting path form), its column scans spread over the lanes, minima taken with
// the smallest index on ties so that the result is deterministic.
#include <cfloat>
#include <vector>

#include "common.cuh"

namespace usbs {
namespace {

constexpr int QAP_MAXN = 64;   // largest nq

__global__ void __launch_bounds__(32) k_qap_round(int nq, int r, const double* __restrict__ U,
                                                  const double* __restrict__ W, const double* __restrict__ D,
                                                  int* __restrict__ perms, double* __restrict__ scores,
                                                  double* __restrict__ costs) {
  __shared__ double M[QAP_MAXN * QAP_MAXN];
  __shared__ double u[QAP_MAXN + 1], v[QAP_MAXN + 1], minv[QAP_MAXN + 1];
  __shared__ int p[QAP_MAXN + 1], way[QAP_MAXN + 1], used[QAP_MAXN + 1], ans[QAP_MAXN];
  const int k = blockIdx.x, lane = threadIdx.x;
  const double sgn = U[k] >= 0.0 ? 1.0 : -1.0;      // row 0 of U, column k
  for (int t = lane; t < nq * nq; t += 32) {
    const int i = t % nq, j = t / nq;               // column-major reshape of U[1:, k]
    M[i * nq + j] = sgn * U[(size_t)(1 + t) * r + k];
  }
  for (int j = lane; j <= nq; j += 32) { u[j] = 0.0; v[j] = 0.0; p[j] = 0; way[j] = 0; }
  __syncwarp();
  // minimum-cost assignment of the cost a(i, j) = -M(i, j), rows and columns 1..nq
  for (int i = 1; i <= nq; ++i) {
    if (lane == 0) p[0] = i;
    for (int j = lane; j <= nq; j += 32) { minv[j] = DBL_MAX; used[j] = 0; }
    __syncwarp();
    int j0 = 0;
    for (int guard = 0; guard <= nq; ++guard) {
      if (lane == 0) used[j0] = 1;
      __syncwarp();
      const int i0 = p[j0];
      double best = DBL_MAX;
      int bj = 0;
      for (int j = 1 + lane; j <= nq; j += 32) {
        if (!used[j]) {
          const double cur = -M[(i0 - 1) * nq + (j - 1)] - u[i0] - v[j];
          if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
          if (minv[j] < best || (minv[j] == best && j < bj)) { best = minv[j]; bj = j; }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob < best || (ob == best && oj != 0 && (bj == 0 || oj < bj))) { best = ob; bj = oj; }
      }
      const double delta = best;
      __syncwarp();
      for (int j = lane; j <= nq; j += 32) {
        if (used[j]) { u[p[j]] += delta; v[j] -= delta; }
        else minv[j] -= delta;
      }
      __syncwarp();
      j0 = bj;
      if (j0 == 0 || p[j0] == 0) break;
    }
    if (lane == 0) {
      // augment along the path (at most nq steps)
      for (int guard = 0; guard <= nq && j0 != 0; ++guard) {
        const int j1 = way[j0];
        p[j0] = p[j1];
        j0 = j1;
      }
    }
    __syncwarp();
  }
  for (int j = 1 + lane; j <= nq; j += 32) ans[p[j] - 1] = j - 1;   // row p[j] takes column j
  __syncwarp();
  // <M, Pi> and tr(W Pi D Pi^T) = sum_{a, b} W(a, b) D(perm(b), perm(a)), fixed order
  double sc = 0.0, cost = 0.0;
  for (int a = lane; a < nq; a += 32) sc += M[a * nq + ans[a]];
  for (int t = lane; t < nq * nq; t += 32) {
    const int a = t / nq, b = t % nq;
    cost += W[a * nq + b] * D[ans[b] * nq + ans[a]];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sc += __shfl_xor_sync(0xffffffffu, sc, o);
    cost += __shfl_xor_sync(0xffffffffu, cost, o);
  }
  if (lane == 0) {
    scores[k] = sc;
    costs[k] = cost;
  }
  for (int a = lane; a < nq; a += 32) perms[k * nq + a] = ans[a];
}

}  // namespace
}  // namespace usbs

extern "C" int usbs_qap_round(usbs_ctx* ctx, int nq, const double* W, const double* D, double* costs,
                              double* scores, int* perms, int* best) {
  using namespace usbs;
  if (!ctx || !W || !D || !costs) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (nq < 1 || nq > QAP_MAXN || c->n != (int64_t)nq * nq + 1 || c->r < 1) {
    c->err = "usbs_qap_round needs n = nq^2 + 1 (nq <= 64) and a sketch (r > 0)";
    return USBS_EINVAL;
  }
  const int r = c->r;
  const int64_t n = c->n;
  std::vector<double> lam(r), U((size_t)n * r);
  USBS_TRY(usbs_nystrom_round(ctx, lam.data(), U.data(), nullptr, nullptr, nullptr));
  double *dU = nullptr, *dW = nullptr, *dD = nullptr, *dsc = nullptr, *dco = nullptr;
  int* dp = nullptr;
  int rc = USBS_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == USBS_OK) {
      c->err = std::string("usbs_qap_round: ") + cudaGetErrorString(e);
      rc = USBS_ECUDA;
    }
  };
  ck(cudaMalloc(&dU, sizeof(double) * U.size()));
  ck(cudaMalloc(&dW, sizeof(double) * nq * nq));
  ck(cudaMalloc(&dD, sizeof(double) * nq * nq));
  ck(cudaMalloc(&dsc, sizeof(double) * r));
  ck(cudaMalloc(&dco, sizeof(double) * r));
  ck(cudaMalloc(&dp, sizeof(int) * r * nq));
  std::vector<int> hp((size_t)r * nq);
  std::vector<double> hs(r);
  if (rc == USBS_OK) {
    ck(cudaMemcpyAsync(dU, U.data(), sizeof(double) * U.size(), cudaMemcpyHostToDevice, c->stream));
    ck(cudaMemcpyAsync(dW, W, sizeof(double) * nq * nq, cudaMemcpyHostToDevice, c->stream));
    ck(cudaMemcpyAsync(dD, D, sizeof(double) * nq * nq, cudaMemcpyHostToDevice, c->stream));
    {
      USBS_LAUNCH(c, USBS_KIND_SMALL);
      k_qap_round<<<r, 32, 0, c->stream>>>(nq, r, dU, dW, dD, dp, dsc, dco);
    }
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(costs, dco, sizeof(double) * r, cudaMemcpyDeviceToHost, c->stream));
    ck(cudaMemcpyAsync(hs.data(), dsc, sizeof(double) * r, cudaMemcpyDeviceToHost, c->stream));
    ck(cudaMemcpyAsync(hp.data(), dp, sizeof(int) * r * nq, cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  }
  if (rc == USBS_OK) {
    int b = 0;
    for (int k = 1; k < r; ++k)
      if (costs[k] < costs[b]) b = k;
    if (best) *best = b;
    if (scores)
      for (int k = 0; k < r; ++k) scores[k] = hs[k];
    if (perms)
      for (size_t t = 0; t < hp.size(); ++t) perms[t] = hp[t];
  }
  for (void* q : {(void*)dU, (void*)dW, (void*)dD, (void*)dsc, (void*)dco, (void*)dp})
    if (q) cudaFree(q);
  return rc;
}
