// Reconstruction of the primal from its Nystrom sketch, and MaxCut rounding
// (App. C, eq. nystrom_approx; App. E, MaxCut rounding).
//
// The sketch P = Xbar Psi (n x r, FP32, scaled units) and the test matrix Psi give
// X_hat = P (Psi^T P)^+ P^T.  It is computed by the numerically stable method the paper
// adopts (Tropp, Yurtsever, Udell and Cevher 2017, Algorithm 3):
//   nu = sqrt(n) eps(||P||_2), Y = P + nu Psi, B = Psi^T Y = R^T R,
//   E = Y R^-1 = U Sigma W^T, Lambda = max(Sigma^2 - nu I, 0), X_hat = U Lambda U^T.
// The singular value decomposition of the n x r matrix E is taken through its r x r Gram
// matrix: E^T E = W Sigma^2 W^T and U = E W Sigma^-1.  The sign vector z_k = sgn(U[:, k])
// (0 -> +1) of every column is a cut, valued <C, z_k z_k^T>.
//
// Kernels: three bulk passes over the n rows (FP32 sketch in, FP64 arithmetic) and two
// single-CTA FP64 steps on r x r matrices (Jacobi eigen-decompositions, a Cholesky factor
// and its inverse).  An output stage: it runs once per call, outside the iteration.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace usbs {
namespace {

constexpr int NY_RMAX = 32;     // sketch rank limit (RMAX)
constexpr int NY_T = 256;       // threads of every kernel here
constexpr int NY_ROWS = 64;     // rows of a staged chunk in the bulk passes
constexpr int NY_LD = NY_RMAX + 1;

// Result of the r x r steps, in device memory.
struct NyState {
  double nu;                    // the shift
  double normP;                 // ||P||_2
  int status;                   // 0, or USBS_ENUMERIC when B is not positive definite
  int pad;
  double Rinv[NY_RMAX * NY_RMAX];   // R^-1 (upper), row-major r x r
  double M[NY_RMAX * NY_RMAX];      // W Sigma^-1, row-major r x r (columns by descending sigma)
  double lam[NY_RMAX];              // max(sigma^2 - nu, 0), descending
};

// ---- bulk: partial Gram matrices over row chunks ---------------------------------------
// nmat = 3: G0 = X^T X, G1 = Z^T X, G2 = Z^T Z for X = P, Z = Psi (the first pass);
// nmat = 1: G0 = X^T X for X = E (the second pass, X given in FP64).
// Thread t owns the entries e = t, t + 256, ... < r * r; rows are staged in shared memory.
__device__ __forceinline__ void ny_gram_chunk(int rows, int r, const double* sx, const double* sz, int nmat,
                                              double (&g)[3][4]) {
  const int rr = r * r;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + q * NY_T;
    if (e < rr) {
      const int a = e / r, b = e - (e / r) * r;
      double x0 = 0.0, x1 = 0.0, x2 = 0.0;
      for (int i = 0; i < rows; ++i) {
        const double xb = sx[i * NY_LD + b];
        x0 = fma(sx[i * NY_LD + a], xb, x0);
        if (nmat == 3) {
          const double za = sz[i * NY_LD + a];
          x1 = fma(za, xb, x1);
          x2 = fma(za, sz[i * NY_LD + b], x2);
        }
      }
      g[0][q] += x0;
      g[1][q] += x1;
      g[2][q] += x2;
    }
  }
}

__device__ __forceinline__ void ny_store_parts(int r, int nmat, const double (&g)[3][4], double* parts) {
  const int rr = r * r;
  double* out = parts + (size_t)blockIdx.x * nmat * rr;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + q * NY_T;
    if (e < rr)
      for (int k = 0; k < nmat; ++k) out[k * rr + e] = g[k][q];
  }
}

// pass 1: partial G0 = P^T P, G1 = Psi^T P, G2 = Psi^T Psi
__global__ void __launch_bounds__(NY_T) k_ny_gram_sketch(int64_t n, int r, const float* __restrict__ P,
                                                         const float* __restrict__ Psi, double* __restrict__ parts) {
  __shared__ double sx[NY_ROWS * NY_LD], sz[NY_ROWS * NY_LD];
  double g[3][4] = {};
  for (int64_t base = (int64_t)blockIdx.x * NY_ROWS; base < n; base += (int64_t)gridDim.x * NY_ROWS) {
    const int rows = (n - base < NY_ROWS) ? (int)(n - base) : NY_ROWS;
    for (int t = threadIdx.x; t < rows * r; t += NY_T) {
      const int i = t / r, a = t - (t / r) * r;
      sx[i * NY_LD + a] = (double)P[base * r + t];
      sz[i * NY_LD + a] = (double)Psi[base * r + t];
    }
    __syncthreads();
    ny_gram_chunk(rows, r, sx, sz, 3, g);
    __syncthreads();
  }
  ny_store_parts(r, 3, g, parts);
}

// pass 2: E = (P + nu Psi) R^-1 (written, FP64) and partial G0 = E^T E
__global__ void __launch_bounds__(NY_T) k_ny_apply_rinv(int64_t n, int r, const float* __restrict__ P,
                                                        const float* __restrict__ Psi, const NyState* __restrict__ st,
                                                        double* __restrict__ E, double* __restrict__ parts) {
  __shared__ double sy[NY_ROWS * NY_LD], se[NY_ROWS * NY_LD];
  __shared__ double sR[NY_RMAX * NY_RMAX];
  for (int t = threadIdx.x; t < r * r; t += NY_T) sR[t] = st->Rinv[t];
  const double nu = st->nu;
  double g[3][4] = {};
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * NY_ROWS; base < n; base += (int64_t)gridDim.x * NY_ROWS) {
    const int rows = (n - base < NY_ROWS) ? (int)(n - base) : NY_ROWS;
    for (int t = threadIdx.x; t < rows * r; t += NY_T) {
      const int i = t / r, a = t - (t / r) * r;
      sy[i * NY_LD + a] = fma(nu, (double)Psi[base * r + t], (double)P[base * r + t]);
    }
    __syncthreads();
    // e_b = sum_{a <= b} y_a Rinv[a][b]
    for (int t = threadIdx.x; t < rows * r; t += NY_T) {
      const int i = t / r, b = t - (t / r) * r;
      double e = 0.0;
      for (int a = 0; a <= b; ++a) e = fma(sy[i * NY_LD + a], sR[a * r + b], e);
      se[i * NY_LD + b] = e;
      E[base * r + t] = e;
    }
    __syncthreads();
    ny_gram_chunk(rows, r, se, se, 1, g);
    __syncthreads();
  }
  ny_store_parts(r, 1, g, parts);
}

// pass 3: U = E M in place (row by row), and the sign bits of every row (bit k set when
// U[i, k] < 0)
__global__ void __launch_bounds__(NY_T) k_ny_apply_m(int64_t n, int r, const NyState* __restrict__ st,
                                                     double* __restrict__ EU, uint32_t* __restrict__ bits) {
  __shared__ double sM[NY_RMAX * NY_RMAX];
  for (int t = threadIdx.x; t < r * r; t += NY_T) sM[t] = st->M[t];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * NY_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * NY_T) {
    double e[NY_RMAX];
#pragma unroll
    for (int a = 0; a < NY_RMAX; ++a) e[a] = (a < r) ? EU[i * r + a] : 0.0;
    uint32_t bs = 0u;
    for (int k = 0; k < r; ++k) {
      double u = 0.0;
#pragma unroll
      for (int a = 0; a < NY_RMAX; ++a)
        if (a < r) u = fma(e[a], sM[a * r + k], u);
      EU[i * r + k] = u;
      if (u < 0.0) bs |= 1u << k;
    }
    bits[i] = bs;
  }
}

// pass 4: partial values v_k = sum_i z_ik (C z_k)_i over the CSR rows of C (scaled):
// diagonal entries add diagC[i], an off-diagonal entry adds +-valC[e] (+ when the two
// ends have the same sign in column k)
__global__ void __launch_bounds__(NY_T) k_ny_cut(int64_t n, int r, const int* __restrict__ rowptr,
                                                 const int* __restrict__ col, const double* __restrict__ valC,
                                                 const double* __restrict__ diagC, const uint32_t* __restrict__ bits,
                                                 double* __restrict__ parts) {
  __shared__ double red[NY_T / 32][NY_RMAX];
  double acc[NY_RMAX];
#pragma unroll
  for (int k = 0; k < NY_RMAX; ++k) acc[k] = 0.0;
  double dsum = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NY_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * NY_T) {
    dsum += diagC[i];
    const uint32_t bi = bits[i];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double v = valC[e];
      if (v == 0.0) continue;
      const uint32_t x = bi ^ bits[col[e]];
#pragma unroll
      for (int k = 0; k < NY_RMAX; ++k)
        if (k < r) acc[k] += ((x >> k) & 1u) ? -v : v;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NY_RMAX; ++k) {
    double s = acc[k] + dsum;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < r) {
    double s = 0.0;
    for (int w = 0; w < NY_T / 32; ++w) s += red[w][threadIdx.x];
    parts[(size_t)blockIdx.x * r + threadIdx.x] = s;
  }
}

// out[v] = sum over CTAs c (in order) of parts[c * nv + v]
__global__ void k_ny_reduce(const double* __restrict__ parts, int nparts, int nv, double* __restrict__ out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += parts[(size_t)c * nv + v];
    out[v] = s;
  }
}

// ---- single CTA: cyclic Jacobi on a symmetric m x m matrix (m even, m <= 32) ------------
// A (m x NY_LD) is diagonalised in place; V (m x NY_LD) receives the eigenvectors as
// columns.  Circle ordering: the m/2 rotations of a round act on disjoint pairs; their
// parameters are formed first, then every 2 x 2 block of A and every row of V is updated.
__device__ void ny_jacobi(double* A, double* V, int m) {
  __shared__ double cs[NY_RMAX / 2], sn[NY_RMAX / 2];
  __shared__ int pp[NY_RMAX / 2], qq[NY_RMAX / 2];
  __shared__ double wred[2][NY_T / 32];
  __shared__ int stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int half = m / 2;
  for (int t = tid; t < m * m; t += NY_T) V[(t / m) * NY_LD + t % m] = (t / m == t % m) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = tid; t < m * m; t += NY_T) {
      const int i = t / m, j = t % m;
      const double x = A[i * NY_LD + j];
      tot += x * x;
      if (i != j) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) { wred[0][warp] = off; wred[1][warp] = tot; }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, t2 = 0.0;
      for (int w = 0; w < NY_T / 32; ++w) { o2 += wred[0][w]; t2 += wred[1][w]; }
      stop = (o2 <= 1e-30 * t2) ? 1 : 0;
    }
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < m - 1; ++round) {
      if (tid < half) {
        const int k = tid;
        const int pa = k == 0 ? 0 : 1 + ((k - 1 + round) % (m - 1));
        const int pb = 1 + ((m - 1 - k - 1 + round) % (m - 1));
        const int p = min(pa, pb), q = max(pa, pb);
        pp[k] = p;
        qq[k] = q;
        const double apq = A[p * NY_LD + q], app = A[p * NY_LD + p], aqq = A[q * NY_LD + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (fabs(tau) > 1e150) ? 0.5 / tau
                           : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(tau * tau + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      const int nblk = half * half;
      for (int t = tid; t < nblk + m * half; t += NY_T) {
        if (t < nblk) {
          const int k1 = t / half, k2 = t % half;
          const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
          const double c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
          const double a = A[p1 * NY_LD + p2], b = A[p1 * NY_LD + q2];
          const double cc = A[q1 * NY_LD + p2], d = A[q1 * NY_LD + q2];
          const double ra = c1 * a - s1 * cc, rb = c1 * b - s1 * d;
          const double rc = s1 * a + c1 * cc, rd = s1 * b + c1 * d;
          A[p1 * NY_LD + p2] = c2 * ra - s2 * rb;
          A[p1 * NY_LD + q2] = s2 * ra + c2 * rb;
          A[q1 * NY_LD + p2] = c2 * rc - s2 * rd;
          A[q1 * NY_LD + q2] = s2 * rc + c2 * rd;
        } else {
          const int u = t - nblk;
          const int k = u / m, row = u % m;
          const double c = cs[k], s = sn[k];
          const int p = pp[k], q = qq[k];
          const double vp = V[row * NY_LD + p], vq = V[row * NY_LD + q];
          V[row * NY_LD + p] = c * vp - s * vq;
          V[row * NY_LD + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
}

// order[rank] = index for the diagonal of A (m entries) by descending value, ties by index
__device__ void ny_sort_desc(const double* A, int m, int* order) {
  const int tid = threadIdx.x;
  if (tid < m) {
    const double x = A[tid * NY_LD + tid];
    int rank = 0;
    for (int u = 0; u < m; ++u) {
      const double y = A[u * NY_LD + u];
      if (y > x || (y == x && u < tid)) ++rank;
    }
    order[rank] = tid;
  }
  __syncthreads();
}

// r x r core: ||P||_2 from G0, nu, B = G1 + nu G2 (symmetrised), its Cholesky factor and R^-1
__global__ void __launch_bounds__(NY_T) k_ny_core(int64_t n, int r, const double* __restrict__ G, NyState* st) {
  __shared__ double A[NY_RMAX * NY_LD], V[NY_RMAX * NY_LD];
  __shared__ double Rm[NY_RMAX * NY_RMAX];
  __shared__ int order[NY_RMAX];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int rr = r * r, m = r + (r & 1);
  // largest eigenvalue of G0 = P^T P (padded to an even size with a zero row and column)
  for (int t = tid; t < m * m; t += NY_T) {
    const int i = t / m, j = t % m;
    A[i * NY_LD + j] = (i < r && j < r) ? 0.5 * (G[i * r + j] + G[j * r + i]) : 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  ny_jacobi(A, V, m);
  ny_sort_desc(A, m, order);
  // nu = sqrt(n) * eps(||P||_2) with the FP32 spacing of the stored sketch,
  // eps(x) = 2^(e - 24) for x = f 2^e, f in [1/2, 1): the shift has to cover the
  // rounding of P itself, or Psi^T (P + nu Psi) comes out indefinite
  const double lmax = fmax(A[order[0] * NY_LD + order[0]], 0.0);
  const double normP = sqrt(lmax);
  int ex = 0;
  frexp(normP, &ex);
  const double nu = (normP > 0.0) ? sqrt((double)n) * ldexp(1.0, ex - 24) : 0.0;
  // B = G1 + nu G2, symmetrised, into Rm; then the upper Cholesky factor B = R^T R
  for (int t = tid; t < rr; t += NY_T) {
    const int i = t / r, j = t % r;
    const double bij = G[rr + i * r + j] + nu * G[2 * rr + i * r + j];
    const double bji = G[rr + j * r + i] + nu * G[2 * rr + j * r + i];
    Rm[t] = 0.5 * (bij + bji);
  }
  __syncthreads();
  if (tid < 32) {
    // column-by-column Cholesky (lane j owns column j of R): R[i][j] for i <= j
    const int lane = tid;
    double rc[NY_RMAX];
#pragma unroll
    for (int i = 0; i < NY_RMAX; ++i) rc[i] = 0.0;
    for (int j = 0; j < r; ++j) {
      double d = 0.0;
      if (lane == j) {
        d = Rm[j * r + j];
#pragma unroll
        for (int l = 0; l < NY_RMAX; ++l)
          if (l < j) d -= rc[l] * rc[l];
      }
      d = __shfl_sync(0xffffffffu, d, j);
      if (!(d > 0.0)) {
        if (lane == 0) bad = 1;
        break;
      }
      const double rjj = sqrt(d);
      double s = (lane > j && lane < r) ? Rm[j * r + lane] : 0.0;
#pragma unroll
      for (int l = 0; l < NY_RMAX; ++l) {
        if (l < j) {
          const double rlj = __shfl_sync(0xffffffffu, rc[l], j);
          s -= rlj * rc[l];
        }
      }
      if (lane == j) rc[j] = rjj;
      else if (lane > j && lane < r) rc[j] = s / rjj;
    }
    __syncwarp();
    // R^-1, column c by back substitution (lane c): R X = I, X upper triangular
    if (!bad && lane < r) {
      for (int i = 0; i < r; ++i) Rm[i * r + lane] = (i <= lane) ? rc[i] : 0.0;
    }
    __syncwarp();
    if (!bad && lane < r) {
      double x[NY_RMAX];
#pragma unroll
      for (int i = 0; i < NY_RMAX; ++i) x[i] = 0.0;
      const int c = lane;
      x[c] = 1.0 / Rm[c * r + c];
      for (int i = c - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1; l <= c; ++l) s += Rm[i * r + l] * x[l];
        x[i] = -s / Rm[i * r + i];
      }
      for (int i = 0; i < r; ++i) st->Rinv[i * r + c] = x[i];
    }
  }
  __syncthreads();
  if (tid == 0) {
    st->nu = nu;
    st->normP = normP;
    st->status = bad ? USBS_ENUMERIC : 0;
  }
}

// r x r decomposition: E^T E = W Sigma^2 W^T; lam = max(sigma^2 - nu, 0) by descending sigma; M = W Sigma^-1
__global__ void __launch_bounds__(NY_T) k_ny_svd(int r, const double* __restrict__ G, NyState* st) {
  __shared__ double A[NY_RMAX * NY_LD], V[NY_RMAX * NY_LD];
  __shared__ int order[NY_RMAX];
  const int tid = threadIdx.x;
  const int m = r + (r & 1);
  for (int t = tid; t < m * m; t += NY_T) {
    const int i = t / m, j = t % m;
    A[i * NY_LD + j] = (i < r && j < r) ? 0.5 * (G[i * r + j] + G[j * r + i]) : 0.0;
  }
  __syncthreads();
  ny_jacobi(A, V, m);
  ny_sort_desc(A, m, order);
  const double nu = st->nu;
  // the padded index (zero row and column) has eigenvalue 0 and sorts last among the
  // non-negative ones; only the first r ranks are kept
  for (int t = tid; t < r * r; t += NY_T) {
    const int a = t / r, k = t % r;
    const int o = order[k];
    const double s2 = A[o * NY_LD + o];
    st->M[a * r + k] = (s2 > 0.0) ? V[a * NY_LD + o] / sqrt(s2) : 0.0;
  }
  if (tid < r) {
    const int o = order[tid];
    st->lam[tid] = fmax(A[o * NY_LD + o] - nu, 0.0);
  }
}

__global__ void k_ny_signs(int64_t n, int k, const uint32_t* __restrict__ bits, int8_t* __restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = ((bits[i] >> k) & 1u) ? (int8_t)-1 : (int8_t)1;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace usbs

using namespace usbs;

extern "C" int usbs_nystrom_round(usbs_ctx* ctx, double* lam, double* U, double* values, int* best,
                                  int8_t* signs) {
  if (!ctx || !lam) return USBS_EINVAL;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  const int r = c->r;
  const int64_t n = c->n;
  if (r <= 0 || r > NY_RMAX) {
    c->err = "usbs_nystrom_round needs a sketch (0 < r <= 32)";
    return USBS_EINVAL;
  }
  const int rr = r * r;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + NY_ROWS - 1) / NY_ROWS, 2 * c->num_sms));
  const int gcut = (int)std::max<int64_t>(1, std::min<int64_t>((n + NY_T - 1) / NY_T, 4 * c->num_sms));
  DevBuf parts, G, EU, bits, st, vals, zb;
  USBS_CUDA_TRY(c, cudaMalloc(&parts.p, sizeof(double) * (size_t)std::max(grid, gcut) * 3 * rr));
  USBS_CUDA_TRY(c, cudaMalloc(&G.p, sizeof(double) * 3 * rr));
  USBS_CUDA_TRY(c, cudaMalloc(&EU.p, sizeof(double) * (size_t)n * r));
  USBS_CUDA_TRY(c, cudaMalloc(&bits.p, sizeof(uint32_t) * (size_t)n));
  USBS_CUDA_TRY(c, cudaMalloc(&st.p, sizeof(NyState)));
  USBS_CUDA_TRY(c, cudaMalloc(&vals.p, sizeof(double) * r));
  double* dparts = (double*)parts.p;
  double* dG = (double*)G.p;
  NyState* dst = (NyState*)st.p;
  {
    USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 8.0 * n * r);
    k_ny_gram_sketch<<<grid, NY_T, 0, c->stream>>>(n, r, c->P, c->Psi, dparts);
  }
  {
    USBS_LAUNCH(c, USBS_KIND_REDUCE);
    k_ny_reduce<<<(3 * rr + 255) / 256, 256, 0, c->stream>>>(dparts, grid, 3 * rr, dG);
  }
  {
    USBS_LAUNCH(c, USBS_KIND_SMALL);
    k_ny_core<<<1, NY_T, 0, c->stream>>>(n, r, dG, dst);
  }
  {
    USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 8.0 * n * r + 8.0 * n * r);
    k_ny_apply_rinv<<<grid, NY_T, 0, c->stream>>>(n, r, c->P, c->Psi, dst, (double*)EU.p, dparts);
  }
  {
    USBS_LAUNCH(c, USBS_KIND_REDUCE);
    k_ny_reduce<<<(rr + 255) / 256, 256, 0, c->stream>>>(dparts, grid, rr, dG);
  }
  {
    USBS_LAUNCH(c, USBS_KIND_SMALL);
    k_ny_svd<<<1, NY_T, 0, c->stream>>>(r, dG, dst);
  }
  {
    USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 16.0 * n * r + 4.0 * n);
    k_ny_apply_m<<<gcut, NY_T, 0, c->stream>>>(n, r, dst, (double*)EU.p, (uint32_t*)bits.p);
  }
  {
    USBS_LAUNCH_B(c, USBS_KIND_SKETCH, 12.0 * c->nnz_off + 4.0 * (n + 1) + 12.0 * n);
    k_ny_cut<<<gcut, NY_T, 0, c->stream>>>(n, r, c->rowptr, c->col, c->valC64, c->diagC64,
                                           (const uint32_t*)bits.p, dparts);
  }
  {
    USBS_LAUNCH(c, USBS_KIND_REDUCE);
    k_ny_reduce<<<1, 256, 0, c->stream>>>(dparts, gcut, r, (double*)vals.p);
  }
  USBS_TRY(check_launch(c, "nystrom"));
  NyState hst;
  std::vector<double> hv(r);
  USBS_CUDA_TRY(c, cudaMemcpyAsync(&hst, dst, sizeof(NyState), cudaMemcpyDeviceToHost, c->stream));
  USBS_CUDA_TRY(c, cudaMemcpyAsync(hv.data(), vals.p, sizeof(double) * r, cudaMemcpyDeviceToHost, c->stream));
  USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (hst.status != 0) {
    c->err = "Nystrom core matrix Psi^T (P + nu Psi) is not positive definite";
    return USBS_ENUMERIC;
  }
  // problem units: X = tau X_s, C = c_scale C_s
  for (int k = 0; k < r; ++k) lam[k] = hst.lam[k] * c->tau;
  int kb = 0;
  for (int k = 1; k < r; ++k)
    if (hv[k] > hv[kb]) kb = k;
  if (values)
    for (int k = 0; k < r; ++k) values[k] = hv[k] * c->c_scale;
  if (best) *best = kb;
  if (U) USBS_CUDA_TRY(c, cudaMemcpy(U, EU.p, sizeof(double) * (size_t)n * r, cudaMemcpyDeviceToHost));
  if (signs) {
    USBS_CUDA_TRY(c, cudaMalloc(&zb.p, (size_t)n));
    {
      USBS_LAUNCH(c, USBS_KIND_SKETCH);
      k_ny_signs<<<gcut, NY_T, 0, c->stream>>>(n, kb, (const uint32_t*)bits.p, (int8_t*)zb.p);
    }
    USBS_TRY(check_launch(c, "nystrom signs"));
    USBS_CUDA_TRY(c, cudaMemcpyAsync(signs, zb.p, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    USBS_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return USBS_OK;
}
