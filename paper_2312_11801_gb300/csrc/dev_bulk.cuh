// Device bodies of the bulk kernels of a USBS iteration: everything whose size grows
// with n, nnz or m.  T is the bulk type (float in mixed precision, double in plain
// FP64); reductions accumulate in T inside a CTA and in FP64 across CTAs.  A body takes
// its CTA index and CTA count as arguments: the __global__ kernels in bulk.cu pass
// blockIdx.x and gridDim.x, and the batched solver calls a body with (0, 1) so that one
// CTA covers every row and writes the final sums where the partials would go.
#pragma once

#include "common.cuh"

namespace usbs {
namespace {

constexpr float SQRT2F = 1.41421356237309504880f;

template <typename T> __device__ __forceinline__ T sqrt2_t();
template <> __device__ __forceinline__ float sqrt2_t<float>() { return SQRT2F; }
template <> __device__ __forceinline__ double sqrt2_t<double>() { return 1.41421356237309504880; }

template <typename T>
__device__ __forceinline__ void load8(const T* USBS_RESTRICT p, T (&v)[8]);
template <>
__device__ __forceinline__ void load8<float>(const float* USBS_RESTRICT p, float (&v)[8]) {
  float4 a = USBS_LDG(reinterpret_cast<const float4*>(p));
  float4 b = USBS_LDG(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void load8<double>(const double* USBS_RESTRICT p, double (&v)[8]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    double2 t = USBS_LDG(q + u);
    v[2 * u] = t.x; v[2 * u + 1] = t.y;
  }
}
template <typename T>
__device__ __forceinline__ void store8(T* USBS_RESTRICT p, const T (&v)[8]);
template <>
__device__ __forceinline__ void store8<float>(float* USBS_RESTRICT p, const float (&v)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void store8<double>(double* USBS_RESTRICT p, const double (&v)[8]) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int u = 0; u < 4; ++u) q[u] = make_double2(v[2 * u], v[2 * u + 1]);
}

__device__ __forceinline__ int bsvec_idx8(int p, int q) {  // p >= q
  return q * 8 - (q * (q - 1)) / 2 + (p - q);
}

// ---- operator setup: diag and effective off-diagonal values of C - A*(y) ------------------
template <typename T>
__device__ __forceinline__ void k_setup_diag_dev(const int cta, const int ncta, int n, const double* USBS_RESTRICT diagC, const int* USBS_RESTRICT dptr,
                             const int* USBS_RESTRICT dcon, const double* USBS_RESTRICT dval,
                             const double* USBS_RESTRICT y, T* USBS_RESTRICT dM) {
  for (int64_t i = (int64_t)cta * blockDim.x + threadIdx.x; i < n; i += (int64_t)ncta * blockDim.x) {
    double s = diagC[i];
    for (int e = dptr[i]; e < dptr[i + 1]; ++e) s -= y[dcon[e]] * dval[e];
    dM[i] = (T)s;
  }
}

template <typename T>
__device__ __forceinline__ void k_setup_off_dev(const int cta, const int ncta, int nnz, const double* USBS_RESTRICT valC, const int* USBS_RESTRICT sptr,
                            const int* USBS_RESTRICT scon, const double* USBS_RESTRICT sval,
                            const double* USBS_RESTRICT y, T* USBS_RESTRICT valM) {
  for (int s = cta * blockDim.x + threadIdx.x; s < nnz; s += ncta * blockDim.x) {
    double v = valC[s];
    for (int e = sptr[s]; e < sptr[s + 1]; ++e) v -= y[scon[e]] * sval[e];
    valM[s] = (T)v;
  }
}

// ---- Y = M X: CSR SpMM over an n x 8 block, diagonal shift fused ---------------------------
template <typename T>
__device__ __forceinline__ void k_spmm_dev(const int cta, const int ncta, int n, const int* USBS_RESTRICT rowptr,
                                              const int* USBS_RESTRICT col,
                                              const T* USBS_RESTRICT val, const T* USBS_RESTRICT d,
                                              const T* USBS_RESTRICT X, T* USBS_RESTRICT Y) {
  for (int64_t i = (int64_t)cta * blockDim.x + threadIdx.x; i < n; i += (int64_t)ncta * blockDim.x) {
    T x[8], acc[8];
    load8(X + (size_t)8 * i, x);
    const T di = d[i];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc[a] = di * x[a];
    const int s0 = rowptr[i], s1 = rowptr[i + 1];
    for (int s = s0; s < s1; ++s) {
      const int j = USBS_LDG(col + s);
      const T v = USBS_LDG(val + s);
      T xj[8];
      load8(X + (size_t)8 * j, xj);
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[a] += v * xj[a];
    }
    store8(Y + (size_t)8 * i, acc);
  }
}

// ---- g_c = svec(V^T A_c V) for one constraint -------------------------------------------
template <typename T>
__device__ __forceinline__ void build_g(int c, const int* USBS_RESTRICT con_ptr,
                                        const int* USBS_RESTRICT ent_i, const int* USBS_RESTRICT ent_j,
                                        const T* USBS_RESTRICT ent_v, const T* USBS_RESTRICT V,
                                        T (&g)[KSV]) {
#pragma unroll
  for (int u = 0; u < KSV; ++u) g[u] = (T)0;
  const int e0 = con_ptr[c], e1 = con_ptr[c + 1];
  for (int e = e0; e < e1; ++e) {
    const int i = ent_i[e], j = ent_j[e];
    const T hv = (T)0.5 * ent_v[e];
    T vi[8], vj[8];
    load8(V + (size_t)8 * i, vi);
    load8(V + (size_t)8 * j, vj);
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int p = q; p < 8; ++p) {
        T t = hv * (vi[p] * vj[q] + vj[p] * vi[q]);
        g[bsvec_idx8(p, q)] += (p == q) ? t : t * sqrt2_t<T>();
      }
  }
}

// ---- augmented Gram [G | A Xbar | w0]^T [G | A Xbar | w0] over all constraints ------------
// 40 x 40 upper-triangular in 4 x 4 tiles: 55 tiles x 16 = 880 values per CTA.
constexpr int GS_ROWS = 128;
template <typename T>
__device__ __forceinline__ void k_gstats_dev(const int cta, const int ncta, int m, const int* USBS_RESTRICT con_ptr,
                                                const int* USBS_RESTRICT ent_i,
                                                const int* USBS_RESTRICT ent_j,
                                                const T* USBS_RESTRICT ent_v, const T* USBS_RESTRICT V,
                                                const double* USBS_RESTRICT ax,
                                                const double* USBS_RESTRICT y,
                                                const double* USBS_RESTRICT b, double inv_rho,
                                                double* USBS_RESTRICT partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Gs = reinterpret_cast<T*>(smem_raw);                    // GS_ROWS x AUG
  double* dred = reinterpret_cast<double*>(smem_raw + sizeof(T) * GS_ROWS * AUG);  // 4 x 880
  const int tid = threadIdx.x;
  const int grp = tid / 55, tile = tid % 55;
  int ti = 0, tj = 0;
  {
    int t = tile;
    for (ti = 0; ti < 10; ++ti) {
      if (t < 10 - ti) { tj = ti + t; break; }
      t -= 10 - ti;
    }
  }
  const bool active = grp < 4;
  double dacc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) dacc[u] = 0.0;
  for (int64_t base = (int64_t)cta * GS_ROWS; base < m; base += (int64_t)ncta * GS_ROWS) {
    if (tid < GS_ROWS) {
      const int64_t c = base + tid;
      T* row = Gs + tid * AUG;
      if (c < m) {
        T g[KSV];
        build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
#pragma unroll
        for (int u = 0; u < KSV; ++u) row[u] = g[u];
        row[36] = (T)ax[c];
        row[37] = (T)(y[c] - b[c] * inv_rho);
      } else {
#pragma unroll
        for (int u = 0; u < 38; ++u) row[u] = (T)0;
      }
      row[38] = (T)0;
      row[39] = (T)0;
    }
    __syncthreads();
    if (active) {
      T acc[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] = (T)0;
      for (int r = grp; r < GS_ROWS; r += 4) {
        const T* row = Gs + r * AUG;
        T li[4], lj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { li[u] = row[ti * 4 + u]; lj[u] = row[tj * 4 + u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u * 4 + v] += li[u] * lj[v];
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) dacc[u] += (double)acc[u];
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int u = 0; u < 16; ++u) dred[grp * 880 + tile * 16 + u] = dacc[u];
  }
  __syncthreads();
  for (int t = tid; t < 880; t += blockDim.x) {
    double s = dred[t] + dred[880 + t] + dred[1760 + t] + dred[2640 + t];
    partials[(size_t)cta * PART_STRIDE + t] = s;
  }
}

// Block reduction of NV doubles per thread into partials[cta][0..NV).
template <int NV>
__device__ __forceinline__ void block_reduce_store(const int cta, double (&v)[NV], double* USBS_RESTRICT partials,
                                                   double* sred /* 8 x NV */) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < NV; ++u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int u = 0; u < NV; ++u) sred[warp * NV + u] = v[u];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NV; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w * NV + t];
    partials[(size_t)cta * PART_STRIDE + t] = s;
  }
}

// svec(S) for an 8 x 8 row-major FP64 matrix
__device__ __forceinline__ void svec8(const double* S, double* s) {
  for (int q = 0; q < 8; ++q)
    for (int p = q; p < 8; ++p)
      s[bsvec_idx8(p, q)] = (p == q) ? S[p * 8 + q] : 1.41421356237309504880 * S[p * 8 + q];
}

// Per-constraint products in the bulk type.  In FP32 the 36-term dot <g_c, svec S> is an
// FP32 dot product and the running sums of G^T w (one term per constraint of the thread)
// are compensated FP32 sums (Kahan summation): FP64-like accuracy for the sums while the
// FP64 pipe, a 64th of the FP32 rate on GB300, is left to the few scalars per constraint.
template <int NV>
struct KahanSums {
  float s[NV], c[NV];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int u = 0; u < NV; ++u) { s[u] = 0.f; c[u] = 0.f; }
  }
  __device__ __forceinline__ void add(int u, float x) {
    const float y = x - c[u];
    const float t = s[u] + y;
    c[u] = (t - s[u]) - y;
    s[u] = t;
  }
  __device__ __forceinline__ double value(int u) const { return (double)s[u] - (double)c[u]; }
};

template <typename T>
__device__ __forceinline__ double dot_svec(const T (&g)[KSV], const double* ssv, const float* ssf) {
  if constexpr (sizeof(T) == 4) {
    float z = 0.f;
#pragma unroll
    for (int u = 0; u < KSV; ++u) z = fmaf(g[u], ssf[u], z);
    return (double)z;
  } else {
    double z = 0.0;
#pragma unroll
    for (int u = 0; u < KSV; ++u) z += g[u] * ssv[u];
    return z;
  }
}

// ---- candidate: A X_{t+1} = eta A Xbar + G svec(S), y~ = proj_Y(y - (b - A X)/rho) -------
// partial layout: [0,36) G^T y~, 36 <b,y~>, 37 <A Xbar, y~>, 38 sum d^2, 39 max|d|
template <typename T>
__device__ __forceinline__ void k_xupdate_dev(const int cta, const int ncta, int m, const int* USBS_RESTRICT con_ptr,
                                                 const int* USBS_RESTRICT ent_i,
                                                 const int* USBS_RESTRICT ent_j,
                                                 const T* USBS_RESTRICT ent_v, const T* USBS_RESTRICT V,
                                                 const DevScalars* USBS_RESTRICT sc,
                                                 const double* USBS_RESTRICT ax,
                                                 const double* USBS_RESTRICT y,
                                                 const double* USBS_RESTRICT b,
                                                 const uint8_t* USBS_RESTRICT ineq, double inv_rho,
                                                 double* USBS_RESTRICT axnew,
                                                 double* USBS_RESTRICT ycand,
                                                 double* USBS_RESTRICT partials) {
  __shared__ double ssv[KSV];
  __shared__ float ssf[KSV];
  __shared__ double sred[8 * 39];
  __shared__ double smax[8];
  __shared__ int finite_ok;
  if (threadIdx.x == 0) {
    svec8(sc->S, ssv);
    int ok = isfinite(sc->eta);
    for (int u = 0; u < KSV; ++u) {
      ok &= isfinite(ssv[u]);
      ssf[u] = (float)ssv[u];
    }
    finite_ok = ok;
  }
  __syncthreads();
  // a non-finite subproblem solution must not reach the eigen solve: stay at y and let
  // the host report USBS_ENUMERIC from the status word
  const bool okS = finite_ok != 0;
  if (!okS && cta == 0 && threadIdx.x == 0) const_cast<DevScalars*>(sc)->status = USBS_ENUMERIC;
  const double eta = okS ? sc->eta : 1.0;
  double acc[39];
  double mx = 0.0;
#pragma unroll
  for (int u = 0; u < 39; ++u) acc[u] = 0.0;
  KahanSums<KSV> kg;
  kg.init();
  for (int64_t c = (int64_t)cta * blockDim.x + threadIdx.x; c < m; c += (int64_t)ncta * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    const double z = dot_svec<T>(g, ssv, ssf);
    const double axc = okS ? eta * ax[c] + z : ax[c];
    const double bc = b[c];
    double yc = okS ? y[c] - (bc - axc) * inv_rho : y[c];
    const bool iq = ineq[c] != 0;
    if (iq && yc < 0.0) yc = 0.0;
    axnew[c] = axc;
    ycand[c] = yc;
    if constexpr (sizeof(T) == 4) {
      const float ycf = (float)yc;
#pragma unroll
      for (int u = 0; u < KSV; ++u) kg.add(u, g[u] * ycf);
    } else {
#pragma unroll
      for (int u = 0; u < KSV; ++u) acc[u] += g[u] * yc;
    }
    acc[36] += bc * yc;
    acc[37] += ax[c] * yc;
    const double proj = iq ? fmin(axc, bc) : bc;
    const double dd = axc - proj;
    acc[38] += dd * dd;
    mx = fmax(mx, fabs(dd));
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int u = 0; u < KSV; ++u) acc[u] = kg.value(u);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smax[warp] = mx;
  block_reduce_store<39>(cta, acc, partials, sred);
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, smax[w]);
    partials[(size_t)cta * PART_STRIDE + 39] = m2;
  }
}

// ---- one alternating-maximisation pass (eq. dual_slack_update) ---------------------------
// A X~ = alpha (eta_hat A Xbar / tr Xbar + G svec(S_hat)); nu = proj_N(b - A X~ - rho y);
// w = y - (b - nu)/rho.  partials: [0,36) G^T w, 36 <A Xbar, w>, 37 sum (d nu)^2.
template <typename T>
__device__ __forceinline__ void k_alt_dev(const int cta, const int ncta, int m, const int* USBS_RESTRICT con_ptr,
                                             const int* USBS_RESTRICT ent_i,
                                             const int* USBS_RESTRICT ent_j,
                                             const T* USBS_RESTRICT ent_v, const T* USBS_RESTRICT V,
                                             const DevScalars* USBS_RESTRICT sc,
                                             const double* USBS_RESTRICT ax,
                                             const double* USBS_RESTRICT y,
                                             const double* USBS_RESTRICT b,
                                             const uint8_t* USBS_RESTRICT ineq, double rho,
                                             double alpha, double* USBS_RESTRICT nu,
                                             double* USBS_RESTRICT partials) {
  __shared__ double ssv[KSV];
  __shared__ float ssf[KSV];
  __shared__ double sred[8 * 38];
  if (threadIdx.x == 0) {
    svec8(sc->S_hat, ssv);
    for (int u = 0; u < KSV; ++u) ssf[u] = (float)ssv[u];
  }
  __syncthreads();
  const double coef = sc->has_eta ? sc->eta_hat / sc->tr : 0.0;
  const double inv_rho = 1.0 / rho;
  double acc[38];
#pragma unroll
  for (int u = 0; u < 38; ++u) acc[u] = 0.0;
  KahanSums<KSV> kg;
  kg.init();
  for (int64_t c = (int64_t)cta * blockDim.x + threadIdx.x; c < m; c += (int64_t)ncta * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    const double z = dot_svec<T>(g, ssv, ssf);
    const double axt = alpha * (coef * ax[c] + z);
    const double bc = b[c];
    double nn = 0.0;
    if (ineq[c]) nn = fmax(bc - axt - rho * y[c], 0.0);
    const double dn = nn - nu[c];
    nu[c] = nn;
    const double wc = y[c] - (bc - nn) * inv_rho;
    if constexpr (sizeof(T) == 4) {
      const float wcf = (float)wc;
#pragma unroll
      for (int u = 0; u < KSV; ++u) kg.add(u, g[u] * wcf);
    } else {
#pragma unroll
      for (int u = 0; u < KSV; ++u) acc[u] += g[u] * wc;
    }
    acc[36] += ax[c] * wc;
    acc[37] += dn * dn;
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int u = 0; u < KSV; ++u) acc[u] = kg.value(u);
  }
  block_reduce_store<38>(cta, acc, partials, sred);
}

// ---- z = A(V S V^T) --------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void k_constraint_eval_dev(const int cta, const int ncta, int m, const int* USBS_RESTRICT con_ptr, const int* USBS_RESTRICT ent_i,
                                  const int* USBS_RESTRICT ent_j, const T* USBS_RESTRICT ent_v,
                                  const T* USBS_RESTRICT V, const double* USBS_RESTRICT S,
                                  double* USBS_RESTRICT z) {
  __shared__ double ssv[KSV];
  __shared__ float ssf[KSV];
  if (threadIdx.x == 0) {
    svec8(S, ssv);
    for (int u = 0; u < KSV; ++u) ssf[u] = (float)ssv[u];
  }
  __syncthreads();
  for (int64_t c = (int64_t)cta * blockDim.x + threadIdx.x; c < m; c += (int64_t)ncta * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    z[c] = dot_svec<T>(g, ssv, ssf);
  }
}

// ---- past information (k_p > 0) ------------------------------------------------------------
// A Xbar_{t+1} = eta A Xbar_t + A(V S_c V^T) (eq. x_bar_def through the constraint values,
// App. C): out[c] = eta ax[c] + <g_c, svec S_c>, eta read from the device scalars.
template <typename T>
__device__ __forceinline__ void k_constraint_axpy_dev(const int cta, const int ncta, int m, const int* USBS_RESTRICT con_ptr,
                                                      const int* USBS_RESTRICT ent_i, const int* USBS_RESTRICT ent_j,
                                                      const T* USBS_RESTRICT ent_v, const T* USBS_RESTRICT V,
                                                      const double* USBS_RESTRICT S, const double* USBS_RESTRICT eta_dev,
                                                      const double* USBS_RESTRICT ax, double* USBS_RESTRICT out) {
  __shared__ double ssv[KSV];
  __shared__ float ssf[KSV];
  if (threadIdx.x == 0) {
    svec8(S, ssv);
    for (int u = 0; u < KSV; ++u) ssf[u] = (float)ssv[u];
  }
  __syncthreads();
  const double eta = *eta_dev;
  for (int64_t c = (int64_t)cta * blockDim.x + threadIdx.x; c < m; c += (int64_t)ncta * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    out[c] = eta * ax[c] + dot_svec<T>(g, ssv, ssf);
  }
}

// W = [V Q_p | v_1 .. v_kc | 0] row by row (eq. v_next_def before its QR): the k_p past
// columns V Q_p (Q_p: 8 x 8 FP64, its first k_p columns), then the first k_c Ritz vectors
// at the candidate, then zeros.
template <typename T>
__device__ __forceinline__ void k_vnext_dev(const int cta, const int ncta, int n, const T* USBS_RESTRICT V,
                                            const double* USBS_RESTRICT Qp, const T* USBS_RESTRICT U,
                                            int kp, int kc, T* USBS_RESTRICT W) {
  __shared__ T qs[64];
  if (threadIdx.x < 64) qs[threadIdx.x] = (T)Qp[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)cta * blockDim.x + threadIdx.x; i < n; i += (int64_t)ncta * blockDim.x) {
    T v[8], u[8], w[8];
    load8(V + 8 * i, v);
    load8(U + 8 * i, u);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      T acc = (T)0;
      if (a < kp) {
#pragma unroll
        for (int b = 0; b < 8; ++b) acc += v[b] * qs[b * 8 + a];
      } else if (a < kp + kc) {
#pragma unroll
        for (int b = 0; b < 8; ++b)
          if (b == a - kp) acc = u[b];
      }
      w[a] = acc;
    }
    store8(W + 8 * i, w);
  }
}

// ---- B = V^T Psi (8 x r) ------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void k_vt_psi_dev(const int cta, const int ncta, int n, int r, const T* USBS_RESTRICT V,
                                                const float* USBS_RESTRICT Psi,
                                                double* USBS_RESTRICT partials) {
  __shared__ float red[8][8 * RMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  float acc[RMAX];
#pragma unroll
  for (int s = 0; s < RMAX; ++s) acc[s] = 0.f;
  for (int64_t base = ((int64_t)cta * 8 + warp) * 4; base < n; base += (int64_t)ncta * 32) {
    const int64_t i = base + rr;
    if (i < n) {
      const float v = (float)V[(size_t)8 * i + a];
      const float* pr = Psi + (size_t)r * i;
#pragma unroll
      for (int s = 0; s < RMAX; ++s)
        if (s < r) acc[s] += v * USBS_LDG(pr + s);
    }
  }
#pragma unroll
  for (int s = 0; s < RMAX; ++s) {
    if (s < r) {
      acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 8);
      acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 16);
    }
  }
  if (rr == 0) {
#pragma unroll
    for (int s = 0; s < RMAX; ++s)
      if (s < r) red[warp][a * r + s] = acc[s];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * r; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += (double)red[w][t];
    partials[(size_t)cta * PART_STRIDE + t] = s;
  }
}

// ---- P <- eta P + V (S B) ----------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void k_sketch_update_dev(const int cta, const int ncta, int n, int r, const T* USBS_RESTRICT V,
                                                       const double* USBS_RESTRICT S,
                                                       const double* USBS_RESTRICT Bsk,
                                                       float* USBS_RESTRICT P,
                                                       const double* USBS_RESTRICT eta_dev,
                                                       double eta_host) {
  __shared__ float Cm[8 * RMAX];
  for (int t = threadIdx.x; t < 8 * r; t += blockDim.x) {
    const int a = t / r, s = t % r;
    double v = 0.0;
    for (int c = 0; c < 8; ++c) v += S[a * 8 + c] * Bsk[c * r + s];
    Cm[t] = (float)v;
  }
  __syncthreads();
  const float eta = (float)(eta_dev ? *eta_dev : eta_host);
  const size_t total = (size_t)n * r;
  for (size_t t = (size_t)cta * blockDim.x + threadIdx.x; t < total;
       t += (size_t)ncta * blockDim.x) {
    const size_t i = t / r;
    const int s = (int)(t % r);
    T vi[8];
    load8(V + 8 * i, vi);
    float acc = eta * P[t];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc += (float)vi[a] * Cm[a * r + s];
    P[t] = acc;
  }
}

// Sum of per-CTA partials, fixed order: a block owns 32 outputs; warp w adds partials
// w, w + 8, ... (coalesced 256-byte rows), then the 8 warp sums are added in order.
__device__ __forceinline__ void k_reduce_dev(const int cta, const int ncta, const double* USBS_RESTRICT partials, int nparts,
                                                int nvals, double* USBS_RESTRICT out,
                                                const int* USBS_RESTRICT mask) {
  if (mask && *mask == 0) return;
  __shared__ double ws[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = cta * 32 + lane;
  double s = 0.0;
  if (t < nvals) {
    int p = warp;
    for (; p + 24 < nparts; p += 32) {
      const double a0 = partials[(size_t)p * PART_STRIDE + t];
      const double a1 = partials[(size_t)(p + 8) * PART_STRIDE + t];
      const double a2 = partials[(size_t)(p + 16) * PART_STRIDE + t];
      const double a3 = partials[(size_t)(p + 24) * PART_STRIDE + t];
      s += a0; s += a1; s += a2; s += a3;
    }
    for (; p < nparts; p += 8) s += partials[(size_t)p * PART_STRIDE + t];
  }
  ws[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && t < nvals) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += ws[w][lane];
    out[t] = tot;
  }
}

// max-reduce one slot (used for the infinity norm)
__device__ __forceinline__ void k_reduce_max_dev(const int cta, const int ncta, const double* USBS_RESTRICT partials, int nparts, int slot,
                             double* USBS_RESTRICT out) {
  if (threadIdx.x != 0 || cta != 0) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s = fmax(s, partials[(size_t)p * PART_STRIDE + slot]);
  *out = s;
}

}  // namespace
}  // namespace usbs
