// Bulk kernels of one USBS iteration: everything whose size grows with n, nnz or m.
// T is the bulk type: float (mixed precision) or double (plain FP64).  Reductions
// accumulate in T inside a CTA and in FP64 across CTAs, in a fixed order.
//
// Row kernels use one warp per 4 rows: lane L works on row (L >> 3) and on column
// a = L & 7 of an n x 8 row-major block, so the 8 lanes of a row read one 32-byte
// (float) or 64-byte (double) row segment together.
#include <mutex>

#include "common.cuh"

namespace usbs {

namespace {

constexpr float SQRT2F = 1.41421356237309504880f;

template <typename T> __device__ __forceinline__ T sqrt2_t();
template <> __device__ __forceinline__ float sqrt2_t<float>() { return SQRT2F; }
template <> __device__ __forceinline__ double sqrt2_t<double>() { return 1.41421356237309504880; }

template <typename T>
__device__ __forceinline__ void load8(const T* __restrict__ p, T (&v)[8]);
template <>
__device__ __forceinline__ void load8<float>(const float* __restrict__ p, float (&v)[8]) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void load8<double>(const double* __restrict__ p, double (&v)[8]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    double2 t = __ldg(q + u);
    v[2 * u] = t.x; v[2 * u + 1] = t.y;
  }
}
template <typename T>
__device__ __forceinline__ void store8(T* __restrict__ p, const T (&v)[8]);
template <>
__device__ __forceinline__ void store8<float>(float* __restrict__ p, const float (&v)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void store8<double>(double* __restrict__ p, const double (&v)[8]) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int u = 0; u < 4; ++u) q[u] = make_double2(v[2 * u], v[2 * u + 1]);
}

// counter-based uniform(-1, 1) from a 64-bit mix (splitmix64 finaliser)
__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t row, uint64_t col) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (row * 16 + col + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__device__ __forceinline__ int svec_idx8(int p, int q) {  // p >= q
  return q * 8 - (q * (q - 1)) / 2 + (p - q);
}

// ---- operator setup: diag and effective off-diagonal values of C - A*(y) ------------------
template <typename T>
__global__ void k_setup_diag(int n, const double* __restrict__ diagC, const int* __restrict__ dptr,
                             const int* __restrict__ dcon, const double* __restrict__ dval,
                             const double* __restrict__ y, T* __restrict__ dM) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = diagC[i];
    for (int e = dptr[i]; e < dptr[i + 1]; ++e) s -= y[dcon[e]] * dval[e];
    dM[i] = (T)s;
  }
}

template <typename T>
__global__ void k_setup_off(int nnz, const double* __restrict__ valC, const int* __restrict__ sptr,
                            const int* __restrict__ scon, const double* __restrict__ sval,
                            const double* __restrict__ y, T* __restrict__ valM) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nnz; s += gridDim.x * blockDim.x) {
    double v = valC[s];
    for (int e = sptr[s]; e < sptr[s + 1]; ++e) v -= y[scon[e]] * sval[e];
    valM[s] = (T)v;
  }
}

// ---- Y = M X: CSR SpMM over an n x 8 block, diagonal shift fused ---------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_spmm(int n, const int* __restrict__ rowptr,
                                              const int* __restrict__ col,
                                              const T* __restrict__ val, const T* __restrict__ d,
                                              const T* __restrict__ X, T* __restrict__ Y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T x[8], acc[8];
    load8(X + (size_t)8 * i, x);
    const T di = d[i];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc[a] = di * x[a];
    const int s0 = rowptr[i], s1 = rowptr[i + 1];
    for (int s = s0; s < s1; ++s) {
      const int j = __ldg(col + s);
      const T v = __ldg(val + s);
      T xj[8];
      load8(X + (size_t)8 * j, xj);
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[a] += v * xj[a];
    }
    store8(Y + (size_t)8 * i, acc);
  }
}

// Reduce a per-lane array over the 4 row-lanes of a warp (lanes with equal L & 7).
template <typename T, int N>
__device__ __forceinline__ void reduce_rowlanes(T (&v)[N]) {
#pragma unroll
  for (int u = 0; u < N; ++u) {
    v[u] += __shfl_xor_sync(0xffffffffu, v[u], 8);
    v[u] += __shfl_xor_sync(0xffffffffu, v[u], 16);
  }
}

// ---- H_blk = Q_blk^T W for blk < nb (first Gram-Schmidt projection) ----------------------
template <typename T>
__global__ void __launch_bounds__(256) k_proj(int n, const T* __restrict__ Q, size_t bstride, int nb,
                                              const T* __restrict__ W, double* __restrict__ partials,
                                              const int* __restrict__ mask) {
  if (mask && *mask == 0) return;
  __shared__ T red[8][8 * 64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  T acc[8][8];
#pragma unroll
  for (int b = 0; b < 8; ++b)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[b][c] = (T)0;
  for (int base = (blockIdx.x * 8 + warp) * 4; base < n; base += gridDim.x * 32) {
    const int i = base + rr;
    if (i < n) {
      T w[8];
      load8(W + (size_t)8 * i, w);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (b < nb) {
          const T q = Q[b * bstride + (size_t)8 * i + a];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[b][c] += q * w[c];
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < nb) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        acc[b][c] += __shfl_xor_sync(0xffffffffu, acc[b][c], 8);
        acc[b][c] += __shfl_xor_sync(0xffffffffu, acc[b][c], 16);
      }
      if (rr == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) red[warp][b * 64 + a * 8 + c] = acc[b][c];
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nb * 64; t += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += (double)red[w][t];
    partials[(size_t)blockIdx.x * PART_STRIDE + t] = s;
  }
}

// ---- W <- W - Q H; then H2 = Q^T W and G = W^T W (second pass + Gram) ---------------------
template <typename T>
__global__ void __launch_bounds__(256) k_update_proj(int n, const T* __restrict__ Q, size_t bstride,
                                                     int nb, T* __restrict__ W,
                                                     const double* __restrict__ Hred,
                                                     double* __restrict__ partials,
                                                     const int* __restrict__ mask) {
  if (mask && *mask == 0) return;
  __shared__ T Hs[8 * 64];
  __shared__ T red[8][8 * 64 + 64];
  for (int t = threadIdx.x; t < nb * 64; t += blockDim.x) Hs[t] = (T)Hred[t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  T acc[8][8], gram[8];
#pragma unroll
  for (int b = 0; b < 8; ++b)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[b][c] = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) gram[c] = (T)0;
  for (int base = (blockIdx.x * 8 + warp) * 4; base < n; base += gridDim.x * 32) {
    const int i = base + rr;
    const bool ok = i < n;
    T x = ok ? W[(size_t)8 * i + a] : (T)0;
    T qa[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      qa[b] = (T)0;
      if (b < nb && ok) {
        T q[8];
        load8(Q + b * bstride + (size_t)8 * i, q);
        qa[b] = q[a];
#pragma unroll
        for (int ap = 0; ap < 8; ++ap) x -= q[ap] * Hs[b * 64 + ap * 8 + a];
      }
    }
    T xr[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xr[c] = __shfl_sync(0xffffffffu, x, (lane & ~7) | c);
    if (ok) {
      W[(size_t)8 * i + a] = x;
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (b < nb) {
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[b][c] += qa[b] * xr[c];
        }
#pragma unroll
      for (int c = 0; c < 8; ++c) gram[c] += x * xr[c];
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < nb) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        acc[b][c] += __shfl_xor_sync(0xffffffffu, acc[b][c], 8);
        acc[b][c] += __shfl_xor_sync(0xffffffffu, acc[b][c], 16);
      }
      if (rr == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) red[warp][b * 64 + a * 8 + c] = acc[b][c];
      }
    }
  }
  reduce_rowlanes<T, 8>(gram);
  if (rr == 0) {
#pragma unroll
    for (int c = 0; c < 8; ++c) red[warp][512 + a * 8 + c] = gram[c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 576; t += blockDim.x) {
    if (t < 512 && t >= nb * 64) continue;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += (double)red[w][t];
    partials[(size_t)blockIdx.x * PART_STRIDE + t] = s;
  }
}

// ---- out = (W - Q H2) R^-1, deficient columns replaced by random vectors ------------------
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(int n, const T* __restrict__ Q, size_t bstride,
                                                  int nb, const T* W, const double* __restrict__ H2red,
                                                  const DevLanczos* __restrict__ lz, T* out,
                                                  const int* __restrict__ mask, uint64_t seed,
                                                  const int* __restrict__ deficient) {
  if (mask && *mask == 0) return;
  __shared__ T Hs[8 * 64];
  __shared__ T Ri[64];
  __shared__ int dfc[8];
  for (int t = threadIdx.x; t < nb * 64; t += blockDim.x) Hs[t] = (T)H2red[t];
  if (threadIdx.x < 64) Ri[threadIdx.x] = (T)lz->Rinv[threadIdx.x];
  if (threadIdx.x < 8) dfc[threadIdx.x] = deficient[threadIdx.x];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  for (int base = (blockIdx.x * 8 + warp) * 4; base < n; base += gridDim.x * 32) {
    const int i = base + rr;
    const bool ok = i < n;
    T x = ok ? W[(size_t)8 * i + a] : (T)0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < nb && ok) {
        T q[8];
        load8(Q + b * bstride + (size_t)8 * i, q);
#pragma unroll
        for (int ap = 0; ap < 8; ++ap) x -= q[ap] * Hs[b * 64 + ap * 8 + a];
      }
    }
    T xr[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xr[c] = __shfl_sync(0xffffffffu, x, (lane & ~7) | c);
    T o = (T)0;
#pragma unroll
    for (int c = 0; c < 8; ++c) o += xr[c] * Ri[c * 8 + a];
    if (dfc[a]) o = (T)hash_uniform(seed, (uint64_t)i, (uint64_t)a);
    if (ok) out[(size_t)8 * i + a] = o;
  }
}

// ---- out[ob] = Q[:, :J] Y[:, 8 ob : 8 ob + 8] (thick restart / Ritz vectors) ---------------
template <typename T>
__global__ void __launch_bounds__(256) k_restart_gemm(int n, const T* __restrict__ Q, size_t bstride,
                                                      int J, int nout, const double* __restrict__ Y,
                                                      T* __restrict__ out, size_t ostride,
                                                      const T* __restrict__ resid, int resid_slot) {
  __shared__ T Ys[JMAX * 32];
  const int ncol = nout * 8;
  for (int t = threadIdx.x; t < J * ncol; t += blockDim.x) {
    const int l = t / ncol, cc = t % ncol;
    Ys[t] = (T)Y[l * JMAX + cc];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  const int nbk = J / 8;
  for (int base = (blockIdx.x * 8 + warp) * 4; base < n; base += gridDim.x * 32) {
    const int i = base + rr;
    if (i >= n) continue;
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
    for (int b = 0; b < nbk; ++b) {
      T q[8];
      load8(Q + b * bstride + (size_t)8 * i, q);
#pragma unroll
      for (int ap = 0; ap < 8; ++ap) {
        const int l = b * 8 + ap;
#pragma unroll
        for (int o = 0; o < 4; ++o)
          if (o < nout) acc[o] += q[ap] * Ys[l * ncol + o * 8 + a];
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o)
      if (o < nout) out[o * ostride + (size_t)8 * i + a] = acc[o];
    if (resid) out[resid_slot * ostride + (size_t)8 * i + a] = resid[(size_t)8 * i + a];
  }
}

// ---- g_c = svec(V^T A_c V) for one constraint -------------------------------------------
template <typename T>
__device__ __forceinline__ void build_g(int c, const int* __restrict__ con_ptr,
                                        const int* __restrict__ ent_i, const int* __restrict__ ent_j,
                                        const T* __restrict__ ent_v, const T* __restrict__ V,
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
        g[svec_idx8(p, q)] += (p == q) ? t : t * sqrt2_t<T>();
      }
  }
}

// ---- augmented Gram [G | A Xbar | w0]^T [G | A Xbar | w0] over all constraints ------------
// 40 x 40 upper-triangular in 4 x 4 tiles: 55 tiles x 16 = 880 values per CTA.
constexpr int GS_ROWS = 128;
template <typename T>
__global__ void __launch_bounds__(256) k_gstats(int m, const int* __restrict__ con_ptr,
                                                const int* __restrict__ ent_i,
                                                const int* __restrict__ ent_j,
                                                const T* __restrict__ ent_v, const T* __restrict__ V,
                                                const double* __restrict__ ax,
                                                const double* __restrict__ y,
                                                const double* __restrict__ b, double inv_rho,
                                                double* __restrict__ partials) {
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
  for (int base = blockIdx.x * GS_ROWS; base < m; base += gridDim.x * GS_ROWS) {
    if (tid < GS_ROWS) {
      const int c = base + tid;
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
    partials[(size_t)blockIdx.x * PART_STRIDE + t] = s;
  }
}

// Block reduction of NV doubles per thread into partials[blockIdx][0..NV).
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* __restrict__ partials,
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
    partials[(size_t)blockIdx.x * PART_STRIDE + t] = s;
  }
}

// svec(S) for an 8 x 8 row-major FP64 matrix
__device__ __forceinline__ void svec8(const double* S, double* s) {
  for (int q = 0; q < 8; ++q)
    for (int p = q; p < 8; ++p)
      s[svec_idx8(p, q)] = (p == q) ? S[p * 8 + q] : 1.41421356237309504880 * S[p * 8 + q];
}

// ---- candidate: A X_{t+1} = eta A Xbar + G svec(S), y~ = proj_Y(y - (b - A X)/rho) -------
// partial layout: [0,36) G^T y~, 36 <b,y~>, 37 <A Xbar, y~>, 38 sum d^2, 39 max|d|
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
  __shared__ double ssv[KSV];
  __shared__ double sred[8 * 39];
  __shared__ double smax[8];
  __shared__ int finite_ok;
  if (threadIdx.x == 0) {
    svec8(sc->S, ssv);
    int ok = isfinite(sc->eta);
    for (int u = 0; u < KSV; ++u) ok &= isfinite(ssv[u]);
    finite_ok = ok;
  }
  __syncthreads();
  // a non-finite subproblem solution must not reach the eigen solve: stay at y and let
  // the host report USBS_ENUMERIC from the status word
  const bool okS = finite_ok != 0;
  if (!okS && blockIdx.x == 0 && threadIdx.x == 0) const_cast<DevScalars*>(sc)->status = USBS_ENUMERIC;
  const double eta = okS ? sc->eta : 1.0;
  double acc[39];
  double mx = 0.0;
#pragma unroll
  for (int u = 0; u < 39; ++u) acc[u] = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    double z = 0.0;
#pragma unroll
    for (int u = 0; u < KSV; ++u) z += (double)g[u] * ssv[u];
    const double axc = okS ? eta * ax[c] + z : ax[c];
    const double bc = b[c];
    double yc = okS ? y[c] - (bc - axc) * inv_rho : y[c];
    const bool iq = ineq[c] != 0;
    if (iq && yc < 0.0) yc = 0.0;
    axnew[c] = axc;
    ycand[c] = yc;
#pragma unroll
    for (int u = 0; u < KSV; ++u) acc[u] += (double)g[u] * yc;
    acc[36] += bc * yc;
    acc[37] += ax[c] * yc;
    const double proj = iq ? fmin(axc, bc) : bc;
    const double dd = axc - proj;
    acc[38] += dd * dd;
    mx = fmax(mx, fabs(dd));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smax[warp] = mx;
  block_reduce_store<39>(acc, partials, sred);
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, smax[w]);
    partials[(size_t)blockIdx.x * PART_STRIDE + 39] = m2;
  }
}

// ---- one alternating-maximisation pass (eq. dual_slack_update) ---------------------------
// A X~ = alpha (eta_hat A Xbar / tr Xbar + G svec(S_hat)); nu = proj_N(b - A X~ - rho y);
// w = y - (b - nu)/rho.  partials: [0,36) G^T w, 36 <A Xbar, w>, 37 sum (d nu)^2.
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
  __shared__ double ssv[KSV];
  __shared__ double sred[8 * 38];
  if (threadIdx.x == 0) svec8(sc->S_hat, ssv);
  __syncthreads();
  const double coef = sc->has_eta ? sc->eta_hat / sc->tr : 0.0;
  const double inv_rho = 1.0 / rho;
  double acc[38];
#pragma unroll
  for (int u = 0; u < 38; ++u) acc[u] = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    double z = 0.0;
#pragma unroll
    for (int u = 0; u < KSV; ++u) z += (double)g[u] * ssv[u];
    const double axt = alpha * (coef * ax[c] + z);
    const double bc = b[c];
    double nn = 0.0;
    if (ineq[c]) nn = fmax(bc - axt - rho * y[c], 0.0);
    const double dn = nn - nu[c];
    nu[c] = nn;
    const double wc = y[c] - (bc - nn) * inv_rho;
#pragma unroll
    for (int u = 0; u < KSV; ++u) acc[u] += (double)g[u] * wc;
    acc[36] += ax[c] * wc;
    acc[37] += dn * dn;
  }
  block_reduce_store<38>(acc, partials, sred);
}

// ---- z = A(V S V^T) --------------------------------------------------------------------
template <typename T>
__global__ void k_constraint_eval(int m, const int* __restrict__ con_ptr, const int* __restrict__ ent_i,
                                  const int* __restrict__ ent_j, const T* __restrict__ ent_v,
                                  const T* __restrict__ V, const double* __restrict__ S,
                                  double* __restrict__ z) {
  __shared__ double ssv[KSV];
  if (threadIdx.x == 0) svec8(S, ssv);
  __syncthreads();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    T g[KSV];
    build_g<T>(c, con_ptr, ent_i, ent_j, ent_v, V, g);
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < KSV; ++u) s += (double)g[u] * ssv[u];
    z[c] = s;
  }
}

// ---- B = V^T Psi (8 x r) ------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_vt_psi(int n, int r, const T* __restrict__ V,
                                                const float* __restrict__ Psi,
                                                double* __restrict__ partials) {
  __shared__ float red[8][8 * RMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  float acc[RMAX];
#pragma unroll
  for (int s = 0; s < RMAX; ++s) acc[s] = 0.f;
  for (int base = (blockIdx.x * 8 + warp) * 4; base < n; base += gridDim.x * 32) {
    const int i = base + rr;
    if (i < n) {
      const float v = (float)V[(size_t)8 * i + a];
      const float* pr = Psi + (size_t)r * i;
#pragma unroll
      for (int s = 0; s < RMAX; ++s)
        if (s < r) acc[s] += v * __ldg(pr + s);
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
    partials[(size_t)blockIdx.x * PART_STRIDE + t] = s;
  }
}

// ---- P <- eta P + V (S B) ----------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sketch_update(int n, int r, const T* __restrict__ V,
                                                       const double* __restrict__ S,
                                                       const double* __restrict__ Bsk,
                                                       float* __restrict__ P,
                                                       const double* __restrict__ eta_dev,
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
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
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
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nparts,
                                                int nvals, double* __restrict__ out,
                                                const int* __restrict__ mask) {
  if (mask && *mask == 0) return;
  __shared__ double ws[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 32 + lane;
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
__global__ void k_reduce_max(const double* __restrict__ partials, int nparts, int slot,
                             double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s = fmax(s, partials[(size_t)p * PART_STRIDE + slot]);
  *out = s;
}

}  // namespace

// =========================================================================================
int red_grid(Ctx* c, int64_t rows, int rows_per_cta) {
  int64_t g = (rows + rows_per_cta - 1) / rows_per_cta;
  if (g < 1) g = 1;
  if (g > RED_GRID_MAX) g = RED_GRID_MAX;
  return (int)g;
}

void reduce_partials(Ctx* c, int nparts, int nvals, double* out, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REDUCE, mask ? 0.0 : 8.0 * nvals * (nparts + 1));
  k_reduce<<<(nvals + 31) / 32, 256, 0, c->stream>>>(c->partials, nparts, nvals, out, mask);
}

// CTAs for kernels whose CTA covers 32 rows per iteration (8 warps x 4 rows)
static int row32_grid(Ctx* c, int64_t n) {
  int64_t g = (n + 31) / 32;
  const int64_t cap = (int64_t)c->num_sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
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
void Bulk<T>::proj(Ctx* c, const void* Qb, int nb, const void* W, int nparts, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 1));
  k_proj<T><<<nparts, 256, 0, c->stream>>>((int)c->n, (const T*)Qb, (size_t)c->n * 8, nb,
                                             (const T*)W, c->partials, mask);
}

template <typename T>
void Bulk<T>::update_proj(Ctx* c, const void* Qb, int nb, void* W, int nparts, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 2));
  k_update_proj<T><<<nparts, 256, 0, c->stream>>>((int)c->n, (const T*)Qb, (size_t)c->n * 8, nb,
                                                    (T*)W, c->red + RED_H, c->partials, mask);
}

template <typename T>
void Bulk<T>::finalize(Ctx* c, const void* Qb, int nb, const void* W, void* out, int nparts,
                       const int* mask, uint64_t seed) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 2));
  (void)nparts;
  k_finalize<T><<<row32_grid(c, c->n), 256, 0, c->stream>>>(
      (int)c->n, (const T*)Qb, (size_t)c->n * 8, nb, (const T*)W, c->red + RED_H2, c->lz,
      (T*)out, mask, seed, DEV_FIELD(c->lz, DevLanczos, dcol, int));
}

template <typename T>
void Bulk<T>::restart_gemm(Ctx* c, const void* Qb, int J, int nout_blocks, const double* Y,
                           void* out, const void* resid, int resid_slot) {
  USBS_LAUNCH_B(c, USBS_KIND_RESTART, 8.0 * sizeof(T) * c->n * (J / 8 + nout_blocks + (resid ? 2 : 0)));
  k_restart_gemm<T><<<row32_grid(c, c->n), 256, 0, c->stream>>>(
      (int)c->n, (const T*)Qb, (size_t)c->n * 8, J, nout_blocks, Y, (T*)out, (size_t)c->n * 8,
      (const T*)resid, resid_slot);
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
void Bulk<T>::gram_xy(Ctx* c, const void* X, const void* Y, int nparts) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, 16.0 * sizeof(T) * c->n);
  k_proj<T><<<nparts, 256, 0, c->stream>>>((int)c->n, (const T*)X, (size_t)c->n * 8, 1,
                                             (const T*)Y, c->partials, nullptr);
}

void reduce_max_slot(Ctx* c, int nparts, int slot, double* out) {
  USBS_LAUNCH(c, USBS_KIND_REDUCE);
  k_reduce_max<<<1, 32, 0, c->stream>>>(c->partials, nparts, slot, out);
}

template struct Bulk<float>;
template struct Bulk<double>;

}  // namespace usbs
