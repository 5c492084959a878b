// Device bodies of the k-sized single-CTA kernels of a USBS iteration (FP64 unless
// stated): Cholesky-QR of a Lanczos block with deflation, Rayleigh-Ritz by parallel
// Jacobi, the App. B.2 interior point method, and the model value, descent test and
// gates.  Each __global__ kernel in small.cu calls one body; the batched solver calls
// them in sequence inside its own CTA.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace usbs {
namespace {

__device__ __forceinline__ int svec_idx(int p, int q, int k) {  // p >= q, k x k matrix
  return q * k - (q * (q - 1)) / 2 + (p - q);
}
__device__ __forceinline__ int svec_idx8(int p, int q) { return svec_idx(p, q, 8); }

constexpr double SQ2 = 1.41421356237309504880;

constexpr unsigned FULL = 0xffffffffu;

// Warp-cooperative Cholesky A = R^T R (R upper) of a k x k matrix, k <= 8, row stride 8.
// All 32 lanes call it; lane l < k keeps column l of R.  Returns false (on every lane)
// if a pivot is not positive.  When R is non-null the factor is stored (row stride 8).
__device__ bool warp_chol(const double* A, double* R, int k) {
  const int lane = threadIdx.x & 31;
  double rc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) rc[i] = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j >= k) break;
    double d = 0.0;
    if (lane == j) {
      d = A[j * 8 + j];
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l < j) d -= rc[l] * rc[l];
    }
    d = __shfl_sync(FULL, d, j);
    if (!(d > 0.0)) return false;
    const double inv = rsqrt(d), rjj = d * inv;
    double sacc = (lane > j && lane < k) ? A[j * 8 + lane] : 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      if (l < j) {
        const double rlj = __shfl_sync(FULL, rc[l], j);
        sacc -= rlj * rc[l];
      }
    }
    if (lane == j) rc[j] = rjj;
    else if (lane > j && lane < k) rc[j] = sacc * inv;
  }
  if (R && lane < 8) {
#pragma unroll
    for (int i = 0; i < 8; ++i) R[i * 8 + lane] = (i <= lane && lane < k) ? rc[i] : 0.0;
  }
  __syncwarp();
  return true;
}

// Largest eigenvalue of a small symmetric matrix (k <= 8, row stride 8): parallel
// Jacobi in FP32 by one warp for the eigenvector, then its FP64 Rayleigh quotient.
__device__ double warp_lambda_max(const double* A, int k, float* Af, float* Vf) {
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < 64; t += 32) {
    const int i = t / 8, j = t % 8;
    Af[t] = (i < k && j < k) ? (float)A[t] : (i == j ? -1e30f : 0.f);
    Vf[t] = (i == j) ? 1.f : 0.f;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 12; ++sweep) {
    for (int round = 0; round < 7; ++round) {
      // circle ordering on 8 indices
      float c = 1.f, sv = 0.f;
      int p = 0, q = 0;
      if (lane < 4) {
        const int pa = lane == 0 ? 0 : 1 + ((lane - 1 + round) % 7);
        const int pb = 1 + ((7 - lane - 1 + round) % 7);
        p = min(pa, pb); q = max(pa, pb);
        const float apq = Af[p * 8 + q];
        if (fabsf(apq) > 1e-30f) {
          const float tau = (Af[q * 8 + q] - Af[p * 8 + p]) / (2.f * apq);
          const float t = fabsf(tau) > 1e18f ? 0.5f / tau
                                              : (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(tau * tau + 1.f));
          c = 1.f / sqrtf(t * t + 1.f);
          sv = t * c;
        }
      }
      float cs[4], sn[4];
      int pp[4], qq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cs[u] = __shfl_sync(FULL, c, u);
        sn[u] = __shfl_sync(FULL, sv, u);
        pp[u] = __shfl_sync(FULL, p, u);
        qq[u] = __shfl_sync(FULL, q, u);
      }
      __syncwarp();
      float na = 0.f, nb = 0.f, nc = 0.f, nd = 0.f;
      int k1 = 0, k2 = 0;
      if (lane < 16) {
        k1 = lane / 4; k2 = lane % 4;
        const float a = Af[pp[k1] * 8 + pp[k2]], b = Af[pp[k1] * 8 + qq[k2]];
        const float cc = Af[qq[k1] * 8 + pp[k2]], d = Af[qq[k1] * 8 + qq[k2]];
        const float ra = cs[k1] * a - sn[k1] * cc, rb = cs[k1] * b - sn[k1] * d;
        const float rcc = sn[k1] * a + cs[k1] * cc, rd = sn[k1] * b + cs[k1] * d;
        na = cs[k2] * ra - sn[k2] * rb; nb = sn[k2] * ra + cs[k2] * rb;
        nc = cs[k2] * rcc - sn[k2] * rd; nd = sn[k2] * rcc + cs[k2] * rd;
      }
      float vp = 0.f, vq = 0.f;
      const int kr = lane / 8, row = lane % 8;
      vp = Vf[row * 8 + pp[kr]];
      vq = Vf[row * 8 + qq[kr]];
      __syncwarp();
      if (lane < 16) {
        Af[pp[k1] * 8 + pp[k2]] = na; Af[pp[k1] * 8 + qq[k2]] = nb;
        Af[qq[k1] * 8 + pp[k2]] = nc; Af[qq[k1] * 8 + qq[k2]] = nd;
      }
      Vf[row * 8 + pp[kr]] = cs[kr] * vp - sn[kr] * vq;
      Vf[row * 8 + qq[kr]] = sn[kr] * vp + cs[kr] * vq;
      __syncwarp();
    }
  }
  // top eigenvector, FP64 Rayleigh quotient
  int best = 0;
  for (int i = 1; i < k; ++i)
    if (Af[i * 8 + i] > Af[best * 8 + best]) best = i;
  double num = 0.0, den = 0.0;
  if (lane < k) {
    const double vi = (double)Vf[lane * 8 + best];
    double av = 0.0;
    for (int j = 0; j < k; ++j) av += A[lane * 8 + j] * (double)Vf[j * 8 + best];
    num = vi * av;
    den = vi * vi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(FULL, num, o);
    den += __shfl_xor_sync(FULL, den, o);
  }
  return num / den;
}

// ---- Cholesky-QR factor of a new block ------------------------------------------------------
// red + RED_H: H (nb blocks x 64), red + RED_H2: H2 (nb x 64), red + RED_GRAM: W'^T W'.
// Gram of the final block: W'^T W' - sum_b H2_b^T H2_b (the correction W' - Q H2 is
// orthogonal to Q).  A column whose squared norm after orthogonalisation falls below
// rel_thr times its squared norm before it is deficient: it is replaced by a random
// vector (k_finalize) and the block is orthogonalised once more (the masked pass).
// pass 0: the new block (writes T, R_last, and the second pass's mask); pass 1: masked by
// defl, replaces still-dependent columns again and sets the third pass's mask; pass 2:
// masked by defl2, zeroes what is still dependent.
__device__ __forceinline__ void k_chol_block_dev(DevLanczos* lz, const double* USBS_RESTRICT red, int j, int nb,
                             int write_T, int is_resid, int defl_pass, double rel_thr) {
  if (defl_pass == 1 && lz->defl == 0) return;
  if (defl_pass == 2 && lz->defl2 == 0) return;
  __shared__ double G[64], pre[8], R[64], Ri[64];
  __shared__ int dc[8];
  const double* H = red + RED_H;
  const double* H2 = red + RED_H2;
  const double* Gram = red + RED_GRAM;
  const int tid = threadIdx.x;
  if (write_T && !defl_pass) {
    for (int t = tid; t < nb * 64; t += blockDim.x) {
      const int b = t / 64, a = (t / 8) % 8, cc = t % 8;
      const int row = b * 8 + a, colT = j * 8 + cc;
      if (b == j) {
        const int tt = b * 64 + cc * 8 + a;
        lz->T[row * JMAX + colT] = 0.5 * (H[t] + H2[t] + H[tt] + H2[tt]);
      } else {
        const double v = H[t] + H2[t];
        lz->T[row * JMAX + colT] = v;
        lz->T[colT * JMAX + row] = v;
      }
    }
  }
  if (tid < 64) {
    const int a = tid / 8, cc = tid % 8;
    double g = Gram[tid];
    for (int b = 0; b < nb; ++b)
      for (int r = 0; r < 8; ++r) g -= H2[b * 64 + r * 8 + a] * H2[b * 64 + r * 8 + cc];
    G[tid] = g;
  }
  __syncthreads();
  __shared__ double premax;
  if (tid < 8) {
    double p = G[tid * 8 + tid];
    for (int b = 0; b < nb; ++b)
      for (int r = 0; r < 8; ++r) {
        const double h = H[b * 64 + r * 8 + tid] + H2[b * 64 + r * 8 + tid];
        p += h * h;
      }
    pre[tid] = p;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int a = 0; a < 8; ++a) m = fmax(m, pre[a]);
    premax = m;
  }
  __syncthreads();
  if (tid < 32) {
    // warp-cooperative Cholesky with deficient columns: lane l owns column l of R
    const int lane = tid;
    double rc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rc[i] = 0.0;
    int badmask = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double d = 0.0;
      if (lane == j) {
        d = G[j * 8 + j];
#pragma unroll
        for (int l = 0; l < 8; ++l)
          if (l < j) d -= rc[l] * rc[l];
      }
      d = __shfl_sync(FULL, d, j);
      // deficient: small against the column's own norm before orthogonalisation, or
      // against the block's largest column (a residual at rounding level)
      const bool bad = !(d > rel_thr * pre[j]) || !(d > rel_thr * rel_thr * premax) || !(pre[j] > 0.0);
      if (bad) {
        badmask |= 1 << j;
        if (lane == j) rc[j] = 1.0;   // row j of R stays e_j^T: the column is replaced
        continue;
      }
      const double inv = rsqrt(d), rjj = d * inv;
      double sacc = (lane > j && lane < 8) ? G[j * 8 + lane] : 0.0;
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        if (l < j) {
          const double rlj = __shfl_sync(FULL, rc[l], j);
          sacc -= rlj * rc[l];
        }
      }
      if (lane == j) rc[j] = rjj;
      else if (lane > j && lane < 8) rc[j] = sacc * inv;
    }
    if (lane < 8) {
#pragma unroll
      for (int i = 0; i < 8; ++i) R[i * 8 + lane] = (i <= lane) ? rc[i] : 0.0;
    }
    __syncwarp();
    // column c of R^-1 by back substitution (lane c), with the reciprocals of R's
    // diagonal shared by shuffles
    const double rd_own = (lane < 8) ? 1.0 / R[lane * 8 + lane] : 0.0;
    double rd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rd[i] = __shfl_sync(FULL, rd_own, i);
    if (lane < 8) {
      const int cidx = lane;
      double x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = 0.0;
      x[cidx] = rd[cidx];
      for (int i = cidx - 1; i >= 0; --i) {
        double sacc = 0.0;
        for (int l = i + 1; l <= cidx; ++l) sacc += R[i * 8 + l] * x[l];
        x[i] = -sacc * rd[i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) Ri[i * 8 + cidx] = x[i];
      const int isbad = (badmask >> lane) & 1;
      dc[lane] = isbad ? (defl_pass < 2 ? 1 : 2) : 0;
    }
    __syncwarp();
    for (int u = lane; u < 64; u += 32) {
      lz->R[u] = R[u];
      lz->Rinv[u] = Ri[u];
      const int i = u / 8, jj = u % 8;
      if (is_resid && defl_pass == 0)
        lz->Rlast[u] = (i == jj && dc[i]) ? 0.0 : R[u];   // deficient rows carry no residual
      else if (is_resid && defl_pass == 2 && dc[i])
        lz->Rlast[u] = 0.0;                              // zeroed columns carry none either
    }
    if (lane < 8) lz->dcol[lane] = dc[lane];
    // each masked pass reads its flag in every one of its kernels, so a flag is only
    // changed by the pass before it
    if (lane == 0) {
      if (defl_pass == 0) {
        lz->defl = (badmask != 0) ? 1 : 0;
        lz->defl2 = 0;
        if (badmask != 0 && write_T) lz->defl_seen = 1;   // a block of a cycle, not the start block
      } else if (defl_pass == 1) {
        lz->defl2 = (badmask != 0) ? 1 : 0;
      }
    }
  }
}

// ---- Rayleigh-Ritz in FP32 (mixed mode) ---------------------------------------------------------
// The same cyclic Jacobi method with circle ordering as the generic body below, arranged so
// that one CTA runs a round at FP32 speed with a single barrier:
//  - every warp forms the J/2 rotations of the round itself (lane l the rotation of pair
//    l mod J/2) and hands them to its lanes by shuffles, so no shared table and no barrier
//    sits between the rotation parameters and the update;
//  - A is double-buffered (read A_cur, write A_next), so the pivots a round reads are never
//    overwritten within it;
//  - the rotation parameters keep IEEE division and square root (with the hardware
//    approximations instead, together with the one-step orthonormalisation below, a
//    mixed-precision solve of a 400-node geometric graph stalled at 2.5e-3 infeasibility;
//    either change alone converges);
//  - T is scaled by an exact power of two (its largest entry to [1/2, 1)), which leaves every
//    rotation unchanged and keeps the sums of squares of the stopping test in FP32 range;
//  - the kept Ritz vectors are made orthonormal by one Newton-Schulz step towards their polar
//    factor, Y_keep <- Y_keep + Y_keep (I - Y_keep^T Y_keep) / 2: the accumulated rotations
//    are orthogonal to about 1e-6, and one step squares that defect (same span as the
//    Gram-Schmidt of the generic body, two barriers instead of four per column).
// The restarted projected matrix is Y_keep^T T Y_keep with the unrotated T, as in the generic
// body, so rounding in the rotations costs convergence speed, not accuracy.
__device__ __forceinline__ int jac_circle(int pos, int round, int J) {
  if (pos == 0) return 0;
  int x = pos - 1 + round;
  if (x >= J - 1) x -= J - 1;
  return 1 + x;
}

__device__ __forceinline__ void jac_rot_f32(float app, float aqq, float apq, float skip2,
                                            float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (apq != 0.f && apq * apq > skip2 * fabsf(app * aqq)) {
    const float tau = (aqq - app) / (2.f * apq);
    float t;
    if (fabsf(tau) > 1e18f) t = 0.5f / tau;
    else t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(tau * tau + 1.f));
    c = 1.f / sqrtf(t * t + 1.f);
    s = t * c;
  }
}

template <int J>
__device__ __forceinline__ void k_ritz_f32_dev(DevLanczos* lz, int kc, double tol, int max_sweeps,
                                                  double jac_eps) {
  constexpr int keep = J / 2;
  constexpr int half = J / 2;
  constexpr int LD = J + 1;
  constexpr int NBLK = half * half, NITEM = half * half + J * half;
  static_assert(NBLK % 32 == 0 && NITEM % 32 == 0 && half <= 32, "warp-uniform work split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* A0 = reinterpret_cast<float*>(smem_raw);   // J x LD: T (scaled), rotated
  float* A1 = A0 + J * LD;                            // J x LD: the other buffer of A
  float* Vv = A1 + J * LD;                            // J x LD: accumulated rotations
  float* Z = Vv + 2 * J * LD;                         // J x keep floats: I - G, then the FP64
                                                      // keep x keep restarted matrix
  __shared__ float key[JMAX], dg[JMAX];
  __shared__ int order[JMAX];
  __shared__ float wsum[2][16];
  __shared__ unsigned wmax[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  // largest |T_ij| by the high word of its bit pattern (integer order = magnitude order)
  unsigned hm = 0;
  for (int t = tid; t < J * J; t += blockDim.x) {
    const double x = lz->T[(t / J) * JMAX + t % J];
    hm = max(hm, (unsigned)__double2hiint(x) & 0x7fffffffu);
  }
  hm = __reduce_max_sync(FULL, hm);
  if (lane == 0) wmax[warp] = hm;
  __syncthreads();
  hm = 0;
  for (int w = 0; w < nw; ++w) hm = max(hm, wmax[w]);
  const int ebits = (int)(hm >> 20);
  if (ebits == 0x7ff) {
    // non-finite projected matrix: report it and stop the eigen solve
    if (tid == 0) {
      lz->status = USBS_ENUMERIC;
      lz->converged = 1;
      lz->cycles += 1;
    }
    for (int t = tid; t < JMAX * JMAX; t += blockDim.x) lz->Y[t] = ((t / JMAX) == (t % JMAX)) ? 1.0 : 0.0;
    if (tid < JMAX) lz->theta[tid] = 0.0;
    return;
  }
  // A = T 2^-esh with the largest entry in [1/2, 1)
  const int esh = (hm == 0) ? 0 : ebits - 1022;
  const bool fscale = esh > -100 && esh < 100;
  const float scf = fscale ? ldexpf(1.f, -esh) : 1.f;
  const double scd = ldexp(1.0, -esh);
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int i = t / J, j = t % J;
    const double x = lz->T[i * JMAX + j];
    const float xf = (float)x;
    A0[i * LD + j] = fscale ? xf * scf : (float)(x * scd);
    Vv[i * LD + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  float* Ac = A0;
  float* An = A1;
  if constexpr (J == 32) {
    // One-sided (Hestenes) Jacobi by warp 0 with every column in registers: lane l holds
    // column l of M = A + sigma I (sigma = 1.0625 ||A||_F makes M positive definite, so its
    // eigenvalues lambda + sigma are distinct wherever A's are) and column l of V.  Round
    // r = 1..31 pairs lane l with lane l ^ r (31 rounds meet every pair once: a sweep) and
    // rotates the two columns of M to orthogonality, V alongside; the two lanes of a pair
    // form the same Gram entries bit for bit (same products, same order), so they agree on
    // the rotation.  At convergence M_0 V has orthogonal columns, V holds the eigenvectors
    // and column l of M_0 V has norm lambda_l + sigma.  No shared memory and no barrier
    // inside the sweeps; a sweep in which no pair rotates ends the iteration.
    if (warp == 0) {
      float fro = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float x = A0[i * LD + lane];
        fro = fmaf(x, x, fro);
      }
      for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(FULL, fro, o);
      const float sigma = 1.0625f * sqrtf(fro) + 1e-30f;
      float m[32], v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        m[i] = A0[i * LD + lane] + (i == lane ? sigma : 0.f);
        v[i] = (i == lane) ? 1.f : 0.f;
      }
      const float eps = (float)jac_eps;
      for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool rotated = false;
        for (int r = 1; r < 32; ++r) {
          float pm[32];
          float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, g0 = 0.f, g1 = 0.f;
#pragma unroll
          for (int i = 0; i < 32; ++i) pm[i] = __shfl_xor_sync(FULL, m[i], r);
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            a0 = fmaf(m[i], m[i], a0);
            a1 = fmaf(m[i + 1], m[i + 1], a1);
            b0 = fmaf(pm[i], pm[i], b0);
            b1 = fmaf(pm[i + 1], pm[i + 1], b1);
            g0 = fmaf(m[i], pm[i], g0);
            g1 = fmaf(m[i + 1], pm[i + 1], g1);
          }
          const bool lo = lane < (lane ^ r);
          const float own = a0 + a1, other = b0 + b1, g = g0 + g1;
          const float al = lo ? own : other, be = lo ? other : own;   // |m_p|^2, |m_q|^2, p < q
          float c = 1.f, sn = 0.f;
          if (g != 0.f && fabsf(g) > eps * sqrtf(al * be)) {
            const float zeta = (be - al) / (2.f * g);
            const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            c = 1.f / sqrtf(fmaf(t, t, 1.f));
            sn = t * c;
            rotated = true;
          }
          // p: c m_p - s m_q;  q: s m_p + c m_q
          const float sq = lo ? -sn : sn;
#pragma unroll
          for (int i = 0; i < 32; ++i) m[i] = fmaf(sq, pm[i], c * m[i]);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float pv = __shfl_xor_sync(FULL, v[i], r);
            v[i] = fmaf(sq, pv, c * v[i]);
          }
        }
        if (lane == 0) lz->sweeps += 1;
        if (!__any_sync(FULL, rotated)) break;
      }
      float nn = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) nn = fmaf(m[i], m[i], nn);
      A0[lane * LD + lane] = sqrtf(nn) - sigma;
#pragma unroll
      for (int i = 0; i < 32; ++i) Vv[i * LD + lane] = v[i];
    }
    __syncthreads();
  } else {
    const float skip2 = (float)(jac_eps * 1e-2) * (float)(jac_eps * 1e-2);
    const float eps2 = (float)jac_eps * (float)jac_eps;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      float off = 0.f, tot = 0.f;
      for (int t = tid; t < J * J; t += blockDim.x) {
        const int i = t / J, j = t % J;
        const float x = Ac[i * LD + j];
        tot = fmaf(x, x, tot);
        if (i != j) off = fmaf(x, x, off);
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(FULL, off, o);
        tot += __shfl_xor_sync(FULL, tot, o);
      }
      if (lane == 0) { wsum[0][warp] = off; wsum[1][warp] = tot; }
      __syncthreads();
      // every thread sums the warps' parts in the same order: one decision, no second barrier
      float o2 = 0.f, t2 = 0.f;
      for (int w = 0; w < nw; ++w) { o2 += wsum[0][w]; t2 += wsum[1][w]; }
      if (o2 <= eps2 * t2) break;
      if (tid == 0) lz->sweeps += 1;
      for (int round = 0; round < J - 1; ++round) {
        // lane l: the rotation of pair l mod half, from the pivots of A_cur
        const int kr = lane & (half - 1);
        const int pa = jac_circle(kr, round, J), pb = jac_circle(J - 1 - kr, round, J);
        const int pr = min(pa, pb), qr = max(pa, pb);
        float cr, sr;
        jac_rot_f32(Ac[pr * LD + pr], Ac[qr * LD + qr], Ac[pr * LD + qr], skip2, cr, sr);
        const int pqr = pr | (qr << 8);
        for (int t0 = warp * 32; t0 < NITEM; t0 += blockDim.x) {   // warp-uniform
          const int t = t0 + lane;
          if (t0 < NBLK) {
            // 2 x 2 block (p1, q1) x (p2, q2): rows by rotation k1, columns by k2
            const int k1 = t / half, k2 = t % half;
            const float c1 = __shfl_sync(FULL, cr, k1), s1 = __shfl_sync(FULL, sr, k1);
            const float c2 = __shfl_sync(FULL, cr, k2), s2 = __shfl_sync(FULL, sr, k2);
            const int pq1 = __shfl_sync(FULL, pqr, k1), pq2 = __shfl_sync(FULL, pqr, k2);
            const int p1 = pq1 & 255, q1 = pq1 >> 8, p2 = pq2 & 255, q2 = pq2 >> 8;
            const float a = Ac[p1 * LD + p2], b = Ac[p1 * LD + q2];
            const float cc = Ac[q1 * LD + p2], d = Ac[q1 * LD + q2];
            const float ra = c1 * a - s1 * cc, rb = c1 * b - s1 * d;
            const float rc = s1 * a + c1 * cc, rd = s1 * b + c1 * d;
            An[p1 * LD + p2] = c2 * ra - s2 * rb;
            An[p1 * LD + q2] = s2 * ra + c2 * rb;
            An[q1 * LD + p2] = c2 * rc - s2 * rd;
            An[q1 * LD + q2] = s2 * rc + c2 * rd;
          } else {
            // V <- V G on row `row`, pair k (each (row, k) owned by one thread: in place)
            const int u = t - NBLK;
            const int k = u / J, row = u % J;
            const float c = __shfl_sync(FULL, cr, k), sv = __shfl_sync(FULL, sr, k);
            const int pq = __shfl_sync(FULL, pqr, k);
            const int p = pq & 255, q = pq >> 8;
            const float vp = Vv[row * LD + p], vq = Vv[row * LD + q];
            Vv[row * LD + p] = c * vp - sv * vq;
            Vv[row * LD + q] = sv * vp + c * vq;
          }
        }
        __syncthreads();
        float* tmp = Ac; Ac = An; An = tmp;
      }
    }
  }
  // descending order under a strict total order (value, then index)
  if (tid < J) {
    const float d = Ac[tid * LD + tid];
    dg[tid] = d;
    key[tid] = isfinite(d) ? d : -FLT_MAX;
  }
  __syncthreads();
  if (tid < J) {
    int rank = 0;
    const float x = key[tid];
    for (int u = 0; u < J; ++u) {
      const float y = key[u];
      if (y > x || (y == x && u < tid)) ++rank;
    }
    order[rank] = tid;
  }
  __syncthreads();
  // A is no longer needed: Y (sorted Ritz vectors) in one buffer, its correction in the other
  float* Y = An;
  float* Yn = Ac;
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int l = t / J, col = t % J;
    Y[l * LD + col] = Vv[l * LD + order[col]];
  }
  __syncthreads();
  // E = I - Y_keep^T Y_keep
  float* E = Z;
  for (int t = tid; t < keep * keep; t += blockDim.x) {
    const int i = t / keep, j = t % keep;
    float g = 0.f;
    for (int r = 0; r < J; ++r) g = fmaf(Y[r * LD + i], Y[r * LD + j], g);
    E[t] = (i == j ? 1.f : 0.f) - g;
  }
  __syncthreads();
  // Y_keep <- Y_keep + Y_keep E / 2; the other columns are copied
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int r = t / J, i = t % J;
    float v = Y[r * LD + i];
    if (i < keep) {
      float acc = 0.f;
      for (int j = 0; j < keep; ++j) acc = fmaf(Y[r * LD + j], E[j * keep + i], acc);
      v = fmaf(0.5f, acc, v);
    }
    Yn[r * LD + i] = v;
  }
  __syncthreads();
  Y = Yn;
  // FP64 finish.  The FP32 rotations only serve to find the Ritz vectors; the quantities
  // that leave the kernel are formed in FP64 from the FP64 projected matrix T and the kept
  // vectors (their FP32 values, exact in FP64): Z = T Y_keep, the restarted projected
  // matrix B = Y_keep^T Z, the Rayleigh quotients theta_i = y_i^T T y_i / y_i^T y_i and the
  // residual norms.  A Rayleigh quotient of an approximate eigenvector with angle error e
  // is off by O(e^2), so the Ritz values carry FP64 accuracy, not the FP32 of the rotations.
  double* Yd = reinterpret_cast<double*>(Vv);                  // J x keep
  double* Zd = reinterpret_cast<double*>(Y == A0 ? A1 : A0);   // J x keep
  double* Bd = reinterpret_cast<double*>(Z);                   // keep x keep
  for (int t = tid; t < J * keep; t += blockDim.x) Yd[t] = (double)Y[(t / keep) * LD + t % keep];
  __syncthreads();
  for (int t = tid; t < J * keep; t += blockDim.x) {
    const int r = t / keep, i = t % keep;
    const double* Tr = lz->T + r * JMAX;
    double z = 0.0;
    for (int c2 = 0; c2 < J; ++c2) z = fma(Tr[c2], Yd[c2 * keep + i], z);
    Zd[t] = z;
  }
  __syncthreads();
  for (int t = tid; t < keep * keep; t += blockDim.x) {
    const int i = t / keep, j = t % keep;
    if (j < i) continue;
    double acc = 0.0;
    for (int r = 0; r < J; ++r) acc = fma(Yd[r * keep + i], Zd[r * keep + j], acc);
    Bd[i * keep + j] = acc;          // symmetric by construction: one value per pair
    Bd[j * keep + i] = acc;
  }
  __syncthreads();
  for (int t = tid; t < JMAX * JMAX; t += blockDim.x) {
    const int i = t / JMAX, j = t % JMAX;
    lz->T[t] = (i < keep && j < keep) ? Bd[i * keep + j] : 0.0;
  }
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int l = t / J, col = t % J;
    lz->Y[l * JMAX + col] = (double)Y[l * LD + col];
  }
  if (warp == 0) {
    // Ritz values in T's units (the diagonal of A scaled back, used for the order), then for
    // the top k_c the FP64 Rayleigh quotients and residual norms
    // ||T y_i - theta_i y_i||^2 + ||R_last E^T y_i||^2 (two orthogonal terms) of y_i / |y_i|
    for (int i = lane; i < J; i += 32) lz->theta[i] = ldexp((double)key[order[i]], esh);
    float m = 0.f;
    for (int i = lane; i < J; i += 32) m = fmaxf(m, fabsf(dg[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    const double normest = fmax(lz->normest, ldexp((double)m, esh));
    double res = 0.0;
    if (lane < kc) {
      const int i = lane;
      double yy = 0.0;
      for (int r = 0; r < J; ++r) yy = fma(Yd[r * keep + i], Yd[r * keep + i], yy);
      const double th = Bd[i * keep + i] / yy;
      double s2 = 0.0;
      for (int r = 0; r < J; ++r) {
        const double e = Zd[r * keep + i] - th * Yd[r * keep + i];
        s2 = fma(e, e, s2);
      }
      for (int a = 0; a < 8; ++a) {
        double v = 0.0;
        for (int c2 = a; c2 < 8; ++c2) v = fma(lz->Rlast[a * 8 + c2], Yd[(J - 8 + c2) * keep + i], v);
        s2 = fma(v, v, s2);
      }
      res = sqrt(s2 / yy);
      lz->res[i] = res;
      lz->theta[i] = th;
    }
    const bool ok = (lane >= kc) || (res <= tol * normest);
    const unsigned all_ok = __all_sync(FULL, ok);
    if (lane == 0) {
      lz->normest = normest;
      lz->converged = all_ok ? 1 : 0;
      lz->cycles += 1;
    }
  }
}

// ---- Rayleigh-Ritz: eigen-decomposition of T by parallel cyclic Jacobi ------------------------
// Generic body, S the arithmetic of the whole Ritz step (the FP64 of the plain mode; FP32 runs
// the restructured body above).  The J/2 rotations of a round act on disjoint index pairs
// (circle ordering), so every 2 x 2 block (p1, q1) x (p2, q2) of A is updated in one pass
// as R1^T [a b; c d] R2.  After the sort, the kept Ritz vectors are orthonormalised
// (classical Gram-Schmidt, two passes) and the restarted projected matrix is
// Y_keep^T T Y_keep, so rounding in the rotations does not leak into the next cycle.
template <typename S, int J>
__device__ __forceinline__ void k_ritz_generic_dev(DevLanczos* lz, int kc, double tol, int max_sweeps,
                                                      double jac_eps) {
  constexpr int keep = J / 2;
  constexpr int half = J / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LD = J + 1;
  S* A = reinterpret_cast<S*>(smem_raw);      // J x LD: T, rotated in place
  S* Vv = A + J * LD;                           // J x LD: accumulated rotations
  S* Tc = Vv + J * LD;                          // J x LD: copy of T
  S* Y = Tc + J * LD;                           // J x LD: sorted Ritz vectors
  S* Z = Y + J * LD;                            // J x keep: T Y_keep
  __shared__ S cs[JMAX / 2], sn[JMAX / 2];
  __shared__ int pp[JMAX / 2], qq[JMAX / 2];
  __shared__ double th[JMAX];
  __shared__ int order[JMAX];
  __shared__ double wred[2][16];
  __shared__ S hbuf[JMAX];
  __shared__ S nrm;
  __shared__ int stop, bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int i = t / J, j = t % J;
    const double x = lz->T[i * JMAX + j];
    if (!isfinite(x)) bad = 1;
    A[i * LD + j] = (S)x;
    Tc[i * LD + j] = (S)x;
    Vv[i * LD + j] = (S)(i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  if (bad) {
    // non-finite projected matrix: report it and stop the eigen solve
    if (tid == 0) {
      lz->status = USBS_ENUMERIC;
      lz->converged = 1;
      lz->cycles += 1;
    }
    for (int t = tid; t < JMAX * JMAX; t += blockDim.x) lz->Y[t] = ((t / JMAX) == (t % JMAX)) ? 1.0 : 0.0;
    if (tid < JMAX) lz->theta[tid] = 0.0;
    return;
  }
  const S skip = (S)(jac_eps * 1e-2), big = (S)1e18;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = tid; t < J * J; t += blockDim.x) {
      const int i = t / J, j = t % J;
      const double x = (double)A[i * LD + j];
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
      for (int w = 0; w < nw; ++w) { o2 += wred[0][w]; t2 += wred[1][w]; }
      stop = (o2 <= jac_eps * jac_eps * t2) ? 1 : 0;
    }
    __syncthreads();
    if (stop) break;
    if (tid == 0) lz->sweeps += 1;
    for (int round = 0; round < J - 1; ++round) {
      if (tid < half) {
        // circle method: position 0 fixed, the others rotate
        const int k = tid;
        const int posA = k, posB = J - 1 - k;
        const int pa = posA == 0 ? 0 : 1 + ((posA - 1 + round) % (J - 1));
        const int pb = 1 + ((posB - 1 + round) % (J - 1));
        const int p = min(pa, pb), q = max(pa, pb);
        pp[k] = p;
        qq[k] = q;
        const S apq = A[p * LD + q];
        S c = (S)1, sv = (S)0;
        const S app = A[p * LD + p], aqq = A[q * LD + q];
        // all in S: an FP64 sqrt here would be a long FP64 sequence every round
        if (apq != (S)0 && fabs(apq) > skip * sqrt(fabs(app * aqq))) {
          const S tau = (aqq - app) / ((S)2 * apq);
          S t;
          if (fabs(tau) > big) t = (S)0.5 / tau;
          else t = (tau >= (S)0 ? (S)1 : (S)-1) / (fabs(tau) + sqrt(tau * tau + (S)1));
          c = (S)1 / sqrt(t * t + (S)1);
          sv = t * c;
        }
        cs[k] = c;
        sn[k] = sv;
      }
      __syncthreads();
      // A <- G^T A G on 2 x 2 blocks; V <- V G (index arithmetic on powers of two)
      constexpr int NBLK = half * half, NITEM = half * half + J * half;
      for (int t = tid; t < NITEM; t += blockDim.x) {
        if (t < NBLK) {
          const int k1 = t / half, k2 = t % half;
          const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
          const S c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
          const S a = A[p1 * LD + p2], b = A[p1 * LD + q2];
          const S cc = A[q1 * LD + p2], d = A[q1 * LD + q2];
          // rows: [p1; q1] <- [c1 -s1; s1 c1] [p1; q1]
          const S ra = c1 * a - s1 * cc, rb = c1 * b - s1 * d;
          const S rc = s1 * a + c1 * cc, rd = s1 * b + c1 * d;
          // cols: [p2 q2] <- [p2 q2] [c2 s2; -s2 c2]
          A[p1 * LD + p2] = c2 * ra - s2 * rb;
          A[p1 * LD + q2] = s2 * ra + c2 * rb;
          A[q1 * LD + p2] = c2 * rc - s2 * rd;
          A[q1 * LD + q2] = s2 * rc + c2 * rd;
        } else {
          const int u = t - NBLK;
          const int k = u / J, row = u % J;
          const S c = cs[k], sv = sn[k];
          const int p = pp[k], q = qq[k];
          const S vp = Vv[row * LD + p], vq = Vv[row * LD + q];
          Vv[row * LD + p] = c * vp - sv * vq;
          Vv[row * LD + q] = sv * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
  // descending order under a strict total order (value, then index)
  if (tid < J) {
    const double d = (double)A[tid * LD + tid];
    th[tid] = isfinite(d) ? d : -DBL_MAX;
  }
  __syncthreads();
  if (tid < J) {
    int rank = 0;
    const double x = th[tid];
    for (int u = 0; u < J; ++u) {
      const double y = th[u];
      if (y > x || (y == x && u < tid)) ++rank;
    }
    order[rank] = tid;
  }
  __syncthreads();
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int l = t / J, col = t % J;
    Y[l * LD + col] = Vv[l * LD + order[col]];
  }
  __syncthreads();
  // orthonormalise Y_keep (two passes of classical Gram-Schmidt per column)
  for (int i = 0; i < keep; ++i) {
    for (int pass = 0; pass < 2; ++pass) {
      // h_l = y_l . y_i for l < i: warp w takes l = w, w + nw, ...
      for (int l = warp; l < i; l += nw) {
        S h = (S)0;
        for (int r = lane; r < J; r += 32) h += Y[r * LD + l] * Y[r * LD + i];
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
        if (lane == 0) hbuf[l] = h;
      }
      __syncthreads();
      if (tid < J) {
        S v = Y[tid * LD + i];
        for (int l = 0; l < i; ++l) v -= Y[tid * LD + l] * hbuf[l];
        Y[tid * LD + i] = v;
      }
      __syncthreads();
    }
    if (warp == 0) {
      S s2 = (S)0;
      for (int r = lane; r < J; r += 32) s2 += Y[r * LD + i] * Y[r * LD + i];
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm = (S)1 / sqrt(s2);
    }
    __syncthreads();
    if (tid < J) Y[tid * LD + i] *= nrm;
    __syncthreads();
  }
  // Z = T Y_keep; restarted projected matrix Y_keep^T T Y_keep
  for (int t = tid; t < J * keep; t += blockDim.x) {
    const int r = t / keep, i = t % keep;
    S z = (S)0;
    for (int c2 = 0; c2 < J; ++c2) z += Tc[r * LD + c2] * Y[c2 * LD + i];
    Z[r * keep + i] = z;
  }
  __syncthreads();
  for (int t = tid; t < JMAX * JMAX; t += blockDim.x) {
    const int i = t / JMAX, j = t % JMAX;
    double v = 0.0;
    if (i < keep && j < keep) {
      S acc = (S)0;
      for (int r = 0; r < J; ++r) acc += Y[r * LD + i] * Z[r * keep + j];
      v = (double)acc;
    }
    lz->T[t] = v;
  }
  for (int t = tid; t < J * J; t += blockDim.x) {
    const int l = t / J, col = t % J;
    lz->Y[l * JMAX + col] = (double)Y[l * LD + col];
  }
  if (tid < J) lz->theta[tid] = th[order[tid]];
  __syncthreads();
  // Ritz values of the orthonormalised vectors (Rayleigh quotients) and residual norms
  // ||R_last E^T y_i|| for the top k_c
  if (tid < kc) {
    // residual of the Ritz pair (theta_i, Q y_i): Q (T y_i - theta_i y_i) + Q_res R E^T y_i,
    // two orthogonal terms (y_i is only an approximate eigenvector of T)
    const int i = tid;
    S zz = (S)0;
    for (int r = 0; r < J; ++r) zz += Y[r * LD + i] * Z[r * keep + i];
    th[i] = (double)zz;
    double s2 = 0.0;
    for (int r = 0; r < J; ++r) {
      const double e = (double)Z[r * keep + i] - (double)zz * (double)Y[r * LD + i];
      s2 += e * e;
    }
    for (int a = 0; a < 8; ++a) {
      double v = 0.0;
      for (int c2 = a; c2 < 8; ++c2) v += lz->Rlast[a * 8 + c2] * (double)Y[(J - 8 + c2) * LD + i];
      s2 += v * v;
    }
    lz->res[i] = sqrt(s2);
  }
  __syncthreads();
  if (tid == 0) {
    double scale = 0.0;
    for (int i = 0; i < J; ++i) scale = fmax(scale, fabs((double)A[i * LD + i]));
    lz->normest = fmax(lz->normest, scale);
    int conv = 1;
    for (int i = 0; i < kc; ++i) {
      lz->theta[i] = th[i];
      if (!(lz->res[i] <= tol * lz->normest)) conv = 0;
    }
    lz->converged = conv;
    lz->cycles += 1;
  }
}

// Rayleigh-Ritz step of one restart cycle: FP32 (mixed mode) by the restructured body, FP64
// by the generic one (where GB300's FP64 rate, not the barriers, sets the time).
template <typename S, int J>
__device__ __forceinline__ void k_ritz_dev(DevLanczos* lz, int kc, double tol, int max_sweeps,
                                              double jac_eps) {
  if constexpr (sizeof(S) == 4) k_ritz_f32_dev<J>(lz, kc, tol, max_sweeps, jac_eps);
  else k_ritz_generic_dev<S, J>(lz, kc, tol, max_sweeps, jac_eps);
}

// ---- App. B.2 interior point method --------------------------------------------------------
// S^-1 for the symmetric positive definite k_c x k_c block of S (an 8 x 8 array) by
// Gauss-Jordan elimination of [S | I] without pivoting (the pivots of an SPD matrix are
// positive).  Threads 0..127 own the 128 entries of [S | I], double-buffered in buf
// (256 doubles), one barrier per pivot; every thread of the CTA calls it.  Each pivot costs
// one FP64 reciprocal and one fused update per entry, all entries at once: a warp-serial
// Cholesky, triangular inverse and product took about seven times as long on GB300's FP64
// rate.  The result is symmetrised; entries outside the k_c x k_c block are the identity's.
__device__ __forceinline__ void cta_spd_inverse8(const double* S, double* buf, double* Sinv, int kc) {
  const int tid = threadIdx.x;
  const int r = (tid >> 4) & 7, c = tid & 15;
  double* cur = buf;
  double* nxt = buf + 128;
  if (tid < 128) {
    double v;
    if (c < 8) v = (r < kc && c < kc) ? S[r * 8 + c] : (r == c ? 1.0 : 0.0);
    else v = (c - 8 == r) ? 1.0 : 0.0;
    cur[tid] = v;
  }
  __syncthreads();
  for (int p = 0; p < kc; ++p) {
    if (tid < 128) {
      const double ip = 1.0 / cur[p * 16 + p];
      const double mpc = cur[p * 16 + c] * ip;
      nxt[tid] = (r == p) ? mpc : fma(-cur[r * 16 + p], mpc, cur[tid]);
    }
    __syncthreads();
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (tid < 64) {
    const int i = tid >> 3, j = tid & 7;
    Sinv[tid] = 0.5 * (cur[i * 16 + 8 + j] + cur[j * 16 + 8 + i]);
  }
  __syncthreads();
}

struct IpmShared {
  double Q[KSV * KSV];
  double TS[KSV * KSV];
  double L[KSV * (KSV + 1)];
  double q12[KSV], h1[KSV], v[KSV], s[KSV], t[KSV], sinv[KSV], F1[KSV], ds[KSV], dt[KSV];
  double fcol[KSV];
  double S[64], T[64], Sinv[64], dS[64], dT[64], St[64], Tt[64];
  double q22, h2, eta, zeta, omega, mu, deta, dzeta, domega, delta, kappa1, kappa2, det, r2, r3;
  int map[KSV];
  int perm[2][KSV];            // row permutations of the elimination (current, next)
  int piv, done, iters, has_eta;
};

// Warp 0 of k_ipm: pivot of column pc of [L | rhs] among the logical rows pc..K-1 of the
// permutation src.  The largest |entry| is found by the high word of its bit pattern
// (exponent and 20 mantissa bits, which order magnitudes to 1e-6, ties to the lowest row)
// with two warp reductions on the integer pipe.  dst = src with the pivot row moved to
// position pc (dst may be src); fcol[pc] = 1 / pivot, or 0 and piv = -1 if it vanishes.
__device__ __forceinline__ void ipm_pivot(IpmShared& sh, const int* src, int* dst, int pc, int K,
                                          int LDL, int lane) {
  unsigned key = 0u;
  int bi = pc;
  for (int r = pc + lane; r < K; r += 32) {
    const unsigned k = (unsigned)__double2hiint(sh.L[src[r] * LDL + pc]) & 0x7fffffffu;
    if (k > key) { key = k; bi = r; }
  }
  const unsigned kmax = __reduce_max_sync(FULL, key);
  bi = (int)__reduce_min_sync(FULL, key == kmax ? (unsigned)bi : 0xffffffffu);
  if (dst != src)
    for (int r = lane; r < K; r += 32) dst[r] = src[r];
  __syncwarp();
  if (lane == 0) {
    const int a = dst[pc], b = dst[bi];
    dst[pc] = b;
    dst[bi] = a;
    // an exactly singular system (possible at degenerate optima): mark the direction
    // unusable instead of dividing by zero
    const double pv = sh.L[b * LDL + pc];
    const bool ok = fabs(pv) > 1e-300;
    sh.fcol[pc] = ok ? 1.0 / pv : 0.0;
    if (!ok) sh.piv = -1;
  }
  __syncwarp();
}

__device__ __forceinline__ double aug_at(const double* aug, int r, int c) {
  if (r > c) { int t = r; r = c; c = t; }
  const int ti = r / 4, tj = c / 4;
  int idx = 0;
  for (int u = 0; u < ti; ++u) idx += 10 - u;
  idx += tj - ti;
  return aug[idx * 16 + (r % 4) * 4 + (c % 4)];
}

// One CTA of 256 threads (8 warps: the phases below hand rows and scalars to fixed warps).
// b1 = 1 solves App. B.1 instead: the model value f^_t(y~) = <b, y~> + max over the model set
// of <C - A*(y~), X>, a linear objective over the same set, i.e. this IPM with Q11 = q12 =
// q22 = 0 and the linear data of y~ (G^T y~ and <A Xbar, y~> from k_xupdate's sums in
// red + RED_VEC); its value goes to sc->f_hat_ipm and the subproblem's S and eta are kept.
__device__ __forceinline__ void k_ipm_dev(DevScalars* sc, const double* USBS_RESTRICT red, int kc,
                                             double alpha, double rho, double mu_tol, int max_iter,
                                             int first_pass, int b1 = 0) {
  __shared__ IpmShared sh;
  const int tid = threadIdx.x;
  const int K = kc * (kc + 1) / 2;
  const double* aug = red + RED_AUG;
  const double* vec = red + RED_VEC;
  const double* vc = red + RED_VC;
  if (tid == 0) {
    int u = 0;
    for (int q = 0; q < kc; ++q)
      for (int p = q; p < kc; ++p) sh.map[u++] = svec_idx8(p, q);
    sh.has_eta = sc->tr > 0.0 ? 1 : 0;
    sc->has_eta = sh.has_eta;
  }
  __syncthreads();
  const int has_eta = sh.has_eta;
  const double tr = sc->tr, cx = sc->cx;
  const double a2r = alpha * alpha / rho;
  for (int t = tid; t < K * K; t += blockDim.x) {
    const int i = t / K, j = t % K;
    sh.Q[t] = b1 ? 0.0 : a2r * aug_at(aug, sh.map[i], sh.map[j]);
  }
  if (tid < K) {
    const int gi = sh.map[tid];
    sh.q12[tid] = (has_eta && !b1) ? a2r / tr * aug_at(aug, gi, 36) : 0.0;
    const double gtw = (first_pass && !b1) ? aug_at(aug, gi, 37) : vec[gi];
    // svec of V^T C V (k_c x k_c block)
    int p = 0, q = 0;
    {
      int u = tid;
      for (q = 0; q < kc; ++q) {
        if (u < kc - q) { p = q + u; break; }
        u -= kc - q;
      }
    }
    const double vcpq = 0.5 * (vc[p * 8 + q] + vc[q * 8 + p]);
    const double svc = (p == q) ? vcpq : SQ2 * vcpq;
    sh.h1[tid] = alpha * (gtw - svc);
    sh.v[tid] = (p == q) ? 1.0 : 0.0;
  }
  if (tid == 0) {
    sh.q22 = (has_eta && !b1) ? a2r / (tr * tr) * aug_at(aug, 36, 36) : 0.0;
    // w = y - (b - nu)/rho for the subproblem; y~ itself for App. B.1 (vec[37] = <A Xbar, y~>)
    const double axw = b1 ? vec[37] : (first_pass ? aug_at(aug, 36, 37) : vec[36]);
    sh.h2 = has_eta ? alpha * (axw - cx) / tr : 0.0;
    // strictly feasible start (App. B.1 leaves it free)
    for (int u = 0; u < 64; ++u) { sh.S[u] = 0.0; sh.T[u] = 0.0; }
    for (int p = 0; p < kc; ++p) { sh.S[p * 8 + p] = 1.0 / (2.0 * kc); sh.T[p * 8 + p] = 1.0; }
    sh.eta = has_eta ? 0.25 : 0.0;
    sh.zeta = 1.0;
    sh.omega = 1.0;
    const double slack = 1.0 - 0.5 - sh.eta;
    double m0 = kc * (1.0 / (2.0 * kc)) + sh.omega * slack;
    if (has_eta) m0 += sh.eta * sh.zeta;
    sh.mu = m0 / (has_eta ? 2.0 * (kc + 2) : 2.0 * (kc + 1));
    sh.done = 0;
    sh.iters = 0;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  for (int it = 1; it <= max_iter; ++it) {
    // S^-1 (Gauss-Jordan over the CTA; the system matrix L is assembled later, so its
    // storage serves as the scratch)
    cta_spd_inverse8(sh.S, sh.L, sh.Sinv, kc);
    if (tid < K) {
      int p = 0, q = 0;
      int u = tid;
      for (q = 0; q < kc; ++q) {
        if (u < kc - q) { p = q + u; break; }
        u -= kc - q;
      }
      const double f = (p == q) ? 1.0 : SQ2;
      sh.s[tid] = f * sh.S[p * 8 + q];
      sh.t[tid] = f * sh.T[p * 8 + q];
      sh.sinv[tid] = f * sh.Sinv[p * 8 + q];
    }
    // T (x)_s S^-1 entry by entry: (1/(s_a s_b)) (H_jk G_il + G_jk H_il + H_jl G_ik + G_jl H_ik)
    // with G = T, H = S^-1, a = (i, j), b = (k, l), s = 2 on the diagonal and sqrt(2) off it
    for (int t = tid; t < K * K; t += blockDim.x) {
      const int ra = t / K, cb = t % K;
      int i = 0, j = 0, k = 0, l = 0;
      {
        int u = ra;
        for (j = 0; j < kc; ++j) { if (u < kc - j) { i = j + u; break; } u -= kc - j; }
        u = cb;
        for (l = 0; l < kc; ++l) { if (u < kc - l) { k = l + u; break; } u -= kc - l; }
      }
      const double inv_s = ((i == j) ? 0.5 : 1.0 / SQ2) * ((k == l) ? 0.5 : 1.0 / SQ2);
      const double* G = sh.T;
      const double* H = sh.Sinv;
      sh.TS[t] = (H[j * 8 + k] * G[i * 8 + l] + G[j * 8 + k] * H[i * 8 + l] +
                  H[j * 8 + l] * G[i * 8 + k] + G[j * 8 + l] * H[i * 8 + k]) * inv_s;
    }
    __syncthreads();
    // The k-sized FP64 chains below are split so that no thread runs a K-long dependent
    // sequence (one FP64 warp instruction occupies a sub-partition for many cycles):
    // F1 = Q s + ... with four threads per row (warps 0-4), the scalars in warp 6.
    if (warp <= 4) {
      const int r = tid >> 2, h = tid & 3;
      double f1 = 0.0;
      if (r < K)
        for (int c = h; c < K; c += 4) f1 = fma(sh.Q[r * K + c], sh.s[c], f1);
      f1 += __shfl_xor_sync(FULL, f1, 1);
      f1 += __shfl_xor_sync(FULL, f1, 2);
      if (r < K && h == 0)
        sh.F1[r] = sh.h1[r] - sh.t[r] + sh.omega * sh.v[r] + sh.eta * sh.q12[r] + f1;
    }
    if (warp == 6) {
      double qs = 0.0;
      for (int c = lane; c < K; c += 32) qs = fma(sh.q12[c], sh.s[c], qs);
      for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(FULL, qs, o);
      if (lane == 0) {
        double trS = 0.0;
        for (int p = 0; p < kc; ++p) trS += sh.S[p * 8 + p];
        const double slack = 1.0 - trS - sh.eta;
        sh.kappa1 = slack / sh.omega;
        sh.r3 = sh.mu / sh.omega - slack;
        if (has_eta) {
          const double F2 = qs + sh.eta * sh.q22 + sh.h2 - sh.zeta + sh.omega;
          sh.kappa2 = sh.zeta / sh.eta + sh.q22;
          sh.r2 = -F2 + sh.mu / sh.eta - sh.zeta;
          sh.det = sh.kappa1 * sh.kappa2 + 1.0;
        }
      }
    }
    __syncthreads();
    // assemble [L | rhs] (eq. delta_S_linear_system2)
    {
      const double idet = has_eta ? 1.0 / sh.det : 0.0, ik1 = has_eta ? 0.0 : 1.0 / sh.kappa1;
      for (int t = tid; t < K * (K + 1); t += blockDim.x) {
        const int i = t / (K + 1), j = t % (K + 1);
        double val;
        if (j < K) {
          val = sh.Q[i * K + j] + sh.TS[i * K + j];
          if (has_eta)
            val -= (sh.q12[i] * (sh.kappa1 * sh.q12[j] + sh.v[j]) +
                    sh.v[i] * (sh.q12[j] - sh.kappa2 * sh.v[j])) * idet;
          else
            val += sh.v[i] * sh.v[j] * ik1;
        } else {
          val = -sh.F1[i] + sh.mu * sh.sinv[i] - sh.t[i];
          if (has_eta)
            val -= (sh.q12[i] * (sh.kappa1 * sh.r2 - sh.r3) + sh.v[i] * (sh.kappa2 * sh.r3 + sh.r2)) * idet;
          else
            val -= sh.v[i] * sh.r3 * ik1;
        }
        sh.L[t] = val;
      }
    }
    __syncthreads();
    // Gaussian elimination with partial pivoting on [L | rhs].  Rows are addressed through
    // a permutation instead of being swapped, so warp 0 can look ahead: at pivot p it
    // updates column p+1 first, picks pivot p+1 and forms its reciprocal while warps
    // 1.. update columns p+2..K (the rhs included).  One barrier per pivot.
    const int LDL = K + 1;
    int* cur = sh.perm[0];
    int* nxt = sh.perm[1];
    if (warp == 0) {
      if (lane == 0) sh.piv = 0;
      for (int r = lane; r < K; r += 32) cur[r] = r;
      __syncwarp();
      ipm_pivot(sh, cur, cur, 0, K, LDL, lane);
    }
    __syncthreads();
    for (int p = 0; p < K; ++p) {
      const int P = cur[p];
      const double ipv = sh.fcol[p];
      if (warp == 0) {
        if (p + 1 < K) {
          for (int r = p + 1 + lane; r < K; r += 32) {
            const int pr = cur[r];
            const double mult = sh.L[pr * LDL + p] * ipv;
            sh.L[pr * LDL + p + 1] = fma(-mult, sh.L[P * LDL + p + 1], sh.L[pr * LDL + p + 1]);
          }
          __syncwarp();
          ipm_pivot(sh, cur, nxt, p + 1, K, LDL, lane);
        }
      } else {
        const int nw1 = (blockDim.x >> 5) - 1;
        for (int r = p + 1 + lane; r < K; r += 32) {
          const int pr = cur[r];
          const double mult = sh.L[pr * LDL + p] * ipv;
          for (int c = p + 1 + warp; c < LDL; c += nw1)
            sh.L[pr * LDL + c] = fma(-mult, sh.L[P * LDL + c], sh.L[pr * LDL + c]);
        }
      }
      __syncthreads();
      if (p + 1 < K) { int* t = cur; cur = nxt; nxt = t; }
    }
    // back substitution (warp 0) with the reciprocal pivots kept in fcol; row r of the
    // triangular factor is physical row cur[r].  Lane i keeps the right-hand sides of rows
    // i and i + 32 in registers, so a step is a shuffle, a multiply and a fused update.
    if (warp == 0) {
      double y0 = (lane < K) ? sh.L[cur[lane] * LDL + K] : 0.0;
      double y1 = (lane + 32 < K) ? sh.L[cur[lane + 32] * LDL + K] : 0.0;
      for (int r = K - 1; r >= 0; --r) {
        const double yr = __shfl_sync(FULL, r < 32 ? y0 : y1, r & 31);
        const double x = yr * sh.fcol[r];
        if (lane == 0) sh.ds[r] = x;
        if (lane < r) y0 = fma(-sh.L[cur[lane] * LDL + r], x, y0);
        if (lane + 32 < r) y1 = fma(-sh.L[cur[lane + 32] * LDL + r], x, y1);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // v^T ds and q12^T ds by warp reductions, then the scalar directions (lane 0)
      double vds = 0.0, qds = 0.0;
      for (int c = lane; c < K; c += 32) {
        vds = fma(sh.v[c], sh.ds[c], vds);
        qds = fma(sh.q12[c], sh.ds[c], qds);
      }
      for (int o = 16; o > 0; o >>= 1) {
        vds += __shfl_xor_sync(FULL, vds, o);
        qds += __shfl_xor_sync(FULL, qds, o);
      }
      if (lane == 0 && has_eta) {
        const double a = sh.r2 - qds, cc = sh.r3 + vds;
        sh.deta = (sh.kappa1 * a - cc) / sh.det;
        sh.domega = (sh.kappa2 * cc + a) / sh.det;
        sh.dzeta = sh.mu / sh.eta - sh.zeta - (sh.zeta / sh.eta) * sh.deta;
      } else if (lane == 0) {
        sh.domega = (sh.r3 + vds) / sh.kappa1;
        sh.deta = 0.0;
        sh.dzeta = 0.0;
      }
    } else if (warp <= 5) {
      // dt = mu S^-1 - t - (T (x)_s S^-1) ds, four threads per row (warps 1-5)
      const int r = (tid - 32) >> 2, h = tid & 3;
      double x = 0.0;
      if (r < K)
        for (int c = h; c < K; c += 4) x = fma(sh.TS[r * K + c], sh.ds[c], x);
      x += __shfl_xor_sync(FULL, x, 1);
      x += __shfl_xor_sync(FULL, x, 2);
      if (r < K && h == 0) sh.dt[r] = sh.mu * sh.sinv[r] - sh.t[r] - x;
    }
    __syncthreads();
    // a non-finite Newton direction (singular system): keep the current strictly
    // feasible iterate and stop
    if (warp == 0) {
      bool fin = true;
      for (int c = lane; c < K; c += 32) fin = fin && isfinite(sh.ds[c]) && isfinite(sh.dt[c]);
      fin = __all_sync(FULL, fin);
      if (lane == 0) {
        fin = fin && isfinite(sh.deta) && isfinite(sh.domega) && isfinite(sh.dzeta) && sh.piv >= 0;
        sh.done = fin ? 0 : 2;
      }
    }
    __syncthreads();
    if (sh.done == 2) break;
    if (tid < 64) {
      // smat of ds, dt
      const int p = tid / 8, q = tid % 8;
      double vs = 0.0, vt = 0.0;
      if (p < kc && q < kc) {
        const int pi = max(p, q), qi = min(p, q);
        const int u = svec_idx(pi, qi, kc);
        const double f = (p == q) ? 1.0 : 1.0 / SQ2;
        vs = f * sh.ds[u];
        vt = f * sh.dt[u];
      }
      sh.dS[tid] = vs;
      sh.dT[tid] = vt;
    }
    if (tid == 0) sh.delta = 1.0;
    __syncthreads();
    // backtracking: halve until strictly feasible (warps 0 and 1 test S and T), then 0.95 delta
    for (int ls = 0; ls < 80; ++ls) {
      const double delta = sh.delta;
      if (tid < 64) {
        const int p = tid / 8, q = tid % 8;
        sh.St[tid] = sh.S[tid] + delta * sh.dS[tid];
        sh.Tt[tid] = sh.T[tid] + delta * sh.dT[tid];
        (void)p; (void)q;
      }
      __syncthreads();
      // warps 0 and 1 test S and T by Cholesky; warp 2 meanwhile tests the trace slack
      // and the scalar variables
      bool okw = true;
      if (warp == 0) okw = warp_chol(sh.St, nullptr, kc);
      if (warp == 1) okw = warp_chol(sh.Tt, nullptr, kc);
      if (warp == 2) {
        double trS = (lane < kc) ? sh.St[lane * 9] : 0.0;
        for (int o = 4; o > 0; o >>= 1) trS += __shfl_xor_sync(FULL, trS, o);
        const double en = sh.eta + delta * sh.deta, zn = sh.zeta + delta * sh.dzeta;
        const double on = sh.omega + delta * sh.domega;
        okw = on > 0.0 && (1.0 - trS - en) > 0.0;
        if (has_eta) okw = okw && en > 0.0 && zn > 0.0;
      }
      if (lane == 0 && warp < 3) sh.fcol[warp] = okw ? 1.0 : 0.0;
      __syncthreads();
      if (tid == 0) {
        const bool ok = sh.fcol[0] > 0.5 && sh.fcol[1] > 0.5 && sh.fcol[2] > 0.5;
        sh.done = ok ? 1 : 0;
        if (!ok) sh.delta = 0.5 * delta;
      }
      __syncthreads();
      if (sh.done) break;
    }
    __syncthreads();
    const double delta = 0.95 * sh.delta;
    if (tid < 64) {
      // each thread reads and writes only its own entry of S and T: in place
      const int p = tid / 8, q = tid % 8;
      if (p < kc && q < kc) {
        sh.S[tid] += 0.5 * delta * (sh.dS[p * 8 + q] + sh.dS[q * 8 + p]);
        sh.T[tid] += 0.5 * delta * (sh.dT[p * 8 + q] + sh.dT[q * 8 + p]);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // <S, T> and tr S by warp reductions (entries outside k_c x k_c are zero)
      double st = fma(sh.S[lane], sh.T[lane], sh.S[lane + 32] * sh.T[lane + 32]);
      double trS = (lane < kc) ? sh.S[lane * 9] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_xor_sync(FULL, st, o);
        trS += __shfl_xor_sync(FULL, trS, o);
      }
      if (lane == 0) {
        sh.omega += delta * sh.domega;
        if (has_eta) {
          sh.eta += delta * sh.deta;
          sh.zeta += delta * sh.dzeta;
        }
        double mest = st + sh.omega * (1.0 - trS - sh.eta);
        if (has_eta) mest += sh.eta * sh.zeta;
        mest /= has_eta ? 2.0 * (kc + 2) : 2.0 * (kc + 1);
        const double gamma = sh.delta * 0.95 <= 0.2 ? 1.0 : 0.5 - 0.4 * delta * delta;
        sh.mu = fmin(sh.mu, gamma * mest);
        sh.iters = it;
        sh.done = (sh.mu < mu_tol || !isfinite(sh.mu)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (sh.done) break;
  }
  if (b1) {
    if (tid == 0) {
      // f^ = <b, y~> - min (h1^T svec S + eta h2)
      double v = has_eta ? sh.eta * sh.h2 : 0.0;
      int u = 0;
      for (int q = 0; q < kc; ++q)
        for (int p = q; p < kc; ++p, ++u) v = fma(sh.h1[u], (p == q ? 1.0 : SQ2) * sh.S[p * 8 + q], v);
      sc->f_hat_ipm = vec[36] - v;
      sc->ipm_iters_b1 = sh.iters;
      if (!isfinite(sc->f_hat_ipm)) sc->status = USBS_ENUMERIC;
    }
    return;
  }
  if (tid == 0) {
    for (int u = 0; u < 64; ++u) {
      sc->S_hat[u] = sh.S[u];
      sc->S[u] = alpha * sh.S[u];
    }
    sc->eta_hat = sh.eta;
    sc->eta = has_eta ? alpha * sh.eta / tr : 0.0;
    sc->theta_ipm[0] = sh.zeta;
    sc->theta_ipm[1] = sh.omega;
    sc->theta_ipm[2] = sh.mu;
    sc->ipm_iters += sh.iters;
    if (!isfinite(sh.mu) || !isfinite(sh.eta)) sc->status = USBS_ENUMERIC;
  }
}

// ---- model value, descent test, implicit primal update and gates ------------------------------
// red + RED_VEC holds the reduced candidate sums of k_xupdate:
// [0,36) G^T y~, 36 <b, y~>, 37 <A Xbar, y~>, 38 sum d^2, 39 max |d|.
__device__ __forceinline__ void k_finish_dev(DevScalars* sc, const DevLanczos* lz, const double* USBS_RESTRICT red, int kc,
                         double alpha, double beta, double bnorm, int use_ipm = 0) {
  __shared__ double Zs[64];
  __shared__ float Af[64], Vf[64];
  const double* vec = red + RED_VEC;
  const double* vc = red + RED_VC;
  // V^T (C - A*(y~)) V = V^T C V - smat(G^T y~)
  for (int t = threadIdx.x; t < 64; t += 32) {
    const int p = t / 8, q = t % 8;
    double z = 0.0;
    if (p < kc && q < kc) {
      const int pi = max(p, q), qi = min(p, q);
      const double g = vec[svec_idx8(pi, qi)];
      z = 0.5 * (vc[p * 8 + q] + vc[q * 8 + p]) - ((p == q) ? g : g / SQ2);
    }
    Zs[t] = z;
  }
  __syncwarp();
  const double lamV = warp_lambda_max(Zs, kc, Af, Vf);
  if (threadIdx.x != 0) return;
  double Vc[64];
  for (int p = 0; p < 8; ++p)
    for (int q = 0; q < 8; ++q) Vc[p * 8 + q] = 0.5 * (vc[p * 8 + q] + vc[q * 8 + p]);
  double cxS = 0.0, trS = 0.0;
  for (int p = 0; p < kc; ++p) {
    trS += sc->S[p * 8 + p];
    for (int q = 0; q < kc; ++q) cxS += Vc[p * 8 + q] * sc->S[p * 8 + q];
  }
  const double cx_new = sc->eta * sc->cx + cxS;
  const double tr_new = sc->eta * sc->tr + trS;
  sc->cx_prev = sc->cx;
  sc->tr_prev = sc->tr;
  const double bty = vec[36], axy = vec[37];
  double best = fmax(0.0, lamV);
  if (sc->has_eta) best = fmax(best, (sc->cx - axy) / sc->tr);
  const double f_hat_closed = bty + alpha * best;
  // App. B.1 by the IPM (launched before this kernel) in place of the closed form
  const double f_hat = use_ipm ? sc->f_hat_ipm : f_hat_closed;
  sc->f_hat_closed = f_hat_closed;
  const double lam = lz->theta[0];
  const double f_cand = alpha * fmax(lam, 0.0) + bty;
  const double f_old = sc->f_y;
  const int descent = (beta * (f_old - f_hat) <= f_old - f_cand) ? 1 : 0;
  sc->descent = descent;
  if (descent) sc->f_y = f_cand;
  sc->f_hat = f_hat;
  sc->f_cand = f_cand;
  sc->lam_max = lam;
  sc->bty = bty;
  sc->axy = axy;
  sc->cx_new = cx_new;
  sc->tr_new = tr_new;
  sc->cx = cx_new;
  sc->tr = tr_new;
  sc->cx_it = cx_new;
  sc->tr_it = tr_new;
  sc->relgap = fabs(sc->f_y - cx_new) / (1.0 + fabs(cx_new));
  sc->relinf = sqrt(fmax(vec[38], 0.0)) / (1.0 + bnorm);
  sc->relinf_max = vec[39];
  sc->t += 1;
  if (!isfinite(sc->f_y) || !isfinite(cx_new)) sc->status = USBS_ENUMERIC;
}

// f(y) at the centre y_t from a longer eigen solve (usbs_solve's certification).  A Ritz
// value never exceeds lambda_max, so of two evaluations of f(y_t) the larger is the more
// accurate; it replaces f(y_t) for the gates and for the next descent tests.
__device__ __forceinline__ void k_certify_dev(DevScalars* sc, const DevLanczos* lz, const double* USBS_RESTRICT red,
                                              double alpha) {
  if (threadIdx.x != 0) return;
  const double lam = lz->theta[0];
  const double f = alpha * fmax(lam, 0.0) + red[RED_CERT];
  sc->f_cert = f;
  sc->lam_cert = lam;
  if (f > sc->f_y) sc->f_y = f;
  sc->relgap = fabs(sc->f_y - sc->cx_it) / (1.0 + fabs(sc->cx_it));
  if (!isfinite(sc->f_y)) sc->status = USBS_ENUMERIC;
}

// ---- past information (k_p > 0; Sec. 3, eq. model_update_eigendecomposition) ----------------
// All eigenpairs of a symmetric k x k matrix (k <= 8, row stride 8) in FP64 by one warp:
// parallel cyclic Jacobi with circle ordering on 8 indices, four disjoint rotations per
// round, until the off-diagonal mass of the k x k block is below 1e-30 of its total or 20
// sweeps.  Aw is overwritten (its diagonal ends as the eigenvalues) and Vw receives the
// eigenvectors as columns.  Entries outside the k x k block must be zero: a rotation of
// such a pair is the identity.
__device__ void warp_eig8_f64(double* Aw, double* Vw, int k) {
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < 64; t += 32) Vw[t] = (t / 8 == t % 8) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 20; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = lane; t < 64; t += 32) {
      const double x = Aw[t];
      tot += x * x;
      if (t / 8 != t % 8) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(FULL, off, o);
      tot += __shfl_xor_sync(FULL, tot, o);
    }
    if (!(off > 1e-30 * tot)) break;
    for (int round = 0; round < 7; ++round) {
      double c = 1.0, sv = 0.0;
      int p = 0, q = 0;
      if (lane < 4) {
        const int pa = lane == 0 ? 0 : 1 + ((lane - 1 + round) % 7);
        const int pb = 1 + ((7 - lane - 1 + round) % 7);
        p = min(pa, pb);
        q = max(pa, pb);
        const double apq = Aw[p * 8 + q];
        if (apq != 0.0) {
          const double tau = (Aw[q * 8 + q] - Aw[p * 8 + p]) / (2.0 * apq);
          const double t = fabs(tau) > 1e150 ? 0.5 / tau
                                             : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(tau * tau + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          sv = t * c;
        }
      }
      double cs[4], sn[4];
      int pp[4], qq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cs[u] = __shfl_sync(FULL, c, u);
        sn[u] = __shfl_sync(FULL, sv, u);
        pp[u] = __shfl_sync(FULL, p, u);
        qq[u] = __shfl_sync(FULL, q, u);
      }
      __syncwarp();
      double na = 0.0, nb = 0.0, nc = 0.0, nd = 0.0;
      const int k1 = (lane & 15) / 4, k2 = lane % 4;
      if (lane < 16) {
        const double a = Aw[pp[k1] * 8 + pp[k2]], b = Aw[pp[k1] * 8 + qq[k2]];
        const double cc = Aw[qq[k1] * 8 + pp[k2]], d = Aw[qq[k1] * 8 + qq[k2]];
        const double ra = cs[k1] * a - sn[k1] * cc, rb = cs[k1] * b - sn[k1] * d;
        const double rc = sn[k1] * a + cs[k1] * cc, rd = sn[k1] * b + cs[k1] * d;
        na = cs[k2] * ra - sn[k2] * rb;
        nb = sn[k2] * ra + cs[k2] * rb;
        nc = cs[k2] * rc - sn[k2] * rd;
        nd = sn[k2] * rc + cs[k2] * rd;
      }
      const int kr = lane / 8, row = lane % 8;
      const double vp = Vw[row * 8 + pp[kr]], vq = Vw[row * 8 + qq[kr]];
      __syncwarp();
      if (lane < 16) {
        Aw[pp[k1] * 8 + pp[k2]] = na;
        Aw[pp[k1] * 8 + qq[k2]] = nb;
        Aw[qq[k1] * 8 + pp[k2]] = nc;
        Aw[qq[k1] * 8 + qq[k2]] = nd;
      }
      Vw[row * 8 + pp[kr]] = cs[kr] * vp - sn[kr] * vq;
      Vw[row * 8 + qq[kr]] = sn[kr] * vp + cs[kr] * vq;
      __syncwarp();
    }
  }
}

// Split of S_{t+1} = Q_p L_p Q_p^T + Q_c L_c Q_c^T with (Q_p, L_p) its k_p largest
// eigenpairs (eq. model_update_eigendecomposition).  Writes S_p, S_c and Q_p (8 x 8, the
// k_p columns first) to sc, and the scalars of Xbar_{t+1} = eta Xbar_t + V S_c V^T (eq.
// x_bar_def), summed from Xbar_t's and S_c's like the sketch, not by cancellation from
// X_{t+1}'s: <C, Xbar> = eta <C, Xbar_t> + <V^T C V, S_c>, tr Xbar = eta tr Xbar_t + tr S_c.
// One warp.
__device__ __forceinline__ void k_kp_split_dev(DevScalars* sc, const double* USBS_RESTRICT red, int kdim, int kp) {
  __shared__ double Aw[64], Vw[64], lam[8];
  __shared__ int ord[8];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  for (int t = lane; t < 64; t += 32) {
    const int i = t / 8, j = t % 8;
    Aw[t] = (i < kdim && j < kdim) ? 0.5 * (sc->S[i * 8 + j] + sc->S[j * 8 + i]) : 0.0;
  }
  __syncwarp();
  warp_eig8_f64(Aw, Vw, kdim);
  if (lane < 8) lam[lane] = Aw[lane * 9];
  __syncwarp();
  if (lane < kdim) {
    // descending order under a strict total order (value, then index)
    int rank = 0;
    for (int u = 0; u < kdim; ++u)
      if (lam[u] > lam[lane] || (lam[u] == lam[lane] && u < lane)) ++rank;
    ord[rank] = lane;
  }
  __syncwarp();
  for (int t = lane; t < 64; t += 32) {
    const int i = t / 8, j = t % 8;
    double sp = 0.0, scv = 0.0;
    if (i < kdim && j < kdim) {
      for (int u = 0; u < kdim; ++u) {
        const int e = ord[u];
        const double x = lam[e] * Vw[i * 8 + e] * Vw[j * 8 + e];
        if (u < kp) sp += x; else scv += x;
      }
    }
    sc->Sp[t] = sp;
    sc->Sc[t] = scv;
    sc->Qp[t] = (i < kdim && j < kp) ? Vw[i * 8 + ord[j]] : 0.0;
  }
  __syncwarp();
  if (lane == 0) {
    const double* vc = red + RED_VC;
    double ccx = 0.0, ctr = 0.0;
    for (int p = 0; p < kdim; ++p) {
      ctr += sc->Sc[p * 8 + p];
      for (int q = 0; q < kdim; ++q) ccx += 0.5 * (vc[p * 8 + q] + vc[q * 8 + p]) * sc->Sc[p * 8 + q];
    }
    sc->cx = sc->eta * sc->cx_prev + ccx;
    sc->tr = sc->eta * sc->tr_prev + ctr;
    if (!isfinite(sc->cx) || !isfinite(sc->tr)) sc->status = USBS_ENUMERIC;
  }
}

__device__ __forceinline__ void k_cold_dev(DevScalars* sc, const DevLanczos* lz, double alpha) {
  if (threadIdx.x != 0) return;
  sc->f_y = alpha * fmax(lz->theta[0], 0.0);
  sc->cx = 0.0;
  sc->tr = 0.0;
  sc->cx_it = 0.0;
  sc->tr_it = 0.0;
  sc->has_eta = 0;
  sc->t = 0;
  sc->status = 0;
  sc->lam_max = lz->theta[0];
}

__device__ __forceinline__ void k_begin_step_dev(DevScalars* sc) {
  if (threadIdx.x != 0) return;
  sc->ipm_iters = 0;
  sc->n_alt = 0;
}

__device__ __forceinline__ void k_commit_dev(const int cta, const int ncta, int m, const DevScalars* USBS_RESTRICT sc, const double* USBS_RESTRICT ycand,
                         double* USBS_RESTRICT y) {
  if (!sc->descent) return;
  for (int64_t c = (int64_t)cta * blockDim.x + threadIdx.x; c < m; c += (int64_t)ncta * blockDim.x) y[c] = ycand[c];
}

__device__ __forceinline__ void k_lanczos_reset_dev(DevLanczos* lz) {
  for (int t = threadIdx.x; t < JMAX * JMAX; t += blockDim.x) lz->T[t] = 0.0;
  if (threadIdx.x == 0) {
    lz->sweeps = 0;
    lz->status = 0;
    lz->defl = 0;
    lz->defl_seen = 0;
    lz->redo = 0;
    lz->converged = 0;
    lz->cycles = 0;
    lz->normest = 0.0;
  }
}

}  // namespace
}  // namespace usbs
