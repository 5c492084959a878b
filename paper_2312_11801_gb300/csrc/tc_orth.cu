// Gram-Schmidt and restart tiles of the mixed-precision (FP32) Lanczos step on the
// 5th-generation tensor cores (tcgen05), staged by bulk tensor copies (TMA).
//
// A CTA of 128 threads walks tiles of 128 rows.  Per tile:
//  1. TMA copies the 128-row tile of each basis block Q_b (and of the new block W) into a
//     double-buffered stage, 32-byte swizzled: as it lands, a block's tile is the K-major
//     tf32 operand of Q H (M = 128 rows, K = 8 columns).
//  2. A split pass writes, from the staged tile, what the tensor core still needs:
//       - lo = x - hi(x) in the same layout (the raw tile is the hi operand: the tensor
//         core truncates to tf32), for products with the rows as M;
//       - hi and lo, each 8 x 8 sub-tile transposed, for products with the rows as K
//         (Gram-type sums over the rows; only K-major operands are taken).
//  3. Phase 1 (update, finalize, restart): D1 = Q [H_hi | H_lo] + Q_lo [H_hi | 0] into TMEM
//     (M = 128, N = 16), so that Q H = D1[:, :8] + D1[:, 8:].  Each thread owns one row: it
//     reads its accumulator lane, forms X = W - Q H (update, finalize) or the restarted
//     vectors, writes them to HBM and, for the update, X's transposed hi/lo planes.
//  4. Phase 2 (projection, update): D2 += [Q_hi; X_hi; Q_lo; X_lo]^T [X_hi | X_lo] over the
//     tile's rows (M = 16 (nb + 1) rows padded to 64 or 128, N = 16, K = 8 rows per MMA),
//     accumulated in TMEM over all tiles of the CTA; at the end the four hi/lo products
//     are added and written as the CTA's FP64 partial sums of H2 = Q^T X and G = X^T X
//     (or H = Q^T W), the layout the reduction kernel expects.
// Every wait is bounded; a wait that runs out sets USBS_ETIMEOUT in the Lanczos status
// word, and the CTA leaves its loop together, waits (bounded) for its copies and MMAs in
// flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dev_orth.cuh"
#include "tc_orth.cuh"

namespace usbs {
namespace {

enum TcMode { TC_PROJ = 0, TC_UPDATE = 1, TC_FINAL = 2, TC_RESTART = 3 };

constexpr int TC_TR = 128;          // rows per tile
constexpr int TC_THREADS = 256;
constexpr int TC_TMEM_COLS = 128;   // D1 at column 0 (up to 64 wide), D2 chunks at 64 and 80
constexpr int TC_D2 = 64;

struct TcArgs {
  int n, nb, ntiles;          // rows, basis blocks used, tiles of 128 rows
  int qblk0, wblk;            // block of Q_0 in the Q map, block of W in the W map
  const double* H;            // update: H (nb x 64); finalize: H2 (nb x 64)
  const DevLanczos* lz;       // finalize: Rinv and the deflation flags
  float* wout;                // update: X (rewrites W); finalize: the new block
  double* partials;           // projection, update: per-CTA FP64 partial sums
  int* status;                // Lanczos status word (USBS_ETIMEOUT on a wait that runs out)
  uint64_t seed;              // finalize: seed of replacement columns
  const double* Y;            // restart: Ritz vectors, J x JMAX row-major
  int nout;                   // restart: output blocks (1..4)
  float* out;                 // restart: first output block
  size_t ostride;             // restart: floats between output blocks
  const float* resid;         // restart: residual block copied to out[resid_slot], or null
  int resid_slot;
  const int* mask;            // masked deflation passes: the launch does nothing if *mask == 0
};

struct TcLayout {
  int stage_bytes, stage, lo, tpl, tgroup, b1, bars, total;
};

// Shared-memory plan of one CTA (bytes, every region 1024-aligned)
__host__ __device__ inline TcLayout tc_layout(int mode, int nb, int nout) {
  TcLayout L{};
  const int nsb = mode == TC_RESTART ? nb : nb + 1;
  L.stage_bytes = nsb * 4096;
  L.stage = 0;
  int off = 2 * L.stage_bytes;
  L.lo = off;                 // the finalize also uses it as a 128 x 8 row buffer
  if (mode != TC_PROJ) off += (mode == TC_FINAL ? (nb > 1 ? nb : 1) : nb) * 4096;
  L.tpl = off;
  L.tgroup = 2 * (nb + 1) * 256;
  if (mode == TC_PROJ || mode == TC_UPDATE) off += 16 * L.tgroup + 4096;   // + reads of padded M
  L.b1 = off;
  if (mode == TC_UPDATE || mode == TC_FINAL) off += nb * 1024;
  if (mode == TC_RESTART) off += nb * 1024 * nout;
  off = (off + 1023) & ~1023;
  L.bars = off;               // 4 mbarriers, the TMEM address, R^-1 (64 floats), 8 flags
  L.total = off + 512;
  return L;
}

// Phase-1 B operands of block b (K = its 8 rows of H, N = 16): B' = [H_hi | H_lo] at
// b1 + 1024 b, B'' = [H_hi | 0] at b1 + 1024 b + 512; stored K-major (row n holds column n
// of H), 32-byte swizzled.  For the restart, N = 16 nout: [Y_hi | Y_lo] and [Y_hi | 0] over
// the nout output blocks, 1024 nout bytes per basis block.
__device__ __forceinline__ void write_b1(float* b1, int nb, int ncol, const double* src, int ld) {
  // src(k, c) = src[(8 b + k) * ld + c] for block b, c < ncol
  const int per = 2 * 2 * ncol * 8;   // floats of B' and B'' of one block
  for (int t = threadIdx.x; t < nb * 2 * ncol * 8; t += blockDim.x) {
    const int b = t / (2 * ncol * 8), rem = t % (2 * ncol * 8);
    const int nrow = rem / 8, k = rem % 8;            // nrow < 2 ncol
    const int c = nrow % ncol, half = nrow / ncol;    // half 0: hi columns, 1: lo columns
    const float x = (float)src[(size_t)(8 * b + k) * ld + c];
    const float hi = tc::tf32_hi(x);
    float* base = b1 + (size_t)b * per;
    base[tc::sw(nrow, k)] = half == 0 ? hi : x - hi;                 // B'
    base[2 * ncol * 8 + tc::sw(nrow, k)] = half == 0 ? hi : 0.f;     // B''
  }
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_tc(const __grid_constant__ CUtensorMap mapQ,
                                                   const __grid_constant__ CUtensorMap mapW, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  if (a.mask && *a.mask == 0) return;
  const int nb = a.nb;
  const TcLayout L = tc_layout(MODE, nb, a.nout);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);   // 0, 1: stages; 2: phase 1; 3: phase 2
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + L.bars + 64);
  float* lo = reinterpret_cast<float*>(smem + L.lo);
  float* T = reinterpret_cast<float*>(smem + L.tpl);
  float* B1 = reinterpret_cast<float*>(smem + L.b1);
  float* Ri = reinterpret_cast<float*>(smem + L.bars + 128);
  int* dcol = reinterpret_cast<int*>(smem + L.bars + 384);
  const int ncol1 = MODE == TC_RESTART ? 8 * a.nout : 8;      // columns of the phase-1 product
  const int N1 = 2 * ncol1;
  const int my_tiles = (int)blockIdx.x < a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::bar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (MODE == TC_UPDATE || MODE == TC_FINAL) write_b1(B1, nb, 8, a.H, 8);
  if (MODE == TC_RESTART) write_b1(B1, nb, ncol1, a.Y, JMAX);
  if (MODE == TC_FINAL) {
    if (tid < 64) Ri[tid] = (float)a.lz->Rinv[tid];
    if (tid < 8) dcol[tid] = a.lz->dcol[tid];
  }
  if (warp == 0) tc::tmem_alloc(slot, TC_TMEM_COLS);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  // TMEM lanes of this warp (warps w and w + 4 share the lanes 32 (w % 4) ..)
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int r_own = (warp & 3) * 32 + lane;       // the tile row this thread works on
  const int chalf = warp >> 2;                    // its half of the 8 columns

  auto issue_tile = [&](int s, int k) {   // k-th tile of this CTA into stage s
    const int tile = blockIdx.x + k * gridDim.x;
    unsigned char* st = smem + L.stage + s * L.stage_bytes;
    tc::fence_async_smem();
    tc::bar_expect_tx(&bars[s], (unsigned)L.stage_bytes);
    for (int b = 0; b < nb; ++b) tc::tma_tile(st + b * 4096, &mapQ, tile * TC_TR, a.qblk0 + b, &bars[s]);
    if (MODE != TC_RESTART) tc::tma_tile(st + nb * 4096, &mapW, tile * TC_TR, a.wblk, &bars[s]);
  };
  if (tid == 0) {
    if (my_tiles > 0) issue_tile(0, 0);
    if (my_tiles > 1) issue_tile(1, 1);
  }

  // phase-2 M chunks: atoms [0, 16) with M = 128 (or 64 if there are at most 8), then the
  // rest with M = 64 or 128
  const int atoms = 2 * (nb + 1);
  const int m2a = atoms <= 8 ? 64 : 128;
  const int atoms_b = atoms > 16 ? atoms - 16 : 0;
  const int m2b = atoms_b <= 8 ? 64 : 128;
  // transposing copies of the split pass: thread -> (m, k) inside an atom and one of 4 atoms
  // per pass; its read and write offsets inside a block's tile and an atom are fixed
  const int tm = (tid >> 3) & 7, tk = tid & 7, tq = tid >> 6;
  const int rd_off = tc::sw(tk, tm);          // (row tk of an 8-row group, column tm)
  const int wr_off = tc::sw(tm, tk);          // (row tm, column tk) of a transposed atom
  const int tg = L.tgroup / 4;                // floats per k-group of atoms

  bool aborted = false;
  int it = 0;
  unsigned ph1 = 0, ph2 = 0;
  bool p1_out = false, p2_out = false;   // committed MMAs not yet waited for
  for (; it < my_tiles; ++it) {
    const int s = it & 1;
    const int tile = blockIdx.x + it * gridDim.x;
    float* st = reinterpret_cast<float*>(smem + L.stage + s * L.stage_bytes);
    // one thread waits (the others sleep in the barrier); afterwards every thread observes
    // the completed phases itself (a test that returns at once) to acquire their writes
    bool ok = true;
    if (tid == 0) {
      ok = tc::bar_wait(&bars[s], (it >> 1) & 1);
      if (ok && p2_out) ok = tc::bar_wait(&bars[3], ph2);
    }
    if (!__syncthreads_and(ok)) { aborted = true; break; }
    tc::bar_test(&bars[s], (it >> 1) & 1);
    if (p2_out) { tc::bar_test(&bars[3], ph2); p2_out = false; ph2 ^= 1; }
    tc::fence_after_sync();

    // ---- split pass ----
    if (MODE == TC_FINAL || MODE == TC_RESTART) {
      // lo of every Q element, in the staged (swizzled) layout
      const int nvec = nb * TC_TR * 2;
      for (int v = tid; v < nvec; v += TC_THREADS) {
        const float4 x = reinterpret_cast<const float4*>(st)[v];
        float4 y;
        y.x = tc::tf32_lo(x.x, tc::tf32_hi(x.x)); y.y = tc::tf32_lo(x.y, tc::tf32_hi(x.y));
        y.z = tc::tf32_lo(x.z, tc::tf32_hi(x.z)); y.w = tc::tf32_lo(x.w, tc::tf32_hi(x.w));
        reinterpret_cast<float4*>(lo)[v] = y;
      }
    } else {
      // transposed hi / lo atoms: atom (ks, h, b) holds, as its row m and column k, the value
      // of column m of block b at tile row 8 ks + k (and the update also writes the lo of the
      // element in the staged layout for phase 1).  Both the reads (8 rows x 4 columns of the
      // swizzled tile) and the transposed writes (128 contiguous bytes) of a warp are free of
      // bank conflicts.
      const int nblk = MODE == TC_PROJ ? nb + 1 : nb;
      const int tlo = (nb + 1) * 64;
      for (int b = 0; b < nblk; ++b) {
        const float* src = st + b * 1024 + tq * 64 + rd_off;
        float* lrow = lo + b * 1024 + tq * 64 + rd_off;
        float* dst = T + tq * tg + b * 64 + wr_off;
#pragma unroll
        for (int ks = 0; ks < 16; ks += 4) {
          const float x = src[ks * 64];
          const float hi = tc::tf32_hi(x);
          const float l = tc::tf32_lo(x, hi);
          if (MODE == TC_UPDATE) lrow[ks * 64] = l;
          dst[ks * tg] = hi;
          dst[ks * tg + tlo] = l;
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    if (MODE != TC_PROJ) {
      // ---- phase 1: D1 = Q B' + Q_lo B'' ----
      const bool run1 = nb > 0;
      if (tid == 0 && run1) {
        const uint32_t id1 = tc::idesc_tf32(128, N1);
        const uint32_t sq = tc::su32(st), sl = tc::su32(lo), sb = tc::su32(B1);
        const int bper = 2 * N1 * 32;      // bytes of B' + B'' of one block
        for (int b = 0; b < nb; ++b) {
          tc::mma_tf32(tmem, tc::desc_k32(sq + b * 4096, 256), tc::desc_k32(sb + b * bper, 256), id1, b > 0);
          tc::mma_tf32(tmem, tc::desc_k32(sl + b * 4096, 256), tc::desc_k32(sb + b * bper + N1 * 32, 256), id1, 1);
        }
        tc::mma_commit(&bars[2]);
      }
      if (run1) p1_out = true;
      ok = !run1 || tid != 0 || tc::bar_wait(&bars[2], ph1);
      if (!__syncthreads_and(ok)) { aborted = true; break; }
      if (run1) { tc::bar_test(&bars[2], ph1); p1_out = false; ph1 ^= 1; }
      tc::fence_after_sync();
      const int r = r_own;
      const int row = tile * TC_TR + r;
      const int c0 = 4 * chalf;
      if (MODE == TC_UPDATE || MODE == TC_FINAL) {
        // X = W - Q H on this thread's row, columns c0 .. c0 + 3
        float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
        if (run1) {
          tc::tmem_ld4(tmem + lane_base + c0, dh);
          tc::tmem_ld4(tmem + lane_base + 8 + c0, dl);
        }
        const float* wr = st + nb * 1024;
        float x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = wr[tc::sw(r, c0 + c)] - (dh[c] + dl[c]);
        if (MODE == TC_UPDATE) {
          if (row < a.n)
            *reinterpret_cast<float4*>(a.wout + (size_t)8 * row + c0) = make_float4(x[0], x[1], x[2], x[3]);
          // X's transposed hi / lo atoms (rows past n are zero: W arrived as zeros there)
          float* at = T + (r >> 3) * tg + nb * 64;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float hi = tc::tf32_hi(x[c]);
            at[tc::sw(c0 + c, r & 7)] = hi;
            at[(nb + 1) * 64 + tc::sw(c0 + c, r & 7)] = tc::tf32_lo(x[c], hi);
          }
        } else {
          // the new block (X R^-1): the row's other half comes through shared memory (the lo
          // plane is free once phase 1 has completed)
          *reinterpret_cast<float4*>(lo + 8 * r + c0) = make_float4(x[0], x[1], x[2], x[3]);
          __syncthreads();
          if (row < a.n) {
            const float4 xa = *reinterpret_cast<const float4*>(lo + 8 * r);
            const float4 xb = *reinterpret_cast<const float4*>(lo + 8 * r + 4);
            const float xr[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float acc = 0.f;
#pragma unroll
              for (int e = 0; e < 8; ++e) acc = fmaf(xr[e], Ri[e * 8 + c0 + c], acc);
              const int dc = dcol[c0 + c];
              if (dc == 1) acc = (float)hash_uniform_o(a.seed, (uint64_t)row, (uint64_t)(c0 + c));
              else if (dc == 2) acc = 0.f;
              o[c] = acc;
            }
            *reinterpret_cast<float4*>(a.wout + (size_t)8 * row + c0) = make_float4(o[0], o[1], o[2], o[3]);
          }
        }
      } else {   // TC_RESTART: out_o = D1[:, 8 o : 8 o + 8] + D1[:, 8 nout + 8 o : ...]
        for (int ob = 0; ob < a.nout; ++ob) {
          float dh[4], dl[4];
          tc::tmem_ld4(tmem + lane_base + 8 * ob + c0, dh);
          tc::tmem_ld4(tmem + lane_base + ncol1 + 8 * ob + c0, dl);
          if (row < a.n)
            *reinterpret_cast<float4*>(a.out + ob * a.ostride + (size_t)8 * row + c0) =
                make_float4(dh[0] + dl[0], dh[1] + dl[1], dh[2] + dl[2], dh[3] + dl[3]);
        }
        if (a.resid && row < a.n)
          *reinterpret_cast<float4*>(a.out + a.resid_slot * a.ostride + (size_t)8 * row + c0) =
              *reinterpret_cast<const float4*>(a.resid + (size_t)8 * row + c0);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }

    if (MODE == TC_PROJ || MODE == TC_UPDATE) {
      // ---- phase 2: D2 += [hi; lo]^T [X_hi | X_lo] over the 16 groups of 8 rows ----
      if (tid == 0) {
        const uint32_t t0 = tc::su32(T);
        for (int ks = 0; ks < 16; ++ks) {
          const uint32_t g = t0 + ks * L.tgroup;
          const uint64_t bdesc = tc::desc_k32(g + nb * 256, (nb + 1) * 256);
          const int acc = (it > 0 || ks > 0) ? 1 : 0;
          tc::mma_tf32(tmem + TC_D2, tc::desc_k32(g, 256), bdesc, tc::idesc_tf32(m2a, 16), acc);
          if (atoms_b > 0)
            tc::mma_tf32(tmem + TC_D2 + 16, tc::desc_k32(g + 16 * 256, 256), bdesc, tc::idesc_tf32(m2b, 16), acc);
        }
        tc::mma_commit(&bars[3]);
      }
      p2_out = true;
    }
    // refill this stage (its raw tile is no longer read: phase 1 and the epilogue are done)
    if (tid == 0 && it + 2 < my_tiles) issue_tile(s, it + 2);
  }

  if (!aborted && p2_out) {
    const bool ok = tid != 0 || tc::bar_wait(&bars[3], ph2);
    if (!__syncthreads_and(ok)) aborted = true;
    else { tc::bar_test(&bars[3], ph2); p2_out = false; ph2 ^= 1; }
  }
  if (aborted) {
    if (tid == 0) atomicExch(a.status, USBS_ETIMEOUT);
    // copies and MMAs that may still be in flight: tiles it and it + 1, the open phases
    for (int k = it; k < it + 2 && k < my_tiles; ++k) tc::bar_wait(&bars[k & 1], (k >> 1) & 1);
    if (p1_out) tc::bar_wait(&bars[2], ph1);
    if (p2_out) tc::bar_wait(&bars[3], ph2);
  } else if ((MODE == TC_PROJ || MODE == TC_UPDATE) && my_tiles > 0) {
    // D2 rows to shared memory (the transposed planes are free now), then the partial sums
    tc::fence_after_sync();
    float* Ds = T;                                         // rows x 16
    if (warp < 4) {
      float d[16];
      tc::tmem_ld16(tmem + lane_base + TC_D2, d);
      const int rr = m2a == 128 ? tid : (lane < 16 ? 16 * warp + lane : -1);
      if (rr >= 0 && rr < atoms * 8)
        for (int c = 0; c < 16; ++c) Ds[rr * 16 + c] = d[c];
      if (atoms_b > 0) {
        tc::tmem_ld16(tmem + lane_base + TC_D2 + 16, d);
        const int rb = m2b == 128 ? tid : (lane < 16 ? 16 * warp + lane : -1);
        if (rb >= 0 && 128 + rb < atoms * 8)
          for (int c = 0; c < 16; ++c) Ds[(128 + rb) * 16 + c] = d[c];
      }
    }
    __syncthreads();
    const int nout_blk = MODE == TC_PROJ ? nb : nb + 1;   // the update adds G = X^T X
    double* part = a.partials + (size_t)blockIdx.x * PART_STRIDE;
    for (int o = tid; o < nout_blk * 64; o += TC_THREADS) {
      const int b = o >> 6, am = (o >> 3) & 7, c = o & 7;
      const int rh = 8 * b + am, rl = 8 * (nb + 1 + b) + am;
      const float sum = (Ds[rh * 16 + c] + Ds[rh * 16 + 8 + c]) + (Ds[rl * 16 + c] + Ds[rl * 16 + 8 + c]);
      part[(b < nb ? b * 64 : 512) + am * 8 + c] = (double)sum;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TC_TMEM_COLS);
  if (tid == 0)
    for (int i = 0; i < 4; ++i) tc::bar_inval(&bars[i]);
}

// ---------------------------------------------------------------------------------------
// Host side: tensor maps of a context's n x 8 FP32 buffers and the launchers
// ---------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

template <int MODE>
void set_smem_attr() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
}

template <int MODE>
int tc_grid(Ctx* c, int ntiles, size_t smem, bool partials) {
  struct Entry { size_t s; int v; };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
      if (e.s == smem) per_sm = e.v;
    if (!per_sm) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc<MODE>, TC_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
      }
      per_sm = std::max(1, std::min(per_sm, 512 / TC_TMEM_COLS));   // TMEM: 512 columns per SM
      cache.push_back({smem, per_sm});
    }
  }
  int64_t g = std::min<int64_t>(ntiles, (int64_t)per_sm * c->num_sms);
  if (partials) g = std::min<int64_t>(g, c->max_parts);
  return (int)std::max<int64_t>(g, 1);
}

template <int MODE>
int tc_launch(Ctx* c, const CUtensorMap& mq, const CUtensorMap& mw, TcArgs a) {
  const TcLayout L = tc_layout(MODE, a.nb, a.nout);
  set_smem_attr<MODE>();
  a.ntiles = (int)((c->n + TC_TR - 1) / TC_TR);
  a.n = (int)c->n;
  a.status = DEV_FIELD(c->lz, DevLanczos, status, int);
  const int g = tc_grid<MODE>(c, a.ntiles, L.total, MODE == TC_PROJ || MODE == TC_UPDATE);
  k_tc<MODE><<<g, TC_THREADS, L.total, c->stream>>>(mq, mw, a);
  return g;
}

}  // namespace

// Registers the tensor maps of the FP32 n x 8 buffers (basis Q and Q2 with NBMAX blocks,
// V, Vnew, W) of a mixed-precision context: a 3-D map {8 values, n rows, blocks} with boxes
// of 8 x 128 x 1 and 32-byte swizzle.  Without the driver's encoder the tiles stay on the
// legacy path.
void tc_register(Ctx* c) {
  c->tma.clear();
  if (c->fp64 || !c->use_tc) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) { c->use_tc = false; return; }
  const size_t bs = (size_t)c->n * 8 * sizeof(float);
  auto add = [&](void* base, int blocks) {
    TmaEntry e;
    e.base = static_cast<const char*>(base);
    e.bytes = bs * blocks;
    cuuint64_t dims[3] = {8, (cuuint64_t)c->n, (cuuint64_t)blocks};
    cuuint64_t strides[2] = {32, (cuuint64_t)bs};
    cuuint32_t box[3] = {8, TC_TR, 1};
    cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) c->use_tc = false;
    c->tma.push_back(e);
  };
  add(c->Q, NBMAX);
  add(c->Q2, NBMAX);
  add(c->V, 1);
  add(c->Vnew, 1);
  add(c->W, 1);
  if (!c->use_tc) c->tma.clear();
}

static const TmaEntry* tc_find(const Ctx* c, const void* p, int* blk) {
  const char* q = static_cast<const char*>(p);
  const size_t bs = (size_t)c->n * 8 * sizeof(float);
  for (const TmaEntry& e : c->tma)
    if (q >= e.base && q < e.base + e.bytes && (size_t)(q - e.base) % bs == 0) {
      *blk = (int)((size_t)(q - e.base) / bs);
      return &e;
    }
  return nullptr;
}

static TcArgs tc_args() {
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nout = 1;
  return a;
}

// H = Q^T W (nb blocks); returns the grid (the partial rows to reduce), or 0 if the buffers
// have no tensor map (the caller takes the legacy path)
int tc_proj(Ctx* c, const void* Q, int nb, const void* W, const int* mask) {
  int qb = 0, wb = 0;
  const TmaEntry* eq = tc_find(c, Q, &qb);
  const TmaEntry* ew = tc_find(c, W, &wb);
  if (!eq || !ew || nb < 1 || nb > 8) return 0;
  TcArgs a = tc_args();
  a.nb = nb; a.qblk0 = qb; a.wblk = wb; a.partials = c->partials; a.mask = mask;
  return tc_launch<TC_PROJ>(c, eq->map, ew->map, a);
}

// X = W - Q H (W rewritten), H2 = Q^T X, G = X^T X; H in red + RED_H
int tc_update(Ctx* c, const void* Q, int nb, void* W, const int* mask) {
  int qb = 0, wb = 0;
  const TmaEntry* eq = tc_find(c, Q, &qb);
  const TmaEntry* ew = tc_find(c, W, &wb);
  if (!eq || !ew || nb < 0 || nb > 8) return 0;
  TcArgs a = tc_args();
  a.nb = nb; a.qblk0 = qb; a.wblk = wb; a.partials = c->partials; a.mask = mask;
  a.H = c->red + RED_H; a.wout = static_cast<float*>(W);
  return tc_launch<TC_UPDATE>(c, eq->map, ew->map, a);
}

// out = (W - Q H2) R^-1 with the deflation replacements; H2 in red + RED_H2
bool tc_final(Ctx* c, const void* Q, int nb, const void* W, void* out, const int* mask, uint64_t seed) {
  int qb = 0, wb = 0;
  const TmaEntry* eq = tc_find(c, Q, &qb);
  const TmaEntry* ew = tc_find(c, W, &wb);
  if (!eq || !ew || nb < 0 || nb > 8) return false;
  TcArgs a = tc_args();
  a.nb = nb; a.qblk0 = qb; a.wblk = wb; a.mask = mask; a.seed = seed;
  a.H = c->red + RED_H2; a.lz = c->lz; a.wout = static_cast<float*>(out);
  tc_launch<TC_FINAL>(c, eq->map, ew->map, a);
  return true;
}

// out[o] = Q[:, :J] Y[:, 8 o : 8 o + 8] for o < nout; the residual block copied to
// out[resid_slot] when given
bool tc_restart(Ctx* c, const void* Q, int J, int nout, const double* Y, void* out, const void* resid,
                int resid_slot) {
  int qb = 0;
  const TmaEntry* eq = tc_find(c, Q, &qb);
  if (!eq || J / 8 < 1 || J / 8 > 8 || nout < 1 || nout > 4) return false;
  TcArgs a = tc_args();
  a.nb = J / 8; a.qblk0 = qb; a.Y = Y; a.nout = nout; a.out = static_cast<float*>(out);
  a.ostride = (size_t)c->n * 8; a.resid = static_cast<const float*>(resid); a.resid_slot = resid_slot;
  tc_launch<TC_RESTART>(c, eq->map, eq->map, a);
  return true;
}

}  // namespace usbs
