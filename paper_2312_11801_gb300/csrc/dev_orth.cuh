// Device bodies of the block Gram-Schmidt kernels, staged through shared memory by bulk
// asynchronous copies (a pipeline of ns tiles of TR rows, 2 <= ns <= NSMAX).  A body takes its CTA index and CTA count
// as arguments: the __global__ kernels in orth.cu pass blockIdx.x and gridDim.x, and the
// batched solver calls a body with (0, 1), one CTA walking every tile.
#pragma once

#include "common.cuh"

namespace usbs {
namespace {

template <typename T> struct TileRows;
template <> struct TileRows<float> { static constexpr int value = 128; };
template <> struct TileRows<double> { static constexpr int value = 64; };
// a staged block is TR rows of 8 values plus 32 bytes: the same row of consecutive blocks
// then falls in different shared-memory banks (TR * 8 values alone is a multiple of 128 B)
template <typename T> struct BlockStride {
  static constexpr int value = TileRows<T>::value * 8 + 32 / (int)sizeof(T);
};

// vector shared-memory accesses: 4 or 8 consecutive values (16-byte aligned), 2 values
// (8-byte aligned for float, 16-byte for double)
template <typename T> __device__ __forceinline__ void lds4(const T* p, T (&v)[4]);
template <> __device__ __forceinline__ void lds4<float>(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <> __device__ __forceinline__ void lds4<double>(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T> __device__ __forceinline__ void lds8(const T* p, T (&v)[8]) {
  T a[4], b[4];
  lds4<T>(p, a);
  lds4<T>(p + 4, b);
#pragma unroll
  for (int u = 0; u < 4; ++u) { v[u] = a[u]; v[4 + u] = b[u]; }
}
template <typename T> __device__ __forceinline__ void lds2(const T* p, T& x, T& y);
template <> __device__ __forceinline__ void lds2<float>(const float* p, float& x, float& y) {
  const float2 a = *reinterpret_cast<const float2*>(p);
  x = a.x; y = a.y;
}
template <> __device__ __forceinline__ void lds2<double>(const double* p, double& x, double& y) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  x = a.x; y = a.y;
}
template <typename T> __device__ __forceinline__ void sts4(T* p, const T (&v)[4]);
template <> __device__ __forceinline__ void sts4<float>(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void sts4<double>(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}



// ---- out = (W - Q H2) R^-1; deficient columns replaced by random vectors -----------------------
__device__ __forceinline__ double hash_uniform_o(uint64_t seed, uint64_t row, uint64_t col) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (row * 16 + col + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}



// ---- TMA staging of tiles ------------------------------------------------------------------
// The tile of one block (rows row0 .. row0 + TR - 1, 8 values each) is contiguous in the
// block-major layout, so one bulk asynchronous copy (cp.async.bulk) moves it; one thread
// issues the copies of a tile and an mbarrier with a transaction count tells the CTA when
// they have landed.  Rows past n are not copied: the threads zero them in shared memory.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The tile pipeline has ns stages (2 <= ns <= NSMAX), each with its own barrier: iteration
// k of a CTA's tile loop (tile cta + k ncta) reads stage k % ns and waits for phase k / ns
// of barrier k % ns; at its top it issues the copies of iteration k + ns - 1 into the stage
// that iteration k - 1 released at its closing __syncthreads.  ns - 1 tiles are thus in
// flight while one is used: deeper pipelines keep more bytes in flight when the stages are
// small (few basis blocks).
constexpr int NSMAX = 4;

// Stage barriers, initialised by thread 0 and published by the barrier that follows.
__device__ __forceinline__ void tiles_begin(uint64_t* bar, int ns) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
}

// Stage indices of the loop: s (the stage read in this iteration) with its barrier phase,
// and sl (the stage the copies issued in this iteration go to, (s + ns - 1) % ns).
struct TileRing {
  int ns, s, ph, sl;
  __device__ explicit TileRing(int ns_) : ns(ns_), s(0), ph(0), sl(ns_ - 1) {}
  __device__ void next() {
    if (++s == ns) { s = 0; ph ^= 1; }
    if (++sl == ns) sl = 0;
  }
};

// Stage rows [row0, row0 + TR) of blocks 0..nq-1 of Q and of W (if given, after them).
template <typename T, int TR>
__device__ __forceinline__ void tile_load(T* stage, const T* Q, size_t bstride, int nq, const T* W, int n,
                                          int row0, uint64_t* bar) {
  constexpr int BS = BlockStride<T>::value;
  const int valid = min(TR, n - row0);
  const int nblk = nq + (W ? 1 : 0);
  if (valid < TR) {
    const int per = (TR - valid) * 8;
    for (int u = threadIdx.x; u < nblk * per; u += blockDim.x) {
      const int b = u / per, rem = u % per;
      stage[(size_t)b * BS + (size_t)valid * 8 + rem] = (T)0;
    }
  }
  if (threadIdx.x == 0) {
    const unsigned bytes = (unsigned)valid * 8u * (unsigned)sizeof(T);
    // the stage may hold generic stores of the previous tile
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, bytes * (unsigned)nblk);
    for (int b = 0; b < nblk; ++b) {
      const T* src = (b < nq ? Q + b * bstride : W) + (size_t)8 * row0;
      bulk_g2s(stage + (size_t)b * BS, src, bytes, bar);
    }
  }
}

// Wait for the copies of one stage: at most 2^20 polls with a short sleep (about 0.1 s);
// false, with USBS_ETIMEOUT in *status, if they did not land.
__device__ __forceinline__ bool tile_wait(uint64_t* bar, unsigned parity, int* status) {
  for (int k = 0; k < (1 << 20); ++k) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(64);
  }
  if (status) atomicExch(status, USBS_ETIMEOUT);
  return false;
}

// The same wait for a whole CTA: thread 0 polls while the others sleep in the barrier (so
// the waiting warps take no issue slots from the other CTA on the SM); afterwards every
// thread observes the completed phase once itself, which makes the copies' bytes visible to
// it.  Every thread of the CTA must call it.
__device__ __forceinline__ bool tile_wait_cta(uint64_t* bar, unsigned parity, int* status) {
  bool ok = true;
  if (threadIdx.x == 0) ok = tile_wait(bar, parity, status);
  ok = __syncthreads_and(ok) != 0;
  if (ok) mbar_test(bar, parity);
  return ok;
}

// After the tile loop: on an abort at iteration it_abort (-1: none), wait (bounded) for the
// copies that may still be landing, those of iterations it_abort .. it_abort + ns - 1 whose
// tiles exist, then release the barriers.
__device__ __forceinline__ void tiles_end(uint64_t* bar, int ns, int it_abort, int cta, int ncta, int ntiles) {
  if (it_abort >= 0) {
    for (int k = it_abort; k < it_abort + ns; ++k)
      if ((int64_t)cta + (int64_t)k * ncta < ntiles) tile_wait(&bar[k % ns], (unsigned)(k / ns) & 1u, nullptr);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) mbar_inval(&bar[s]);
  }
}

// =============================================================================================
// FP32 bodies on the tensor cores.  Every contraction of the tiles is an m16n8k8 TF32 MMA
// (mma.sync) with FP32 accumulation.  TF32 keeps 10 mantissa bits, so each FP32 operand
// is split into a TF32 high part and a TF32 low part (the rounding error of the high
// part) and a product is taken as hi*hi + hi*lo + lo*hi: about 2^-21 relative, the
// accuracy of the FP32 CUDA-core products these replace.
// Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4): A (16 x 8, row-major)
// a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4); B (8 x 8) b0 (t, g), b1 (t+4, g);
// C/D (16 x 8) c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).
// The projection, update and finalize bodies take the number of basis blocks NB (0..8) as a
// template argument (the k_t*_dev bodies dispatch on it): every block loop is then unrolled
// without run-time guards, which takes about a tenth of the update's instructions off.
// =============================================================================================
// x rounded to TF32 (1 sign, 8 exponent, 10 mantissa bits), to nearest with ties away from
// zero: half a unit of the 13 dropped bits is added to the sign-magnitude bit pattern (a
// carry moves into the exponent exactly as rounding up does) and the 13 bits are cleared.
// Two integer operations; for finite x the bits equal cvt.rna.tf32.f32's
// (tests/test_gpu_kernels.py checks it against that instruction), which the tiles called
// once per operand and which cost more issue slots.  Overflow gives inf; a NaN whose
// payload lies in the dropped bits alone would come out as inf (the tiles see finite data).
__device__ __forceinline__ uint32_t tf32_of(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}
__device__ __forceinline__ uint32_t tf32_of_cvt(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// D += A B with A given by four FP32 values and B by two, in split TF32 (small terms first)
struct SplitB { uint32_t h0, h1, l0, l1; };
__device__ __forceinline__ SplitB split_b(float b0, float b1) {
  SplitB s;
  tf32_split(b0, s.h0, s.l0);
  tf32_split(b1, s.h1, s.l1);
  return s;
}
// The two small terms go to ds, the large one to db: two accumulators, so that consecutive
// MMAs of a tile do not wait on one another (an m16n8k8 MMA's result is ready only after its
// full latency); the caller adds ds to db at the end.
__device__ __forceinline__ void mma3s(float (&ds)[4], float (&db)[4], float a0, float a1, float a2, float a3,
                                      const SplitB& b) {
  uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
  tf32_split(a0, h0, l0);
  tf32_split(a1, h1, l1);
  tf32_split(a2, h2, l2);
  tf32_split(a3, h3, l3);
  mma_tf32(ds, l0, l1, l2, l3, b.h0, b.h1);
  mma_tf32(db, h0, h1, h2, h3, b.h0, b.h1);
  mma_tf32(ds, h0, h1, h2, h3, b.l0, b.l1);
}

// shared memory of the warp reduction of tc_reduce_xty with MAXP pairs: 8 x MAXP x 32 x 4
// floats (tproj: 4 pairs, 16 KB; tupdate: 5 pairs, 20 KB)
constexpr size_t tc_red_bytes(int maxp) { return sizeof(float) * 8 * (size_t)maxp * 32 * 4; }

// index of output (m, c) of a 16 x 8 D fragment: lane and register
__device__ __forceinline__ int dfrag_lane(int m, int c) { return (m & 7) * 4 + (c >> 1); }
__device__ __forceinline__ int dfrag_reg(int m, int c) { return ((m >> 3) << 1) | (c & 1); }

// Sums of X_i^T Y over the tile's rows for the blocks of `blocks` (block i at stage
// offset i * BS; block nblk-1 may be Y itself), accumulated per block pair in acc: pair p
// covers blocks 2p and 2p+1 (rows m 0..7 and 8..15 of the MMA).  Warp w takes the 8-row
// k-steps 2w and 2w + 1 of the 128-row tile: rows 16w .. 16w + 15, the rows it owns in the
// row-wise products (X = W - Q H), so the update needs no CTA barrier between the two.
template <int MAXP>
__device__ __forceinline__ void tc_accum_xty(const float* st, int nblk, const float* Y, int warp, int g, int t,
                                             float (&accs)[MAXP][4], float (&accb)[MAXP][4]) {
  constexpr int BS = BlockStride<float>::value;
  const int off = t * 8 + g;   // element (row t, column g) of an 8-row step; + 32 for row t + 4
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int r0 = (2 * warp + kk) * 8;
    const float* y = Y + r0 * 8 + off;
    const SplitB b = split_b(y[0], y[32]);
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
      if (2 * p < nblk) {
        const float* q0 = st + (size_t)(2 * p) * BS + r0 * 8 + off;
        const bool two = 2 * p + 1 < nblk;
        const float a0 = q0[0], a2 = q0[32];
        const float a1 = two ? q0[BS] : 0.f, a3 = two ? q0[BS + 32] : 0.f;
        mma3s(accs[p], accb[p], a0, a1, a2, a3, b);
      }
    }
  }
}

// Reduce acc[p][4] over the 8 warps (fixed order, FP32 like the sums inside a CTA) into
// the CTA's FP64 partials: output index out_of(block, a, c) for block < nblk.
// red: 8 x MAXP x 32 x 4 floats of shared memory.
template <int MAXP, typename OutIdx>
__device__ __forceinline__ void tc_reduce_xty(const float (&acc)[MAXP][4], int nblk, int warp, int lane,
                                              float* red, double* partials, OutIdx out_of) {
#pragma unroll
  for (int p = 0; p < MAXP; ++p)
    *reinterpret_cast<float4*>(red + ((warp * MAXP + p) * 32 + lane) * 4) =
        make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
  __syncthreads();
  for (int o = threadIdx.x; o < nblk * 64; o += blockDim.x) {
    const int blk = o >> 6, a = (o >> 3) & 7, c = o & 7;
    const int p = blk >> 1, m = a + 8 * (blk & 1);
    const int ln = dfrag_lane(m, c), rg = dfrag_reg(m, c);
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += red[((w * MAXP + p) * 32 + ln) * 4 + rg];
    partials[out_of(blk, a, c)] = (double)sum;
  }
}

// H = Q^T W for nb <= 8 blocks
template <int NB>
__device__ __forceinline__ void tc_tproj(const int cta, const int ncta, int n, const float* Q, size_t bstride,
                                         const float* W, double* partials, int* status, int ns) {
  constexpr int nb = NB;
  constexpr int TR = 128, BS = BlockStride<float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>(smem_raw);
  const int sstride = (nb + 1) * BS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[4][4], accb[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[p][u] = accb[p][u] = 0.f;
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<float, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<float, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    const float* st = stages + rg.s * sstride;
    tc_accum_xty<4>(st, nb, st + (size_t)nb * BS, warp, g, t, acc, accb);
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[p][u] = accb[p][u] + acc[p][u];
  tc_reduce_xty<4>(acc, nb, warp, lane, reinterpret_cast<float*>(smem_raw), partials + (size_t)cta * PART_STRIDE,
                   [](int blk, int a, int c) { return blk * 64 + a * 8 + c; });
}

// X = W - Q H (W overwritten, in shared memory and in global memory); then H2 = Q^T X and
// G = X^T X.  H in Hs (nb x 64, FP32).
template <int NB>
__device__ __forceinline__ void tc_tupdate(const int cta, const int ncta, int n, const float* Q, size_t bstride,
                                           float* W, const double* Hred, double* partials, int* status, int ns) {
  constexpr int nb = NB;
  constexpr int TR = 128, BS = BlockStride<float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>(smem_raw);
  const int sstride = (nb + 1) * BS;
  float* Hs = stages + ns * sstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int u = threadIdx.x; u < nb * 64; u += blockDim.x) Hs[u] = (float)Hred[u];
  __syncthreads();
  // B fragments of H, split once for all tiles
  SplitB hb[8];
#pragma unroll
  for (int b = 0; b < 8; ++b)
    hb[b] = (b < nb) ? split_b(Hs[b * 64 + t * 8 + g], Hs[b * 64 + (t + 4) * 8 + g]) : SplitB{0u, 0u, 0u, 0u};
  float acc[5][4], accb[5][4];
#pragma unroll
  for (int p = 0; p < 5; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[p][u] = accb[p][u] = 0.f;
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<float, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<float, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    float* st = stages + rg.s * sstride;
    float* Xs = st + (size_t)nb * BS;
    // phase 1: rows 16 warp .. 16 warp + 15 of X = W - Q H
    {
      const int rb = 16 * warp;
      // four accumulators (small / large terms of even / odd blocks): independent MMA chains
      float d[4] = {0.f, 0.f, 0.f, 0.f}, e0[4] = {0.f, 0.f, 0.f, 0.f};
      float s1[4] = {0.f, 0.f, 0.f, 0.f}, e1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (b < nb) {
          const float* q = st + (size_t)b * BS + (size_t)rb * 8;
          if (b & 1) mma3s(s1, e1, q[g * 8 + t], q[(g + 8) * 8 + t], q[g * 8 + t + 4], q[(g + 8) * 8 + t + 4], hb[b]);
          else mma3s(d, e0, q[g * 8 + t], q[(g + 8) * 8 + t], q[g * 8 + t + 4], q[(g + 8) * 8 + t + 4], hb[b]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) d[u] = (e0[u] + e1[u]) + (d[u] + s1[u]);
      float* x0 = Xs + (size_t)(rb + g) * 8 + 2 * t;
      float* x1 = Xs + (size_t)(rb + g + 8) * 8 + 2 * t;
      const float v0 = x0[0] - d[0], v1 = x0[1] - d[1], v2 = x1[0] - d[2], v3 = x1[1] - d[3];
      x0[0] = v0; x0[1] = v1; x1[0] = v2; x1[1] = v3;
      const int row0 = tile * TR + rb + g, row1 = row0 + 8;
      if (row0 < n) *reinterpret_cast<float2*>(W + (size_t)8 * row0 + 2 * t) = make_float2(v0, v1);
      if (row1 < n) *reinterpret_cast<float2*>(W + (size_t)8 * row1 + 2 * t) = make_float2(v2, v3);
    }
    // phase 2 reads the 16 rows of X this warp wrote in phase 1: a warp barrier suffices
    __syncwarp();
    // phase 2: H2 = Q^T X and G = X^T X (X is block nb of the pair list; rows past n are 0)
    tc_accum_xty<5>(st, nb + 1, Xs, warp, g, t, acc, accb);
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 5; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[p][u] = accb[p][u] + acc[p][u];
  tc_reduce_xty<5>(acc, nb + 1, warp, lane, reinterpret_cast<float*>(smem_raw), partials + (size_t)cta * PART_STRIDE,
                   [nb](int blk, int a, int c) { return (blk < nb ? blk * 64 : 512) + a * 8 + c; });
}

// out = (W - Q H2) R^-1, deficient columns replaced (1: random, 2: zero)
template <int NB>
__device__ __forceinline__ void tc_tfinalize(const int cta, const int ncta, int n, const float* Q, size_t bstride,
                                             const float* W, const double* H2red, const DevLanczos* lz,
                                             float* out, uint64_t seed, int* status, int ns) {
  constexpr int nb = NB;
  constexpr int TR = 128, BS = BlockStride<float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>(smem_raw);
  const int sstride = (nb + 1) * BS;
  float* Hs = stages + ns * sstride;
  float* Ri = Hs + 8 * 64;
  __shared__ int dfc[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  for (int u = tid; u < nb * 64; u += blockDim.x) Hs[u] = (float)H2red[u];
  if (tid < 64) Ri[tid] = (float)lz->Rinv[tid];
  if (tid < 8) dfc[tid] = lz->dcol[tid];
  __syncthreads();
  const SplitB rb0 = split_b(Ri[t * 8 + g], Ri[(t + 4) * 8 + g]);
  // B fragments of H2, split once for all tiles
  SplitB hb[8];
#pragma unroll
  for (int b = 0; b < 8; ++b)
    hb[b] = (b < nb) ? split_b(Hs[b * 64 + t * 8 + g], Hs[b * 64 + (t + 4) * 8 + g]) : SplitB{0u, 0u, 0u, 0u};
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<float, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<float, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    float* st = stages + rg.s * sstride;
    float* Xs = st + (size_t)nb * BS;
    const int rb = 16 * warp;
    float d[4] = {0.f, 0.f, 0.f, 0.f}, e0[4] = {0.f, 0.f, 0.f, 0.f};
    float s1[4] = {0.f, 0.f, 0.f, 0.f}, e1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < nb) {
        const float* q = st + (size_t)b * BS + (size_t)rb * 8;
        if (b & 1) mma3s(s1, e1, q[g * 8 + t], q[(g + 8) * 8 + t], q[g * 8 + t + 4], q[(g + 8) * 8 + t + 4], hb[b]);
        else mma3s(d, e0, q[g * 8 + t], q[(g + 8) * 8 + t], q[g * 8 + t + 4], q[(g + 8) * 8 + t + 4], hb[b]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] = (e0[u] + e1[u]) + (d[u] + s1[u]);
    // X = W - Q H2 back into this warp's own rows, then (X R^-1) as a second MMA
    float* x0 = Xs + (size_t)(rb + g) * 8 + 2 * t;
    float* x1 = Xs + (size_t)(rb + g + 8) * 8 + 2 * t;
    x0[0] -= d[0]; x0[1] -= d[1]; x1[0] -= d[2]; x1[1] -= d[3];
    __syncwarp();
    const float* xr = Xs + (size_t)rb * 8;
    float o[4] = {0.f, 0.f, 0.f, 0.f}, ob[4] = {0.f, 0.f, 0.f, 0.f};
    mma3s(o, ob, xr[g * 8 + t], xr[(g + 8) * 8 + t], xr[g * 8 + t + 4], xr[(g + 8) * 8 + t + 4], rb0);
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = ob[u] + o[u];
    const int row0 = tile * TR + rb + g, row1 = row0 + 8;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = u < 2 ? row0 : row1, a = 2 * t + (u & 1);
      if (dfc[a] == 1) o[u] = (float)hash_uniform_o(seed, (uint64_t)row, (uint64_t)a);
      else if (dfc[a] == 2) o[u] = 0.f;
    }
    if (row0 < n) *reinterpret_cast<float2*>(out + (size_t)8 * row0 + 2 * t) = make_float2(o[0], o[1]);
    if (row1 < n) *reinterpret_cast<float2*>(out + (size_t)8 * row1 + 2 * t) = make_float2(o[2], o[3]);
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
}

// out[o] = Q[:, :J] Y[:, 8o : 8o + 8] for o < nout <= 4; the residual block copied to
// out[resid_slot] when resid is given.  Ys: J x 8 nout split pairs in shared memory.
// NBK / NOUT > 0 fix nbk / nout at compile time (0: taken from the arguments).
template <int NBK, int NOUT>
__device__ __forceinline__ void tc_trestart(const int cta, const int ncta, int n, const float* Q, size_t bstride,
                                            int nbk_rt, int nout_rt, const double* Y, float* out, size_t ostride,
                                            const float* resid, int resid_slot, int* status, int ns) {
  const int nbk = NBK > 0 ? NBK : nbk_rt, nout = NOUT > 0 ? NOUT : nout_rt;
  constexpr int TR = 128, BS = BlockStride<float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>(smem_raw);
  const int sstride = nbk * BS;
  // Y split once per launch into TF32 high and low parts: (hi, lo) pairs, J x 8 nout
  uint2* Ys = reinterpret_cast<uint2*>(stages + ns * sstride);
  const int J = nbk * 8, ncol = nout * 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  for (int u = tid; u < J * ncol; u += blockDim.x) {
    uint32_t hi, lo;
    tf32_split((float)Y[(u / ncol) * JMAX + (u % ncol)], hi, lo);
    Ys[u] = make_uint2(hi, lo);
  }
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<float, TR>(stages + k * sstride, Q, bstride, nbk, nullptr, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<float, TR>(stages + rg.sl * sstride, Q, bstride, nbk, nullptr, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    const float* st = stages + rg.s * sstride;
    const int rb = 16 * warp;
    // small terms in d, large terms in e: independent accumulators per output block
    float d[4][4], e[4][4];
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int u = 0; u < 4; ++u) d[o][u] = e[o][u] = 0.f;
#pragma unroll
    for (int b = 0; b < nbk; ++b) {
      const float* q = st + (size_t)b * BS + (size_t)rb * 8;
      uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
      tf32_split(q[g * 8 + t], h0, l0);
      tf32_split(q[(g + 8) * 8 + t], h1, l1);
      tf32_split(q[g * 8 + t + 4], h2, l2);
      tf32_split(q[(g + 8) * 8 + t + 4], h3, l3);
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        if (o < nout) {
          const uint2 y0 = Ys[(b * 8 + t) * ncol + 8 * o + g], y1 = Ys[(b * 8 + t + 4) * ncol + 8 * o + g];
          mma_tf32(d[o], l0, l1, l2, l3, y0.x, y1.x);
          mma_tf32(e[o], h0, h1, h2, h3, y0.x, y1.x);
          mma_tf32(d[o], h0, h1, h2, h3, y0.y, y1.y);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int u = 0; u < 4; ++u) d[o][u] = e[o][u] + d[o][u];
    const int row0 = tile * TR + rb + g, row1 = row0 + 8;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      if (o < nout) {
        if (row0 < n) *reinterpret_cast<float2*>(out + o * ostride + (size_t)8 * row0 + 2 * t) = make_float2(d[o][0], d[o][1]);
        if (row1 < n) *reinterpret_cast<float2*>(out + o * ostride + (size_t)8 * row1 + 2 * t) = make_float2(d[o][2], d[o][3]);
      }
    }
    if (resid) {
      for (int p = tid; p < TR * 8; p += blockDim.x) {
        const int row = tile * TR + p / 8;
        if (row < n) out[resid_slot * ostride + (size_t)8 * row + (p % 8)] = resid[(size_t)8 * row + (p % 8)];
      }
    }
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
}

// ---- H = Q^T W --------------------------------------------------------------------------
// Items (b, a-pair): 4 nb <= 32.  256 threads = 8 row groups (warps) x 32 slots.  A slot
// owns one item, 2 basis columns x all 8 columns of W (16 accumulators, 3 shared loads
// per 16 FMAs).  When there are fewer items than slots, the spare slots of a warp take
// further rows of the tile: slot = item + nitems * sub, sub < nsub = 32 / nitems, and
// the tile's rows are dealt out over the 8 * nsub (warp, sub) pairs.  The epilogue adds
// the partial sums in a fixed order (warp, then sub).
template <typename T>
__device__ __forceinline__ void accum_pair(const T* USBS_RESTRICT qcol2, const T* USBS_RESTRICT X,
                                           int r0, int rstep, T (&acc)[16]) {
  constexpr int TR = TileRows<T>::value;
  for (int r = r0; r < TR; r += rstep) {
    T q0, q1, xr[8];
    lds2<T>(qcol2 + r * 8, q0, q1);
    lds8<T>(X + r * 8, xr);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      acc[c] += q0 * xr[c];
      acc[8 + c] += q1 * xr[c];
    }
  }
}

// Sum of one output t of the item layout (item = t / 16 of the [b][a][c] block order,
// u = 16 values of a slot) over the 8 warps and the nsub row subgroups, fixed order.
__device__ __forceinline__ double sum_slots(const double* red, int nitems, int nsub, int item,
                                            int u, int nslot) {
  double sum = 0.0;
#pragma unroll
  for (int g = 0; g < 8; ++g)
    for (int sb = 0; sb < nsub; ++sb) sum += red[((size_t)g * nslot + item + nitems * sb) * 16 + u];
  return sum;
}

template <typename T>
__device__ __forceinline__ void k_tproj_dev(const int cta, const int ncta, int n, const T* USBS_RESTRICT Q, size_t bstride, int nb,
                                               const T* USBS_RESTRICT W, double* USBS_RESTRICT partials,
                                               const int* USBS_RESTRICT mask, int* status, int ns = 2) {
  if constexpr (sizeof(T) == 4) {
    if (mask && *mask == 0) return;
    switch (nb) {
      case 0: tc_tproj<0>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 1: tc_tproj<1>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 2: tc_tproj<2>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 3: tc_tproj<3>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 4: tc_tproj<4>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 5: tc_tproj<5>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 6: tc_tproj<6>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      case 7: tc_tproj<7>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
      default: tc_tproj<8>(cta, ncta, n, Q, bstride, W, partials, status, ns); break;
    }
    return;
  }
  if (mask && *mask == 0) return;
  constexpr int TR = TileRows<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  const int sstride = (nb + 1) * BlockStride<T>::value;
  const int tid = threadIdx.x, grp = tid >> 5, slot = tid & 31;
  const int nitems = 4 * nb;
  const int nsub = nitems > 0 ? 32 / nitems : 1;
  const int item = nitems > 0 ? slot % nitems : 0, sub = nitems > 0 ? slot / nitems : 0;
  const bool active = nitems > 0 && sub < nsub;
  T acc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = (T)0;
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<T, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<T, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    const T* st = stages + rg.s * sstride;
    if (active) {
      const int b = item >> 2, a0 = 2 * (item & 3);
      accum_pair<T>(st + (size_t)b * BlockStride<T>::value + a0, st + (size_t)nb * BlockStride<T>::value, grp + 8 * sub, 8 * nsub, acc);
    }
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);     // 8 warps x 32 slots x 16
  if (active) {
#pragma unroll
    for (int u = 0; u < 16; ++u) red[((size_t)grp * 32 + slot) * 16 + u] = (double)acc[u];
  }
  __syncthreads();
  for (int t = tid; t < nb * 64; t += blockDim.x) {
    // t = b * 64 + a * 8 + c  ->  item b * 4 + a / 2, value (a % 2) * 8 + c
    const int b = t >> 6, a = (t >> 3) & 7, c = t & 7;
    partials[(size_t)cta * PART_STRIDE + t] = sum_slots(red, nitems, nsub, b * 4 + (a >> 1), (a & 1) * 8 + c, 32);
  }
}

// ---- X = W - Q H; H2 = Q^T X; G = X^T X -----------------------------------------------------
template <typename T>
__device__ __forceinline__ void k_tupdate_dev(const int cta, const int ncta, int n, const T* USBS_RESTRICT Q, size_t bstride, int nb,
                                                 T* USBS_RESTRICT W, const double* USBS_RESTRICT Hred,
                                                 double* USBS_RESTRICT partials,
                                                 const int* USBS_RESTRICT mask, int* status, int ns = 2) {
  if constexpr (sizeof(T) == 4) {
    if (mask && *mask == 0) return;
    switch (nb) {
      case 0: tc_tupdate<0>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 1: tc_tupdate<1>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 2: tc_tupdate<2>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 3: tc_tupdate<3>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 4: tc_tupdate<4>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 5: tc_tupdate<5>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 6: tc_tupdate<6>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      case 7: tc_tupdate<7>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
      default: tc_tupdate<8>(cta, ncta, n, Q, bstride, W, Hred, partials, status, ns); break;
    }
    return;
  }
  if (mask && *mask == 0) return;
  constexpr int TR = TileRows<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  const int sstride = (nb + 1) * BlockStride<T>::value;
  T* Hs = stages + ns * sstride;                             // nb x 8 x 8
  const int tid = threadIdx.x, grp = tid >> 5, slot = tid & 31;
  for (int t = tid; t < nb * 64; t += blockDim.x) Hs[t] = (T)Hred[t];
  const int nitems = 4 * (nb + 1);                          // item b == nb: the Gram matrix
  // up to 32 items: one per slot, spare slots split the rows; more (nb = 8): two per slot
  const int nsub = nitems <= 32 ? 32 / nitems : 1;
  const int nslot = nitems <= 32 ? 32 : 64;
  const int sub = nitems <= 32 ? slot / nitems : 0;
  T acc[2][16];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 16; ++v) acc[u][v] = (T)0;
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<T, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<T, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    T* st = stages + rg.s * sstride;
    T* Xs = st + (size_t)nb * BlockStride<T>::value;                               // W tile, overwritten by X
    // phase 1: X = W - Q H, 4 columns per thread
    for (int p = tid; p < TR * 2; p += blockDim.x) {
      const int r = p >> 1, c0 = 4 * (p & 1);
      T x[4];
      lds4<T>(Xs + r * 8 + c0, x);
      for (int b = 0; b < nb; ++b) {
        T q[8];
        lds8<T>(st + (size_t)b * BlockStride<T>::value + (size_t)r * 8, q);
        const T* hb = Hs + b * 64 + c0;
#pragma unroll
        for (int ap = 0; ap < 8; ++ap) {
          T h[4];
          lds4<T>(hb + ap * 8, h);
#pragma unroll
          for (int v = 0; v < 4; ++v) x[v] -= q[ap] * h[v];
        }
      }
      sts4<T>(Xs + r * 8 + c0, x);
      const int row = tile * TR + r;
      if (row < n) {
#pragma unroll
        for (int v = 0; v < 4; ++v) W[(size_t)8 * row + c0 + v] = x[v];
      }
    }
    __syncthreads();
    // phase 2: H2 += Q^T X and G += X^T X (rows past n are zero in X)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int item = nitems <= 32 ? slot % nitems : slot + 32 * u;
      const bool act = nitems <= 32 ? (u == 0 && sub < nsub) : item < nitems;
      if (act) {
        const int b = item >> 2, a0 = 2 * (item & 3);
        accum_pair<T>((b < nb ? st + (size_t)b * BlockStride<T>::value : Xs) + a0, Xs, grp + 8 * sub, 8 * nsub, acc[u]);
      }
    }
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);     // 8 warps x nslot x 16
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const bool act = nitems <= 32 ? (u == 0 && sub < nsub) : slot + 32 * u < nitems;
    if (act) {
#pragma unroll
      for (int v = 0; v < 16; ++v) red[((size_t)grp * nslot + slot + 32 * u) * 16 + v] = (double)acc[u][v];
    }
  }
  __syncthreads();
  for (int t = tid; t < 576; t += blockDim.x) {
    if (t < 512 && t >= nb * 64) continue;
    // t < 512: H2 block b = t / 64; t >= 512: the Gram matrix, item block nb
    const int b = t < 512 ? (t >> 6) : nb, a = (t >> 3) & 7, c = t & 7;
    partials[(size_t)cta * PART_STRIDE + t] =
        sum_slots(red, nitems <= 32 ? nitems : 0, nitems <= 32 ? nsub : 1, b * 4 + (a >> 1),
                  (a & 1) * 8 + c, nslot);
  }
}

template <typename T>
__device__ __forceinline__ void k_tfinalize_dev(const int cta, const int ncta, int n, const T* USBS_RESTRICT Q, size_t bstride,
                                                   int nb, const T* W, const double* USBS_RESTRICT H2red,
                                                   const DevLanczos* USBS_RESTRICT lz, T* out,
                                                   const int* USBS_RESTRICT mask, uint64_t seed, int* status, int ns = 2) {
  if constexpr (sizeof(T) == 4) {
    if (mask && *mask == 0) return;
    switch (nb) {
      case 0: tc_tfinalize<0>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 1: tc_tfinalize<1>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 2: tc_tfinalize<2>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 3: tc_tfinalize<3>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 4: tc_tfinalize<4>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 5: tc_tfinalize<5>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 6: tc_tfinalize<6>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      case 7: tc_tfinalize<7>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
      default: tc_tfinalize<8>(cta, ncta, n, Q, bstride, W, H2red, lz, out, seed, status, ns); break;
    }
    return;
  }
  if (mask && *mask == 0) return;
  constexpr int TR = TileRows<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  const int sstride = (nb + 1) * BlockStride<T>::value;
  T* Hs = stages + ns * sstride;
  T* Ri = Hs + 8 * 64;
  __shared__ int dfc[8];
  const int tid = threadIdx.x;
  for (int t = tid; t < nb * 64; t += blockDim.x) Hs[t] = (T)H2red[t];
  if (tid < 64) Ri[tid] = (T)lz->Rinv[tid];
  if (tid < 8) dfc[tid] = lz->dcol[tid];
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<T, TR>(stages + k * sstride, Q, bstride, nb, W, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<T, TR>(stages + rg.sl * sstride, Q, bstride, nb, W, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    T* st = stages + rg.s * sstride;
    T* Xs = st + (size_t)nb * BlockStride<T>::value;
    for (int p = tid; p < TR * 2; p += blockDim.x) {
      const int r = p >> 1, c0 = 4 * (p & 1);
      T x[4];
      lds4<T>(Xs + r * 8 + c0, x);
      for (int b = 0; b < nb; ++b) {
        T q[8];
        lds8<T>(st + (size_t)b * BlockStride<T>::value + (size_t)r * 8, q);
        const T* hb = Hs + b * 64 + c0;
#pragma unroll
        for (int ap = 0; ap < 8; ++ap) {
          T h[4];
          lds4<T>(hb + ap * 8, h);
#pragma unroll
          for (int v = 0; v < 4; ++v) x[v] -= q[ap] * h[v];
        }
      }
      __syncwarp();
      sts4<T>(Xs + r * 8 + c0, x);
    }
    __syncthreads();
    for (int p = tid; p < TR * 2; p += blockDim.x) {
      const int r = p >> 1, c0 = 4 * (p & 1);
      const int row = tile * TR + r;
      if (row >= n) continue;
      const T* xr = Xs + r * 8;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int a = c0 + v;
        T o = (T)0;
#pragma unroll
        for (int c = 0; c < 8; ++c) o += xr[c] * Ri[c * 8 + a];
        if (dfc[a] == 1) o = (T)hash_uniform_o(seed, (uint64_t)row, (uint64_t)a);
        else if (dfc[a] == 2) o = (T)0;
        out[(size_t)8 * row + a] = o;
      }
    }
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
}


// ---- out[o] = Q[:, :J] Y[:, 8o : 8o + 8], o < nout (thick restart, Ritz vectors) -------------
// Optionally copies the residual block into out[resid_slot].  Y (J x 8 nout) sits in shared
// memory; a thread owns (row, 4 output columns) items.
template <typename T>
__device__ __forceinline__ void k_trestart_dev(const int cta, const int ncta, int n, const T* USBS_RESTRICT Q, size_t bstride, int nbk,
                                                  int nout, const double* USBS_RESTRICT Y,
                                                  T* USBS_RESTRICT out, size_t ostride,
                                                  const T* USBS_RESTRICT resid, int resid_slot, int* status, int ns = 2) {
  if constexpr (sizeof(T) == 4) {
    // the shapes of the 16-, 32- and 64-column bases (restart: keep = J / 2; final: 1 block)
    const int shape = nbk * 8 + nout;
    if (shape == 4 * 8 + 2) tc_trestart<4, 2>(cta, ncta, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
    else if (shape == 4 * 8 + 1) tc_trestart<4, 1>(cta, ncta, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
    else if (shape == 8 * 8 + 4) tc_trestart<8, 4>(cta, ncta, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
    else if (shape == 8 * 8 + 1) tc_trestart<8, 1>(cta, ncta, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
    else tc_trestart<0, 0>(cta, ncta, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
    return;
  }
  constexpr int TR = TileRows<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  const int sstride = nbk * BlockStride<T>::value;
  T* Ys = stages + ns * sstride;                       // J x ncol
  const int J = nbk * 8, ncol = nout * 8;
  const int tid = threadIdx.x;
  for (int t = tid; t < J * ncol; t += blockDim.x) Ys[t] = (T)Y[(t / ncol) * JMAX + (t % ncol)];
  const int ntiles = (n + TR - 1) / TR;
  __shared__ uint64_t tbar[NSMAX];
  tiles_begin(tbar, ns);
  for (int k = 0; k < ns - 1; ++k)
    if (cta + k * ncta < ntiles)
      tile_load<T, TR>(stages + k * sstride, Q, bstride, nbk, nullptr, n, (cta + k * ncta) * TR, &tbar[k]);
  int it_abort = -1;
  TileRing rg(ns);
  for (int it = 0, tile = cta; tile < ntiles; ++it, tile += ncta, rg.next()) {
    const int ahead = tile + (ns - 1) * ncta;
    if (ahead < ntiles) tile_load<T, TR>(stages + rg.sl * sstride, Q, bstride, nbk, nullptr, n, ahead * TR, &tbar[rg.sl]);
    if (!tile_wait_cta(&tbar[rg.s], rg.ph, status)) {
      it_abort = it;
      break;
    }
    const T* st = stages + rg.s * sstride;
    // items (row pair, output block, column group): with nout < 4 the 8 columns of an
    // output block are split into 4 / nout groups so that every thread has work
    const int ngrp = nout >= 4 ? 1 : 4 / nout, ncols = 8 / ngrp;
    for (int p = tid; p < (TR / 2) * nout * ngrp; p += blockDim.x) {
      const int pair = p / (nout * ngrp), rem = p % (nout * ngrp);
      const int o = rem / ngrp, c0 = (rem % ngrp) * ncols;
      const int r0 = 2 * pair;
      T acc0[8], acc1[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) { acc0[v] = (T)0; acc1[v] = (T)0; }
      for (int b = 0; b < nbk; ++b) {
        const T* qr0 = st + (size_t)b * BlockStride<T>::value + (size_t)r0 * 8;
        const T* qr1 = qr0 + 8;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const T q0 = qr0[a], q1 = qr1[a];
          const T* yr = Ys + (b * 8 + a) * ncol + 8 * o + c0;
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            if (v < ncols) {
              acc0[v] += q0 * yr[v];
              acc1[v] += q1 * yr[v];
            }
          }
        }
      }
      const int row0 = tile * TR + r0;
      if (row0 < n) {
#pragma unroll
        for (int v = 0; v < 8; ++v)
          if (v < ncols) out[o * ostride + (size_t)8 * row0 + c0 + v] = acc0[v];
      }
      if (row0 + 1 < n) {
#pragma unroll
        for (int v = 0; v < 8; ++v)
          if (v < ncols) out[o * ostride + (size_t)8 * (row0 + 1) + c0 + v] = acc1[v];
      }
    }
    if (resid) {
      for (int p = tid; p < TR * 8; p += blockDim.x) {
        const int row = tile * TR + p / 8;
        if (row < n) out[resid_slot * ostride + (size_t)8 * row + (p % 8)] = resid[(size_t)8 * row + (p % 8)];
      }
    }
    __syncthreads();
  }
  tiles_end(tbar, ns, it_abort, cta, ncta, ntiles);
}

}  // namespace
}  // namespace usbs
