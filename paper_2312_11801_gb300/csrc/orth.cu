// Block Gram-Schmidt kernels of the Lanczos step, staged through shared memory.
//
// A CTA walks tiles of TR consecutive rows.  For each tile it copies the rows of every
// basis block Q_0..Q_{nb-1} and of the new block W into shared memory with bulk
// asynchronous copies (in the block-major layout the tile of one block is TR * 8
// contiguous values), in a pipeline of 2 to 4 stages (as many as fit while two CTAs share
// an SM), so that the next tiles stream in while the current one is used.
// The arithmetic then runs from shared memory as small register-blocked GEMMs:
//   proj     : H  += Q^T W                                   (first projection)
//   update   : X = W - Q H (written back), H2 += Q^T X, G += X^T X   (second pass, Gram)
//   finalize : out = (W - Q H2) R^-1                          (normalised new block)
// Cross-CTA sums go to per-CTA FP64 partials in the same layout as before
// ([b*64 + a*8 + c] for H_b[a][c]; [512 + a*8 + c] for the Gram matrix).
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dev_orth.cuh"

namespace usbs {
namespace {

template <typename T>
__global__ void __launch_bounds__(256, 2) k_tproj(int n, const T* __restrict__ Q, size_t bstride, int nb,
                                               const T* __restrict__ W, double* __restrict__ partials,
                                               const int* __restrict__ mask, int* status, int ns) {
  k_tproj_dev<T>(blockIdx.x, gridDim.x, n, Q, bstride, nb, W, partials, mask, status, ns);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_tupdate(int n, const T* __restrict__ Q, size_t bstride, int nb,
                                                 T* __restrict__ W, const double* __restrict__ Hred,
                                                 double* __restrict__ partials,
                                                 const int* __restrict__ mask, int* status, int ns) {
  k_tupdate_dev<T>(blockIdx.x, gridDim.x, n, Q, bstride, nb, W, Hred, partials, mask, status, ns);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_tfinalize(int n, const T* __restrict__ Q, size_t bstride,
                                                   int nb, const T* W, const double* __restrict__ H2red,
                                                   const DevLanczos* __restrict__ lz, T* out,
                                                   const int* __restrict__ mask, uint64_t seed, int* status, int ns) {
  k_tfinalize_dev<T>(blockIdx.x, gridDim.x, n, Q, bstride, nb, W, H2red, lz, out, mask, seed, status, ns);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_trestart(int n, const T* __restrict__ Q, size_t bstride, int nbk,
                                                  int nout, const double* __restrict__ Y,
                                                  T* __restrict__ out, size_t ostride,
                                                  const T* __restrict__ resid, int resid_slot, int* status, int ns) {
  k_trestart_dev<T>(blockIdx.x, gridDim.x, n, Q, bstride, nbk, nout, Y, out, ostride, resid, resid_slot, status, ns);
}

// Dynamic shared memory of one CTA: a budget under which two CTAs still share an SM
// (228 KB per SM, 1 KB of it reserved per CTA), so the pipeline depth never costs occupancy.
constexpr size_t PIPE_BUDGET = 110 * 1024;

// Stages of the tile pipeline for one launch: as many as fit the budget, 2 to NSMAX.
static int pipe_stages(size_t stage_bytes, size_t fixed_bytes) {
  int ns = 2;
  while (ns < NSMAX && (size_t)(ns + 1) * stage_bytes + fixed_bytes <= PIPE_BUDGET) ++ns;
  return ns;
}

// bytes of one stage of nb + 1 staged blocks, and the pipeline depth with `extra` values after it
template <typename T>
size_t stage_bytes(int nblk) { return sizeof(T) * (size_t)nblk * BlockStride<T>::value; }
template <typename T>
int tile_stages(int nb, int extra) { return pipe_stages(stage_bytes<T>(nb + 1), sizeof(T) * (size_t)extra); }
template <typename T>
size_t tile_smem(int nb, int extra, int ns) {
  return (size_t)ns * stage_bytes<T>(nb + 1) + sizeof(T) * (size_t)extra;
}

template <typename T>
void set_attrs() {
  static std::once_flag once;
  std::call_once(once, [] {
    // the largest launch: two stages of nine blocks (nb = 8) or the budget
    const int mx = (int)std::max(tile_smem<T>(8, 8 * 64 + 64, 2), PIPE_BUDGET);
    cudaFuncSetAttribute(k_tproj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_tupdate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_tfinalize<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_trestart<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)std::max(2 * stage_bytes<T>(8) + 8 * JMAX * 32, PIPE_BUDGET));
  });
}

}  // namespace

int64_t parts_needed(int64_t n, int64_t m) {
  const int64_t g = (std::max(n, m) + 63) / 64 + 1;
  return std::min<int64_t>(g, RED_GRID_MAX);
}

// resident CTAs per SM of a kernel at a dynamic shared-memory size, cached (one device)
static int resident_ctas(const void* kernel, size_t smem) {
  struct Entry { const void* k; size_t s; int v; };
  static std::mutex mu;
  static std::vector<Entry> cache;
  std::lock_guard<std::mutex> lk(mu);
  for (const Entry& e : cache)
    if (e.k == kernel && e.s == smem) return e.v;
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, 256, smem) != cudaSuccess) {
    cudaGetLastError();
    v = 1;
  }
  v = std::max(v, 1);
  cache.push_back({kernel, smem, v});
  return v;
}

int orth_grid(Ctx* c, int64_t rows, const void* kernel, size_t smem) {
  const int TR = c->fp64 ? TileRows<double>::value : TileRows<float>::value;
  int64_t g = (rows + TR - 1) / TR;
  // at most 2 CTAs per SM: the tiles are issue-bound, more CTAs only lengthen the
  // reduction of their partials
  const int per_sm = std::min(resident_ctas(kernel, smem), 2);
  const int64_t cap = std::min<int64_t>(c->max_parts, (int64_t)per_sm * c->num_sms);
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// FP32 contexts take the tcgen05 tiles (tc_orth.cu) when their buffers have tensor maps
template <typename T>
static bool on_tc(const Ctx* c) {
  return sizeof(T) == 4 && c->use_tc && !c->tma.empty();
}

template <typename T>
int Orth<T>::proj(Ctx* c, const void* Qb, int nb, const void* W, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 1));
  if (on_tc<T>(c)) {
    const int g = tc_proj(c, Qb, nb, W, mask);
    if (g > 0) return g;
  }
  set_attrs<T>();
  // the epilogue reuses the stage buffers for its warp partials
  const int ns = tile_stages<T>(nb, 0);
  const size_t sm = std::max(tile_smem<T>(nb, 0, ns), sizeof(double) * 8 * 512);
  const int g = orth_grid(c, c->n, (const void*)k_tproj<T>, sm);
  k_tproj<T><<<g, 256, sm, c->stream>>>((int)c->n, (const T*)Qb, (size_t)c->n * 8, nb, (const T*)W,
                                        c->partials, mask, DEV_FIELD(c->lz, DevLanczos, status, int), ns);
  return g;
}

template <typename T>
int Orth<T>::gram_xy(Ctx* c, const void* X, const void* Y) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH, 16.0 * sizeof(T) * c->n);
  if (on_tc<T>(c)) {
    const int g = tc_proj(c, X, 1, Y, nullptr);
    if (g > 0) return g;
  }
  set_attrs<T>();
  const int ns = tile_stages<T>(1, 0);
  const size_t sm = std::max(tile_smem<T>(1, 0, ns), sizeof(double) * 8 * 512);
  const int g = orth_grid(c, c->n, (const void*)k_tproj<T>, sm);
  k_tproj<T><<<g, 256, sm, c->stream>>>((int)c->n, (const T*)X, (size_t)c->n * 8, 1, (const T*)Y,
                                        c->partials, nullptr, DEV_FIELD(c->lz, DevLanczos, status, int), ns);
  return g;
}

template <typename T>
int Orth<T>::update(Ctx* c, const void* Qb, int nb, void* W, const int* mask) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH_UPDATE, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 2));
  if (on_tc<T>(c)) {
    const int g = tc_update(c, Qb, nb, W, mask);
    if (g > 0) return g;
  }
  set_attrs<T>();
  // the epilogue reuses the stage buffers for its warp partials: FP32 (tensor cores)
  // 8 warps x 5 pairs x 32 x 4 floats; FP64 8 warps x (32 or 64) slots x 16 doubles
  const size_t red = sizeof(T) == 4 ? tc_red_bytes(5)
                                    : sizeof(double) * 8 * (4 * (nb + 1) <= 32 ? 32 : 64) * 16;
  const int ns = tile_stages<T>(nb, 8 * 64);
  const size_t sm = std::max(tile_smem<T>(nb, 8 * 64, ns), red);
  const int g = orth_grid(c, c->n, (const void*)k_tupdate<T>, sm);
  k_tupdate<T><<<g, 256, sm, c->stream>>>((int)c->n, (const T*)Qb, (size_t)c->n * 8, nb, (T*)W,
                                          c->red + RED_H, c->partials, mask, DEV_FIELD(c->lz, DevLanczos, status, int),
                                          ns);
  return g;
}

template <typename T>
void Orth<T>::finalize(Ctx* c, const void* Qb, int nb, const void* W, void* out, const int* mask,
                       uint64_t seed) {
  USBS_LAUNCH_B(c, USBS_KIND_REORTH_FINAL, mask ? 0.0 : 8.0 * sizeof(T) * c->n * (nb + 2));
  if (on_tc<T>(c) && tc_final(c, Qb, nb, W, out, mask, seed)) return;
  set_attrs<T>();
  const int ns = tile_stages<T>(nb, 8 * 64 + 64);
  const size_t sm = tile_smem<T>(nb, 8 * 64 + 64, ns);
  k_tfinalize<T><<<orth_grid(c, c->n, (const void*)k_tfinalize<T>, sm), 256, sm, c->stream>>>(
      (int)c->n, (const T*)Qb, (size_t)c->n * 8, nb, (const T*)W, c->red + RED_H2, c->lz, (T*)out,
      mask, seed, DEV_FIELD(c->lz, DevLanczos, status, int), ns);
}

template <typename T>
void Orth<T>::restart(Ctx* c, const void* Qb, int J, int nout, const double* Y, void* out,
                      const void* resid, int resid_slot) {
  USBS_LAUNCH_B(c, USBS_KIND_RESTART, 8.0 * sizeof(T) * c->n * (J / 8 + nout + (resid ? 2 : 0)));
  if (on_tc<T>(c) && tc_restart(c, Qb, J, nout, Y, out, resid, resid_slot)) return;
  set_attrs<T>();
  // stages, then Y: J x 8 nout values (FP64), or (hi, lo) TF32 pairs (FP32), 8 bytes each
  const size_t ybytes = 8 * (size_t)J * nout * 8;
  const int ns = pipe_stages(stage_bytes<T>(J / 8), ybytes);
  const size_t sm = (size_t)ns * stage_bytes<T>(J / 8) + ybytes;
  k_trestart<T><<<orth_grid(c, c->n, (const void*)k_trestart<T>, sm), 256, sm, c->stream>>>(
      (int)c->n, (const T*)Qb, (size_t)c->n * 8, J / 8, nout, Y, (T*)out, (size_t)c->n * 8,
      (const T*)resid, resid_slot, DEV_FIELD(c->lz, DevLanczos, status, int), ns);
}

template struct Orth<float>;
template struct Orth<double>;

namespace {
// The bounded wait of the staged tiles, run alone: one CTA arms a stage barrier for a 1 KB
// bulk copy and waits for it as every tile kernel does.  deliver = 0 issues no copy, so the
// wait runs out, USBS_ETIMEOUT is written to *status and the abort path (a second bounded
// wait, then the barriers released) runs; deliver = 1 issues the copy and the kernel ends
// with *status untouched.
__global__ void k_selftest_tile_wait(const float* __restrict__ src, int deliver, int* status) {
  __shared__ __align__(128) float buf[256];
  __shared__ uint64_t tbar[2];
  tiles_begin(tbar, 2);
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&tbar[0], 1024u);
    if (deliver) bulk_g2s(buf, src, 1024u, &tbar[0]);
  }
  const bool ok = tile_wait_cta(&tbar[0], 0, status);
  tiles_end(tbar, 2, ok ? -1 : 0, 0, 1, 1);
}

// the tiles' TF32 rounding and the PTX conversion, side by side
__global__ void k_selftest_tf32(int64_t count, const float* __restrict__ x, uint32_t* __restrict__ ours,
                                uint32_t* __restrict__ ref) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    ours[i] = tf32_of(x[i]);
    ref[i] = tf32_of_cvt(x[i]);
  }
}
}  // namespace

}  // namespace usbs

extern "C" int usbs_selftest_tile_wait(int deliver) {
  using namespace usbs;
  float* src = nullptr;
  int* st = nullptr;
  if (cudaMalloc(&src, 1024) != cudaSuccess || cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (src) cudaFree(src);
    return USBS_ENOMEM;
  }
  int status = 0;
  cudaError_t e = cudaMemset(src, 0, 1024);
  if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_selftest_tile_wait<<<1, 128>>>(src, deliver ? 1 : 0, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&status, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(src);
  cudaFree(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return USBS_ECUDA;
  }
  return status == USBS_ETIMEOUT ? USBS_ETIMEOUT : USBS_OK;
}

extern "C" int usbs_selftest_tf32_round(int64_t count, const float* x, uint32_t* ours, uint32_t* ref) {
  using namespace usbs;
  if (count < 0 || (count > 0 && (!x || !ours || !ref))) return USBS_EINVAL;
  if (count == 0) return USBS_OK;
  float* dx = nullptr;
  uint32_t* dout = nullptr;
  if (cudaMalloc(&dx, sizeof(float) * count) != cudaSuccess ||
      cudaMalloc(&dout, sizeof(uint32_t) * 2 * count) != cudaSuccess) {
    cudaGetLastError();
    if (dx) cudaFree(dx);
    return USBS_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(dx, x, sizeof(float) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    k_selftest_tf32<<<(int)blocks, 256>>>(count, dx, dout, dout + count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(ours, dout, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, dout + count, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dout);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return USBS_ECUDA;
  }
  return USBS_OK;
}
