// usbs_sketch_update_static: the sketch update of usbs_op_sketch_update for callers
// that must not allocate device memory.  Its scratch (the per-CTA partial sums of
// V^T Psi and their total) lives in one file-scope __device__ array instead of the
// context's cudaMalloc'ed buffers, and no context is needed.
#include <mutex>

#include "common.cuh"

namespace usbs {
namespace {

constexpr int NA_PARTS = 128;                 // CTAs of the V^T Psi reduction
constexpr int NA_RMAX = 32;                   // largest sketch rank accepted
constexpr int NA_PART_STRIDE = 8 * NA_RMAX;   // doubles per CTA partial
constexpr int NA_DOUBLES = NA_PARTS * NA_PART_STRIDE + 8 * NA_RMAX;
constexpr int NA_MAX_DEVICES = 64;

// 128 x 256 partial sums + the 8 x 32 result: 264,192 bytes on every GPU that loads
// the library, for the life of the process.
static __device__ __align__(256) double g_na_scratch[NA_DOUBLES];

// per-CTA partial sums of B = V^T Psi (8 x r), V n x 8 FP32, Psi n x r FP32
__global__ void __launch_bounds__(256) k_na_vt_psi(int n, int r, const float* __restrict__ V,
                                                   const float* __restrict__ Psi,
                                                   double* __restrict__ partials) {
  __shared__ float red[8][8 * NA_RMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane >> 3, a = lane & 7;
  float acc[NA_RMAX];
#pragma unroll
  for (int s = 0; s < NA_RMAX; ++s) acc[s] = 0.f;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 4; base < n; base += (int64_t)gridDim.x * 32) {
    const int64_t i = base + rr;
    if (i < n) {
      const float v = V[(size_t)8 * i + a];
      const float* pr = Psi + (size_t)r * i;
#pragma unroll
      for (int s = 0; s < NA_RMAX; ++s)
        if (s < r) acc[s] += v * pr[s];
    }
  }
#pragma unroll
  for (int s = 0; s < NA_RMAX; ++s) {
    acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 8);
    acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 16);
  }
  if (rr == 0) {
#pragma unroll
    for (int s = 0; s < NA_RMAX; ++s)
      if (s < r) red[warp][a * r + s] = acc[s];
  }
  __syncthreads();
  // every slot this call will read is written here, so stale contents never leak
  for (int t = threadIdx.x; t < 8 * r; t += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += (double)red[w][t];
    partials[(size_t)blockIdx.x * NA_PART_STRIDE + t] = sum;
  }
}

__global__ void k_na_reduce(const double* __restrict__ partials, int nparts, int nvals,
                            double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvals) return;
  double sum = 0.0;
  for (int p = 0; p < nparts; ++p) sum += partials[(size_t)p * NA_PART_STRIDE + t];
  out[t] = sum;
}

// P <- eta P + V (S B)
__global__ void __launch_bounds__(256) k_na_sketch(int n, int r, const float* __restrict__ V,
                                                   const double* __restrict__ S,
                                                   const double* __restrict__ B,
                                                   float* __restrict__ P, float eta) {
  __shared__ float Cm[8 * NA_RMAX];
  for (int t = threadIdx.x; t < 8 * r; t += blockDim.x) {
    const int a = t / r, s = t % r;
    double v = 0.0;
    for (int c = 0; c < 8; ++c) v += S[a * 8 + c] * B[c * r + s];
    Cm[t] = (float)v;
  }
  __syncthreads();
  const size_t total = (size_t)n * r;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / r;
    const int s = (int)(t % r);
    const float* vi = V + 8 * i;
    float acc = eta * P[t];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc += vi[a] * Cm[a * r + s];
    P[t] = acc;
  }
}

// Device address of g_na_scratch and the SM count, looked up once per device with that
// device current.
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {};
int g_na_sms[NA_MAX_DEVICES] = {};

int scratch_address(double** out, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return USBS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return USBS_ECUDA;
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
      cudaGetLastError();
      return USBS_ECUDA;
    }
    g_na_sms[dev] = nsm;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  *sms = g_na_sms[dev];
  return USBS_OK;
}

}  // namespace
}  // namespace usbs

extern "C" int usbs_sketch_update_static(int64_t n, int r, const float* V_dev,
                                         const double* S_dev, const float* Psi_dev,
                                         float* P_dev, double eta, void* stream) {
  using namespace usbs;
  if (n < 1 || n > 0x7fffffff - 1 || r < 1 || r > NA_RMAX || !V_dev || !S_dev || !Psi_dev ||
      !P_dev)
    return USBS_EINVAL;
  double* scratch = nullptr;
  int sms = 0;
  const int rc = scratch_address(&scratch, &sms);
  if (rc != USBS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* partials = scratch;
  double* B = scratch + NA_PARTS * NA_PART_STRIDE;
  k_na_vt_psi<<<NA_PARTS, 256, 0, st>>>((int)n, r, V_dev, Psi_dev, partials);
  k_na_reduce<<<1, 256, 0, st>>>(partials, NA_PARTS, 8 * r, B);
  int64_t g = (n * r + 255) / 256;
  if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;   // eight 256-thread CTAs per SM
  k_na_sketch<<<(int)g, 256, 0, st>>>((int)n, r, V_dev, S_dev, B, P_dev, (float)eta);
  if (cudaGetLastError() != cudaSuccess) return USBS_ECUDA;
  return USBS_OK;
}
