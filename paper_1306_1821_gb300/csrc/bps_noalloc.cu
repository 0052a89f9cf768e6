// k-bin power of a half spectrum without any device allocation.
//
// The same quantity as the sigma_m reduction behind bps_sample_power, for
// callers that are not allowed to allocate device memory themselves or through
// this library: the per-block partial sums live in a file-scope device array
// of fixed size instead of a buffer from cudaMalloc.  See bps_bin_power_noalloc
// in include/bps.h for the contract.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "bps_internal.h"
#include "bps_passes.cuh"

namespace bps {
namespace {

constexpr int NA_BLOCKS = 1024;                 // blocks of the first kernel (fixed grid)
constexpr int NA_THREADS = 256;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr int NA_MAX_N = 512;

// Scratch shared by every call on a device: NA_BLOCKS x MAXB partial sums
// (512 KiB), held by each GPU that loads the library until the process exits.
static __device__ __align__(256) double g_na_scratch[NA_BLOCKS * MAXB];

struct Thr {
  int t[MAXB];
};

// One warp per half-spectrum row (fixed ix, iy; all iz): along iz the bin is
// monotone, so the segmented shuffle sum of bin_accumulate applies with groups
// of 32 lanes.  Every block writes all MAXB of its partials on every call.
__global__ void __launch_bounds__(NA_THREADS) k_na_partials(const float2* __restrict__ spec, int N, Thr thr,
                                                            double* part) {
  __shared__ int s_thr[MAXB];
  __shared__ double s_wb[NA_WARPS][MAXB];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < MAXB; i += NA_THREADS) {
    s_thr[i] = thr.t[i];
    for (int k = 0; k < NA_WARPS; ++k) s_wb[k][i] = 0.0;
  }
  __syncthreads();
  const int H = N / 2, rowlen = H + 1;
  const long long rows = (long long)N * N;
  const long long gw = (long long)blockIdx.x * NA_WARPS + w, nw = (long long)gridDim.x * NA_WARPS;
  for (long long r = gw; r < rows; r += nw) {
    const int ix = (int)(r / N), iy = (int)(r % N);
    const int nx = ix <= H ? ix : ix - N, ny = iy <= H ? iy : iy - N;
    const int n2xy = nx * nx + ny * ny;
    const float2* row = spec + r * rowlen;
    for (int z0 = 0; z0 < rowlen; z0 += 32) {
      const int iz = z0 + lane;
      float e = 0.f;
      int m = -1;
      if (iz < rowlen) {
        const float2 x = row[iz];
        m = bin_of(n2xy + iz * iz, s_thr);
        const float wk = (iz == 0 || iz == H) ? 1.f : 2.f;
        e = wk * (x.x * x.x + x.y * x.y);
      }
      bin_accumulate<32>(e, m, s_wb[w]);
    }
  }
  __syncthreads();
  for (int m = t; m < MAXB; m += NA_THREADS) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NA_WARPS; ++k) s += s_wb[k][m];
    part[(size_t)m * NA_BLOCKS + blockIdx.x] = s;
  }
}

// block m: sigma_m = scale * sum over the NA_BLOCKS partials (fixed order)
__global__ void __launch_bounds__(256) k_na_finish(const double* part, double scale, double* sigma) {
  __shared__ double sh[32];
  const int m = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < NA_BLOCKS; i += 256) v += part[(size_t)m * NA_BLOCKS + i];
  v = block_sum<256>(v, sh);
  if (threadIdx.x == 0) sigma[m] = v * scale;
}

std::mutex g_na_mu;
double* g_na_ptr[64] = {nullptr};

}  // namespace
}  // namespace bps

using namespace bps;

extern "C" bps_status bps_bin_power_noalloc(int grid_n, double box_len, int n_bins, const float* spec_dev,
                                            double* sigma_dev, void* cuda_stream) {
  if (!spec_dev || !sigma_dev) {
    set_last_error("null argument");
    return BPS_EINVAL;
  }
  if (grid_n < 4 || grid_n > NA_MAX_N || (grid_n & 1)) {
    set_last_error("grid size must be even and in 4..512");
    return BPS_EINVAL;
  }
  if (n_bins < 1 || n_bins > MAXB) {
    set_last_error("n_bins must be in 1..64 (the static scratch holds 64 bins per block)");
    return BPS_EINVAL;
  }
  if (!(box_len > 0.0) || !std::isfinite(box_len)) {
    set_last_error("box length must be positive");
    return BPS_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(spec_dev) & 7) || (reinterpret_cast<uintptr_t>(sigma_dev) & 7)) {
    set_last_error("spec_dev and sigma_dev must be 8-byte aligned (complex64 and double arrays)");
    return BPS_EINVAL;
  }
  // the bins of bps_create, with the same validation: every bin needs a
  // threshold and at least one wave vector of the grid
  Thr thr;
  if (!bin_tables(grid_n, n_bins, thr.t, nullptr) || !bins_have_modes(grid_n, n_bins, thr.t)) {
    set_last_error("a bin holds no mode of the grid; use fewer bins");
    return BPS_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("no current CUDA device");
    return BPS_ECUDA;
  }
  double* part = nullptr;
  {
    // once per device, with that device current: the device address of the
    // static scratch (its host-side name is not a device address)
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p) {
        set_last_error("cudaGetSymbolAddress of the static scratch failed");
        return BPS_ECUDA;
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    part = g_na_ptr[dev];
  }
  // an error left by earlier, unrelated work is reported as such and left in
  // place, not taken for a failure of these launches
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "a CUDA error was already pending before this call: %s",
                  cudaGetErrorName(pending));
    set_last_error(msg);
    return BPS_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const double vc = std::pow(box_len / grid_n, 3);
  const double scale = vc / ((double)grid_n * grid_n * grid_n);
  k_na_partials<<<NA_BLOCKS, NA_THREADS, 0, s>>>(reinterpret_cast<const float2*>(spec_dev), grid_n, thr, part);
  k_na_finish<<<n_bins, 256, 0, s>>>(part, scale, sigma_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("kernel launch failed");
    return BPS_ECUDA;
  }
  return BPS_OK;
}

