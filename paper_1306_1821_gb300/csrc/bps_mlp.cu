// Mass-preconditioner network: a multilayer perceptron (ReLU hidden layers,
// linear output) trained by mean squared error with Adam, all on the device.
// The matrix products run on the tensor cores as BF16 operands with FP32
// accumulation (mma.sync m16n8k16); parameters, Adam moments and every other
// quantity stay FP32.  The paper's HMC uses the diagonal Fourier mass of Eq.
// Mass_matrix; the mass affects efficiency only (Sec. 4.1.2), and the network
// predicts per-bin log multipliers of it from binned features of the problem.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bps_internal.h"

namespace bps {
namespace {

constexpr int MLP_MAX_LAYERS = 4;
constexpr int MLP_MAX_WIDTH = 512;
constexpr float MASSNET_ZMAX = 4.0f;   // clamp of the standardised network-mass features

// ------------------------------------------------------------------ GEMM
// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]) (ReLU if act), FP32 in and
// out, BF16 operands.  TA: A is stored K x M (element (m,k) at A[k*lda + m]);
// TB: B is stored N x K (element (k,n) at B[n*ldb + k]).  One warp computes one
// 16 x 8 tile of C; operands are converted to BF16 as they are loaded.
// With `mask` (same layout as C) the result is multiplied by (mask > 0): the
// ReLU derivative of a backward pass.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const float* __restrict__ bias, int act,
                                              const float* __restrict__ mask) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;
  const int g = lane >> 2, q = lane & 3;
  auto a_at = [&](int m, int k) -> float {
    if (m >= M || k >= K) return 0.f;
    return TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k];
  };
  auto b_at = [&](int k, int n) -> float {
    if (k >= K || n >= N) return 0.f;
    return TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n];
  };
  const int m0 = tm * 16, n0 = tn * 8;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    a[0] = pack_bf16(a_at(m0 + g, k0 + 2 * q), a_at(m0 + g, k0 + 2 * q + 1));
    a[1] = pack_bf16(a_at(m0 + g + 8, k0 + 2 * q), a_at(m0 + g + 8, k0 + 2 * q + 1));
    a[2] = pack_bf16(a_at(m0 + g, k0 + 2 * q + 8), a_at(m0 + g, k0 + 2 * q + 9));
    a[3] = pack_bf16(a_at(m0 + g + 8, k0 + 2 * q + 8), a_at(m0 + g + 8, k0 + 2 * q + 9));
    b[0] = pack_bf16(b_at(k0 + 2 * q, n0 + g), b_at(k0 + 2 * q + 1, n0 + g));
    b[1] = pack_bf16(b_at(k0 + 2 * q + 8, n0 + g), b_at(k0 + 2 * q + 9, n0 + g));
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + g + (i >= 2 ? 8 : 0);
    const int n = n0 + 2 * q + (i & 1);
    if (m < M && n < N) {
      float v = c[i];
      if (bias) v += bias[n];
      if (act) v = fmaxf(v, 0.f);
      if (mask && !(mask[(long long)m * ldc + n] > 0.f)) v = 0.f;
      C[(long long)m * ldc + n] = v;
    }
  }
}

// column sums of G [M x N] into out[N] (bias gradients)
__global__ void k_colsum(int M, int N, const float* __restrict__ G, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += G[(long long)m * N + n];
  out[n] = s;
}

// d loss / d y = 2 (y - t) / (M N) and the loss sum (per-block FP64 partials)
__global__ void k_mse(int total, float scale, const float* __restrict__ y, const float* __restrict__ t,
                      float* __restrict__ g, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const float r = y[i] - t[i];
    g[i] = 2.f * r * scale;
    acc += (double)r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s * scale;
  }
}

// Adam with bias correction, in place on the FP32 parameter vector
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// rows idx[0..B) of X [n x d] into out [B x d]; idx drawn from Philox
__global__ void k_gather(int B, int d, int n, uint64_t seed, uint64_t step, const float* __restrict__ X,
                         const float* __restrict__ T, int dt, float* __restrict__ xo, float* __restrict__ to) {
  const int r = blockIdx.x;
  if (r >= B) return;
  __shared__ int src;
  if (threadIdx.x == 0) {
    P4 w = philox((uint64_t)r, step, 100, 0, seed);
    src = (int)(w.w[0] % (uint64_t)n);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) xo[(long long)r * d + j] = X[(long long)src * d + j];
  for (int j = threadIdx.x; j < dt; j += blockDim.x) to[(long long)r * dt + j] = T[(long long)src * dt + j];
}

__global__ void k_sum(const double* part, int n, double* out) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  *out = s;
}

__global__ void k_to_bf16(long long n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

}  // namespace

// ------------------------------------------------------------------ in-graph inference
// One device allocation: this header, then per layer the BF16 weights and the
// FP32 biases at the byte offsets below (16-byte aligned).
struct MassNet {
  int n_layers;
  int sizes[MLP_MAX_LAYERS + 1];
  long long off_w[MLP_MAX_LAYERS], off_b[MLP_MAX_LAYERS];
  float mean[MLP_MAX_WIDTH], sd[MLP_MAX_WIDTH];
  float log_clamp;
};

namespace {

// One block per chain: the features [ln P_m, ln W_m] of the chain's current
// state, standardised and clamped to +-MASSNET_ZMAX (a state far outside the
// training range, e.g. a bin whose P drifts, must not drive the network to
// arbitrary outputs), through the network with the numerics of the training
// kernels (operands rounded to BF16, FP32 accumulation, FP32 bias and ReLU),
// then s_j = exp(clamp(y_j)) into the chain's mass scales.  A matrix-vector
// product per layer (at most 512 x 512): FP32 FMAs over coalesced weight rows.
__global__ void __launch_bounds__(256) k_mass_net(ScalarArgs a, const MassNet* __restrict__ m) {
  DevState* ds = a.ds + blockIdx.y;
  __shared__ float h[2][MLP_MAX_WIDTH];
  const int t = threadIdx.x, nb = a.n_bins;
  const char* base = reinterpret_cast<const char*>(m);
  const int n0 = m->sizes[0];
  for (int i = t; i < n0; i += blockDim.x) {
    const float f = i < nb ? (float)log(ds->P[i]) : ds->wfeat[i - nb];
    const float z = (f - m->mean[i]) / m->sd[i];
    h[0][i] = bf16_round(fminf(fmaxf(z, -MASSNET_ZMAX), MASSNET_ZMAX));
  }
  __syncthreads();
  int cur = 0;
  const int L = m->n_layers;
  for (int l = 0; l < L; ++l) {
    const int ni = m->sizes[l], no = m->sizes[l + 1];
    const __nv_bfloat16* W = reinterpret_cast<const __nv_bfloat16*>(base + m->off_w[l]);
    const float* b = reinterpret_cast<const float*>(base + m->off_b[l]);
    for (int j = t; j < no; j += blockDim.x) {
      float acc = 0.f;
      for (int i = 0; i < ni; ++i) acc = fmaf(h[cur][i], __bfloat162float(W[(long long)i * no + j]), acc);
      float v = acc + b[j];
      if (l < L - 1) v = bf16_round(fmaxf(v, 0.f));
      h[cur ^ 1][j] = v;
    }
    __syncthreads();
    cur ^= 1;
  }
  const float c = m->log_clamp;
  for (int j = t; j < m->sizes[L]; j += blockDim.x) ds->mass_scale[j] = exp((double)fminf(fmaxf(h[cur][j], -c), c));
}

}  // namespace

int massnet_width(const bps_mlp* net, int output);
bps_status massnet_create(const bps_mlp* net, const float* mean, const float* sd, double log_clamp, MassNet** out);
void massnet_destroy(MassNet* m) { cudaFree(m); }

void launch_mass_net(const ScalarArgs& a, const MassNet* m, int nch, cudaStream_t s) {
  k_mass_net<<<dim3(1, nch), 256, 0, s>>>(a, m);
}

}  // namespace bps

using namespace bps;

struct bps_mlp {
  int L = 0;                       // number of layers
  int sizes[MLP_MAX_LAYERS + 1] = {0};
  size_t n_params = 0;
  size_t off_w[MLP_MAX_LAYERS] = {0}, off_b[MLP_MAX_LAYERS] = {0};
  cudaStream_t stream = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  // activations for a batch of up to cap rows
  int cap = 0;
  float* act[MLP_MAX_LAYERS + 1] = {nullptr};   // act[0] = input copy, act[l] = layer output
  float* grad_act[MLP_MAX_LAYERS + 1] = {nullptr};
  float *xb = nullptr, *tb = nullptr;           // minibatch buffers of the trainer
  double* part = nullptr;
  double* loss_dev = nullptr;
  long long adam_t = 0;
  std::string err;
};

namespace {

bps_status mfail(bps_mlp* n, bps_status s, const char* msg) {
  if (n) n->err = msg;
  set_last_error(msg);
  return s;
}

void gemm(bps_mlp* net, bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
          float* C, int ldc, const float* bias, int act, const float* mask) {
  const int warps = ((M + 15) / 16) * ((N + 7) / 8);
  const int blocks = (warps * 32 + 127) / 128;
  if (!ta && !tb) k_gemm<false, false><<<blocks, 128, 0, net->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, mask);
  else if (ta && !tb) k_gemm<true, false><<<blocks, 128, 0, net->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, mask);
  else if (!ta && tb) k_gemm<false, true><<<blocks, 128, 0, net->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, mask);
  else k_gemm<true, true><<<blocks, 128, 0, net->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, mask);
}

bps_status ensure_cap(bps_mlp* net, int B) {
  if (B <= net->cap) return BPS_OK;
  for (int l = 0; l <= net->L; ++l) {
    cudaFree(net->act[l]);
    cudaFree(net->grad_act[l]);
    net->act[l] = net->grad_act[l] = nullptr;
  }
  cudaFree(net->xb);
  cudaFree(net->tb);
  cudaFree(net->part);
  bool ok = true;
  for (int l = 0; l <= net->L && ok; ++l) {
    ok = cudaMalloc((void**)&net->act[l], (size_t)B * net->sizes[l] * sizeof(float)) == cudaSuccess &&
         cudaMalloc((void**)&net->grad_act[l], (size_t)B * net->sizes[l] * sizeof(float)) == cudaSuccess;
  }
  ok = ok && cudaMalloc((void**)&net->xb, (size_t)B * net->sizes[0] * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&net->tb, (size_t)B * net->sizes[net->L] * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&net->part, 256 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    net->cap = 0;
    return mfail(net, BPS_ENOMEM, "network buffers do not fit");
  }
  net->cap = B;
  return BPS_OK;
}

// forward pass of B rows from x (device, B x n0); outputs in act[L]
void forward(bps_mlp* net, int B, const float* x) {
  const float* h = x;
  for (int l = 0; l < net->L; ++l) {
    const int ni = net->sizes[l], no = net->sizes[l + 1];
    gemm(net, false, false, B, no, ni, h, ni, net->p + net->off_w[l], no, net->act[l + 1], no,
         net->p + net->off_b[l], l < net->L - 1 ? 1 : 0, nullptr);
    h = net->act[l + 1];
  }
}

// loss and gradients for B rows (x, t device); gradients into net->g
void backward(bps_mlp* net, int B, const float* x, const float* t) {
  const int L = net->L, no = net->sizes[L];
  const int total = B * no;
  k_mse<<<64, 256, 0, net->stream>>>(total, 1.f / (float)total, net->act[L], t, net->grad_act[L], net->part);
  k_sum<<<1, 1, 0, net->stream>>>(net->part, 64, net->loss_dev);
  for (int l = L - 1; l >= 0; --l) {
    const int ni = net->sizes[l], nl = net->sizes[l + 1];
    const float* hin = l == 0 ? x : net->act[l];
    // dW_l = h_l^T G_{l+1}  (K = B)
    gemm(net, true, false, ni, nl, B, hin, ni, net->grad_act[l + 1], nl, net->g + net->off_w[l], nl, nullptr, 0,
         nullptr);
    k_colsum<<<(nl + 127) / 128, 128, 0, net->stream>>>(B, nl, net->grad_act[l + 1], net->g + net->off_b[l]);
    if (l > 0) {
      // G_l = (G_{l+1} W_l^T) * relu'(z_l)
      gemm(net, false, true, B, ni, nl, net->grad_act[l + 1], nl, net->p + net->off_w[l], nl, net->grad_act[l], ni,
           nullptr, 0, net->act[l]);
    }
  }
}

void adam(bps_mlp* net, float lr) {
  net->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)net->adam_t), c2 = 1.f - powf(b2, (float)net->adam_t);
  const int n = (int)net->n_params;
  k_adam<<<(n + 255) / 256, 256, 0, net->stream>>>(n, net->p, net->g, net->m, net->v, lr, b1, b2, 1e-8f, c1, c2);
}

}  // namespace

extern "C" {

bps_status bps_mlp_create(int n_layers, const int* sizes, void* cuda_stream, bps_mlp** out) {
  if (!out || !sizes) return mfail(nullptr, BPS_EINVAL, "null argument");
  *out = nullptr;
  if (n_layers < 1 || n_layers > MLP_MAX_LAYERS) return mfail(nullptr, BPS_EINVAL, "1..4 layers");
  for (int l = 0; l <= n_layers; ++l)
    if (sizes[l] < 1 || sizes[l] > MLP_MAX_WIDTH) return mfail(nullptr, BPS_EINVAL, "layer widths must be in 1..512");
  bps_mlp* net = new bps_mlp();
  net->L = n_layers;
  net->stream = (cudaStream_t)cuda_stream;
  size_t off = 0;
  for (int l = 0; l <= n_layers; ++l) net->sizes[l] = sizes[l];
  for (int l = 0; l < n_layers; ++l) {
    net->off_w[l] = off;
    off += (size_t)sizes[l] * sizes[l + 1];
    net->off_b[l] = off;
    off += sizes[l + 1];
  }
  net->n_params = off;
  bool ok = cudaMalloc((void**)&net->p, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&net->g, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&net->m, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&net->v, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&net->loss_dev, sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    delete net;
    return mfail(nullptr, BPS_ENOMEM, "network allocation failed");
  }
  cudaMemsetAsync(net->p, 0, off * sizeof(float), net->stream);
  cudaMemsetAsync(net->m, 0, off * sizeof(float), net->stream);
  cudaMemsetAsync(net->v, 0, off * sizeof(float), net->stream);
  *out = net;
  return BPS_OK;
}

void bps_mlp_destroy(bps_mlp* net) {
  if (!net) return;
  cudaStreamSynchronize(net->stream);
  for (int l = 0; l <= net->L; ++l) {
    cudaFree(net->act[l]);
    cudaFree(net->grad_act[l]);
  }
  cudaFree(net->xb);
  cudaFree(net->tb);
  cudaFree(net->part);
  cudaFree(net->p);
  cudaFree(net->g);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->loss_dev);
  delete net;
}

size_t bps_mlp_num_params(const bps_mlp* net) { return net ? net->n_params : 0; }

bps_status bps_mlp_set_params(bps_mlp* net, const float* params) {
  if (!net || !params) return mfail(net, BPS_EINVAL, "null argument");
  if (cudaMemcpy(net->p, params, net->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->m, 0, net->n_params * sizeof(float)) != cudaSuccess ||
      cudaMemset(net->v, 0, net->n_params * sizeof(float)) != cudaSuccess)
    return mfail(net, BPS_ECUDA, "parameter upload failed");
  net->adam_t = 0;
  return BPS_OK;
}

bps_status bps_mlp_get_params(bps_mlp* net, float* params) {
  if (!net || !params) return mfail(net, BPS_EINVAL, "null argument");
  cudaStreamSynchronize(net->stream);
  if (cudaMemcpy(params, net->p, net->n_params * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(net, BPS_ECUDA, "parameter download failed");
  return BPS_OK;
}

bps_status bps_mlp_forward(bps_mlp* net, int batch, const float* x_dev, float* y_dev) {
  if (!net || !x_dev || !y_dev || batch < 1) return mfail(net, BPS_EINVAL, "bad argument");
  bps_status st = ensure_cap(net, batch);
  if (st != BPS_OK) return st;
  forward(net, batch, x_dev);
  const int no = net->sizes[net->L];
  cudaMemcpyAsync(y_dev, net->act[net->L], (size_t)batch * no * sizeof(float), cudaMemcpyDeviceToDevice,
                  net->stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess)
    return mfail(net, BPS_ECUDA, "forward pass failed");
  return BPS_OK;
}

bps_status bps_mlp_loss_grad(bps_mlp* net, int batch, const float* x_dev, const float* t_dev, double* loss,
                             float* grads) {
  if (!net || !x_dev || !t_dev || batch < 1) return mfail(net, BPS_EINVAL, "bad argument");
  bps_status st = ensure_cap(net, batch);
  if (st != BPS_OK) return st;
  forward(net, batch, x_dev);
  backward(net, batch, x_dev, t_dev);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess)
    return mfail(net, BPS_ECUDA, "backward pass failed");
  if (loss) cudaMemcpy(loss, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost);
  if (grads) cudaMemcpy(grads, net->g, net->n_params * sizeof(float), cudaMemcpyDeviceToHost);
  return BPS_OK;
}

bps_status bps_mlp_adam_step(bps_mlp* net, float lr) {
  if (!net) return mfail(nullptr, BPS_EINVAL, "null argument");
  adam(net, lr);
  if (cudaGetLastError() != cudaSuccess) return mfail(net, BPS_ECUDA, "Adam step failed");
  return BPS_OK;
}

bps_status bps_mlp_export(bps_mlp* net, const float* feat_mean, const float* feat_std, double log_clamp, void* blob,
                          size_t* bytes) {
  if (!net || !bytes) return mfail(net, BPS_EINVAL, "null argument");
  const size_t need = 12 + 4 * (size_t)(net->L + 1) + 8 + 2 * 4 * (size_t)net->sizes[0] + 4 * net->n_params;
  if (!blob) {
    *bytes = need;
    return BPS_OK;
  }
  if (*bytes < need) return mfail(net, BPS_EINVAL, "buffer too small for the preconditioner");
  if (!feat_mean || !feat_std) return mfail(net, BPS_EINVAL, "null argument");
  unsigned char* b = static_cast<unsigned char*>(blob);
  size_t off = 0;
  auto put = [&](const void* src, size_t n) {
    std::memcpy(b + off, src, n);
    off += n;
  };
  const uint32_t version = 1, L = (uint32_t)net->L;
  put("BPSM", 4);
  put(&version, 4);
  put(&L, 4);
  for (int l = 0; l <= net->L; ++l) {
    const uint32_t w = (uint32_t)net->sizes[l];
    put(&w, 4);
  }
  put(&log_clamp, 8);
  put(feat_mean, 4 * (size_t)net->sizes[0]);
  put(feat_std, 4 * (size_t)net->sizes[0]);
  std::vector<float> p(net->n_params);
  bps_status st = bps_mlp_get_params(net, p.data());
  if (st != BPS_OK) return st;
  put(p.data(), 4 * net->n_params);
  *bytes = need;
  return BPS_OK;
}

bps_status bps_mlp_train(bps_mlp* net, int n_examples, const float* x_dev, const float* t_dev, int batch, int steps,
                         float lr, uint64_t seed, double* last_loss) {
  if (!net || !x_dev || !t_dev || n_examples < 1 || batch < 1 || steps < 0)
    return mfail(net, BPS_EINVAL, "bad argument");
  bps_status st = ensure_cap(net, batch);
  if (st != BPS_OK) return st;
  const int d = net->sizes[0], dt = net->sizes[net->L];
  for (int s = 0; s < steps; ++s) {
    k_gather<<<batch, 64, 0, net->stream>>>(batch, d, n_examples, seed, (uint64_t)net->adam_t, x_dev, t_dev, dt,
                                            net->xb, net->tb);
    forward(net, batch, net->xb);
    backward(net, batch, net->xb, net->tb);
    adam(net, lr);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess)
    return mfail(net, BPS_ECUDA, "training failed");
  if (last_loss) cudaMemcpy(last_loss, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost);
  return BPS_OK;
}

}  // extern "C"

namespace bps {

int massnet_width(const bps_mlp* net, int output) { return output ? net->sizes[net->L] : net->sizes[0]; }

bps_status massnet_create(const bps_mlp* net, const float* mean, const float* sd, double log_clamp, MassNet** out) {
  *out = nullptr;
  MassNet h{};
  h.n_layers = net->L;
  auto up16 = [](long long x) { return (x + 15) & ~15LL; };
  long long off = up16((long long)sizeof(MassNet));
  for (int l = 0; l <= net->L; ++l) h.sizes[l] = net->sizes[l];
  for (int l = 0; l < net->L; ++l) {
    h.off_w[l] = off;
    off = up16(off + 2LL * net->sizes[l] * net->sizes[l + 1]);
    h.off_b[l] = off;
    off = up16(off + 4LL * net->sizes[l + 1]);
  }
  for (int i = 0; i < net->sizes[0]; ++i) {
    h.mean[i] = mean[i];
    h.sd[i] = sd[i];
  }
  h.log_clamp = (float)log_clamp;
  char* blob = nullptr;
  if (cudaMalloc((void**)&blob, (size_t)off) != cudaSuccess) {
    cudaGetLastError();
    return mfail(nullptr, BPS_ENOMEM, "network copy allocation failed");
  }
  cudaStream_t s = net->stream;
  bool ok = cudaMemcpyAsync(blob, &h, sizeof(MassNet), cudaMemcpyHostToDevice, s) == cudaSuccess;
  for (int l = 0; l < net->L && ok; ++l) {
    const long long nw = (long long)net->sizes[l] * net->sizes[l + 1];
    k_to_bf16<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(nw, net->p + net->off_w[l],
                                                          reinterpret_cast<__nv_bfloat16*>(blob + h.off_w[l]));
    ok = cudaMemcpyAsync(blob + h.off_b[l], net->p + net->off_b[l], 4 * (size_t)net->sizes[l + 1],
                         cudaMemcpyDeviceToDevice, s) == cudaSuccess;
  }
  ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaFree(blob);
    return mfail(nullptr, BPS_ECUDA, "network copy failed");
  }
  *out = reinterpret_cast<MassNet*>(blob);
  return BPS_OK;
}

}  // namespace bps
