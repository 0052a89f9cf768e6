// Host side of the bps C ABI: context life cycle, data and state transfer, and
// the launch sequences of the sampler's stages (the ABI is declared and
// documented in include/bps.h).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bps_internal.h"
#include "bps_passes.cuh"

using namespace bps;

struct bps_ctx {
  int N = 0, n_sub = 0, zp = 0;
  double box = 0, Vc = 0;
  bps_config cfg{};
  cudaStream_t stream = nullptr;
  PassTable pt{};
  long long nv = 0;
  size_t n_spec = 0;          // complex elements of one padded half spectrum
  float2* dh[2] = {nullptr, nullptr};
  float2* ph = nullptr;
  float2* W = nullptr;
  float* a = nullptr;
  float* c = nullptr;
  uint16_t* cnt = nullptr;
  float* R = nullptr;
  float2* tw = nullptr;
  double* part = nullptr;
  int part_stride = 0;
  DevState* ds = nullptr;
  double* chain_dev = nullptr;
  int chain_cap = 0;
  double* host_buf = nullptr;   // pinned staging for small reads
  int n_mass = 0;
  bool have_data = false;
  int rebuild_blocks = 0;
  int n_sm = 0;
  uint64_t launches = 0;
  // leapfrog kernel timing (bps_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev[4];
  size_t ev_used[4] = {0, 0, 0, 0};
  double prof_ms[4] = {0, 0, 0, 0};
  uint64_t prof_n[4] = {0, 0, 0, 0};
  std::string err;
};

namespace {

std::string g_err;

// partial-sum regions (offsets in doubles into ctx->part)
enum Region { RG_INIT = 0, RG_LIK0, RG_FINAL, RG_LIK1, RG_BIN, RG_SUMS, RG_RB, RG_JGRAD, RG_JLIK, RG_GRAD, RG_COUNT };
// quantities per region
int region_width(Region r) {
  switch (r) {
    case RG_INIT: case RG_FINAL: return 2;
    case RG_BIN: case RG_JGRAD: return MAXB;
    case RG_SUMS: return 3 * MAXS;
    default: return 1;
  }
}
int region_offset(const bps_ctx* c, Region r) {
  int off = 0;
  for (int i = 0; i < (int)r; ++i) off += region_width((Region)i);
  return off * c->part_stride;
}
int region_total() {
  int w = 0;
  for (int i = 0; i < RG_COUNT; ++i) w += region_width((Region)i);
  return w;
}

bps_status fail(bps_ctx* c, bps_status s, const std::string& msg) {
  if (c) c->err = msg;
  g_err = msg;
  return s;
}

bps_status cuda_check(bps_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BPS_OK;
  return fail(c, BPS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    bps_status _s = cuda_check(ctx, (call), #call);           \
    if (_s != BPS_OK) return _s;                              \
  } while (0)

#define LAUNCHED(ctx, n)                                      \
  do {                                                        \
    (ctx)->launches += (n);                                   \
    bps_status _s = cuda_check((ctx), cudaGetLastError(), "kernel launch"); \
    if (_s != BPS_OK) return _s;                              \
  } while (0)

Fields fields(bps_ctx* c) {
  Fields f;
  f.dh[0] = c->dh[0];
  f.dh[1] = c->dh[1];
  f.ph = c->ph;
  f.W = c->W;
  f.a = c->a;
  f.c = c->c;
  f.cnt = c->cnt;
  f.R = c->R;
  f.n_sub = c->n_sub;
  f.ds = c->ds;
  f.part = c->part;
  f.part_stride = c->part_stride;
  f.tw = c->tw;
  f.inv_nv = (float)(1.0 / (double)c->nv);
  f.mass_mode = c->cfg.mass_mode;
  f.n_sm = c->n_sm;
  return f;
}

ScalarArgs scalars(bps_ctx* c) {
  ScalarArgs a;
  a.ds = c->ds;
  a.part = c->part;
  a.stride = c->part_stride;
  a.n_bins = c->cfg.n_bins;
  a.n_sub = c->n_sub;
  a.n_mass = c->n_mass;
  a.Vc = c->Vc;
  a.inv_nv = 1.0 / (double)c->nv;
  a.alpha = c->cfg.alpha;
  a.eps_max = c->cfg.eps_max;
  a.jeps_max = c->cfg.jump_eps_max;
  a.seed = c->cfg.seed;
  a.fixed_bias = c->cfg.fixed_bias_index;
  return a;
}

// bin of integer |n|^2 for n_bins linear bins over (0, sqrt(3) N / 2]
int bin_of_host(long long n2, int N, int nb) {
  double b = std::floor((double)nb * std::sqrt((double)n2) / (std::sqrt(3.0) * (double)N / 2.0));
  int m = (int)b;
  return m > nb - 1 ? nb - 1 : m;
}

// thresholds (smallest n2 of each bin) and full-grid mode counts; false if a bin is empty
bool bin_tables(int N, int nb, int* thr, double* nmodes) {
  for (int m = 0; m < MAXB; ++m) {
    thr[m] = 0x7fffffff;
    if (nmodes) nmodes[m] = 0.0;
  }
  thr[0] = 0;
  const long long maxn2 = 3LL * (N / 2) * (N / 2);
  int prev = 0;
  for (long long n2 = 1; n2 <= maxn2; ++n2) {
    int m = bin_of_host(n2, N, nb);
    while (prev < m) {
      ++prev;
      thr[prev] = (int)n2;
    }
  }
  if (nmodes) {
    const int H = N / 2;
    for (int ix = 0; ix < N; ++ix) {
      const long long nx = ix <= H ? ix : ix - N;
      for (int iy = 0; iy < N; ++iy) {
        const long long ny = iy <= H ? iy : iy - N;
        for (int iz = 0; iz <= H; ++iz) {
          const long long n2 = nx * nx + ny * ny + (long long)iz * iz;
          if (n2 == 0) continue;
          const double w = (iz == 0 || iz == H) ? 1.0 : 2.0;
          nmodes[bin_of_host(n2, N, nb)] += w;
        }
      }
    }
    for (int m = 0; m < nb; ++m)
      if (nmodes[m] <= 0.0) return false;
  }
  for (int m = 1; m < nb; ++m)
    if (thr[m] == 0x7fffffff) return false;
  return true;
}

bps_status ds_write_bytes(bps_ctx* ctx, size_t off, const void* src, size_t n) {
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->ds) + off, src, n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status ds_read_bytes(bps_ctx* ctx, size_t off, void* dst, size_t n) {
  CK(cudaMemcpyAsync(ctx->host_buf, reinterpret_cast<char*>(ctx->ds) + off, n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(dst, ctx->host_buf, n);
  return BPS_OK;
}

#define DS_OFF(member) offsetof(DevState, member)

bps_status check_status(bps_ctx* ctx) {
  int st = 0;
  bps_status s = ds_read_bytes(ctx, DS_OFF(status), &st, sizeof(int));
  if (s != BPS_OK) return s;
  if (st != 0) {
    int zero = 0;
    ds_write_bytes(ctx, DS_OFF(status), &zero, sizeof(int));
    if (st & ST_TIMEOUT) return fail(ctx, BPS_ETIMEOUT, "a tile copy did not complete within the wait limit");
    if (st & ST_NONFINITE) return fail(ctx, BPS_ENUMERIC, "non-finite energy difference; move rejected");
    return fail(ctx, BPS_ENUMERIC, "a scalar draw failed (no acceptance within the attempt bound or a non-positive sum)");
  }
  return BPS_OK;
}

// ------------------------------------------------------------------ stages
bps_status rebuild(bps_ctx* ctx) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  launch_rebuild(f, ctx->nv, region_offset(ctx, RG_RB), ctx->rebuild_blocks, ctx->stream);
  launch_abar(sa, region_offset(ctx, RG_RB), ctx->rebuild_blocks, ctx->stream);
  LAUNCHED(ctx, 2);
  return BPS_OK;
}

constexpr size_t PROF_CAP = 8192;   // event pairs per kernel kind before folding

void prof_fold(bps_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < 4; ++k) {
    for (size_t i = 0; i + 1 < ctx->ev_used[k]; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev[k][i], ctx->ev[k][i + 1]) == cudaSuccess) {
        ctx->prof_ms[k] += ms;
        ctx->prof_n[k] += 1;
      }
    }
    ctx->ev_used[k] = 0;
  }
}

// record one event of kernel kind k (start or end); no-op unless profiling
void prof_mark(bps_ctx* ctx, int k) {
  if (!ctx->prof) return;
  if (ctx->ev_used[k] >= PROF_CAP && ctx->ev_used[k] % 2 == 0) prof_fold(ctx);
  if (ctx->ev_used[k] == ctx->ev[k].size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ctx->ev[k].push_back(e);
  }
  cudaEventRecord(ctx->ev[k][ctx->ev_used[k]++], ctx->stream);
}

// force of the current state into W (Fourier), likelihood energy partials in `lik_region`
bps_status hmc_move(bps_ctx* ctx, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const PassTable& P = ctx->pt;
  const int L = ctx->cfg.n_leapfrog;
  launch_move_begin(sa, s);
  P.z_noise(f, ctx->cfg.seed, s);
  P.y_fwd(f, BUF_PH, s);
  P.x_init(f, region_offset(ctx, RG_INIT), s);
  P.y_inv(f, BUF_W, s);
  P.z_grad(f, region_offset(ctx, RG_LIK0), s);
  P.y_fwd(f, BUF_W, s);
  for (int st = 1; st <= L; ++st) {
    prof_mark(ctx, 0);
    P.x_leap(f, st == 1 ? 1 : 0, s);
    prof_mark(ctx, 0);
    prof_mark(ctx, 1);
    P.y_inv(f, BUF_W, s);
    prof_mark(ctx, 1);
    prof_mark(ctx, 2);
    P.z_grad(f, st == L ? region_offset(ctx, RG_LIK1) : -1, s);
    prof_mark(ctx, 2);
    prof_mark(ctx, 3);
    P.y_fwd(f, BUF_W, s);
    prof_mark(ctx, 3);
  }
  P.x_final(f, region_offset(ctx, RG_FINAL), s);
  launch_move_end(sa, region_offset(ctx, RG_INIT), region_offset(ctx, RG_LIK0), region_offset(ctx, RG_FINAL),
                  region_offset(ctx, RG_LIK1), P.x_tiles, P.z_tiles, s);
  int n = 9 + 4 * L;
  if (advance) {
    launch_advance(ctx->ds, s);
    ++n;
  }
  LAUNCHED(ctx, n);
  return BPS_OK;
}

bps_status power_stage(bps_ctx* ctx, bool draw, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  ctx->pt.x_binpow(f, region_offset(ctx, RG_BIN), ctx->stream);
  launch_power(sa, region_offset(ctx, RG_BIN), ctx->pt.x_tiles, draw ? 1 : 0, ctx->stream);
  int n = 2;
  if (advance) {
    launch_advance(ctx->ds, ctx->stream);
    ++n;
  }
  LAUNCHED(ctx, n);
  return BPS_OK;
}

bps_status bias_stage(bps_ctx* ctx, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  // delta = C2R(delta_hat) (x and y inverse into W), the per-subsample sums in the z pass
  ctx->pt.x_inv(f, -1, ctx->W, s);
  ctx->pt.y_inv(f, BUF_W, s);
  ctx->pt.z_sums(f, region_offset(ctx, RG_SUMS), s);
  launch_bias_nbar(sa, region_offset(ctx, RG_SUMS), ctx->pt.z_tiles, s);
  LAUNCHED(ctx, 4);
  bps_status st = rebuild(ctx);
  if (st != BPS_OK) return st;
  if (advance) {
    launch_advance(ctx->ds, s);
    LAUNCHED(ctx, 1);
  }
  return BPS_OK;
}

// force evaluation of the jump at the current theta (scales js on the device)
bps_status jump_gradient(bps_ctx* ctx) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const PassTable& P = ctx->pt;
  P.x_jinv(f, s);
  P.y_inv(f, BUF_W, s);
  P.z_grad(f, region_offset(ctx, RG_JLIK), s);
  P.y_fwd(f, BUF_W, s);
  P.x_jgrad(f, region_offset(ctx, RG_JGRAD), s);
  launch_jump_reduce(sa, region_offset(ctx, RG_JGRAD), P.x_tiles, region_offset(ctx, RG_JLIK), P.z_tiles, s);
  LAUNCHED(ctx, 6);
  return BPS_OK;
}

bps_status jump_stage(bps_ctx* ctx, bool advance) {
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  bps_status st = power_stage(ctx, false, false);   // sigma of the current field (mass of the jump)
  if (st != BPS_OK) return st;
  launch_jump_begin(sa, s);
  LAUNCHED(ctx, 1);
  const int L = ctx->cfg.jump_leapfrog;
  st = jump_gradient(ctx);
  if (st != BPS_OK) return st;
  launch_jump_update(sa, J_FIRST, s);
  LAUNCHED(ctx, 1);
  for (int k = 0; k < L; ++k) {
    st = jump_gradient(ctx);
    if (st != BPS_OK) return st;
    launch_jump_update(sa, k == L - 1 ? J_LAST : J_MID, s);
    LAUNCHED(ctx, 1);
  }
  Fields f = fields(ctx);
  ctx->pt.x_scale(f, s);   // delta_k <- sqrt(P'/P) delta_k if accepted (Eq. det_trans)
  LAUNCHED(ctx, 1);
  if (advance) {
    launch_advance(ctx->ds, s);
    LAUNCHED(ctx, 1);
  }
  return BPS_OK;
}

bps_status need_data(bps_ctx* ctx) {
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  if (!ctx->have_data) return fail(ctx, BPS_ESTATE, "bps_set_data has not been called");
  return BPS_OK;
}

bps_status copy_spec_out(bps_ctx* ctx, const float2* src, float* dst) {
  const size_t H1 = (size_t)ctx->N / 2 + 1;
  CK(cudaMemcpy2DAsync(dst, H1 * sizeof(float2), src, (size_t)ctx->zp * sizeof(float2), H1 * sizeof(float2),
                       (size_t)ctx->N * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
  return BPS_OK;
}

bps_status copy_spec_in(bps_ctx* ctx, const float* src, float2* dst) {
  const size_t H1 = (size_t)ctx->N / 2 + 1;
  CK(cudaMemcpy2DAsync(dst, (size_t)ctx->zp * sizeof(float2), src, H1 * sizeof(float2), H1 * sizeof(float2),
                       (size_t)ctx->N * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
  return BPS_OK;
}

int current_buffer(bps_ctx* ctx, bps_status* st) {
  int cur = 0;
  *st = ds_read_bytes(ctx, DS_OFF(cur), &cur, sizeof(int));
  return cur;
}

void free_all(bps_ctx* c) {
  for (int k = 0; k < 4; ++k)
    for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
  cudaFree(c->dh[0]);
  cudaFree(c->dh[1]);
  cudaFree(c->ph);
  cudaFree(c->W);
  cudaFree(c->a);
  cudaFree(c->c);
  cudaFree(c->cnt);
  cudaFree(c->R);
  cudaFree(c->tw);
  cudaFree(c->part);
  cudaFree(c->ds);
  cudaFree(c->chain_dev);
  if (c->host_buf) cudaFreeHost(c->host_buf);
}

}  // namespace

void bps::set_last_error(const char* msg) { g_err = msg; }

// =================================================================== C ABI
extern "C" {

const char* bps_version(void) { return "bps 0.1 (sm_103a)"; }

const char* bps_last_error(const bps_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

uint64_t bps_kernel_launches(const bps_ctx* ctx) { return ctx ? ctx->launches : 0; }

bps_status bps_profile(bps_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  if (ctx->prof && !enable) prof_fold(ctx);
  ctx->prof = enable != 0;
  return BPS_OK;
}

bps_status bps_profile_read(bps_ctx* ctx, double* ms, uint64_t* n) {
  if (!ctx || !ms || !n) return fail(ctx, BPS_EINVAL, "null argument");
  prof_fold(ctx);
  for (int k = 0; k < 4; ++k) {
    ms[k] = ctx->prof_ms[k];
    n[k] = ctx->prof_n[k];
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  return BPS_OK;
}

bps_status bps_create(int grid_n, double box_len, int n_sub, const bps_config* cfg, void* cuda_stream,
                      bps_ctx** out) {
  if (!out || !cfg) return fail(nullptr, BPS_EINVAL, "null argument");
  *out = nullptr;
  PassTable pt;
  if (!pass_table(grid_n, &pt)) return fail(nullptr, BPS_EINVAL, "unsupported grid size (8,16,32,64,96,128,256)");
  if (!(box_len > 0.0) || !std::isfinite(box_len)) return fail(nullptr, BPS_EINVAL, "box length must be positive");
  if (n_sub < 1 || n_sub > MAXS) return fail(nullptr, BPS_EINVAL, "n_sub must be in 1..16");
  if (cfg->n_bins < 1 || cfg->n_bins > MAXB) return fail(nullptr, BPS_EINVAL, "n_bins must be in 1..64");
  if (cfg->n_leapfrog < 1 || !(cfg->eps_max > 0.0)) return fail(nullptr, BPS_EINVAL, "bad leapfrog settings");
  if (cfg->jump && (cfg->jump_leapfrog < 1 || !(cfg->jump_eps_max > 0.0)))
    return fail(nullptr, BPS_EINVAL, "bad jump settings");
  if (cfg->fixed_bias_index >= n_sub) return fail(nullptr, BPS_EINVAL, "fixed_bias_index out of range");
  if (cfg->mass_mode != 0 && cfg->mass_mode != 1) return fail(nullptr, BPS_EINVAL, "mass_mode must be 0 or 1");

  DevState h;
  std::memset(&h, 0, sizeof(h));
  if (!bin_tables(grid_n, cfg->n_bins, h.thr, h.nmodes))
    return fail(nullptr, BPS_EINVAL, "a power-spectrum bin holds no mode; use fewer bins");
  bin_tables(grid_n, cfg->n_bins, h.mthr, nullptr);

  bps_ctx* ctx = new bps_ctx();
  ctx->N = grid_n;
  ctx->n_sub = n_sub;
  ctx->box = box_len;
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->pt = pt;
  ctx->zp = pt.zp;
  ctx->nv = (long long)grid_n * grid_n * grid_n;
  ctx->Vc = std::pow(box_len / grid_n, 3);
  ctx->n_spec = (size_t)grid_n * grid_n * pt.zp;
  ctx->n_mass = cfg->n_bins;
  ctx->chain_cap = 1024;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ctx->rebuild_blocks = sms > 0 ? 4 * sms : 512;
  ctx->n_sm = sms > 0 ? sms : 148;
  ctx->part_stride = std::max(std::max(pt.x_tiles, pt.z_tiles), ctx->rebuild_blocks);

  auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
  const size_t sb = ctx->n_spec * sizeof(float2), rb = (size_t)ctx->nv * sizeof(float);
  bool ok = alloc((void**)&ctx->dh[0], sb) && alloc((void**)&ctx->dh[1], sb) && alloc((void**)&ctx->ph, sb) &&
            alloc((void**)&ctx->W, sb) && alloc((void**)&ctx->a, rb) && alloc((void**)&ctx->c, rb) &&
            alloc((void**)&ctx->tw, grid_n * sizeof(float2)) &&
            alloc((void**)&ctx->part, (size_t)region_total() * ctx->part_stride * sizeof(double)) &&
            alloc((void**)&ctx->ds, sizeof(DevState)) &&
            alloc((void**)&ctx->chain_dev, (size_t)1024 * (cfg->n_bins + 2 * n_sub + 2) * sizeof(double)) &&
            cudaMallocHost((void**)&ctx->host_buf, 64 * 1024) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ENOMEM, "device allocation failed");
  }
  // twiddles W_N^j = exp(-2 pi i j / N), FP64 rounded to FP32
  std::vector<float2> tw(grid_n);
  for (int j = 0; j < grid_n; ++j) {
    const double ang = -2.0 * M_PI * (double)j / (double)grid_n;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  for (int m = 0; m < MAXB; ++m) {
    h.P[m] = 1.0;
    h.P_ref[m] = 1.0;
    h.mass_scale[m] = 1.0;
    h.js[m] = 1.f;
  }
  for (int l = 0; l < MAXS; ++l) {
    h.b[l] = 1.0;
    h.nbar[l] = 1.0;
  }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(ctx->tw, tw.data(), grid_n * sizeof(float2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ds, &h, sizeof(DevState), cudaMemcpyHostToDevice, s);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(ctx->dh[i], 0, sb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ph, 0, sb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->W, 0, sb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->a, 0, rb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->c, 0, rb, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    std::string msg = std::string("initialisation failed: ") + cudaGetErrorString(e);
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ECUDA, msg);
  }
  *out = ctx;
  return BPS_OK;
}

void bps_destroy(bps_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

static bps_status set_data_impl(bps_ctx* ctx, const int32_t* counts, const float* R, bool host) {
  if (!ctx || !counts || !R) return fail(ctx, BPS_EINVAL, "null argument");
  cudaStream_t s = ctx->stream;
  const size_t total = (size_t)ctx->n_sub * ctx->nv;
  if (!ctx->cnt) {
    if (cudaMalloc((void**)&ctx->cnt, total * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->R, total * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->cnt);
      cudaFree(ctx->R);
      ctx->cnt = nullptr;
      ctx->R = nullptr;
      return fail(ctx, BPS_ENOMEM, "device allocation of the survey data failed");
    }
  }
  const int32_t* cdev = counts;
  const float* rdev = R;
  int32_t* ctmp = nullptr;
  float* rtmp = nullptr;
  if (host) {
    // stage through the spectrum work buffers (each at least N^3 * 8 bytes)
    ctmp = reinterpret_cast<int32_t*>(ctx->ph);
    rtmp = reinterpret_cast<float*>(ctx->W);
  }
  const int blocks = ctx->rebuild_blocks;
  std::vector<double> hp(4 * (size_t)blocks);
  std::vector<double> sR(ctx->n_sub), sB(ctx->n_sub), no(ctx->n_sub);
  double bad = 0.0;
  for (int l = 0; l < ctx->n_sub; ++l) {
    const int32_t* cl = cdev + (size_t)l * ctx->nv;
    const float* rl = rdev + (size_t)l * ctx->nv;
    if (host) {
      CK(cudaMemcpyAsync(ctmp, counts + (size_t)l * ctx->nv, ctx->nv * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(rtmp, R + (size_t)l * ctx->nv, ctx->nv * sizeof(float), cudaMemcpyHostToDevice, s));
      cl = ctmp;
      rl = rtmp;
    }
    launch_data(cl, rl, ctx->cnt + (size_t)l * ctx->nv, ctx->R + (size_t)l * ctx->nv, ctx->nv, ctx->part, blocks,
                blocks, s);
    LAUNCHED(ctx, 1);
    CK(cudaMemcpyAsync(hp.data(), ctx->part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double v[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int b = 0; b < blocks; ++b) v[q] += hp[(size_t)q * blocks + b];
    sR[l] = v[0];
    sB[l] = v[1];
    no[l] = v[2];
    bad += v[3];
  }
  if (host) {
    CK(cudaMemsetAsync(ctx->ph, 0, ctx->n_spec * sizeof(float2), s));
    CK(cudaMemsetAsync(ctx->W, 0, ctx->n_spec * sizeof(float2), s));
  }
  if (bad > 0.0) {
    ctx->have_data = false;
    return fail(ctx, BPS_EINVAL, "invalid survey data: R < 0 or non-finite, a count outside 0..65535, or a count > 0 where R = 0");
  }
  for (int l = 0; l < ctx->n_sub; ++l)
    if (!(no[l] > 0.0)) return fail(ctx, BPS_EINVAL, "a subsample has no observed voxel (R > 0)");
  bps_status st = ds_write_bytes(ctx, DS_OFF(sumR), sR.data(), ctx->n_sub * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(sumB), sB.data(), ctx->n_sub * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(nobs), no.data(), ctx->n_sub * sizeof(double));
  if (st != BPS_OK) return st;
  ctx->have_data = true;
  st = rebuild(ctx);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(s));
  return BPS_OK;
}

bps_status bps_set_data(bps_ctx* ctx, const int32_t* counts_dev, const float* R_dev) {
  return set_data_impl(ctx, counts_dev, R_dev, false);
}

bps_status bps_set_data_host(bps_ctx* ctx, const int32_t* counts, const float* R) {
  return set_data_impl(ctx, counts, R, true);
}

bps_status bps_set_state(bps_ctx* ctx, const float* delta_dev, const double* P, const double* b, const double* nbar,
                         uint64_t iteration) {
  if (!ctx || !P || !b || !nbar) return fail(ctx, BPS_EINVAL, "null argument");
  const int nb = ctx->cfg.n_bins;
  for (int m = 0; m < nb; ++m)
    if (!(P[m] > 0.0) || !std::isfinite(P[m])) return fail(ctx, BPS_EINVAL, "P must be positive and finite");
  for (int l = 0; l < ctx->n_sub; ++l)
    if (!std::isfinite(b[l]) || !(nbar[l] > 0.0) || !std::isfinite(nbar[l]))
      return fail(ctx, BPS_EINVAL, "b must be finite and nbar positive");
  bps_status st = ds_write_bytes(ctx, DS_OFF(P), P, nb * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(P_ref), P, nb * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(b), b, ctx->n_sub * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(nbar), nbar, ctx->n_sub * sizeof(double));
  unsigned long long it = iteration;
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(iteration), &it, sizeof(it));
  if (st != BPS_OK) return st;
  Fields f = fields(ctx);
  if (delta_dev) {
    ctx->pt.z_r2c(f, delta_dev, ctx->W, ctx->stream);
    ctx->pt.y_fwd(f, BUF_W, ctx->stream);
    ctx->pt.x_fwd(f, BUF_W, nullptr, ctx->stream);
    LAUNCHED(ctx, 3);
    int cur = current_buffer(ctx, &st);
    if (st != BPS_OK) return st;
    launch_zero_dc(ctx->dh[cur], ctx->stream);
    LAUNCHED(ctx, 1);
  }
  if (ctx->have_data) {
    st = rebuild(ctx);
    if (st != BPS_OK) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_get_state(bps_ctx* ctx, float* delta_dev, double* P, double* b, double* nbar, uint64_t* iteration) {
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  bps_status st = BPS_OK;
  if (delta_dev) {
    Fields f = fields(ctx);
    ctx->pt.x_inv(f, -1, ctx->W, ctx->stream);
    ctx->pt.y_inv(f, BUF_W, ctx->stream);
    ctx->pt.z_c2r(f, ctx->W, delta_dev, ctx->stream);
    LAUNCHED(ctx, 3);
  }
  if (P) st = ds_read_bytes(ctx, DS_OFF(P), P, ctx->cfg.n_bins * sizeof(double));
  if (st == BPS_OK && b) st = ds_read_bytes(ctx, DS_OFF(b), b, ctx->n_sub * sizeof(double));
  if (st == BPS_OK && nbar) st = ds_read_bytes(ctx, DS_OFF(nbar), nbar, ctx->n_sub * sizeof(double));
  if (st == BPS_OK && iteration) {
    unsigned long long it = 0;
    st = ds_read_bytes(ctx, DS_OFF(iteration), &it, sizeof(it));
    *iteration = it;
  }
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_get_spectrum(bps_ctx* ctx, float* spec_dev) {
  if (!ctx || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument");
  bps_status st;
  int cur = current_buffer(ctx, &st);
  if (st != BPS_OK) return st;
  st = copy_spec_out(ctx, ctx->dh[cur], spec_dev);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_set_spectrum(bps_ctx* ctx, const float* spec_dev) {
  if (!ctx || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument");
  bps_status st;
  int cur = current_buffer(ctx, &st);
  if (st != BPS_OK) return st;
  st = copy_spec_in(ctx, spec_dev, ctx->dh[cur]);
  if (st != BPS_OK) return st;
  launch_zero_dc(ctx->dh[cur], ctx->stream);
  LAUNCHED(ctx, 1);
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_hmc_step(bps_ctx* ctx, bps_move_info* info) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = hmc_move(ctx, true);
  if (st != BPS_OK) return st;
  if (info) {
    int acc = 0;
    double dH = 0, eps = 0;
    st = ds_read_bytes(ctx, DS_OFF(accepted), &acc, sizeof(int));
    if (st == BPS_OK) st = ds_read_bytes(ctx, DS_OFF(dH), &dH, sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, DS_OFF(eps), &eps, sizeof(double));
    if (st != BPS_OK) return st;
    info->accepted = acc;
    info->dH = dH;
    info->eps = eps;
    return check_status(ctx);
  }
  return BPS_OK;
}

bps_status bps_sample_power(bps_ctx* ctx, double* P_out, double* sigma_out) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = power_stage(ctx, true, true);
  if (st != BPS_OK) return st;
  if (P_out) st = ds_read_bytes(ctx, DS_OFF(P), P_out, ctx->cfg.n_bins * sizeof(double));
  if (st == BPS_OK && sigma_out) st = ds_read_bytes(ctx, DS_OFF(sigma), sigma_out, ctx->cfg.n_bins * sizeof(double));
  if (st != BPS_OK) return st;
  if (P_out || sigma_out) return check_status(ctx);
  return BPS_OK;
}

bps_status bps_sample_bias_norm(bps_ctx* ctx, double* b_out, double* nbar_out, double* sums_out) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = bias_stage(ctx, true);
  if (st != BPS_OK) return st;
  if (b_out) st = ds_read_bytes(ctx, DS_OFF(b), b_out, ctx->n_sub * sizeof(double));
  if (st == BPS_OK && nbar_out) st = ds_read_bytes(ctx, DS_OFF(nbar), nbar_out, ctx->n_sub * sizeof(double));
  if (st == BPS_OK && sums_out) {
    std::vector<double> tmp(3 * MAXS);
    st = ds_read_bytes(ctx, DS_OFF(sums), tmp.data(), tmp.size() * sizeof(double));
    for (int i = 0; i < 3 * ctx->n_sub; ++i) sums_out[i] = tmp[i];
  }
  if (st != BPS_OK) return st;
  if (b_out || nbar_out || sums_out) return check_status(ctx);
  return BPS_OK;
}

bps_status bps_jump(bps_ctx* ctx, bps_move_info* info) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (ctx->cfg.jump_leapfrog < 1 || !(ctx->cfg.jump_eps_max > 0.0))
    return fail(ctx, BPS_EINVAL, "jump settings are not set");
  st = jump_stage(ctx, true);
  if (st != BPS_OK) return st;
  if (info) {
    int acc = 0;
    double dH = 0, eps = 0;
    st = ds_read_bytes(ctx, DS_OFF(jaccepted), &acc, sizeof(int));
    if (st == BPS_OK) st = ds_read_bytes(ctx, DS_OFF(jdH), &dH, sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, DS_OFF(jeps), &eps, sizeof(double));
    if (st != BPS_OK) return st;
    info->accepted = acc;
    info->dH = dH;
    info->eps = eps;
    return check_status(ctx);
  }
  return BPS_OK;
}

bps_status bps_gibbs_iterate(bps_ctx* ctx, int n_iter, double* chain_out) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (n_iter < 0) return fail(ctx, BPS_EINVAL, "n_iter must be >= 0");
  const int rec = ctx->cfg.n_bins + 2 * ctx->n_sub + 2;
  if (chain_out && n_iter > ctx->chain_cap) {
    cudaFree(ctx->chain_dev);
    ctx->chain_dev = nullptr;
    ctx->chain_cap = 0;
    if (cudaMalloc((void**)&ctx->chain_dev, (size_t)n_iter * rec * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BPS_ENOMEM, "chain buffer allocation failed");
    }
    ctx->chain_cap = n_iter;
  }
  ScalarArgs sa = scalars(ctx);
  for (int i = 0; i < n_iter; ++i) {
    st = hmc_move(ctx, false);
    if (st == BPS_OK) st = power_stage(ctx, true, false);
    if (st == BPS_OK && ctx->cfg.jump) st = jump_stage(ctx, false);
    if (st == BPS_OK) st = bias_stage(ctx, false);
    if (st != BPS_OK) return st;
    if (chain_out) {
      launch_record(sa, ctx->chain_dev + (size_t)i * rec, ctx->stream);
      LAUNCHED(ctx, 1);
    }
    launch_advance(ctx->ds, ctx->stream);
    LAUNCHED(ctx, 1);
  }
  if (chain_out && n_iter > 0) {
    CK(cudaMemcpyAsync(chain_out, ctx->chain_dev, (size_t)n_iter * rec * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

bps_status bps_set_mass_scale(bps_ctx* ctx, int n_mass_bins, const double* scales) {
  if (!ctx || !scales) return fail(ctx, BPS_EINVAL, "null argument");
  if (n_mass_bins < 1 || n_mass_bins > MAXB) return fail(ctx, BPS_EINVAL, "n_mass_bins must be in 1..64");
  for (int j = 0; j < n_mass_bins; ++j)
    if (!(scales[j] > 0.0) || !std::isfinite(scales[j])) return fail(ctx, BPS_EINVAL, "scales must be positive");
  int thr[MAXB];
  if (!bin_tables(ctx->N, n_mass_bins, thr, nullptr))
    return fail(ctx, BPS_EINVAL, "a mass bin holds no |n|^2 value; use fewer mass bins");
  bps_status st = ds_write_bytes(ctx, DS_OFF(mthr), thr, sizeof(thr));
  if (st == BPS_OK) st = ds_write_bytes(ctx, DS_OFF(mass_scale), scales, n_mass_bins * sizeof(double));
  if (st != BPS_OK) return st;
  ctx->n_mass = n_mass_bins;
  return BPS_OK;
}

bps_status bps_fft_r2c(bps_ctx* ctx, const float* real_dev, float* spec_dev) {
  if (!ctx || !real_dev || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument");
  Fields f = fields(ctx);
  ctx->pt.z_r2c(f, real_dev, ctx->W, ctx->stream);
  ctx->pt.y_fwd(f, BUF_W, ctx->stream);
  ctx->pt.x_fwd(f, BUF_W, ctx->W, ctx->stream);
  LAUNCHED(ctx, 3);
  bps_status st = copy_spec_out(ctx, ctx->W, spec_dev);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_fft_c2r(bps_ctx* ctx, const float* spec_dev, float* real_dev) {
  if (!ctx || !real_dev || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument");
  bps_status st = copy_spec_in(ctx, spec_dev, ctx->W);
  if (st != BPS_OK) return st;
  Fields f = fields(ctx);
  ctx->pt.x_inv(f, BUF_W, ctx->W, ctx->stream);
  ctx->pt.y_inv(f, BUF_W, ctx->stream);
  ctx->pt.z_c2r(f, ctx->W, real_dev, ctx->stream);
  LAUNCHED(ctx, 3);
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_gradient(bps_ctx* ctx, float* grad_dev, double* energies) {
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (!grad_dev) return fail(ctx, BPS_EINVAL, "null argument");
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  launch_move_begin(sa, s);   // per-bin tables of the current P and abar
  ctx->pt.x_inv(f, -1, ctx->W, s);
  ctx->pt.y_inv(f, BUF_W, s);
  ctx->pt.z_grad(f, region_offset(ctx, RG_LIK0), s);
  ctx->pt.y_fwd(f, BUF_W, s);
  ctx->pt.x_grad(f, ctx->W, region_offset(ctx, RG_GRAD), s);
  launch_reduce_to(sa, region_offset(ctx, RG_GRAD), ctx->pt.x_tiles, 1, 0.5 / (double)ctx->nv,
                   reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->ds) + DS_OFF(scratch)), s);
  launch_reduce_to(sa, region_offset(ctx, RG_LIK0), ctx->pt.z_tiles, 1, 1.0,
                   reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->ds) + DS_OFF(scratch)) + 1, s);
  LAUNCHED(ctx, 8);
  st = copy_spec_out(ctx, ctx->W, grad_dev);
  if (st != BPS_OK) return st;
  if (energies) {
    st = ds_read_bytes(ctx, DS_OFF(scratch), energies, 2 * sizeof(double));
    if (st != BPS_OK) return st;
  }
  CK(cudaStreamSynchronize(s));
  return BPS_OK;
}

bps_status bps_philox_words(uint64_t seed, uint64_t iteration, uint64_t stage, uint64_t sub, uint64_t block0,
                            size_t n_words, uint64_t* out_dev, void* cuda_stream) {
  if (!out_dev) return fail(nullptr, BPS_EINVAL, "null argument");
  if (n_words == 0) return BPS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  launch_philox_words(seed, iteration, stage, sub, block0, n_words, out_dev, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, BPS_ECUDA, cudaGetErrorString(e));
  return BPS_OK;
}

bps_status bps_voxel_normals(uint64_t seed, uint64_t iteration, size_t n, float* out_dev, void* cuda_stream) {
  if (!out_dev) return fail(nullptr, BPS_EINVAL, "null argument");
  if (n == 0) return BPS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  launch_voxel_normals(seed, iteration, n, out_dev, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, BPS_ECUDA, cudaGetErrorString(e));
  return BPS_OK;
}

}  // extern "C"
