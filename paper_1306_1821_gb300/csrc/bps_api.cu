// Host side of the bps C ABI: context life cycle, data and state transfer, and
// the launch sequences of the sampler's stages (the ABI is declared and
// documented in include/bps.h).
//
// A context is a group of `batch` chains on one grid size: every chain has its
// own buffers at fixed strides in shared arenas and its own DevState, and each
// field pass or scalar stage is one launch over all chains (gridDim.y).  A
// single-chain context is a group of one.  A batch context (bps_create_batch)
// owns one group per distinct grid size.
#include <algorithm>
#include <bitset>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <nvtx3/nvToolsExt.h>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <unistd.h>

#include "bps_internal.h"
#include "bps_passes.cuh"

using namespace bps;

struct bps_ctx {
  // ---- batch of groups (bps_create_batch) ----
  bool is_batch = false;
  std::vector<bps_ctx*> groups;
  std::vector<std::pair<int, int>> chain_map;   // chain -> (group, index in group)
  int rec_len_all = 0;
  // ---- group of chains on one grid ----
  int N = 0, batch = 1, max_sub = 0, zp = 0;
  std::vector<int> nsub;                        // per chain
  std::vector<double> box;                      // per chain
  std::vector<int> chain_id;                    // per chain: slot in the batch record
  bps_config cfg{};
  cudaStream_t stream = nullptr;
  PassTable pt{};
  long long nv = 0;
  size_t n_spec = 0;          // complex elements of one padded half spectrum
  float2* dh[2] = {nullptr, nullptr};
  float2* ph = nullptr;
  float2* W = nullptr;
  float2* acc = nullptr;      // running sum of the state (bps_mass_stats), allocated on first use
  float* a = nullptr;
  float* c = nullptr;
  int2* span = nullptr;         // per-line support of a and c (grids with N % 32 == 0)
  uint16_t* cnt = nullptr;
  float* R = nullptr;
  float2* tw = nullptr;
  double* part = nullptr;
  int part_stride = 0;
  long long part_cstride = 0;
  DevState* ds = nullptr;
  double* chain_dev = nullptr;
  int chain_cap = 0;
  double* host_buf = nullptr;   // pinned staging for small reads
  int n_mass = 0;
  // the force z pass in use (line pairs per tile chosen by the autotuner) and
  // the number of likelihood-energy partials it writes
  void (*zgrad)(const Fields&, int region, int nch, cudaStream_t) = nullptr;
  int zgrad_tiles = 0;
  int zgrad_pairs = 8;
  YzEntry yz{};                 // fused y^-1 / z / y stage (run == nullptr: three passes)
  // leapfrog x pass with tensor-copy staged tiles (nullptr: the direct-load pass)
  XLeapTma xleap = nullptr;
  XMaps xmaps{};
  MassNet* mnet = nullptr;      // network mass (bps_set_mass_net): scales recomputed before every move
  std::vector<char> have_data;
  int rebuild_blocks = 0;
  int n_sm = 0;
  uint64_t launches = 0;
  uint8_t* pbin = nullptr;   // k bin of every half-spectrum mode (Fields::pbin)
  // CUDA graph of one Gibbs iteration (captured on first use)
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream the graph is captured on
  // host upload of survey data (bps_set_data_host): two device staging slots of
  // one subsample's counts and response, filled on a copy stream while the
  // data kernel of the previous subsample runs (allocated on first use)
  char* stage = nullptr;
  cudaStream_t copy_stream[2] = {nullptr, nullptr};   // counts, response: two copies in flight
  cudaEvent_t stage_copied[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t stage_free[2] = {nullptr, nullptr};
  // staged surveys (bps_stage_data_host_u16): each chain has two data slots;
  // an upload fills the slot after the last one used, on up_stream, and waits
  // (FIFO, at most two) until an operation that uses the data activates it
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_after_main = nullptr;     // orders an upload after earlier work on the main stream
  std::vector<cudaEvent_t> slot_ready;     // [chain][slot]: the upload into that slot is complete
  std::vector<std::vector<int>> pending;   // per chain: staged slots, oldest first
  std::vector<int> next_slot;              // per chain: the slot the next upload fills
  double* dpart = nullptr;                 // data-kernel partials [slot][chain][MAXS][4][blocks]
  long long dpart_cstride = 0;
  bool graph_jump = false;
  uint64_t graph_launches = 0;   // kernels in one replay of the graph
  // leapfrog kernel timing (bps_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev[4];
  size_t ev_used[4] = {0, 0, 0, 0};
  // the iteration captured with event-record nodes around the leapfrog
  // kernels: profiled iterations replay it instead of launching one by one
  cudaGraphExec_t prof_graph = nullptr;
  bool prof_graph_jump = false;
  uint64_t prof_graph_launches = 0;
  size_t prof_graph_events[4] = {0, 0, 0, 0};
  bool capturing = false;
  double prof_ms[4] = {0, 0, 0, 0};
  uint64_t prof_n[4] = {0, 0, 0, 0};
  // running posterior moments (bps_posterior_moments): per-voxel sums of delta
  // and delta^2 [2 N^3], and of the chain parameters [1 + D + D^2], D = n_bins + 2 n_sub
  bool mom_on = false;
  double* mom = nullptr;
  double* pmom = nullptr;
  // device table of the mock calls (amplitudes, selection), grown on demand
  void* mock_buf = nullptr;
  size_t mock_bytes = 0;
  std::string err;
};

namespace bps {

// ------------------------------------------------------------------ k bins (one definition, shared)
// bin of integer |n|^2 for n_bins linear bins over (0, sqrt(3) N / 2]
int bin_of_host(long long n2, int N, int nb) {
  double b = std::floor((double)nb * std::sqrt((double)n2) / (std::sqrt(3.0) * (double)N / 2.0));
  int m = (int)b;
  return m > nb - 1 ? nb - 1 : m;
}

// thresholds (smallest n2 of each bin) and, when nmodes is given, the full-grid
// mode counts; false if a bin has no threshold or (with nmodes) no mode
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


// true when every bin [thr[m], thr[m+1]) holds at least one integer wave vector
// of the grid, |n_x|, |n_y|, |n_z| <= N/2 (N <= 512).  Cheaper than counting the
// modes: a bitmap of the values n_x^2 + n_y^2, then for each bin the first
// |n|^2 of its range that is such a value plus some n_z^2.  A bin can have
// thresholds and still no mode (every |n|^2 in it of the form 4^a (8b + 7)).
bool bins_have_modes(int N, int nb, const int* thr) {
  constexpr int HMAX = 256;
  const int H = N / 2;
  if (H > HMAX || H < 1) return false;
  std::bitset<2 * HMAX * HMAX + 1> two;   // 16 KB on the stack, nothing allocated
  for (int x = 0; x <= H; ++x)
    for (int y = x; y <= H; ++y) two.set((size_t)(x * x + y * y));
  const long long maxn2 = 3LL * H * H;
  for (int m = 0; m < nb; ++m) {
    const long long lo = m == 0 ? 1 : thr[m];
    const long long hi = m + 1 < nb ? thr[m + 1] : maxn2 + 1;
    bool found = false;
    for (long long n2 = lo; n2 < hi && !found; ++n2)
      for (int z = 0; z <= H && (long long)z * z <= n2 && !found; ++z) {
        const long long r = n2 - (long long)z * z;
        if (r <= 2LL * H * H && two.test((size_t)r)) found = true;
      }
    if (!found) return false;
  }
  return true;
}

}  // namespace bps

namespace {

// the last error message of the calling thread (each thread reads only its own)
thread_local std::string g_err;

// A named NVTX range over a public call or a set-up phase: a profiler's timeline
// shows it around the call's host work and launches; without a tool attached
// the push and pop do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// partial-sum regions (offsets in doubles into one chain's part of ctx->part)
enum Region { RG_INIT = 0, RG_LIK0, RG_FINAL, RG_LIK1, RG_BIN, RG_SUMS, RG_RB, RG_JGRAD, RG_JLIK, RG_GRAD, RG_COUNT };
int region_width(Region r) {
  switch (r) {
    case RG_INIT: case RG_FINAL: return 3;   // kinetic, prior, g^T M^-1 g
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
  f.acc = c->acc;
  f.a = c->a;
  f.c = c->c;
  f.cnt = c->cnt;
  f.R = c->R;
  f.span = c->span;
  f.span_stride = (long long)c->N * c->N;
  f.data_slot = (long long)c->max_sub * c->nv * c->batch;
  f.span_slot = (long long)c->N * c->N * c->batch;
  f.n_sub = c->max_sub;
  f.ds = c->ds;
  f.part = c->part;
  f.part_stride = c->part_stride;
  f.tw = c->tw;
  f.pbin = c->pbin;
  f.grid_n = c->N;
  f.inv_nv = (float)(1.0 / (double)c->nv);
  f.mass_mode = (c->cfg.mass_mode != 0 || c->mnet) ? 1 : 0;
  f.n_bins = c->cfg.n_bins;
  f.n_mass = c->n_mass;
  f.n_sm = c->n_sm;
  f.spec_stride = (long long)c->n_spec;
  f.real_stride = c->nv;
  f.data_stride = (long long)c->max_sub * c->nv;
  f.part_cstride = c->part_cstride;
  return f;
}

Fields fields_at(bps_ctx* c, int ch) { return at_chain(fields(c), ch); }

ScalarArgs scalars(bps_ctx* c) {
  ScalarArgs a;
  a.ds = c->ds;
  a.part = c->part;
  a.stride = c->part_stride;
  a.cstride = c->part_cstride;
  a.n_bins = c->cfg.n_bins;
  a.max_sub = c->max_sub;
  a.n_mass = c->n_mass;
  a.inv_nv = 1.0 / (double)c->nv;
  a.alpha = c->cfg.alpha;
  a.eps_max = c->cfg.eps_max;
  a.jeps_max = c->cfg.jump_eps_max;
  a.fixed_bias = c->cfg.fixed_bias_index;
  return a;
}

ScalarArgs scalars_at(bps_ctx* c, int ch) {
  ScalarArgs a = scalars(c);
  a.ds += ch;
  a.part += ch * a.cstride;
  return a;
}

#define DS_OFF(member) offsetof(DevState, member)

char* ds_addr(bps_ctx* ctx, int ch, size_t off) { return reinterpret_cast<char*>(ctx->ds + ch) + off; }

bps_status ds_write_bytes(bps_ctx* ctx, int ch, size_t off, const void* src, size_t n) {
  CK(cudaMemcpyAsync(ds_addr(ctx, ch, off), src, n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status ds_read_bytes(bps_ctx* ctx, int ch, size_t off, void* dst, size_t n) {
  CK(cudaMemcpyAsync(ctx->host_buf, ds_addr(ctx, ch, off), n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(dst, ctx->host_buf, n);
  return BPS_OK;
}

// status words of all chains; cleared after reading
bps_status check_status(bps_ctx* ctx) {
  int any = 0;
  for (int ch = 0; ch < ctx->batch; ++ch) {
    int st = 0;
    bps_status s = ds_read_bytes(ctx, ch, DS_OFF(status), &st, sizeof(int));
    if (s != BPS_OK) return s;
    if (st != 0) {
      int zero = 0;
      ds_write_bytes(ctx, ch, DS_OFF(status), &zero, sizeof(int));
      any |= st;
      if (st & ST_BADDATA) {
        // a chain whose surveys were all invalid has none: only a valid commit
        // writes the observed-voxel counts
        double nobs0 = 0.0;
        if (ds_read_bytes(ctx, ch, DS_OFF(nobs), &nobs0, sizeof(double)) == BPS_OK && !(nobs0 > 0.0))
          ctx->have_data[ch] = 0;
      }
    }
  }
  if (any & ST_BADDATA)
    return fail(ctx, BPS_EINVAL,
                "invalid survey data (R < 0 or non-finite, a count outside 0..65535, a count > 0 where R = 0, "
                "or a subsample without observed voxels); the previous survey stays active");
  if (any & ST_TIMEOUT) return fail(ctx, BPS_ETIMEOUT, "a tile copy did not complete within the wait limit");
  if (any & ST_NONFINITE) return fail(ctx, BPS_ENUMERIC, "non-finite energy difference; move rejected");
  if (any) return fail(ctx, BPS_ENUMERIC, "a scalar draw failed (no acceptance within the attempt bound or a non-positive sum)");
  return BPS_OK;
}

// ------------------------------------------------------------------ profiling
constexpr size_t PROF_CAP = 8192;   // event pairs per kernel kind before folding

void prof_fold(bps_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < 4; ++k) {
    for (size_t i = 0; i + 1 < ctx->ev_used[k]; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev[k][i], ctx->ev[k][i + 1]) == cudaSuccess) {
        ctx->prof_ms[k] += ms;
        ctx->prof_n[k] += 1;
      } else {
        cudaGetLastError();   // a pair without a time is left out
      }
    }
    ctx->ev_used[k] = 0;
  }
}

// record one event of kernel kind k (start or end); no-op unless profiling.
// Under stream capture the record becomes an event-record node of the graph
// (the events were created beforehand, see capture_iteration).
void prof_mark(bps_ctx* ctx, int k) {
  if (!ctx->prof) return;
  if (ctx->capturing) {
    if (ctx->ev_used[k] < ctx->ev[k].size())
      cudaEventRecordWithFlags(ctx->ev[k][ctx->ev_used[k]++], ctx->stream, cudaEventRecordExternal);
    return;
  }
  if (ctx->ev_used[k] >= PROF_CAP && ctx->ev_used[k] % 2 == 0) prof_fold(ctx);
  if (ctx->ev_used[k] == ctx->ev[k].size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ctx->ev[k].push_back(e);
  }
  cudaEventRecord(ctx->ev[k][ctx->ev_used[k]++], ctx->stream);
}

// ------------------------------------------------------------------ stages (all chains of a group)
bps_status rebuild_chain(bps_ctx* ctx, int ch) {
  launch_rebuild(fields_at(ctx, ch), ctx->nv, region_offset(ctx, RG_RB), ctx->rebuild_blocks, 1, ctx->stream);
  launch_abar(scalars_at(ctx, ch), region_offset(ctx, RG_RB), ctx->rebuild_blocks, 1, ctx->stream);
  LAUNCHED(ctx, 2);
  return BPS_OK;
}

bps_status rebuild_all(bps_ctx* ctx) {
  launch_rebuild(fields(ctx), ctx->nv, region_offset(ctx, RG_RB), ctx->rebuild_blocks, ctx->batch, ctx->stream);
  launch_abar(scalars(ctx), region_offset(ctx, RG_RB), ctx->rebuild_blocks, ctx->batch, ctx->stream);
  LAUNCHED(ctx, 2);
  return BPS_OK;
}

// Likelihood-energy partials written by one force stage.
int lik_tiles(const bps_ctx* ctx) { return ctx->yz.run ? ctx->yz.tiles : ctx->zgrad_tiles; }

// The y^-1 / z / y stage of one force evaluation (C2R, local force
// g = a delta - c and its energy partials into `region` when >= 0, R2C): the
// fused plane kernel where the grid has one, else the three passes.
// Profiling kind 2 times the fused kernel; kinds 1 and 3 the y passes.
bps_status force_stage(bps_ctx* ctx, const Fields& f, int region, bool prof, cudaStream_t s) {
  const PassTable& P = ctx->pt;
  const int B = ctx->batch;
  if (ctx->yz.run) {
    if (prof) prof_mark(ctx, 2);
    ctx->yz.run(f, region, B, s);
    if (prof) prof_mark(ctx, 2);
    LAUNCHED(ctx, 1);
    return BPS_OK;
  }
  if (prof) prof_mark(ctx, 1);
  P.y_inv(f, BUF_W, B, s);
  if (prof) prof_mark(ctx, 1);
  if (prof) prof_mark(ctx, 2);
  ctx->zgrad(f, region, B, s);
  if (prof) prof_mark(ctx, 2);
  if (prof) prof_mark(ctx, 3);
  P.y_fwd(f, BUF_W, B, s);
  if (prof) prof_mark(ctx, 3);
  LAUNCHED(ctx, 3);
  return BPS_OK;
}

bps_status hmc_move(bps_ctx* ctx, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const PassTable& P = ctx->pt;
  const int L = ctx->cfg.n_leapfrog, B = ctx->batch;
  if (ctx->mnet) launch_mass_net(sa, ctx->mnet, B, s);
  launch_move_begin(sa, B, s);
  P.z_noise(f, B, s);
  P.y_fwd(f, BUF_PH, B, s);
  P.x_init(f, region_offset(ctx, RG_INIT), B, s);
  bps_status sf = force_stage(ctx, f, region_offset(ctx, RG_LIK0), false, s);
  if (sf != BPS_OK) return sf;
  for (int st = 1; st <= L; ++st) {
    prof_mark(ctx, 0);
    if (st == 1) P.x_leapg(f, region_offset(ctx, RG_INIT) + 2 * ctx->part_stride, B, s);
    else if (ctx->xleap) ctx->xleap(f, ctx->xmaps, 0, B, s);
    else P.x_leap(f, 0, B, s);
    prof_mark(ctx, 0);
    sf = force_stage(ctx, f, st == L ? region_offset(ctx, RG_LIK1) : -1, true, s);
    if (sf != BPS_OK) return sf;
  }
  P.x_final(f, region_offset(ctx, RG_FINAL), B, s);
  launch_move_end(sa, region_offset(ctx, RG_INIT), region_offset(ctx, RG_LIK0), region_offset(ctx, RG_FINAL),
                  region_offset(ctx, RG_LIK1), P.x_tiles, lik_tiles(ctx), B, s);
  int n = 7 + L + (ctx->mnet ? 1 : 0);   // launch_move_end is two kernels
  if (advance) {
    launch_advance(ctx->ds, B, s);
    ++n;
  }
  LAUNCHED(ctx, n);
  return BPS_OK;
}

bps_status power_stage(bps_ctx* ctx, bool draw, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  const int B = ctx->batch;
  ctx->pt.x_binpow(f, region_offset(ctx, RG_BIN), B, ctx->stream);
  launch_power(sa, region_offset(ctx, RG_BIN), ctx->pt.x_tiles, draw ? 1 : 0, B, ctx->stream);
  int n = 2;
  if (advance) {
    launch_advance(ctx->ds, B, ctx->stream);
    ++n;
  }
  LAUNCHED(ctx, n);
  return BPS_OK;
}

bps_status bias_stage(bps_ctx* ctx, bool advance) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const int B = ctx->batch;
  // delta = C2R(delta_hat) (x and y inverse into W), the per-subsample sums in the z pass
  ctx->pt.x_inv(f, -1, nullptr, B, s);
  ctx->pt.y_inv(f, BUF_W, B, s);
  ctx->pt.z_sums(f, region_offset(ctx, RG_SUMS), B, s);
  launch_bias_nbar(sa, region_offset(ctx, RG_SUMS), ctx->pt.z_tiles, B, s);
  LAUNCHED(ctx, 4);
  bps_status st = rebuild_all(ctx);
  if (st != BPS_OK) return st;
  if (advance) {
    launch_advance(ctx->ds, B, s);
    LAUNCHED(ctx, 1);
  }
  return BPS_OK;
}

// force evaluation of the jump at the current theta (scales js on the device)
// One gradient evaluation of the jump's HMC at the current theta, followed by
// the leapfrog update of `kind` (the reduction and the update share a launch).
bps_status jump_gradient(bps_ctx* ctx, int kind) {
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const PassTable& P = ctx->pt;
  const int B = ctx->batch;
  P.x_jinv(f, B, s);
  // the likelihood energy enters only the Hamiltonian at the two ends of the
  // trajectory: a middle step's force stage skips its energy sums
  bps_status sf = force_stage(ctx, f, kind == J_MID ? -1 : region_offset(ctx, RG_JLIK), false, s);
  if (sf != BPS_OK) return sf;
  P.x_jgrad(f, region_offset(ctx, RG_JGRAD), B, s);
  launch_jump_step(sa, region_offset(ctx, RG_JGRAD), P.x_tiles, region_offset(ctx, RG_JLIK),
                   region_offset(ctx, RG_LIK1), lik_tiles(ctx), kind, B, s);
  LAUNCHED(ctx, 3);
  return BPS_OK;
}

// sigma_current: DevState::sigma already holds the k-bin power of the current
// field (the power draw of the same Gibbs iteration computed it, and the field
// has not moved since), so the jump's mass needs no second reduction.
bps_status jump_stage(bps_ctx* ctx, bool advance, bool sigma_current = false) {
  ScalarArgs sa = scalars(ctx);
  cudaStream_t s = ctx->stream;
  const int B = ctx->batch;
  bps_status st = BPS_OK;
  if (!sigma_current) st = power_stage(ctx, false, false);   // sigma of the current field (mass of the jump)
  if (st != BPS_OK) return st;
  // inside the Gibbs scan the jump follows the HMC move and the power draw, which
  // leave W and the likelihood partials of the move's last force evaluation
  launch_jump_begin(sa, sigma_current ? 1 : 0, B, s);
  LAUNCHED(ctx, 1);
  const int L = ctx->cfg.jump_leapfrog;
  st = jump_gradient(ctx, J_FIRST);
  if (st != BPS_OK) return st;
  for (int k = 0; k < L; ++k) {
    st = jump_gradient(ctx, k == L - 1 ? J_LAST : J_MID);
    if (st != BPS_OK) return st;
  }
  Fields f = fields(ctx);
  ctx->pt.x_scale(f, B, s);   // delta_k <- sqrt(P'/P) delta_k if accepted (Eq. det_trans)
  LAUNCHED(ctx, 1);
  if (advance) {
    launch_advance(ctx->ds, B, s);
    LAUNCHED(ctx, 1);
  }
  return BPS_OK;
}

// One Gibbs iteration of every chain of the group, recording each chain's
// sample into `rec` (slot DevState::rec_idx, layout [slot][chain][rec_len]).
bps_status gibbs_once(bps_ctx* ctx, double* rec, int rec_len, long long iter_stride, bool jump) {
  bps_status st = hmc_move(ctx, false);
  if (st == BPS_OK) st = power_stage(ctx, true, false);
  if (st == BPS_OK && jump) st = jump_stage(ctx, false, true);
  if (st == BPS_OK) st = bias_stage(ctx, false);
  if (st != BPS_OK) return st;
  if (ctx->mom_on) {
    // running posterior moments of this iteration's sample: W holds the x and y
    // inverse transforms of the field (bias stage), so one z pass gives delta
    ctx->pt.z_mom(fields_at(ctx, 0), ctx->mom, ctx->stream);
    launch_param_moments(scalars_at(ctx, 0), ctx->pmom, ctx->stream);
    LAUNCHED(ctx, 2);
  }
  launch_record(scalars(ctx), rec, rec_len, iter_stride, ctx->chain_id.empty() ? 0 : ctx->chain_id[0], ctx->batch,
                ctx->stream);
  launch_advance(ctx->ds, ctx->batch, ctx->stream);
  LAUNCHED(ctx, 2);
  return BPS_OK;
}

bps_status commit_data(bps_ctx* ctx, int ch);

// Activates the oldest staged survey of each chain, then requires data.
bps_status need_data(bps_ctx* ctx) {
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  if (ctx->is_batch) return fail(ctx, BPS_EINVAL, "a batch context takes the bps_batch_* calls");
  for (int ch = 0; ch < ctx->batch; ++ch) {
    bps_status st = commit_data(ctx, ch);
    if (st != BPS_OK) return st;
    if (!ctx->have_data[ch]) return fail(ctx, BPS_ESTATE, "bps_set_data has not been called");
  }
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

int current_buffer(bps_ctx* ctx, int ch, bps_status* st) {
  int cur = 0;
  *st = ds_read_bytes(ctx, ch, DS_OFF(cur), &cur, sizeof(int));
  return cur;
}

float2* state_buffer(bps_ctx* ctx, int ch, int cur) { return ctx->dh[cur] + (size_t)ch * ctx->n_spec; }

void drop_graph(bps_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->prof_graph) cudaGraphExecDestroy(c->prof_graph);
  c->graph = nullptr;
  c->prof_graph = nullptr;
}

void free_streams(bps_ctx* c) {
  // staged uploads may still be writing the data slots
  if (c->up_stream) cudaStreamSynchronize(c->up_stream);
  for (int i = 0; i < 2; ++i)
    if (c->copy_stream[i]) cudaStreamSynchronize(c->copy_stream[i]);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (int i = 0; i < 2; ++i) {
    if (c->copy_stream[i]) cudaStreamDestroy(c->copy_stream[i]);
    c->copy_stream[i] = nullptr;
    for (int k = 0; k < 2; ++k) {
      if (c->stage_copied[i][k]) cudaEventDestroy(c->stage_copied[i][k]);
      c->stage_copied[i][k] = nullptr;
    }
    if (c->stage_free[i]) cudaEventDestroy(c->stage_free[i]);
    c->stage_free[i] = nullptr;
  }
  cudaFree(c->stage);
  c->stage = nullptr;
  if (c->up_stream) cudaStreamDestroy(c->up_stream);
  c->up_stream = nullptr;
  if (c->up_after_main) cudaEventDestroy(c->up_after_main);
  c->up_after_main = nullptr;
  for (cudaEvent_t& e : c->slot_ready)
    if (e) cudaEventDestroy(e);
  c->slot_ready.clear();
  cudaFree(c->dpart);
  c->dpart = nullptr;
}

void free_all(bps_ctx* c) {
  if (c->mom) cudaFree(c->mom);
  if (c->pmom) cudaFree(c->pmom);
  c->mom = c->pmom = nullptr;
  if (c->mock_buf) cudaFree(c->mock_buf);
  c->mock_buf = nullptr;
  drop_graph(c);
  free_streams(c);
  for (int k = 0; k < 4; ++k)
    for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
  cudaFree(c->dh[0]);
  cudaFree(c->dh[1]);
  cudaFree(c->ph);
  cudaFree(c->W);
  cudaFree(c->acc);
  cudaFree(c->a);
  cudaFree(c->c);
  cudaFree(c->span);
  cudaFree(c->cnt);
  cudaFree(c->R);
  cudaFree(c->tw);
  cudaFree(c->pbin);
  cudaFree(c->part);
  cudaFree(c->ds);
  cudaFree(c->chain_dev);
  massnet_destroy(c->mnet);
  if (c->host_buf) cudaFreeHost(c->host_buf);
}

// ------------------------------------------------------------------ tile autotuner
// The force z pass can run with 4, 8 or 16 line pairs per tile; which is
// fastest depends on the grid and on how many chains share a launch.  The
// first context of a (GPU, N, chains) kind times each candidate on its own
// buffers (before any data is set: W is scratch) and keeps the fastest; the
// choice is cached for the process and in a JSON file (BPS_TUNE_CACHE, else
// $HOME/.cache/bps_tune.json) so later runs reuse it and give the same
// chains.  BPS_AUTOTUNE=0 keeps 8 line pairs.  The choice changes only the
// grouping of the likelihood-energy terms into per-block partial sums
// (compensated FP32 pairs, one FP64 value per block).
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  if (const char* p = std::getenv("BPS_TUNE_CACHE")) return p;
  if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/bps_tune.json";
  return "";
}

// flat JSON object of string keys and integer values
void tune_load() {
  g_tune_loaded = true;
  const std::string path = tune_path();
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
  std::fclose(f);
  size_t i = 0;
  while ((i = txt.find('"', i)) != std::string::npos) {
    const size_t j = txt.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = txt.substr(i + 1, j - i - 1);
    const size_t c = txt.find(':', j);
    if (c == std::string::npos) break;
    g_tune[key] = std::atoi(txt.c_str() + c + 1);
    i = txt.find_first_of(",}", c);
    if (i == std::string::npos) break;
  }
}

void tune_save() {
  const std::string path = tune_path();
  if (path.empty()) return;
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);   // one level; failure is harmless
  const std::string tmp = path + ".tmp." + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{");
  bool first = true;
  for (const auto& kv : g_tune) {
    std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  std::fprintf(f, "\n}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

bps_status choose_zgrad(bps_ctx* ctx) {
  TraceRange trace_("bps autotune: force z tiles");
  int pick = 1;   // 8 line pairs
  const char* e = std::getenv("BPS_AUTOTUNE");
  if (!(e && std::atoi(e) == 0)) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    const std::string key = std::string(prop.name) + " N=" + std::to_string(ctx->N) + " chains=" +
                            std::to_string(ctx->batch) + " zpairs";
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) tune_load();
    auto it = g_tune.find(key);
    int lp = it != g_tune.end() ? it->second : 0;
    if (lp == 4 || lp == 8 || lp == 16) {
      pick = lp == 4 ? 0 : lp == 8 ? 1 : 2;
    } else {
      // The buffers hold no survey yet.  Each tile size is timed twice: on the
      // dense pass (every line transformed, a full-sky survey) and with the line
      // supports of a centred ball of radius 0.45 N (about 64% of the lines,
      // each over its chord), where tiles without support are skipped and small
      // tiles skip more; the smallest total wins.
      cudaStream_t s = ctx->stream;
      const int N = ctx->N, B = ctx->batch;
      std::vector<int2> ball((size_t)N * N * B);
      const double rho = 0.45 * N, mid = 0.5 * N;
      for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
          const double dx = x + 0.5 - mid, dy = y + 0.5 - mid, r2 = dx * dx + dy * dy;
          int2 sp = make_int2(0, 0);   // empty line
          if (r2 < rho * rho) {
            const double h = std::sqrt(rho * rho - r2);
            const int lo = std::max(0, (int)std::floor((mid - h) / 4.0) * 4);
            const int hi = std::min(N, (int)std::ceil((mid + h) / 4.0) * 4);
            sp = make_int2(N - lo, hi);
          }
          for (int ch = 0; ch < B; ++ch) ball[((size_t)ch * N + x) * N + y] = sp;
        }
      int2* span_dev = nullptr;
      if (cudaMalloc((void**)&span_dev, ball.size() * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, BPS_ENOMEM, "tile autotuning: device allocation failed");
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t err = cudaMemcpy(span_dev, ball.data(), ball.size() * sizeof(int2), cudaMemcpyHostToDevice);
      if (err == cudaSuccess) err = cudaEventCreate(&e0);
      if (err == cudaSuccess) err = cudaEventCreate(&e1);
      float best = 1e30f;
      for (int c = 0; c < 3 && err == cudaSuccess; ++c) {
        float total = 0.f;
        for (int pattern = 0; pattern < 2 && err == cudaSuccess; ++pattern) {
          Fields f = fields(ctx);
          f.span = pattern ? span_dev : nullptr;
          f.span_stride = (long long)N * N;
          f.span_slot = 0;
          for (int w = 0; w < 2; ++w) ctx->pt.z_grad_lp[c](f, -1, B, s);
          cudaEventRecord(e0, s);
          for (int r = 0; r < 5; ++r) ctx->pt.z_grad_lp[c](f, -1, B, s);
          cudaEventRecord(e1, s);
          err = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
          total += ms;
        }
        if (err == cudaSuccess && total < best) {
          best = total;
          pick = c;
        }
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaFree(span_dev);
      CK(err);
      CK(cudaGetLastError());
      g_tune[key] = 4 << pick;
      tune_save();
    }
  }
  ctx->zgrad = ctx->pt.z_grad_lp[pick];
  ctx->zgrad_tiles = ctx->pt.z_lp_tiles[pick];
  ctx->zgrad_pairs = 4 << pick;
  return BPS_OK;
}

// The leapfrog x pass has seven implementations with bit-identical results: the
// direct-load pass, three with tensor-copy staged tiles (W, delta and p; W and
// delta; W only) and three that stream delta and p through a ring of quarter
// tiles (filled by tensor copies, by 16-byte copies of every thread, or by each
// warp for its own rows, without block barriers).  Which
// is fastest depends on the GPU, the grid and the number of chains sharing a
// launch, so the first context of a kind times them on its own (still empty)
// buffers like the z-pass tiles above and caches the choice ("... xleap" keys).
// BPS_XTMA = 0..6 forces one; BPS_AUTOTUNE=0 keeps the direct pass.
bps_status choose_xleap(bps_ctx* ctx) {
  TraceRange trace_("bps autotune: x pass");
  ctx->xleap = nullptr;
  int which = 0;
  const char* xe = std::getenv("BPS_XTMA");
  const char* ae = std::getenv("BPS_AUTOTUNE");
  const bool tune = !xe && !(ae && std::atoi(ae) == 0);
  if (xe) which = std::atoi(xe);
  if (!xe && !tune) return BPS_OK;
  if (!make_xmaps(fields(ctx), ctx->N, ctx->batch, &ctx->xmaps)) return BPS_OK;   // no tensor maps: direct
  if (tune) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    const std::string key = std::string(prop.name) + " N=" + std::to_string(ctx->N) + " chains=" +
                            std::to_string(ctx->batch) + " xleap";
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && it->second >= 0 && it->second <= 6) {
      which = it->second;
    } else {
      cudaStream_t s = ctx->stream;
      const Fields f = fields(ctx);
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      float best = 1e30f;
      for (int c = 0; c < 7; ++c) {
        XLeapTma fn = c ? xleap_tma(ctx->N, c) : nullptr;
        if (c && !fn) continue;
        auto run = [&] {
          if (c) fn(f, ctx->xmaps, 0, ctx->batch, s);
          else ctx->pt.x_leap(f, 0, ctx->batch, s);
        };
        for (int w = 0; w < 2; ++w) run();
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 5; ++r) run();
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          which = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      CK(cudaGetLastError());
      g_tune[key] = which;
      tune_save();
    }
  }
  if (which > 0) ctx->xleap = xleap_tma(ctx->N, which);
  return BPS_OK;
}

// ------------------------------------------------------------------ group construction
bps_status check_config(const bps_config* cfg, int min_sub) {
  if (cfg->n_bins < 1 || cfg->n_bins > MAXB) return fail(nullptr, BPS_EINVAL, "n_bins must be in 1..64");
  if (cfg->n_leapfrog < 1 || !(cfg->eps_max > 0.0)) return fail(nullptr, BPS_EINVAL, "bad leapfrog settings");
  if (cfg->jump && (cfg->jump_leapfrog < 1 || !(cfg->jump_eps_max > 0.0)))
    return fail(nullptr, BPS_EINVAL, "bad jump settings");
  if (cfg->fixed_bias_index >= min_sub) return fail(nullptr, BPS_EINVAL, "fixed_bias_index out of range");
  if (cfg->mass_mode != 0 && cfg->mass_mode != 1) return fail(nullptr, BPS_EINVAL, "mass_mode must be 0 or 1");
  return BPS_OK;
}

// One group: chains j with box[j], nsub[j], seeds[j]; ids[j] = record slot (empty: a single chain).
bps_status create_group(int grid_n, const std::vector<double>& box, const std::vector<int>& nsub,
                        const std::vector<uint64_t>& seeds, const std::vector<int>& ids, const bps_config* cfg,
                        cudaStream_t stream, bps_ctx** out) {
  *out = nullptr;
  PassTable pt;
  if (!pass_table(grid_n, &pt)) return fail(nullptr, BPS_EINVAL, "unsupported grid size (8,16,32,64,96,128,256)");
  const int B = (int)box.size();
  int max_sub = 0;
  for (int j = 0; j < B; ++j) {
    if (!(box[j] > 0.0) || !std::isfinite(box[j])) return fail(nullptr, BPS_EINVAL, "box length must be positive");
    if (nsub[j] < 1 || nsub[j] > MAXS) return fail(nullptr, BPS_EINVAL, "n_sub must be in 1..16");
    max_sub = std::max(max_sub, nsub[j]);
  }
  bps_status cs = check_config(cfg, *std::min_element(nsub.begin(), nsub.end()));
  if (cs != BPS_OK) return cs;

  DevState h;
  std::memset(&h, 0, sizeof(h));
  if (!bin_tables(grid_n, cfg->n_bins, h.thr, h.nmodes))
    return fail(nullptr, BPS_EINVAL, "a power-spectrum bin holds no mode; use fewer bins");
  bin_tables(grid_n, cfg->n_bins, h.mthr, nullptr);
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

  bps_ctx* ctx = new bps_ctx();
  ctx->N = grid_n;
  ctx->batch = B;
  ctx->max_sub = max_sub;
  ctx->nsub = nsub;
  ctx->box = box;
  ctx->chain_id = ids;
  ctx->cfg = *cfg;
  ctx->stream = stream;
  ctx->pt = pt;
  ctx->zp = pt.zp;
  ctx->nv = (long long)grid_n * grid_n * grid_n;
  ctx->n_spec = (size_t)grid_n * grid_n * pt.zp;
  ctx->n_mass = cfg->n_bins;
  ctx->chain_cap = ids.empty() ? 1024 : 0;
  ctx->have_data.assign(B, 0);
  ctx->pending.assign(B, std::vector<int>());
  ctx->next_slot.assign(B, 1);   // slot 0 (all zero) stays active until a first survey is valid
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ctx->n_sm = sms > 0 ? sms : 148;
  // the voxel kernels of a batch run B chains side by side: fewer blocks each
  ctx->rebuild_blocks = std::max(1, std::min(4 * ctx->n_sm / B + 1, (int)(ctx->nv / 1024) + 1));
  // fused y^-1 / z / y stage where the grid has one; BPS_FUSED_YZ=0 keeps the three passes
  {
    const char* e = std::getenv("BPS_FUSED_YZ");
    if (!(e && std::atoi(e) == 0) && !yz_table(grid_n, &ctx->yz)) ctx->yz = YzEntry{};
  }
  ctx->part_stride = std::max(std::max(std::max(pt.x_tiles, pt.z_tiles), pt.z_lp_tiles[0]), ctx->rebuild_blocks);
  ctx->part_stride = std::max(ctx->part_stride, ctx->yz.tiles);
  ctx->part_cstride = (long long)region_total() * ctx->part_stride;

  auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
  const size_t sb = ctx->n_spec * sizeof(float2) * B, rb = (size_t)ctx->nv * sizeof(float) * B;
  const size_t span_bytes = 2 * (size_t)grid_n * grid_n * sizeof(int2) * B;   // two data slots
  const int rec_len = cfg->n_bins + 2 * max_sub + 2;
  bool ok = alloc((void**)&ctx->dh[0], sb) && alloc((void**)&ctx->dh[1], sb) && alloc((void**)&ctx->ph, sb) &&
            alloc((void**)&ctx->W, sb) && alloc((void**)&ctx->a, rb) && alloc((void**)&ctx->c, rb) &&
            (grid_n % 32 != 0 || alloc((void**)&ctx->span, span_bytes)) &&
            alloc((void**)&ctx->tw, grid_n * sizeof(float2)) && alloc((void**)&ctx->pbin, ctx->n_spec) &&
            alloc((void**)&ctx->part, (size_t)ctx->part_cstride * B * sizeof(double)) &&
            alloc((void**)&ctx->ds, sizeof(DevState) * B) &&
            (!ids.empty() || alloc((void**)&ctx->chain_dev, (size_t)ctx->chain_cap * rec_len * sizeof(double))) &&
            cudaMallocHost((void**)&ctx->host_buf, 64 * 1024) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ENOMEM, "device allocation failed");
  }
  // the k bin of every half-spectrum mode, from the same integer rule as the
  // bin thresholds (255 for the DC mode and the pad column)
  std::vector<uint8_t> pbin(ctx->n_spec, 255);
  {
    const int H = grid_n / 2, ZP = pt.zp;
    std::vector<uint8_t> of_n2(3 * (size_t)H * H + 1, 255);
    for (size_t n2 = 1; n2 < of_n2.size(); ++n2) of_n2[n2] = (uint8_t)bin_of_host((long long)n2, grid_n, cfg->n_bins);
    for (int kx = 0; kx < grid_n; ++kx) {
      const int nx = kx <= H ? kx : kx - grid_n;
      for (int ky = 0; ky < grid_n; ++ky) {
        const int ny = ky <= H ? ky : ky - grid_n;
        uint8_t* row = pbin.data() + ((size_t)kx * grid_n + ky) * ZP;
        for (int kz = 0; kz <= H; ++kz) row[kz] = of_n2[(size_t)(nx * nx + ny * ny + kz * kz)];
      }
    }
  }
  // twiddles W_N^j = exp(-2 pi i j / N), FP64 rounded to FP32
  std::vector<float2> tw(grid_n);
  for (int j = 0; j < grid_n; ++j) {
    const double ang = -2.0 * M_PI * (double)j / (double)grid_n;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  std::vector<DevState> hs(B, h);
  for (int j = 0; j < B; ++j) {
    hs[j].vc = std::pow(box[j] / grid_n, 3);
    hs[j].seed = seeds[j];
    hs[j].nsub = nsub[j];
  }
  cudaError_t e = cudaMemcpyAsync(ctx->tw, tw.data(), grid_n * sizeof(float2), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->pbin, pbin.data(), ctx->n_spec, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ds, hs.data(), sizeof(DevState) * B, cudaMemcpyHostToDevice, stream);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(ctx->dh[i], 0, sb, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ph, 0, sb, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->W, 0, sb, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->a, 0, rb, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->c, 0, rb, stream);
  if (e == cudaSuccess && ctx->span) e = cudaMemsetAsync(ctx->span, 0, span_bytes, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    std::string msg = std::string("initialisation failed: ") + cudaGetErrorString(e);
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ECUDA, msg);
  }
  if (choose_xleap(ctx) != BPS_OK) {
    std::string msg = "x-pass autotuning failed: " + ctx->err;
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ECUDA, msg);
  }
  if (choose_zgrad(ctx) != BPS_OK) {
    std::string msg = "tile autotuning failed: " + ctx->err;
    free_all(ctx);
    delete ctx;
    return fail(nullptr, BPS_ECUDA, msg);
  }
  *out = ctx;
  return BPS_OK;
}

// ------------------------------------------------------------------ per-chain operations
// Starts the upload of one chain's survey into its next data slot: (host
// arrays) copies through the two staging slots on the copy streams, then the
// check-and-compress kernel of each subsample on up_stream, which also widens
// the slot's per-line supports and leaves its partial sums in dpart.  Nothing
// waits on the host; commit_data activates the slot.
bps_status stage_data(bps_ctx* ctx, int ch, const void* counts, const float* R, bool host, bool c16) {
  if (!counts || !R) return fail(ctx, BPS_EINVAL, "null argument");
  if (ctx->pending[ch].size() >= 2)
    return fail(ctx, BPS_ESTATE, "two surveys are already staged; run an operation that uses the data first");
  const int ns = ctx->nsub[ch];
  const int B = ctx->batch;
  const int blocks = ctx->rebuild_blocks;
  if (!ctx->cnt) {
    const size_t total = 2 * (size_t)ctx->max_sub * ctx->nv * B;   // two data slots
    if (cudaMalloc((void**)&ctx->cnt, total * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->R, total * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->cnt);
      cudaFree(ctx->R);
      ctx->cnt = nullptr;
      ctx->R = nullptr;
      return fail(ctx, BPS_ENOMEM, "device allocation of the survey data failed");
    }
    CK(cudaMemsetAsync(ctx->cnt, 0, total * sizeof(uint16_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->R, 0, total * sizeof(float), ctx->stream));
  }
  if (!ctx->up_stream) {
    ctx->dpart_cstride = (long long)MAXS * 4 * blocks;
    bool ok = cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->up_after_main, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc((void**)&ctx->dpart, (size_t)2 * B * ctx->dpart_cstride * sizeof(double)) == cudaSuccess;
    ctx->slot_ready.assign(2 * (size_t)B, nullptr);
    for (size_t i = 0; i < ctx->slot_ready.size() && ok; ++i)
      ok = cudaEventCreateWithFlags(&ctx->slot_ready[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_streams(ctx);
      return fail(ctx, BPS_ENOMEM, "upload streams and buffers could not be allocated");
    }
  }
  const size_t slot_bytes = (size_t)ctx->nv * (sizeof(int32_t) + sizeof(float));
  // copy streams for host uploads; the staging buffer only for 32-bit counts
  // (16-bit counts are copied straight into the data slot)
  if (host && !ctx->copy_stream[0]) {
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i)
      ok = cudaStreamCreateWithFlags(&ctx->copy_stream[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ctx->stage_copied[i][0], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&ctx->stage_copied[i][1], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&ctx->stage_free[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_streams(ctx);
      return fail(ctx, BPS_ENOMEM, "copy streams for the host upload could not be created");
    }
  }
  if (host && !c16 && !ctx->stage) {
    if (cudaMalloc((void**)&ctx->stage, 2 * slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->stage = nullptr;
      return fail(ctx, BPS_ENOMEM, "staging buffers for the host upload could not be allocated");
    }
  }
  const int slot = ctx->next_slot[ch];
  Fields f = fields_at(ctx, ch);
  uint16_t* cnt_ch = const_cast<uint16_t*>(f.cnt) + slot * f.data_slot;
  float* R_ch = const_cast<float*>(f.R) + slot * f.data_slot;
  int2* span_ch = f.span ? const_cast<int2*>(f.span) + slot * f.span_slot : nullptr;
  double* part = ctx->dpart + ((size_t)slot * B + ch) * ctx->dpart_cstride;
  cudaStream_t up = ctx->up_stream;
  // the slot may hold the survey that work already queued on the main stream reads
  CK(cudaEventRecord(ctx->up_after_main, ctx->stream));
  CK(cudaStreamWaitEvent(up, ctx->up_after_main, 0));
  // the data kernels widen the slot's per-line supports from empty
  if (span_ch) CK(cudaMemsetAsync(span_ch, 0, (size_t)ctx->N * ctx->N * sizeof(int2), up));
  if (host) CK(cudaEventRecord(ctx->stage_free[0], up));   // orders the copies after earlier uploads
  if (host) CK(cudaEventRecord(ctx->stage_free[1], up));
  const size_t csz = c16 ? sizeof(uint16_t) : sizeof(int32_t);
  for (int l = 0; l < ns; ++l) {
    const void* cl = static_cast<const char*>(counts) + (size_t)l * ctx->nv * csz;
    const float* rl = R + (size_t)l * ctx->nv;
    if (host && c16) {
      // 16-bit counts are the storage format: copy straight into the slot, then
      // check in place (no staging round trip through device memory)
      uint16_t* cdst = cnt_ch + (size_t)l * ctx->nv;
      float* rdst = R_ch + (size_t)l * ctx->nv;
      const int sl = l & 1;
      for (int k = 0; k < 2; ++k) CK(cudaStreamWaitEvent(ctx->copy_stream[k], ctx->stage_free[sl], 0));
      CK(cudaMemcpyAsync(cdst, cl, ctx->nv * csz, cudaMemcpyHostToDevice, ctx->copy_stream[0]));
      CK(cudaMemcpyAsync(rdst, rl, ctx->nv * sizeof(float), cudaMemcpyHostToDevice, ctx->copy_stream[1]));
      for (int k = 0; k < 2; ++k) {
        CK(cudaEventRecord(ctx->stage_copied[sl][k], ctx->copy_stream[k]));
        CK(cudaStreamWaitEvent(up, ctx->stage_copied[sl][k], 0));
      }
      launch_data16(cdst, rdst, nullptr, nullptr, ctx->nv, part + (size_t)l * 4 * blocks, blocks, blocks, span_ch,
                    ctx->N, up);
      LAUNCHED(ctx, 1);
      continue;
    }
    if (host) {
      // copy subsample l into staging slot l % 2 once the data kernel of subsample l - 2 has read it
      const int sl = l & 1;
      void* ctmp = ctx->stage + sl * slot_bytes;
      float* rtmp = reinterpret_cast<float*>(ctx->stage + sl * slot_bytes + (size_t)ctx->nv * sizeof(int32_t));
      for (int k = 0; k < 2; ++k) CK(cudaStreamWaitEvent(ctx->copy_stream[k], ctx->stage_free[sl], 0));
      CK(cudaMemcpyAsync(ctmp, cl, ctx->nv * csz, cudaMemcpyHostToDevice, ctx->copy_stream[0]));
      CK(cudaMemcpyAsync(rtmp, rl, ctx->nv * sizeof(float), cudaMemcpyHostToDevice, ctx->copy_stream[1]));
      for (int k = 0; k < 2; ++k) {
        CK(cudaEventRecord(ctx->stage_copied[sl][k], ctx->copy_stream[k]));
        CK(cudaStreamWaitEvent(up, ctx->stage_copied[sl][k], 0));
      }
      cl = ctmp;
      rl = rtmp;
    }
    if (c16)
      launch_data16(static_cast<const uint16_t*>(cl), rl, cnt_ch + (size_t)l * ctx->nv, R_ch + (size_t)l * ctx->nv,
                    ctx->nv, part + (size_t)l * 4 * blocks, blocks, blocks, span_ch, ctx->N, up);
    else
      launch_data(static_cast<const int32_t*>(cl), rl, cnt_ch + (size_t)l * ctx->nv, R_ch + (size_t)l * ctx->nv,
                  ctx->nv, part + (size_t)l * 4 * blocks, blocks, blocks, span_ch, ctx->N, up);
    LAUNCHED(ctx, 1);
    if (host) CK(cudaEventRecord(ctx->stage_free[l & 1], up));
  }
  CK(cudaEventRecord(ctx->slot_ready[2 * (size_t)ch + slot], up));
  ctx->pending[ch].push_back(slot);
  ctx->next_slot[ch] = 1 - slot;
  return BPS_OK;
}

// Activates the oldest staged survey of chain `ch`, in order on the main
// stream: waits for its upload, then the commit kernel (data constants, or
// ST_BADDATA and the previous slot kept), then a and c rebuilt on the active
// slot (zeroed first where the supports limit the rebuild).
bps_status commit_data(bps_ctx* ctx, int ch) {
  if (ctx->pending[ch].empty()) return BPS_OK;
  const int slot = ctx->pending[ch].front();
  ctx->pending[ch].erase(ctx->pending[ch].begin());
  cudaStream_t s = ctx->stream;
  CK(cudaStreamWaitEvent(s, ctx->slot_ready[2 * (size_t)ch + slot], 0));
  launch_commit_data(ctx->ds + ch, ctx->dpart + ((size_t)slot * ctx->batch + ch) * ctx->dpart_cstride,
                     ctx->dpart_cstride, ctx->rebuild_blocks, slot, 1, s);
  LAUNCHED(ctx, 1);
  Fields f = fields_at(ctx, ch);
  if (f.span) {
    CK(cudaMemsetAsync(f.a, 0, (size_t)ctx->nv * sizeof(float), s));
    CK(cudaMemsetAsync(f.c, 0, (size_t)ctx->nv * sizeof(float), s));
  }
  ctx->have_data[ch] = 1;
  return rebuild_chain(ctx, ch);
}

// The synchronous upload: stage, activate every staged survey in order, and
// report invalid data.
bps_status set_data_chain(bps_ctx* ctx, int ch, const void* counts, const float* R, bool host, bool c16 = false) {
  bps_status st = stage_data(ctx, ch, counts, R, host, c16);
  while (st == BPS_OK && !ctx->pending[ch].empty()) st = commit_data(ctx, ch);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  st = check_status(ctx);
  if (st != BPS_OK) ctx->have_data[ch] = 0;
  return st;
}

bps_status set_state_chain(bps_ctx* ctx, int ch, const float* delta_dev, const double* P, const double* b,
                           const double* nbar, uint64_t iteration) {
  if (!P || !b || !nbar) return fail(ctx, BPS_EINVAL, "null argument");
  const int nb = ctx->cfg.n_bins, ns = ctx->nsub[ch];
  for (int m = 0; m < nb; ++m)
    if (!(P[m] > 0.0) || !std::isfinite(P[m])) return fail(ctx, BPS_EINVAL, "P must be positive and finite");
  for (int l = 0; l < ns; ++l)
    if (!std::isfinite(b[l]) || !(nbar[l] > 0.0) || !std::isfinite(nbar[l]))
      return fail(ctx, BPS_EINVAL, "b must be finite and nbar positive");
  bps_status st = ds_write_bytes(ctx, ch, DS_OFF(P), P, nb * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, ch, DS_OFF(P_ref), P, nb * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, ch, DS_OFF(b), b, ns * sizeof(double));
  if (st == BPS_OK) st = ds_write_bytes(ctx, ch, DS_OFF(nbar), nbar, ns * sizeof(double));
  unsigned long long it = iteration;
  if (st == BPS_OK) st = ds_write_bytes(ctx, ch, DS_OFF(iteration), &it, sizeof(it));
  if (st != BPS_OK) return st;
  Fields f = fields_at(ctx, ch);
  if (delta_dev) {
    ctx->pt.z_r2c(f, delta_dev, f.W, ctx->stream);
    ctx->pt.y_fwd(f, BUF_W, 1, ctx->stream);
    ctx->pt.x_fwd(f, BUF_W, nullptr, 1, ctx->stream);
    LAUNCHED(ctx, 3);
    int cur = current_buffer(ctx, ch, &st);
    if (st != BPS_OK) return st;
    launch_zero_dc(state_buffer(ctx, ch, cur), ctx->stream);
    LAUNCHED(ctx, 1);
  }
  if (ctx->have_data[ch]) {
    st = rebuild_chain(ctx, ch);
    if (st != BPS_OK) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status get_state_chain(bps_ctx* ctx, int ch, float* delta_dev, double* P, double* b, double* nbar,
                           uint64_t* iteration) {
  bps_status st = BPS_OK;
  if (delta_dev) {
    Fields f = fields_at(ctx, ch);
    ctx->pt.x_inv(f, -1, f.W, 1, ctx->stream);
    ctx->pt.y_inv(f, BUF_W, 1, ctx->stream);
    ctx->pt.z_c2r(f, f.W, delta_dev, ctx->stream);
    LAUNCHED(ctx, 3);
  }
  const int ns = ctx->nsub[ch];
  if (P) st = ds_read_bytes(ctx, ch, DS_OFF(P), P, ctx->cfg.n_bins * sizeof(double));
  if (st == BPS_OK && b) st = ds_read_bytes(ctx, ch, DS_OFF(b), b, ns * sizeof(double));
  if (st == BPS_OK && nbar) st = ds_read_bytes(ctx, ch, DS_OFF(nbar), nbar, ns * sizeof(double));
  if (st == BPS_OK && iteration) {
    unsigned long long it = 0;
    st = ds_read_bytes(ctx, ch, DS_OFF(iteration), &it, sizeof(it));
    *iteration = it;
  }
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

// Captures one Gibbs iteration of every chain of the groups into *out (kernels
// counted per replay in *launches).  With `prof` the captured iteration also
// holds event-record nodes around the leapfrog kernels of top (one group).
bps_status capture_iteration(bps_ctx* top, const std::vector<bps_ctx*>& groups, double* rec_dev, int rec_len,
                             long long iter_stride, bool jump, bool prof, cudaGraphExec_t* out, uint64_t* launches) {
  TraceRange trace_(prof ? "bps graph capture (profiled)" : "bps graph capture");
  bps_ctx* ctx = top;
  cudaStream_t s = top->stream;
  // capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is replayed on the caller's
  if (!top->cap_stream) CK(cudaStreamCreateWithFlags(&top->cap_stream, cudaStreamNonBlocking));
  if (prof) {
    prof_fold(top);   // also synchronises
    // event-record nodes need their events before capture: two per leapfrog
    // step and kernel kind
    const size_t need = 2 * (size_t)top->cfg.n_leapfrog;
    for (int k = 0; k < 4; ++k)
      while (top->ev[k].size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        top->ev[k].push_back(e);
      }
  } else {
    CK(cudaStreamSynchronize(s));
  }
  std::vector<uint64_t> before;
  for (bps_ctx* gr : groups) before.push_back(gr->launches);
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(top->cap_stream, cudaStreamCaptureModeThreadLocal));
  for (bps_ctx* gr : groups) gr->stream = top->cap_stream;
  top->capturing = prof;
  bps_status st = BPS_OK;
  for (bps_ctx* gr : groups) {
    st = gibbs_once(gr, rec_dev, rec_len, iter_stride, jump);
    if (st != BPS_OK) break;
  }
  top->capturing = false;
  for (bps_ctx* gr : groups) gr->stream = s;
  cudaError_t e = cudaStreamEndCapture(top->cap_stream, &g);
  // the kernels were captured, not launched: count them per replay instead
  uint64_t captured = 0;
  for (size_t i = 0; i < groups.size(); ++i) {
    captured += groups[i]->launches - before[i];
    groups[i]->launches = before[i];
  }
  if (prof)
    for (int k = 0; k < 4; ++k) {
      top->prof_graph_events[k] = top->ev_used[k];
      top->ev_used[k] = 0;
    }
  if (st != BPS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  CK(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  *launches = captured;
  return BPS_OK;
}

// Run n_iter Gibbs iterations of every chain of the groups, recording into
// `rec_dev` [n_iter][chains][rec_len].  Iterations replay one captured CUDA
// graph (captured on first use, or again after a change that alters the
// launches).  With kernel timing on, a single-chain context replays a second
// graph that also records the leapfrog kernels' events, reading the timings
// after every replay; a batch launches directly.
bps_status run_iterations(bps_ctx* top, const std::vector<bps_ctx*>& groups, int n_iter, double* rec_dev,
                          int rec_len, int n_chains, bool jump) {
  bps_ctx* ctx = top;
  cudaStream_t s = top->stream;
  for (bps_ctx* g : groups) {
    launch_reset_rec(g->ds, g->batch, s);
    LAUNCHED(g, 1);
  }
  const long long iter_stride = (long long)n_chains * rec_len;
  bool prof = false;
  for (bps_ctx* g : groups) prof = prof || g->prof;
  if (prof && groups.size() != 1) {
    for (int i = 0; i < n_iter; ++i)
      for (bps_ctx* g : groups) {
        bps_status st = gibbs_once(g, rec_dev, rec_len, iter_stride, jump);
        if (st != BPS_OK) return st;
      }
    return BPS_OK;
  }
  if (prof) {
    if (top->prof_graph && top->prof_graph_jump != jump) {
      cudaGraphExecDestroy(top->prof_graph);
      top->prof_graph = nullptr;
    }
    if (!top->prof_graph) {
      bps_status st = capture_iteration(top, groups, rec_dev, rec_len, iter_stride, jump, true, &top->prof_graph,
                                        &top->prof_graph_launches);
      if (st != BPS_OK) return st;
      top->prof_graph_jump = jump;
    }
    for (int i = 0; i < n_iter; ++i) {
      CK(cudaGraphLaunch(top->prof_graph, s));
      for (int k = 0; k < 4; ++k) top->ev_used[k] = top->prof_graph_events[k];
      prof_fold(top);   // the replay re-records the same events: read them now
    }
    top->launches += (uint64_t)n_iter * top->prof_graph_launches;
    return BPS_OK;
  }
  if (top->graph && top->graph_jump != jump) {
    cudaGraphExecDestroy(top->graph);
    top->graph = nullptr;
  }
  if (!top->graph) {
    bps_status st =
        capture_iteration(top, groups, rec_dev, rec_len, iter_stride, jump, false, &top->graph, &top->graph_launches);
    if (st != BPS_OK) return st;
    top->graph_jump = jump;
  }
  for (int i = 0; i < n_iter; ++i) CK(cudaGraphLaunch(top->graph, s));
  top->launches += (uint64_t)n_iter * top->graph_launches;
  return BPS_OK;
}

// Posterior statistics of the density modes for the mass preconditioner: run
// n_moves HMC moves of every chain (the hyperparameters stay fixed) and return,
// per chain and mass bin j, V_j = mean over the bin's full-grid modes of
// Var(delta_k) / N^3 (comparable with lambda_k = P/V_cell) and Mbar_j = mean of
// the diagonal mass 1/lambda_k + abar over the same modes.
bps_status mass_stats(bps_ctx* ctx, int n_moves, int n_mass, double* out, int out_stride, const std::vector<int>& slot) {
  int thr[MAXB];
  double nm[MAXB];
  if (!bin_tables(ctx->N, n_mass, thr, nm))
    return fail(ctx, BPS_EINVAL, "a mass bin holds no mode; use fewer mass bins");
  if (ctx->mnet && n_mass != ctx->n_mass)
    return fail(ctx, BPS_EINVAL, "with a network mass, n_mass_bins must equal the network's output width");
  cudaStream_t s = ctx->stream;
  const int B = ctx->batch;
  if (!ctx->acc) {
    if (cudaMalloc((void**)&ctx->acc, ctx->n_spec * sizeof(float2) * B) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BPS_ENOMEM, "accumulator allocation failed");
    }
  }
  CK(cudaMemsetAsync(ctx->acc, 0, ctx->n_spec * sizeof(float2) * B, s));
  std::vector<double> zero(MAXB, 0.0);
  for (int ch = 0; ch < B; ++ch) {
    bps_status st = ds_write_bytes(ctx, ch, DS_OFF(mthr), thr, sizeof(thr));
    if (st == BPS_OK) st = ds_write_bytes(ctx, ch, DS_OFF(mstat), zero.data(), MAXB * sizeof(double));
    if (st != BPS_OK) return st;
  }
  ctx->n_mass = n_mass;   // the mass-bin table now has n_mass bins
  drop_graph(ctx);
  Fields f = fields(ctx);
  ScalarArgs sa = scalars(ctx);
  for (int i = 0; i < n_moves; ++i) {
    bps_status st = hmc_move(ctx, true);
    if (st != BPS_OK) return st;
    ctx->pt.x_macc(f, region_offset(ctx, RG_BIN), B, s);
    launch_mstat(sa, region_offset(ctx, RG_BIN), ctx->pt.x_tiles, n_mass, 0, B, s);
    LAUNCHED(ctx, 2);
  }
  ctx->pt.x_mmean(f, region_offset(ctx, RG_BIN), B, s);
  launch_mstat(sa, region_offset(ctx, RG_BIN), ctx->pt.x_tiles, n_mass, 1, B, s);
  LAUNCHED(ctx, 2);
  CK(cudaStreamSynchronize(s));
  // mode counts per (power bin, mass bin), full-grid weights
  const int nb = ctx->cfg.n_bins, N = ctx->N, H = N / 2;
  std::vector<double> cnt((size_t)nb * n_mass, 0.0), nj(n_mass, 0.0);
  for (int ix = 0; ix < N; ++ix) {
    const long long nx = ix <= H ? ix : ix - N;
    for (int iy = 0; iy < N; ++iy) {
      const long long ny = iy <= H ? iy : iy - N;
      for (int iz = 0; iz <= H; ++iz) {
        const long long n2 = nx * nx + ny * ny + (long long)iz * iz;
        if (n2 == 0) continue;
        const double w = (iz == 0 || iz == H) ? 1.0 : 2.0;
        const int m = bin_of_host(n2, N, nb), j = bin_of_host(n2, N, n_mass);
        cnt[(size_t)m * n_mass + j] += w;
        nj[j] += w;
      }
    }
  }
  const double S = (double)n_moves, nv = (double)ctx->nv;
  for (int ch = 0; ch < B; ++ch) {
    std::vector<double> m1(MAXB), m2(MAXB), P(MAXB);
    double abar = 0.0, vc = 0.0;
    bps_status st = ds_read_bytes(ctx, ch, DS_OFF(mstat), m1.data(), MAXB * sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, ch, DS_OFF(mstat2), m2.data(), MAXB * sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, ch, DS_OFF(P), P.data(), MAXB * sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, ch, DS_OFF(abar), &abar, sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, ch, DS_OFF(vc), &vc, sizeof(double));
    if (st != BPS_OK) return st;
    double* o = out + (size_t)slot[ch] * out_stride;
    for (int j = 0; j < n_mass; ++j) {
      const double var = (m1[j] / S - m2[j] / (S * S)) / (nj[j] * nv);
      double mb = 0.0;
      for (int m = 0; m < nb; ++m) mb += cnt[(size_t)m * n_mass + j] * (vc / P[m] + abar);
      o[j] = var;
      o[n_mass + j] = mb / nj[j];
    }
  }
  return BPS_OK;
}

// Binned power of the survey window: sigma_m of a / abar (the local curvature
// a = sum_l b_l^2 Nbar_l R^l over its voxel mean), one chain per slot.
bps_status window_power(bps_ctx* ctx, double* out, int out_stride, const std::vector<int>& slot) {
  cudaStream_t s = ctx->stream;
  const int nb = ctx->cfg.n_bins;
  for (int ch = 0; ch < ctx->batch; ++ch) {
    Fields f = fields_at(ctx, ch);
    ctx->pt.z_r2c(f, f.a, f.W, s);
    ctx->pt.y_fwd(f, BUF_W, 1, s);
    ctx->pt.x_fwd(f, BUF_W, f.W, 1, s);
    ctx->pt.x_wpow(f, region_offset(ctx, RG_BIN), 1, s);
    launch_power(scalars_at(ctx, ch), region_offset(ctx, RG_BIN), ctx->pt.x_tiles, 0, 1, s);
    LAUNCHED(ctx, 5);
    std::vector<double> sig(MAXB);
    double abar = 0.0;
    bps_status st = ds_read_bytes(ctx, ch, DS_OFF(sigma), sig.data(), MAXB * sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, ch, DS_OFF(abar), &abar, sizeof(double));
    if (st != BPS_OK) return st;
    double* o = out + (size_t)slot[ch] * out_stride;
    for (int m = 0; m < nb; ++m) o[m] = sig[m] / (abar * abar);
  }
  return BPS_OK;
}

}  // namespace

void bps::set_last_error(const char* msg) { g_err = msg; }

// =================================================================== C ABI
extern "C" {

const char* bps_version(void) { return "bps 0.3 (sm_103a)"; }

const char* bps_last_error(const bps_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

uint64_t bps_kernel_launches(const bps_ctx* ctx) {
  if (!ctx) return 0;
  uint64_t n = ctx->launches;
  for (const bps_ctx* g : ctx->groups) n += g->launches;
  return n;
}

int bps_x_pass_variant(const bps_ctx* ctx) {
  if (!ctx) return -1;
  const bps_ctx* g = ctx->is_batch ? (ctx->groups.empty() ? nullptr : ctx->groups[0]) : ctx;
  if (!g || !g->xleap) return 0;
  for (int c = 1; c <= 6; ++c)
    if (xleap_tma(g->N, c) == g->xleap) return c;
  return 0;
}

int bps_z_line_pairs(const bps_ctx* ctx) {
  if (!ctx) return 0;
  return ctx->is_batch ? (ctx->groups.empty() ? 0 : ctx->groups[0]->zgrad_pairs) : ctx->zgrad_pairs;
}

bps_status bps_profile(bps_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  if (ctx->is_batch) return fail(ctx, BPS_EINVAL, "kernel timing is per single-chain context");
  if (ctx->prof && !enable) prof_fold(ctx);
  ctx->prof = enable != 0;
  return BPS_OK;
}

bps_status bps_profile_read(bps_ctx* ctx, double* ms, uint64_t* n) {
  if (!ctx || !ms || !n) return fail(ctx, BPS_EINVAL, "null argument");
  if (ctx->is_batch) return fail(ctx, BPS_EINVAL, "kernel timing is per single-chain context");
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
  TraceRange trace_("bps_create");
  if (!out || !cfg) return fail(nullptr, BPS_EINVAL, "null argument");
  *out = nullptr;
  if (n_sub < 1 || n_sub > MAXS) return fail(nullptr, BPS_EINVAL, "n_sub must be in 1..16");
  return create_group(grid_n, {box_len}, {n_sub}, {cfg->seed}, {}, cfg, (cudaStream_t)cuda_stream, out);
}

void bps_destroy(bps_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (bps_ctx* g : ctx->groups) bps_destroy(g);
  free_all(ctx);
  delete ctx;
}

bps_status bps_set_data(bps_ctx* ctx, const int32_t* counts_dev, const float* R_dev) {
  TraceRange trace_("bps_set_data");
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return set_data_chain(ctx, 0, counts_dev, R_dev, false);
}

bps_status bps_set_data_host(bps_ctx* ctx, const int32_t* counts, const float* R) {
  TraceRange trace_("bps_set_data_host");
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return set_data_chain(ctx, 0, counts, R, true);
}

bps_status bps_set_data_host_u16(bps_ctx* ctx, const uint16_t* counts, const float* R) {
  TraceRange trace_("bps_set_data_host_u16");
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return set_data_chain(ctx, 0, counts, R, true, true);
}

bps_status bps_stage_data_host_u16(bps_ctx* ctx, const uint16_t* counts, const float* R) {
  TraceRange trace_("bps_stage_data_host_u16");
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return stage_data(ctx, 0, counts, R, true, true);
}

bps_status bps_set_state(bps_ctx* ctx, const float* delta_dev, const double* P, const double* b, const double* nbar,
                         uint64_t iteration) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return set_state_chain(ctx, 0, delta_dev, P, b, nbar, iteration);
}

bps_status bps_get_state(bps_ctx* ctx, float* delta_dev, double* P, double* b, double* nbar, uint64_t* iteration) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "single-chain call on a null or batch context");
  return get_state_chain(ctx, 0, delta_dev, P, b, nbar, iteration);
}

bps_status bps_get_spectrum(bps_ctx* ctx, float* spec_dev) {
  if (!ctx || ctx->is_batch || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  bps_status st;
  int cur = current_buffer(ctx, 0, &st);
  if (st != BPS_OK) return st;
  st = copy_spec_out(ctx, ctx->dh[cur], spec_dev);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_set_spectrum(bps_ctx* ctx, const float* spec_dev) {
  if (!ctx || ctx->is_batch || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  bps_status st;
  int cur = current_buffer(ctx, 0, &st);
  if (st != BPS_OK) return st;
  st = copy_spec_in(ctx, spec_dev, ctx->dh[cur]);
  if (st != BPS_OK) return st;
  launch_zero_dc(ctx->dh[cur], ctx->stream);
  LAUNCHED(ctx, 1);
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

// ---- checkpoint of one chain (bps_save_chain / bps_load_chain)
namespace {
constexpr char CHAIN_MAGIC[8] = {'B', 'P', 'S', 'C', 'H', 'A', 'I', 'N'};
struct ChainHeader {
  char magic[8];
  uint32_t version;
  int32_t N, n_sub, n_bins, n_mass, pad;
  double box, eps_max;
  uint64_t iteration;
  double P[MAXB], P_ref[MAXB], b[MAXS], nbar[MAXS], mass_scale[MAXB];
};
size_t chain_blob_bytes(const bps_ctx* ctx) {
  return sizeof(ChainHeader) + (size_t)ctx->N * ctx->N * (ctx->N / 2 + 1) * sizeof(float2);
}
}  // namespace

bps_status bps_save_chain(bps_ctx* ctx, void* blob, size_t* bytes) {
  TraceRange trace_("bps_save_chain");
  if (!ctx || ctx->is_batch || !bytes) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  const size_t need = chain_blob_bytes(ctx);
  if (!blob) {
    *bytes = need;
    return BPS_OK;
  }
  if (*bytes < need) return fail(ctx, BPS_EINVAL, "checkpoint buffer too small");
  ChainHeader h{};
  std::memcpy(h.magic, CHAIN_MAGIC, 8);
  h.version = 1;
  h.N = ctx->N;
  h.n_sub = ctx->nsub[0];
  h.n_bins = ctx->cfg.n_bins;
  h.n_mass = ctx->n_mass;
  h.box = ctx->box[0];
  h.eps_max = ctx->cfg.eps_max;
  unsigned long long it = 0;
  bps_status st = ds_read_bytes(ctx, 0, DS_OFF(P), h.P, sizeof(h.P));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(P_ref), h.P_ref, sizeof(h.P_ref));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(b), h.b, sizeof(h.b));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(nbar), h.nbar, sizeof(h.nbar));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(mass_scale), h.mass_scale, sizeof(h.mass_scale));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(iteration), &it, sizeof(it));
  if (st != BPS_OK) return st;
  h.iteration = it;
  int cur = current_buffer(ctx, 0, &st);
  if (st != BPS_OK) return st;
  const size_t H1 = (size_t)ctx->N / 2 + 1;
  char* out = static_cast<char*>(blob);
  std::memcpy(out, &h, sizeof h);
  CK(cudaMemcpy2DAsync(out + sizeof h, H1 * sizeof(float2), ctx->dh[cur], (size_t)ctx->zp * sizeof(float2),
                       H1 * sizeof(float2), (size_t)ctx->N * ctx->N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *bytes = need;
  return BPS_OK;
}

bps_status bps_load_chain(bps_ctx* ctx, const void* blob, size_t bytes) {
  TraceRange trace_("bps_load_chain");
  if (!ctx || ctx->is_batch || !blob) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  ChainHeader h;
  if (bytes < sizeof h) return fail(ctx, BPS_EINVAL, "not a chain checkpoint (too short)");
  std::memcpy(&h, blob, sizeof h);
  if (std::memcmp(h.magic, CHAIN_MAGIC, 8) != 0 || h.version != 1)
    return fail(ctx, BPS_EINVAL, "not a chain checkpoint of this library version");
  if (h.N != ctx->N || h.n_sub != ctx->nsub[0] || h.n_bins != ctx->cfg.n_bins || h.box != ctx->box[0])
    return fail(ctx, BPS_EINVAL, "checkpoint of another grid, box, subsample or bin count");
  if (bytes != chain_blob_bytes(ctx)) return fail(ctx, BPS_EINVAL, "checkpoint size does not match the grid");
  if (h.n_mass < 0 || h.n_mass > MAXB || !(h.eps_max > 0.0) || !std::isfinite(h.eps_max))
    return fail(ctx, BPS_EINVAL, "corrupt checkpoint header");
  for (int m = 0; m < h.n_bins; ++m)
    if (!(h.P[m] > 0.0) || !std::isfinite(h.P[m]) || !(h.P_ref[m] > 0.0) || !std::isfinite(h.P_ref[m]))
      return fail(ctx, BPS_EINVAL, "corrupt checkpoint spectrum");
  bps_status st = BPS_OK;
  if (h.n_mass > 0) {
    double sc[MAXB];
    std::memcpy(sc, h.mass_scale, sizeof sc);
    st = bps_set_mass_scale(ctx, h.n_mass, sc);
    if (st != BPS_OK) return st;
  }
  st = ds_write_bytes(ctx, 0, DS_OFF(P), h.P, sizeof(h.P));
  if (st == BPS_OK) st = ds_write_bytes(ctx, 0, DS_OFF(P_ref), h.P_ref, sizeof(h.P_ref));
  if (st == BPS_OK) st = ds_write_bytes(ctx, 0, DS_OFF(b), h.b, sizeof(h.b));
  if (st == BPS_OK) st = ds_write_bytes(ctx, 0, DS_OFF(nbar), h.nbar, sizeof(h.nbar));
  unsigned long long it = h.iteration;
  if (st == BPS_OK) st = ds_write_bytes(ctx, 0, DS_OFF(iteration), &it, sizeof(it));
  if (st != BPS_OK) return st;
  if (h.eps_max != ctx->cfg.eps_max) {
    ctx->cfg.eps_max = h.eps_max;
    drop_graph(ctx);   // eps_max is a launch argument of the captured iteration
  }
  int cur = current_buffer(ctx, 0, &st);
  if (st != BPS_OK) return st;
  const size_t H1 = (size_t)ctx->N / 2 + 1;
  CK(cudaMemcpy2DAsync(ctx->dh[cur], (size_t)ctx->zp * sizeof(float2), static_cast<const char*>(blob) + sizeof h,
                       H1 * sizeof(float2), H1 * sizeof(float2), (size_t)ctx->N * ctx->N, cudaMemcpyHostToDevice,
                       ctx->stream));
  if (ctx->have_data[0]) {
    st = rebuild_chain(ctx, 0);
    if (st != BPS_OK) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

// ---- artificial surveys (bps_mock.cu)
namespace {
bps_status mock_scratch(void* owner, size_t bytes, void** out) {
  bps_ctx* ctx = static_cast<bps_ctx*>(owner);
  if (ctx->mock_bytes < bytes) {
    if (ctx->mock_buf) {
      CK(cudaStreamSynchronize(ctx->stream));   // earlier mock kernels may still read it
      cudaFree(ctx->mock_buf);
      ctx->mock_buf = nullptr;
      ctx->mock_bytes = 0;
    }
    if (cudaMalloc(&ctx->mock_buf, bytes) != cudaSuccess) return fail(ctx, BPS_ENOMEM, "mock table buffer");
    ctx->mock_bytes = bytes;
  }
  *out = ctx->mock_buf;
  return BPS_OK;
}
bps_status mock_view(bps_ctx* ctx, MockView* v, Fields* f) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  *f = fields_at(ctx, 0);
  v->N = ctx->N;
  v->zp = ctx->zp;
  v->n_sub = ctx->nsub[0];
  v->n_sm = ctx->n_sm > 0 ? ctx->n_sm : 152;
  v->box = ctx->box[0];
  v->stream = ctx->stream;
  v->pt = &ctx->pt;
  v->f = f;
  v->launches = &ctx->launches;
  v->owner = ctx;
  v->scratch = mock_scratch;
  return BPS_OK;
}
bps_status mock_result(bps_ctx* ctx, bps_status st) {
  if (st != BPS_OK && ctx) ctx->err = bps_last_error(nullptr);
  return st;
}
}  // namespace

bps_status bps_mock_field(bps_ctx* ctx, uint64_t seed, const double* P_n2, float* delta_dev) {
  TraceRange trace_("bps_mock_field");
  MockView v;
  Fields f;
  bps_status st = mock_view(ctx, &v, &f);
  if (st != BPS_OK) return st;
  if (!P_n2 || !delta_dev) return fail(ctx, BPS_EINVAL, "null argument");
  return mock_result(ctx, mock_field(v, seed, P_n2, delta_dev));
}

bps_status bps_mock_counts(bps_ctx* ctx, uint64_t seed, const float* delta_dev, const float* R_dev, const double* b,
                           const double* nbar, int noise, int32_t* counts_dev) {
  TraceRange trace_("bps_mock_counts");
  MockView v;
  Fields f;
  bps_status st = mock_view(ctx, &v, &f);
  if (st != BPS_OK) return st;
  if (!delta_dev || !R_dev || !b || !nbar || !counts_dev) return fail(ctx, BPS_EINVAL, "null argument");
  if (noise != 0 && noise != 1) return fail(ctx, BPS_EINVAL, "noise must be 0 (Poisson) or 1 (Gaussian)");
  return mock_result(ctx, mock_counts(v, seed, delta_dev, R_dev, b, nbar, noise, counts_dev));
}

bps_status bps_mock_response(bps_ctx* ctx, double f_sky, const double* axis, int n_r, const double* table,
                             float* R_dev) {
  TraceRange trace_("bps_mock_response");
  MockView v;
  Fields f;
  bps_status st = mock_view(ctx, &v, &f);
  if (st != BPS_OK) return st;
  if (!axis || !table || !R_dev) return fail(ctx, BPS_EINVAL, "null argument");
  return mock_result(ctx, mock_response(v, f_sky, axis, n_r, table, R_dev));
}

// ---- posterior analysis (Secs. 6.2 and 7)
bps_status bps_posterior_moments(bps_ctx* ctx, int enable) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  if (enable) {
    const size_t D = (size_t)ctx->cfg.n_bins + 2 * (size_t)ctx->nsub[0];
    const size_t nm = 2 * (size_t)ctx->nv, np = 1 + D + D * D;
    if (!ctx->mom && cudaMalloc(&ctx->mom, nm * sizeof(double)) != cudaSuccess) {
      ctx->mom = nullptr;
      return fail(ctx, BPS_ENOMEM, "posterior moment buffers");
    }
    if (!ctx->pmom && cudaMalloc(&ctx->pmom, np * sizeof(double)) != cudaSuccess) {
      ctx->pmom = nullptr;
      return fail(ctx, BPS_ENOMEM, "posterior moment buffers");
    }
    CK(cudaMemsetAsync(ctx->mom, 0, nm * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(ctx->pmom, 0, np * sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if ((enable != 0) != ctx->mom_on) drop_graph(ctx);   // the iteration's launches change
  ctx->mom_on = enable != 0;
  return BPS_OK;
}

bps_status bps_posterior_read(bps_ctx* ctx, double* mean_dev, double* var_dev, double* param_mean,
                              double* param_cov, uint64_t* n_samples) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  if (!ctx->mom || !ctx->pmom) return fail(ctx, BPS_ESTATE, "bps_posterior_moments has not been enabled");
  const size_t D = (size_t)ctx->cfg.n_bins + 2 * (size_t)ctx->nsub[0];
  std::vector<double> acc(1 + D + D * D);
  CK(cudaMemcpyAsync(acc.data(), ctx->pmom, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double n = acc[0];
  if (n_samples) *n_samples = (uint64_t)n;
  if (!(n > 0.0)) return fail(ctx, BPS_ESTATE, "no Gibbs iteration has been accumulated yet");
  if (mean_dev || var_dev) {
    launch_moments_finish(ctx->mom, ctx->nv, n, mean_dev, var_dev, ctx->n_sm * 8, ctx->stream);
    LAUNCHED(ctx, 1);
  }
  for (size_t i = 0; i < D; ++i) {
    const double mi = acc[1 + i] / n;
    if (param_mean) param_mean[i] = mi;
    if (param_cov)
      for (size_t j = 0; j < D; ++j) param_cov[i * D + j] = acc[1 + D + i * D + j] / n - mi * (acc[1 + j] / n);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_selftest_wait(bps_ctx* ctx, uint64_t limit_ns) {
  if (!ctx || ctx->is_batch) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  if (limit_ns < 1 || limit_ns > 1000000000ULL) return fail(ctx, BPS_EINVAL, "limit_ns must be in 1..1e9");
  bps_status st = check_status(ctx);   // report (and clear) anything earlier first
  if (st != BPS_OK) return st;
  launch_wait_probe(ctx->ds, (unsigned long long)limit_ns, ctx->stream);
  LAUNCHED(ctx, 1);
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

bps_status bps_hmc_step(bps_ctx* ctx, bps_move_info* info) {
  TraceRange trace_("bps_hmc_step");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = hmc_move(ctx, true);
  if (st != BPS_OK) return st;
  if (info) {
    int acc = 0;
    double dH = 0, eps = 0;
    st = ds_read_bytes(ctx, 0, DS_OFF(accepted), &acc, sizeof(int));
    if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(dH), &dH, sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(eps), &eps, sizeof(double));
    if (st != BPS_OK) return st;
    info->accepted = acc;
    info->dH = dH;
    info->eps = eps;
    return check_status(ctx);
  }
  return BPS_OK;
}

bps_status bps_adapt_step_size(bps_ctx* ctx, int n_rounds, int moves_per_round, double target,
                               double* eps_max_out) {
  TraceRange trace_("bps_adapt_step_size");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (n_rounds < 1 || moves_per_round < 1 || !(target > 0.0 && target < 1.0))
    return fail(ctx, BPS_EINVAL, "need n_rounds >= 1, moves_per_round >= 1 and 0 < target < 1");
  unsigned long long m0 = 0, a0 = 0;
  st = ds_read_bytes(ctx, 0, DS_OFF(n_moves), &m0, sizeof(m0));
  if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(n_accepted), &a0, sizeof(a0));
  if (st != BPS_OK) return st;
  for (int r = 0; r < n_rounds; ++r) {
    for (int i = 0; i < moves_per_round; ++i) {
      st = hmc_move(ctx, true);
      if (st != BPS_OK) return st;
    }
    unsigned long long m1 = 0, a1 = 0;
    st = ds_read_bytes(ctx, 0, DS_OFF(n_moves), &m1, sizeof(m1));
    if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(n_accepted), &a1, sizeof(a1));
    if (st == BPS_OK) st = check_status(ctx);
    if (st != BPS_OK) return st;
    const double acc = m1 > m0 ? (double)(a1 - a0) / (double)(m1 - m0) : target;
    m0 = m1;
    a0 = a1;
    // Robbins-Monro step on ln eps_max with a decreasing gain, at most a factor 2 per round
    const double gain = 2.0 / std::sqrt((double)(r + 1));
    const double step = std::max(-std::log(2.0), std::min(std::log(2.0), gain * (acc - target)));
    ctx->cfg.eps_max *= std::exp(step);
  }
  drop_graph(ctx);   // eps_max is a launch argument of the captured iteration
  if (eps_max_out) *eps_max_out = ctx->cfg.eps_max;
  return BPS_OK;
}

bps_status bps_sample_power(bps_ctx* ctx, double* P_out, double* sigma_out) {
  TraceRange trace_("bps_sample_power");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = power_stage(ctx, true, true);
  if (st != BPS_OK) return st;
  if (P_out) st = ds_read_bytes(ctx, 0, DS_OFF(P), P_out, ctx->cfg.n_bins * sizeof(double));
  if (st == BPS_OK && sigma_out) st = ds_read_bytes(ctx, 0, DS_OFF(sigma), sigma_out, ctx->cfg.n_bins * sizeof(double));
  if (st != BPS_OK) return st;
  if (P_out || sigma_out) return check_status(ctx);
  return BPS_OK;
}

bps_status bps_sample_bias_norm(bps_ctx* ctx, double* b_out, double* nbar_out, double* sums_out) {
  TraceRange trace_("bps_sample_bias_norm");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  st = bias_stage(ctx, true);
  if (st != BPS_OK) return st;
  const int ns = ctx->nsub[0];
  if (b_out) st = ds_read_bytes(ctx, 0, DS_OFF(b), b_out, ns * sizeof(double));
  if (st == BPS_OK && nbar_out) st = ds_read_bytes(ctx, 0, DS_OFF(nbar), nbar_out, ns * sizeof(double));
  if (st == BPS_OK && sums_out) {
    std::vector<double> tmp(3 * MAXS);
    st = ds_read_bytes(ctx, 0, DS_OFF(sums), tmp.data(), tmp.size() * sizeof(double));
    for (int i = 0; i < 3 * ns; ++i) sums_out[i] = tmp[i];
  }
  if (st != BPS_OK) return st;
  if (b_out || nbar_out || sums_out) return check_status(ctx);
  return BPS_OK;
}

bps_status bps_jump(bps_ctx* ctx, bps_move_info* info) {
  TraceRange trace_("bps_jump");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (ctx->cfg.jump_leapfrog < 1 || !(ctx->cfg.jump_eps_max > 0.0))
    return fail(ctx, BPS_EINVAL, "jump settings are not set");
  st = jump_stage(ctx, true);
  if (st != BPS_OK) return st;
  if (info) {
    int acc = 0;
    double dH = 0, eps = 0;
    st = ds_read_bytes(ctx, 0, DS_OFF(jaccepted), &acc, sizeof(int));
    if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(jdH), &dH, sizeof(double));
    if (st == BPS_OK) st = ds_read_bytes(ctx, 0, DS_OFF(jeps), &eps, sizeof(double));
    if (st != BPS_OK) return st;
    info->accepted = acc;
    info->dH = dH;
    info->eps = eps;
    return check_status(ctx);
  }
  return BPS_OK;
}

bps_status bps_gibbs_iterate(bps_ctx* ctx, int n_iter, double* chain_out) {
  TraceRange trace_("bps_gibbs_iterate");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (n_iter < 0) return fail(ctx, BPS_EINVAL, "n_iter must be >= 0");
  if (n_iter == 0) return BPS_OK;
  const int rec = ctx->cfg.n_bins + 2 * ctx->max_sub + 2;
  // the record buffer holds up to chain_cap iterations; longer runs go in pieces
  int done = 0;
  while (done < n_iter) {
    const int k = std::min(n_iter - done, ctx->chain_cap);
    st = run_iterations(ctx, {ctx}, k, ctx->chain_dev, rec, 1, ctx->cfg.jump != 0);
    if (st != BPS_OK) return st;
    if (chain_out)
      CK(cudaMemcpyAsync(chain_out + (size_t)done * rec, ctx->chain_dev, (size_t)k * rec * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->stream));
    done += k;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

bps_status bps_set_mass_scale(bps_ctx* ctx, int n_mass_bins, const double* scales) {
  if (!ctx || !scales) return fail(ctx, BPS_EINVAL, "null argument");
  if (n_mass_bins < 1 || n_mass_bins > MAXB) return fail(ctx, BPS_EINVAL, "n_mass_bins must be in 1..64");
  for (int j = 0; j < n_mass_bins; ++j)
    if (!(scales[j] > 0.0) || !std::isfinite(scales[j])) return fail(ctx, BPS_EINVAL, "scales must be positive");
  std::vector<bps_ctx*> gs = ctx->is_batch ? ctx->groups : std::vector<bps_ctx*>{ctx};
  for (bps_ctx* g : gs) {
    int thr[MAXB];
    if (!bin_tables(g->N, n_mass_bins, thr, nullptr))
      return fail(ctx, BPS_EINVAL, "a mass bin holds no |n|^2 value; use fewer mass bins");
    for (int ch = 0; ch < g->batch; ++ch) {
      bps_status st = ds_write_bytes(g, ch, DS_OFF(mthr), thr, sizeof(thr));
      if (st == BPS_OK) st = ds_write_bytes(g, ch, DS_OFF(mass_scale), scales, n_mass_bins * sizeof(double));
      if (st != BPS_OK) return st;
    }
    g->n_mass = n_mass_bins;
  }
  drop_graph(ctx);   // the number of mass bins is a launch argument
  return BPS_OK;
}

bps_status bps_set_mass_net(bps_ctx* ctx, const bps_mlp* net, const float* feat_mean, const float* feat_std,
                            double log_clamp) {
  TraceRange trace_("bps_set_mass_net");
  if (!ctx) return fail(nullptr, BPS_EINVAL, "null context");
  std::vector<bps_ctx*> gs = ctx->is_batch ? ctx->groups : std::vector<bps_ctx*>{ctx};
  drop_graph(ctx);
  if (!net) {
    for (bps_ctx* g : gs) {
      massnet_destroy(g->mnet);
      g->mnet = nullptr;
    }
    return BPS_OK;
  }
  const int nb = ctx->cfg.n_bins, n_out = massnet_width(net, 1);
  if (!feat_mean || !feat_std) return fail(ctx, BPS_EINVAL, "null argument");
  if (massnet_width(net, 0) != 2 * nb) return fail(ctx, BPS_EINVAL, "the network must take 2 n_bins inputs");
  if (n_out < 1 || n_out > MAXB) return fail(ctx, BPS_EINVAL, "the network must give 1..64 outputs");
  if (!(log_clamp > 0.0) || !std::isfinite(log_clamp)) return fail(ctx, BPS_EINVAL, "log_clamp must be positive");
  for (int i = 0; i < 2 * nb; ++i)
    if (!(feat_std[i] > 0.f) || !std::isfinite(feat_mean[i])) return fail(ctx, BPS_EINVAL, "bad feature standardisation");
  for (bps_ctx* g : gs) {
    int thr[MAXB];
    if (!bin_tables(g->N, n_out, thr, nullptr))
      return fail(ctx, BPS_EINVAL, "a mass bin holds no |n|^2 value; use fewer network outputs");
    for (int ch = 0; ch < g->batch; ++ch)
      if (!g->have_data[ch]) return fail(ctx, BPS_ESTATE, "a chain has no data");
  }
  for (bps_ctx* g : gs) {
    // window features of every chain: ln of the binned power of a / abar
    std::vector<double> wp((size_t)g->batch * nb);
    std::vector<int> slot(g->batch);
    for (int ch = 0; ch < g->batch; ++ch) slot[ch] = ch;
    bps_status st = window_power(g, wp.data(), nb, slot);
    if (st != BPS_OK) return st;
    int thr[MAXB];
    bin_tables(g->N, n_out, thr, nullptr);
    for (int ch = 0; ch < g->batch && st == BPS_OK; ++ch) {
      float wf[MAXB] = {0.f};
      for (int m = 0; m < nb; ++m) wf[m] = (float)std::log(std::max(wp[(size_t)ch * nb + m], 1e-30));
      st = ds_write_bytes(g, ch, DS_OFF(wfeat), wf, sizeof(wf));
      if (st == BPS_OK) st = ds_write_bytes(g, ch, DS_OFF(mthr), thr, sizeof(thr));
    }
    if (st != BPS_OK) return st;
    MassNet* m = nullptr;
    st = massnet_create(net, feat_mean, feat_std, log_clamp, &m);
    if (st != BPS_OK) return fail(ctx, st, "network copy failed");
    massnet_destroy(g->mnet);
    g->mnet = m;
    g->n_mass = n_out;
  }
  return BPS_OK;
}

// Library format of a trained preconditioner (bps_mlp_export): "BPSM", version
// 1, n_layers, widths[n_layers + 1] (uint32 each), log_clamp (double), feature
// means and standard deviations (float [width 0] each), parameters (float,
// layout of bps_mlp_set_params); host byte order.
bps_status bps_set_preconditioner(bps_ctx* ctx, const void* blob, size_t bytes) {
  TraceRange trace_("bps_set_preconditioner");
  if (!ctx || !blob) return fail(ctx, BPS_EINVAL, "null argument");
  const unsigned char* b = static_cast<const unsigned char*>(blob);
  auto rd32 = [&](size_t off) {
    uint32_t v;
    std::memcpy(&v, b + off, 4);
    return v;
  };
  if (bytes < 12 || std::memcmp(b, "BPSM", 4) != 0 || rd32(4) != 1u)
    return fail(ctx, BPS_EINVAL, "not a preconditioner in the library format");
  const uint32_t L = rd32(8);
  if (L < 1 || L > 4) return fail(ctx, BPS_EINVAL, "preconditioner: 1..4 layers");
  size_t off = 12;
  if (bytes < off + 4 * (L + 1) + 8) return fail(ctx, BPS_EINVAL, "preconditioner: truncated");
  int sizes[5];
  for (uint32_t l = 0; l <= L; ++l) sizes[l] = (int)rd32(off + 4 * l);
  off += 4 * (L + 1);
  double clamp;
  std::memcpy(&clamp, b + off, 8);
  off += 8;
  size_t n_params = 0;
  for (uint32_t l = 0; l < L; ++l) {
    if (sizes[l] < 1 || sizes[l] > 512 || sizes[l + 1] < 1 || sizes[l + 1] > 512)
      return fail(ctx, BPS_EINVAL, "preconditioner: layer widths must be in 1..512");
    n_params += (size_t)sizes[l] * sizes[l + 1] + sizes[l + 1];
  }
  const size_t need = off + 2 * 4 * (size_t)sizes[0] + 4 * n_params;
  if (bytes != need) return fail(ctx, BPS_EINVAL, "preconditioner: size does not match its layout");
  std::vector<float> mean(sizes[0]), sd(sizes[0]), params(n_params);
  std::memcpy(mean.data(), b + off, 4 * (size_t)sizes[0]);
  off += 4 * (size_t)sizes[0];
  std::memcpy(sd.data(), b + off, 4 * (size_t)sizes[0]);
  off += 4 * (size_t)sizes[0];
  std::memcpy(params.data(), b + off, 4 * n_params);
  bps_mlp* net = nullptr;
  bps_status st = bps_mlp_create((int)L, sizes, ctx->is_batch ? ctx->groups[0]->stream : ctx->stream, &net);
  if (st != BPS_OK) return fail(ctx, st, "preconditioner: network allocation failed");
  st = bps_mlp_set_params(net, params.data());
  if (st == BPS_OK) st = bps_set_mass_net(ctx, net, mean.data(), sd.data(), clamp);
  bps_mlp_destroy(net);   // the context keeps its own copy
  return st;
}

bps_status bps_get_mass_scale(bps_ctx* ctx, int chain, int* n_mass_bins, double* scales) {
  if (!ctx || !n_mass_bins || !scales) return fail(ctx, BPS_EINVAL, "null argument");
  bps_ctx* g = ctx;
  int ch = chain;
  if (ctx->is_batch) {
    if (chain < 0 || chain >= (int)ctx->chain_map.size()) return fail(ctx, BPS_EINVAL, "chain out of range");
    g = ctx->groups[ctx->chain_map[chain].first];
    ch = ctx->chain_map[chain].second;
  } else if (chain != 0) {
    return fail(ctx, BPS_EINVAL, "chain must be 0 for a single-chain context");
  }
  *n_mass_bins = g->n_mass;
  return ds_read_bytes(g, ch, DS_OFF(mass_scale), scales, (size_t)g->n_mass * sizeof(double));
}

bps_status bps_fft_r2c(bps_ctx* ctx, const float* real_dev, float* spec_dev) {
  if (!ctx || ctx->is_batch || !real_dev || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  Fields f = fields_at(ctx, 0);
  ctx->pt.z_r2c(f, real_dev, ctx->W, ctx->stream);
  ctx->pt.y_fwd(f, BUF_W, 1, ctx->stream);
  ctx->pt.x_fwd(f, BUF_W, ctx->W, 1, ctx->stream);
  LAUNCHED(ctx, 3);
  bps_status st = copy_spec_out(ctx, ctx->W, spec_dev);
  if (st != BPS_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_fft_c2r(bps_ctx* ctx, const float* spec_dev, float* real_dev) {
  if (!ctx || ctx->is_batch || !real_dev || !spec_dev) return fail(ctx, BPS_EINVAL, "null argument or batch context");
  bps_status st = copy_spec_in(ctx, spec_dev, ctx->W);
  if (st != BPS_OK) return st;
  Fields f = fields_at(ctx, 0);
  ctx->pt.x_inv(f, BUF_W, ctx->W, 1, ctx->stream);
  ctx->pt.y_inv(f, BUF_W, 1, ctx->stream);
  ctx->pt.z_c2r(f, ctx->W, real_dev, ctx->stream);
  LAUNCHED(ctx, 3);
  CK(cudaStreamSynchronize(ctx->stream));
  return BPS_OK;
}

bps_status bps_gradient(bps_ctx* ctx, float* grad_dev, double* energies) {
  TraceRange trace_("bps_gradient");
  bps_status st = need_data(ctx);
  if (st != BPS_OK) return st;
  if (!grad_dev) return fail(ctx, BPS_EINVAL, "null argument");
  Fields f = fields_at(ctx, 0);
  ScalarArgs sa = scalars_at(ctx, 0);
  cudaStream_t s = ctx->stream;
  launch_move_begin(sa, 1, s);   // per-bin tables of the current P and abar
  ctx->pt.x_inv(f, -1, ctx->W, 1, s);
  bps_status sf = force_stage(ctx, f, region_offset(ctx, RG_LIK0), false, s);
  if (sf != BPS_OK) return sf;
  ctx->pt.x_grad(f, ctx->W, region_offset(ctx, RG_GRAD), 1, s);
  double* scratch = reinterpret_cast<double*>(ds_addr(ctx, 0, DS_OFF(scratch)));
  launch_reduce_to(sa, region_offset(ctx, RG_GRAD), ctx->pt.x_tiles, 1, 0.5 / (double)ctx->nv, scratch, s);
  launch_reduce_to(sa, region_offset(ctx, RG_LIK0), lik_tiles(ctx), 1, 1.0, scratch + 1, s);
  LAUNCHED(ctx, 5);
  st = copy_spec_out(ctx, ctx->W, grad_dev);
  if (st != BPS_OK) return st;
  if (energies) {
    st = ds_read_bytes(ctx, 0, DS_OFF(scratch), energies, 2 * sizeof(double));
    if (st != BPS_OK) return st;
  }
  CK(cudaStreamSynchronize(s));
  return BPS_OK;
}

// ------------------------------------------------------------------ batches
bps_status bps_create_batch(int n_chains, const int* grid_n, const double* box_len, const int* n_sub,
                            const bps_config* cfg, void* cuda_stream, bps_ctx** out) {
  TraceRange trace_("bps_create_batch");
  if (!out || !cfg || !grid_n || !box_len || !n_sub) return fail(nullptr, BPS_EINVAL, "null argument");
  *out = nullptr;
  if (n_chains < 1) return fail(nullptr, BPS_EINVAL, "n_chains must be >= 1");
  std::map<int, std::vector<int>> by_n;
  int max_sub = 0;
  for (int j = 0; j < n_chains; ++j) {
    by_n[grid_n[j]].push_back(j);
    if (n_sub[j] < 1 || n_sub[j] > MAXS) return fail(nullptr, BPS_EINVAL, "n_sub must be in 1..16");
    max_sub = std::max(max_sub, n_sub[j]);
  }
  bps_ctx* top = new bps_ctx();
  top->is_batch = true;
  top->cfg = *cfg;
  top->stream = (cudaStream_t)cuda_stream;
  top->max_sub = max_sub;
  top->rec_len_all = cfg->n_bins + 2 * max_sub + 2;
  top->chain_map.assign(n_chains, {-1, -1});
  top->batch = 0;
  int slot = 0;
  for (auto& kv : by_n) {
    std::vector<double> box;
    std::vector<int> ns, ids;
    std::vector<uint64_t> seeds;
    for (size_t i = 0; i < kv.second.size(); ++i) {
      const int j = kv.second[i];
      box.push_back(box_len[j]);
      ns.push_back(n_sub[j]);
      seeds.push_back(cfg->seed + (uint64_t)j);
      ids.push_back(slot + (int)i);   // the records of one group occupy consecutive slots
    }
    bps_ctx* g = nullptr;
    bps_status st = create_group(kv.first, box, ns, seeds, ids, cfg, top->stream, &g);
    if (st != BPS_OK) {
      bps_destroy(top);
      return st;
    }
    const int gi = (int)top->groups.size();
    top->groups.push_back(g);
    for (size_t i = 0; i < kv.second.size(); ++i) top->chain_map[kv.second[i]] = {gi, (int)i};
    slot += (int)kv.second.size();
  }
  top->chain_cap = 256;
  if (cudaMalloc((void**)&top->chain_dev, (size_t)top->chain_cap * n_chains * top->rec_len_all * sizeof(double)) !=
          cudaSuccess ||
      cudaMallocHost((void**)&top->host_buf, 64 * 1024) != cudaSuccess) {
    cudaGetLastError();
    bps_destroy(top);
    return fail(nullptr, BPS_ENOMEM, "device allocation failed");
  }
  *out = top;
  return BPS_OK;
}

int bps_batch_record_len(const bps_ctx* batch) { return batch && batch->is_batch ? batch->rec_len_all : 0; }

int bps_batch_record_slot(const bps_ctx* batch, int chain) {
  if (!batch || !batch->is_batch || chain < 0 || chain >= (int)batch->chain_map.size()) return -1;
  const auto& cm = batch->chain_map[chain];
  return batch->groups[cm.first]->chain_id[cm.second];
}

bps_status bps_batch_set_chain(bps_ctx* batch, int chain, const int32_t* counts_dev, const float* R_dev,
                               const float* delta_dev, const double* P, const double* b, const double* nbar,
                               uint64_t iteration) {
  if (!batch || !batch->is_batch) return fail(batch, BPS_EINVAL, "not a batch context");
  if (chain < 0 || chain >= (int)batch->chain_map.size()) return fail(batch, BPS_EINVAL, "chain out of range");
  bps_ctx* g = batch->groups[batch->chain_map[chain].first];
  const int ch = batch->chain_map[chain].second;
  bps_status st = set_data_chain(g, ch, counts_dev, R_dev, false);
  if (st == BPS_OK) st = set_state_chain(g, ch, delta_dev, P, b, nbar, iteration);
  if (st != BPS_OK) batch->err = g->err;
  return st;
}

bps_status bps_batch_get_chain(bps_ctx* batch, int chain, float* delta_dev, double* P, double* b, double* nbar,
                               uint64_t* iteration) {
  if (!batch || !batch->is_batch) return fail(batch, BPS_EINVAL, "not a batch context");
  if (chain < 0 || chain >= (int)batch->chain_map.size()) return fail(batch, BPS_EINVAL, "chain out of range");
  bps_ctx* g = batch->groups[batch->chain_map[chain].first];
  bps_status st = get_state_chain(g, batch->chain_map[chain].second, delta_dev, P, b, nbar, iteration);
  if (st != BPS_OK) batch->err = g->err;
  return st;
}

bps_status bps_batch_gibbs_iterate(bps_ctx* batch, int n_iter, double* chain_out) {
  TraceRange trace_("bps_batch_gibbs_iterate");
  if (!batch || !batch->is_batch) return fail(batch, BPS_EINVAL, "not a batch context");
  if (n_iter < 0) return fail(batch, BPS_EINVAL, "n_iter must be >= 0");
  for (bps_ctx* g : batch->groups)
    for (int ch = 0; ch < g->batch; ++ch)
      if (!g->have_data[ch]) return fail(batch, BPS_ESTATE, "a chain has no data (bps_batch_set_chain)");
  bps_ctx* ctx = batch;
  const int n_chains = (int)batch->chain_map.size();
  const int rec = batch->rec_len_all;
  int done = 0;
  while (done < n_iter) {
    const int k = std::min(n_iter - done, batch->chain_cap);
    bps_status st = run_iterations(batch, batch->groups, k, batch->chain_dev, rec, n_chains, batch->cfg.jump != 0);
    if (st != BPS_OK) return st;
    if (chain_out)
      CK(cudaMemcpyAsync(chain_out + (size_t)done * n_chains * rec, batch->chain_dev,
                         (size_t)k * n_chains * rec * sizeof(double), cudaMemcpyDeviceToHost, batch->stream));
    done += k;
  }
  CK(cudaStreamSynchronize(batch->stream));
  for (bps_ctx* g : batch->groups) {
    bps_status st = check_status(g);
    if (st != BPS_OK) {
      batch->err = g->err;
      return st;
    }
  }
  return BPS_OK;
}

bps_status bps_mass_stats(bps_ctx* ctx, int n_moves, int n_mass_bins, double* out) {
  TraceRange trace_("bps_mass_stats");
  if (!ctx || !out) return fail(ctx, BPS_EINVAL, "null argument");
  if (n_moves < 2) return fail(ctx, BPS_EINVAL, "n_moves must be >= 2");
  if (n_mass_bins < 1 || n_mass_bins > MAXB) return fail(ctx, BPS_EINVAL, "n_mass_bins must be in 1..64");
  if (!ctx->is_batch) {
    bps_status st = need_data(ctx);
    if (st != BPS_OK) return st;
    st = mass_stats(ctx, n_moves, n_mass_bins, out, 2 * n_mass_bins, {0});
    if (st != BPS_OK) return st;
    return check_status(ctx);
  }
  for (bps_ctx* g : ctx->groups) {
    for (int ch = 0; ch < g->batch; ++ch)
      if (!g->have_data[ch]) return fail(ctx, BPS_ESTATE, "a chain has no data (bps_batch_set_chain)");
    std::vector<int> slot(g->chain_id.begin(), g->chain_id.end());
    bps_status st = mass_stats(g, n_moves, n_mass_bins, out, 2 * n_mass_bins, slot);
    if (st == BPS_OK) st = check_status(g);
    if (st != BPS_OK) {
      ctx->err = g->err;
      return st;
    }
  }
  drop_graph(ctx);
  return BPS_OK;
}

bps_status bps_window_power(bps_ctx* ctx, double* out) {
  TraceRange trace_("bps_window_power");
  if (!ctx || !out) return fail(ctx, BPS_EINVAL, "null argument");
  if (!ctx->is_batch) {
    bps_status st = need_data(ctx);
    if (st != BPS_OK) return st;
    return window_power(ctx, out, ctx->cfg.n_bins, {0});
  }
  for (bps_ctx* g : ctx->groups) {
    for (int ch = 0; ch < g->batch; ++ch)
      if (!g->have_data[ch]) return fail(ctx, BPS_ESTATE, "a chain has no data (bps_batch_set_chain)");
    bps_status st = window_power(g, out, ctx->cfg.n_bins, std::vector<int>(g->chain_id.begin(), g->chain_id.end()));
    if (st != BPS_OK) {
      ctx->err = g->err;
      return st;
    }
  }
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
