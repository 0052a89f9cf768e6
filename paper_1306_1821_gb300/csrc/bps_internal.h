// Internal interfaces between the translation units of the bps library.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "bps_common.cuh"
#include "bps_tma.cuh"

namespace bps {

struct Fields;

// Launchers of the field passes of one grid size (bps_passes.cu).  The `nch`
// argument is the number of chains of a batch (gridDim.y); a single-chain
// operation passes fields already moved to its chain and nch = 1.
struct PassTable {
  int N, zp, F, x_tiles, z_tiles;
  void (*x_init)(const Fields&, int region, int nch, cudaStream_t);
  void (*x_leap)(const Fields&, int first, int nch, cudaStream_t);
  // the first leapfrog step, also reducing sum w |g|^2 / M of the start force into `region`
  void (*x_leapg)(const Fields&, int region, int nch, cudaStream_t);
  void (*x_final)(const Fields&, int region, int nch, cudaStream_t);
  void (*x_inv)(const Fields&, int src_buf, float2* dst, int nch, cudaStream_t);   // src_buf -1: current state; dst NULL: W
  void (*x_fwd)(const Fields&, int src_buf, float2* dst, int nch, cudaStream_t);   // dst NULL: current state
  void (*x_grad)(const Fields&, float2* dst, int region, int nch, cudaStream_t);
  void (*x_jinv)(const Fields&, int nch, cudaStream_t);
  void (*x_jgrad)(const Fields&, int region, int nch, cudaStream_t);
  void (*x_scale)(const Fields&, int nch, cudaStream_t);
  void (*x_binpow)(const Fields&, int region, int nch, cudaStream_t);
  void (*x_macc)(const Fields&, int region, int nch, cudaStream_t);    // acc += delta, mass-bin power
  void (*x_mmean)(const Fields&, int region, int nch, cudaStream_t);   // mass-bin power of acc
  void (*x_wpow)(const Fields&, int region, int nch, cudaStream_t);    // power-bin power of W
  void (*y_fwd)(const Fields&, int buf, int nch, cudaStream_t);
  void (*y_inv)(const Fields&, int buf, int nch, cudaStream_t);
  void (*z_grad)(const Fields&, int region, int nch, cudaStream_t);
  void (*z_noise)(const Fields&, int nch, cudaStream_t);
  void (*z_r2c)(const Fields&, const float* rin, float2* dst, cudaStream_t);   // one chain
  void (*z_c2r)(const Fields&, const float2* src, float* rout, cudaStream_t);  // one chain
  // one chain: delta = C2R_z(W) added to the running sums mom[0..N^3) (delta) and mom[N^3..) (delta^2)
  void (*z_mom)(const Fields&, double* mom, cudaStream_t);
  void (*z_sums)(const Fields&, int region, int nch, cudaStream_t);
  // z_grad with 4, 8 or 16 line pairs per tile (autotuned per grid) and the
  // number of tiles (likelihood-energy partials) of each
  void (*z_grad_lp[3])(const Fields&, int region, int nch, cudaStream_t);
  int z_lp_tiles[3];
};

bool pass_table(int N, PassTable* out);

// Tensor maps of the half spectra of a group (4D: kz, ky, kx, chain; 8-byte
// elements) for the TMA-staged leapfrog x pass; box 16 (or F) columns x 1 x N
// rows x 1 chain.  ok = false when the driver offers no tensor-map encoder.
struct XMaps {
  CUtensorMap W, d0, d1, ph;   // boxes of a whole tile (F columns x N rows)
  CUtensorMap d0q, d1q, phq;   // boxes of a quarter tile (F columns x N/4 rows)
  bool ok = false;
};
bool make_xmaps(const Fields& f, int N, int nch, XMaps* out);
// the leapfrog x pass with its tiles staged by tensor copies (first: the first
// kick of a trajectory); nullptr where a grid has none
using XLeapTma = void (*)(const Fields&, const XMaps&, int first, int nch, cudaStream_t);
// which: 1 stages W, delta and p; 2 W and delta; 3 W only; 4 streams delta and p
// through a ring of quarter tiles filled by tensor copies, 5 the same ring filled
// by 16-byte copies of every thread, 6 warp-private rings (0 or other: none)
XLeapTma xleap_tma(int N, int which);

// The fused y^-1 / z / y stage of a force evaluation (bps_yz.cu): one CTA per
// x plane holds the plane in shared memory, so W is read and written once.
// `tiles` is the number of likelihood-energy partials it writes (one per CTA).
// Grids without a fused kernel keep the three passes.
struct YzEntry {
  void (*run)(const Fields&, int region, int nch, cudaStream_t) = nullptr;
  int tiles = 0;
};
bool yz_table(int N, YzEntry* out);
void launch_rebuild(const Fields& fp, long long nv, int region, int blocks, int nch, cudaStream_t s);
// Data check of one subsample; with `span` (N a multiple of 32) it also widens
// the per-line support of R > 0 (Fields::span encoding).
void launch_data(const int32_t* cin, const float* rin, uint16_t* cout, float* rout, long long nv, double* part,
                 int stride, int blocks, int2* span, int n_grid, cudaStream_t s);
// the same from 16-bit counts
void launch_data16(const uint16_t* cin, const float* rin, uint16_t* cout, float* rout, long long nv, double* part,
                   int stride, int blocks, int2* span, int n_grid, cudaStream_t s);
void launch_philox_words(uint64_t seed, uint64_t it, uint64_t stage, uint64_t sub, uint64_t blk0, size_t n,
                         uint64_t* out, cudaStream_t s);
void launch_voxel_normals(uint64_t seed, uint64_t it, size_t n, float* out, cudaStream_t s);

// Scalar stages of the Gibbs scan (bps_draws.cu).  Chain j of a batch uses
// ds + j and part + j * cstride (blockIdx.y); per-chain constants (seed, cell
// volume, number of subsamples) live in its DevState.
struct ScalarArgs {
  DevState* ds;
  const double* part;
  int stride;
  long long cstride;
  int n_bins, max_sub, n_mass;
  double inv_nv, alpha, eps_max, jeps_max;
  int fixed_bias;
};
void launch_move_begin(const ScalarArgs& a, int nch, cudaStream_t s);
void launch_move_end(const ScalarArgs& a, int r_init, int r_lik0, int r_final, int r_lik1, int nx, int nz, int nch,
                     cudaStream_t s);
void launch_power(const ScalarArgs& a, int region, int nx, int draw, int nch, cudaStream_t s);
void launch_bias_nbar(const ScalarArgs& a, int region, int nz, int nch, cudaStream_t s);
void launch_abar(const ScalarArgs& a, int region, int nblk, int nch, cudaStream_t s);
// reuse = 1: after an accepted HMC move the first gradient takes the move's last force stage
void launch_jump_begin(const ScalarArgs& a, int reuse, int nch, cudaStream_t s);
// reduce the jump gradient and likelihood partials, then the leapfrog update of `kind` (one launch)
void launch_jump_step(const ScalarArgs& a, int r_grad, int nx, int r_lik, int r_lik_move, int nz, int kind,
                      int nch, cudaStream_t s);
void launch_reduce_to(const ScalarArgs& a, int region, int nblk, int count, double scale, double* out_dev,
                      cudaStream_t s);
void launch_record(const ScalarArgs& a, double* rec_dev, int rec_len, long long iter_stride, int chain0, int nch,
                   cudaStream_t s);
void launch_advance(DevState* ds, int nch, cudaStream_t s);
// running sums of the chain parameters x = (P, b, Nbar) of one chain: acc[0] += 1,
// acc[1 + i] += x_i, acc[1 + D + i D + j] += x_i x_j, D = n_bins + 2 nsub
void launch_param_moments(const ScalarArgs& a, double* acc, cudaStream_t s);
// per voxel mean = mom[i] / n and var = mom[nv + i] / n - mean^2 (either output may be NULL)
void launch_moments_finish(const double* mom, long long nv, double n, double* mean, double* var, int blocks,
                           cudaStream_t s);
// activate an uploaded survey: data constants from the data kernel's partials
// (4 x nblk per subsample, chains cstride apart) and DevState::dslot = slot, or
// ST_BADDATA for invalid data
void launch_commit_data(DevState* ds, const double* part, long long cstride, int nblk, int slot, int nch,
                        cudaStream_t s);
void launch_reset_rec(DevState* ds, int nch, cudaStream_t s);
// per mass bin j < n_mass: DevState::mstat[j] += (or mstat2[j] =, when `final`) the sum of partials
void launch_mstat(const ScalarArgs& a, int region, int nblk, int n_mass, int final_, int nch, cudaStream_t s);
void launch_zero_dc(float2* spec, cudaStream_t s);

enum JumpKind { J_FIRST = 0, J_MID = 1, J_LAST = 2 };

// bounded-wait self-test: a wait that no copy completes, limited to limit_ns;
// sets ST_TIMEOUT in ds->status (bps_draws.cu)
void launch_wait_probe(DevState* ds, unsigned long long limit_ns, cudaStream_t s);

// Device copy of the mass-preconditioner network for inference inside the
// Gibbs iteration (bps_mlp.cu).  Before a move, launch_mass_net writes
// DevState::mass_scale[j] = exp(clamp(net(z)_j)) per chain, with z the
// standardised features [ln P_m, wfeat_m] of the chain's current state.
struct MassNet;
bps_status massnet_create(const bps_mlp* net, const float* mean, const float* sd, double log_clamp, MassNet** out);
void massnet_destroy(MassNet* m);
int massnet_width(const bps_mlp* net, int output);   // input width (output = 0) or output width (1)
void launch_mass_net(const ScalarArgs& a, const MassNet* m, int nch, cudaStream_t s);

// Power-spectrum bins (bps_api.cu), the one definition every entry point uses:
// n_bins linear bins in |n| over (0, sqrt(3) N / 2], binned on the integer |n|^2.
int bin_of_host(long long n2, int N, int nb);
// thresholds thr[m] = smallest |n|^2 of bin m (and full-grid mode counts when
// nmodes is not NULL); false when a bin has no threshold or, with nmodes, no mode
bool bin_tables(int N, int nb, int* thr, double* nmodes);
// every bin holds at least one wave vector of the grid (N <= 512; no allocation)
bool bins_have_modes(int N, int nb, const int* thr);

// Artificial surveys (bps_mock.cu): what the context-bound mock calls need of
// a single-chain context (its transforms, W as scratch, a small table buffer).
struct MockView {
  int N, zp, n_sub, n_sm;
  double box;
  cudaStream_t stream;
  const PassTable* pt;
  const Fields* f;
  uint64_t* launches;
  void* owner;
  bps_status (*scratch)(void* owner, size_t bytes, void** out);   // device buffer of >= bytes
  bps_status get_scratch(size_t bytes, void** out) const { return scratch(owner, bytes, out); }
};
bps_status mock_field(const MockView& v, uint64_t seed, const double* P_n2, float* delta_dev);
bps_status mock_counts(const MockView& v, uint64_t seed, const float* delta_dev, const float* R_dev, const double* b,
                       const double* nbar, int noise, int32_t* counts_dev);
bps_status mock_response(const MockView& v, double f_sky, const double* axis, int n_r, const double* table,
                         float* R_dev);

// Text returned by bps_last_error(NULL) for context-free calls.
void set_last_error(const char* msg);

}  // namespace bps
