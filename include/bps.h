/*
 * bps.h - C ABI of the GB300 sampler for joint Bayesian inference of a 3D
 * density field, its power spectrum, galaxy biases and normalisations
 * (Jasche & Wandelt, arXiv:1306.1821).
 *
 * Scope: the data-parallel hot path of the paper's multiple-block sampler
 * (Sec. 3.2, Eq. multiblock; Fig. 1):
 *   - the Hybrid Monte Carlo move of the density field (Sec. 4.1, Eqs.
 *     Potential..acceptance_rule, Wiener_Posterior_psi, Wiener_Posterior_force,
 *     Mass_matrix), whose force alternates 3D real-to-complex FFTs that apply the
 *     inverse-power-spectrum prior per mode with the voxel-local likelihood of
 *     the data model N = Nbar R (1 + b delta) + noise (Eq. data_model,
 *     Eq. LH_all_dataset);
 *   - the k-binned power and per-subsample reductions that feed the power
 *     spectrum draw (Sec. 3.4, Eq. INVERSE_GAMMA; Sec. 4.2, Eq. XI_SQUARE), the
 *     bias draw (Sec. 3.5, App. B), the normalisation draw (Sec. 3.6, Eq.
 *     GIG_post, App. A) and the deterministic P-delta jump (Sec. 4.3, Eqs.
 *     det_trans, mixing_pdf; App. C).
 *
 * Conventions (App. C.1): forward transform unnormalised, inverse 1/N^3.
 * Grid: N^3 voxels, x slowest, z fastest.  Fourier fields are half spectra
 * [N][N][N/2+1] complex (interleaved re, im).  Power-spectrum bins are
 * n_bins linear bins in |n| over (0, sqrt(3) N / 2], |n| the integer wave
 * vector; the k = 0 mode is held at zero.
 *
 * Memory: every pointer named *_dev is a CUDA device pointer on the current
 * device; every other array pointer is host memory.  The caller keeps
 * ownership of what it passes; the library copies what it keeps.  The library
 * owns all of its internal device buffers (allocated in bps_create and
 * bps_set_data, released in bps_destroy).  All work is ordered on the stream
 * given to bps_create; a call that returns host values synchronises that
 * stream before returning.
 *
 * Errors: every call returns a bps_status; nothing is thrown across the ABI.
 * After an error the context keeps the last accepted state and
 * bps_last_error() describes the failure.
 *
 * Random numbers: Philox4x64-10 (Salmon et al., SC'11) with counter
 * (element block, iteration, stage, sub) and key (seed, 0).  Each public step
 * call draws at the context's current iteration and then advances it by one;
 * bps_gibbs_iterate runs all stages of one iteration at one counter value.
 */
#ifndef BPS_H
#define BPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bps_ctx bps_ctx;

typedef enum {
  BPS_OK = 0,
  BPS_EINVAL = 1,    /* invalid argument, size, layout or data */
  BPS_ENOMEM = 2,    /* device allocation failed */
  BPS_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
  BPS_ENUMERIC = 4,  /* a non-finite energy or draw; the move was rejected */
  BPS_ETIMEOUT = 5,  /* a bounded device wait expired */
  BPS_ESTATE = 6     /* call out of order (e.g. a step before bps_set_data) */
} bps_status;

/* Sampler settings (Sec. 4.1.2 trajectory, Sec. 3.4 prior exponent alpha). */
typedef struct {
  int n_bins;              /* power-spectrum bins, 1..64 */
  double alpha;            /* power-law prior P^-alpha (alpha = 1: Jeffreys, Sec. 3.4) */
  int n_leapfrog;          /* leapfrog steps per HMC move */
  double eps_max;          /* step size eps = eps_max * u, u ~ U(0,1) per move */
  int jump;                /* 1: run the P-delta jump in bps_gibbs_iterate (Sec. 4.3) */
  int jump_leapfrog;       /* leapfrog steps of the jump's HMC in ln P */
  double jump_eps_max;     /* step size bound of the jump's HMC */
  int fixed_bias_index;    /* bias held fixed (b-P degeneracy gauge); -1: none */
  int mass_mode;           /* 0: diagonal Fourier mass of Eq. Mass_matrix;
                              1: that mass times per-bin scales (bps_set_mass_scale);
                              bps_set_mass_net installs a network mass in either mode */
  uint64_t seed;           /* Philox key */
} bps_config;

typedef struct {
  int accepted;            /* 1 if the proposal was accepted (Eq. acceptance_rule) */
  double dH;               /* H(proposal) - H(start), FP64 */
  double eps;              /* step size used */
} bps_move_info;

/* Create a context for an N^3 grid of side box_len (Mpc/h) with n_sub galaxy
 * subsamples (Sec. 2, Sec. 3.3.2).  N in {8, 16, 32, 64, 96, 128, 256};
 * 1 <= n_sub <= 16.  cuda_stream is a cudaStream_t (NULL: the legacy default
 * stream).  Returns BPS_EINVAL for an unsupported N, a bin layout with an empty
 * bin, or out-of-range settings; BPS_ENOMEM if the device buffers do not fit.
 * Creation also picks the tile size of the force z pass (bps_z_line_pairs). */
bps_status bps_create(int grid_n, double box_len, int n_sub, const bps_config* cfg,
                      void* cuda_stream, bps_ctx** out);

/* Survey data (Eq. data_model): counts_dev int32 [n_sub][N][N][N] (galaxy
 * counts N^l_i, 0..65535) and R_dev float32 [n_sub][N][N][N] (survey response
 * R^l_i = C^l_i F^l_i >= 0).  Copied into library buffers; the per-subsample
 * constants sum R, sum N^2/R and N_obs (Sec. 3.6) are computed here, and so is
 * the support of each z line (the range of voxels with R > 0 in some
 * subsample), outside which a = c = 0 and the kernels read no data.  Waits for
 * the upload and for any survey staged before it (bps_stage_data_host_u16).
 * BPS_EINVAL if R < 0 or non-finite, a count is negative or above 65535, a
 * voxel has R = 0 and a count > 0, or a subsample has no observed voxel; the
 * chain then has no data until a valid survey is set. */
bps_status bps_set_data(bps_ctx* ctx, const int32_t* counts_dev, const float* R_dev);

/* Same as bps_set_data from host arrays (pageable or pinned).  Subsamples are
 * copied one at a time through two device staging slots on copy streams, the
 * copy of one overlapping the check of the previous. */
bps_status bps_set_data_host(bps_ctx* ctx, const int32_t* counts, const float* R);

/* Same with the counts as uint16 [n_sub][N][N][N] (the library's own storage
 * width; counts are bounded by 65535 in any case): a quarter less to copy, and
 * the arrays are copied straight into the library's buffers and checked there. */
bps_status bps_set_data_host_u16(bps_ctx* ctx, const uint16_t* counts, const float* R);

/* Starts the upload of a survey (counts uint16 and R float32 [n_sub][N][N][N],
 * host arrays, as for bps_set_data_host_u16) into the context's second data
 * slot and returns without waiting: copies and data check run on the
 * context's own streams, beside whatever the caller queues next.  The next
 * call that uses the data (bps_gibbs_iterate, bps_hmc_step, bps_sample_*,
 * bps_jump, bps_gradient, ...) first activates the oldest staged survey: it
 * waits for the upload, takes the data constants of Sec. 3.6 from the check
 * and rebuilds a and c (Eq. Wiener_Posterior_force).  A survey that fails the
 * checks of bps_set_data is not activated; the call that met it returns
 * BPS_EINVAL, having run on the previous survey.  At most two surveys can be
 * staged ahead (BPS_ESTATE otherwise); the host arrays must stay unchanged
 * until the call that activates them returns.  With pinned host memory the
 * copies overlap the Gibbs iterations queued after them, so the upload of
 * survey k + 1 can run during iteration k. */
bps_status bps_stage_data_host_u16(bps_ctx* ctx, const uint16_t* counts, const float* R);

/* Chain state (Sec. 3.2): delta_dev float32 [N][N][N] real field (its mean is
 * dropped: the k = 0 mode is held at zero), P [n_bins], b [n_sub], nbar [n_sub]
 * host FP64, and the iteration counter of the random streams.  P also becomes
 * the reference spectrum of the jump's mass.  Rebuilds the local fields
 * a = sum_l b_l^2 Nbar_l R^l and c = sum_l b_l (N^l - Nbar_l R^l)
 * (Eq. Wiener_Posterior_force).  delta_dev may be NULL (keeps the field). */
bps_status bps_set_state(bps_ctx* ctx, const float* delta_dev, const double* P, const double* b,
                         const double* nbar, uint64_t iteration);

/* Read the state back.  Any output pointer may be NULL. */
bps_status bps_get_state(bps_ctx* ctx, float* delta_dev, double* P, double* b, double* nbar,
                         uint64_t* iteration);

/* Half spectrum of the current field, complex64 [N][N][N/2+1] (device). */
bps_status bps_get_spectrum(bps_ctx* ctx, float* spec_dev);
/* Replace the current field by a half spectrum (device); k = 0 is zeroed. */
bps_status bps_set_spectrum(bps_ctx* ctx, const float* spec_dev);

/* Checkpoint and resume of one chain (Sec. 3.2: the state of the multiple-block
 * scan).  The checkpoint holds the field's half spectrum (its exact FP32 bits),
 * P, b, Nbar, the jump's reference spectrum (bps_set_state), the iteration
 * counter of the random streams, eps_max (bps_adapt_step_size may have changed
 * it) and the mass multipliers of bps_set_mass_scale.  Loaded into a context
 * created with the same grid, box, subsamples and settings, holding the same
 * survey, the chain continues bit for bit as if it had not been interrupted.
 * The survey and a network mass (bps_set_mass_net, bps_set_preconditioner) are
 * not part of it: set them on the new context first.  bps_save_chain: blob
 * NULL makes *bytes receive the size needed; otherwise *bytes is the capacity
 * of blob (host) and receives the size written.  bps_load_chain returns
 * BPS_EINVAL for a blob of another format, grid, box, subsample or bin count.
 * Single-chain contexts. */
bps_status bps_save_chain(bps_ctx* ctx, void* blob, size_t* bytes);
bps_status bps_load_chain(bps_ctx* ctx, const void* blob, size_t bytes);

/* One HMC move of the density field (Sec. 4.1): momenta drawn afresh
 * (p ~ N(0, M), M diagonal in Fourier space, M_k = V_cell/P_k + abar),
 * n_leapfrog kick-drift-kick steps of size eps_max * u, Metropolis accept in
 * FP64 (Eq. acceptance_rule).  info may be NULL (then nothing synchronises). */
bps_status bps_hmc_step(bps_ctx* ctx, bps_move_info* info);

/* Burn-in adaptation of the step size (the paper's chains settle at about 92%
 * acceptance after burn-in, Fig. accept_rat; it gives no tuning rule, so this
 * one is the library's): n_rounds rounds of moves_per_round HMC moves
 * (real moves of the chain, advancing its iteration counter), after each a
 * Robbins-Monro step on ln eps_max toward the acceptance rate `target`
 * (0 < target < 1) with gain 2 / sqrt(round), at most a factor 2 per round.
 * The adapted eps_max replaces the configured one from then on;
 * eps_max_out (host, may be NULL) receives it.  Single-chain contexts. */
bps_status bps_adapt_step_size(bps_ctx* ctx, int n_rounds, int moves_per_round, double target,
                               double* eps_max_out);

/* Power-spectrum draw (Sec. 4.2): sigma_m = (V_cell/N^3) sum_{k in m} |delta_k|^2
 * over the full grid, x_m ~ chi^2 with beta_m = n_m + 2 alpha - 2 degrees of
 * freedom, P_m = sigma_m / x_m.  P_out [n_bins] and sigma_out [n_bins] (host)
 * may be NULL. */
bps_status bps_sample_power(bps_ctx* ctx, double* P_out, double* sigma_out);

/* Bias and normalisation draws (Secs. 3.5-3.6, Apps. A-B): b_l ~ N(D/C, 1/C)
 * with C = Nbar sum R delta^2, D = sum (N - Nbar R) delta (except the fixed
 * index), then Nbar_l ~ GIG(1 - N_obs/2, sum R (1 + b delta)^2, sum N^2 / R),
 * sums over R > 0; then the local fields are rebuilt.  Outputs (host, may be
 * NULL): b_out [n_sub], nbar_out [n_sub], sums_out [n_sub][3] = (sum N delta,
 * sum R delta, sum R delta^2). */
bps_status bps_sample_bias_norm(bps_ctx* ctx, double* b_out, double* nbar_out, double* sums_out);

/* Deterministic P-delta jump (Sec. 4.3, App. C): with u = delta/sqrt(lambda)
 * fixed, an HMC in theta = ln P of jump_leapfrog steps targets
 * P^-alpha x likelihood(delta(u, P)); on acceptance delta_k <- sqrt(P'/P) delta_k
 * (Eq. det_trans).  info may be NULL. */
bps_status bps_jump(bps_ctx* ctx, bps_move_info* info);

/* n_iter full Gibbs iterations: HMC -> P -> [jump] -> b -> Nbar (Sec. 3.2).
 * chain_out (host, may be NULL) receives per iteration n_bins P values, n_sub
 * b, n_sub Nbar, then dH and accepted of the HMC move:
 * n_iter * (n_bins + 2 n_sub + 2) doubles. */
bps_status bps_gibbs_iterate(bps_ctx* ctx, int n_iter, double* chain_out);

/* ---- batches of independent chains (many small surveys in one launch) ----
 * A batch holds n_chains chains, each with its own grid (grid_n[j] in the set
 * of bps_create), box (box_len[j]), subsamples (n_sub[j]) and Philox key
 * cfg->seed + j; every other setting of cfg is shared.  Chains of equal grid
 * size form one group whose field passes and scalar stages are single launches
 * over all of the group's chains, and one Gibbs iteration of the whole batch is
 * one CUDA graph replay.  The single-chain calls above do not accept a batch
 * context; bps_destroy and bps_set_mass_scale do. */
bps_status bps_create_batch(int n_chains, const int* grid_n, const double* box_len, const int* n_sub,
                            const bps_config* cfg, void* cuda_stream, bps_ctx** out);

/* Data and state of chain `chain` (as bps_set_data followed by bps_set_state). */
bps_status bps_batch_set_chain(bps_ctx* batch, int chain, const int32_t* counts_dev, const float* R_dev,
                               const float* delta_dev, const double* P, const double* b,
                               const double* nbar, uint64_t iteration);

/* State of chain `chain` (as bps_get_state). */
bps_status bps_batch_get_chain(bps_ctx* batch, int chain, float* delta_dev, double* P, double* b,
                               double* nbar, uint64_t* iteration);

/* n_iter Gibbs iterations of every chain.  chain_out (host, may be NULL):
 * [n_iter][n_chains][bps_batch_record_len] doubles; the record of chain j sits
 * in slot bps_batch_record_slot(j) and holds n_bins P, n_sub(j) b, n_sub(j)
 * Nbar, dH, accepted (the tail beyond a chain's record is unused). */
bps_status bps_batch_gibbs_iterate(bps_ctx* batch, int n_iter, double* chain_out);
int bps_batch_record_len(const bps_ctx* batch);
int bps_batch_record_slot(const bps_ctx* batch, int chain);

/* Posterior statistics of the density modes, the training targets of the
 * mass preconditioner: n_moves HMC moves of every chain (ctx single or batch;
 * the power spectrum, biases and normalisations stay fixed), then per chain and
 * mass bin j (n_mass_bins linear bins in |n|, as for P) out receives
 *   V_j    = mean over the bin's full-grid modes of Var(delta_k) / N^3 and
 *   Mbar_j = mean of the diagonal mass V_cell / P_k + abar over the same modes,
 * at out[slot * 2 n_mass_bins + j] and out[slot * 2 n_mass_bins + n_mass_bins + j]
 * (host; slot 0 for a single context, bps_batch_record_slot(j) for a batch).
 * The variance estimate is the sample variance of the chain's states.  Also
 * installs n_mass_bins as the mass-bin layout (as bps_set_mass_scale does).
 * BPS_EINVAL if a mass bin holds no mode (the first bin must reach |n| = 1,
 * so n_mass_bins < sqrt(3) N / 2), or if a network mass is installed and n_mass_bins
 * differs from its output width. */
bps_status bps_mass_stats(bps_ctx* ctx, int n_moves, int n_mass_bins, double* out);

/* Binned power of the survey window, a feature of the mass preconditioner:
 * out[slot * n_bins + m] = sigma_m of a / abar, with a = sum_l b_l^2 Nbar_l R^l
 * the local curvature of Eq. Wiener_Posterior_force and sigma_m as in
 * bps_sample_power (host; slots as in bps_mass_stats). */
bps_status bps_window_power(bps_ctx* ctx, double* out);

/* Per-bin multipliers s_m of the diagonal mass for mass_mode = 1 (a
 * preconditioner choice: the mass affects efficiency, not validity,
 * Sec. 4.1.2).  scales [n_mass_bins] host, 1 <= n_mass_bins <= 64, bins
 * linear in |n| as for P. */
bps_status bps_set_mass_scale(bps_ctx* ctx, int n_mass_bins, const double* scales);

/* Network mass: from now on, before every HMC move of every chain (ctx single
 * or batch), the per-bin multipliers s_j of the diagonal mass are recomputed on
 * the device by `net` from the chain's current state, inside the Gibbs
 * iteration's launch sequence (no host round trip):
 *   z = clamp((f - feat_mean) / feat_std, -4, 4),
 *   f = [ln P_0 .. ln P_{n_bins-1}, ln W_0 .. ln W_{n_bins-1}],
 *   s_j = exp(clamp(net(z)_j, -log_clamp, log_clamp)),
 * with W_m the binned window power of bps_window_power, computed here once per
 * chain.  The mass depends on P, not on delta, so each move still leaves the
 * conditional of delta invariant (Sec. 4.1.2: the mass changes efficiency
 * only).  net: input width 2 n_bins, output width = number of mass bins
 * (1..64, linear in |n| as for P); its parameters are copied (later training
 * of `net` does not affect ctx).  feat_mean, feat_std: host float [2 n_bins].
 * net = NULL returns ctx to the mass of its configuration.  The data of every
 * chain must be set. */
typedef struct bps_mlp bps_mlp;
bps_status bps_set_mass_net(bps_ctx* ctx, const bps_mlp* net, const float* feat_mean, const float* feat_std,
                            double log_clamp);

/* Install a trained preconditioner saved with bps_mlp_export (the library's
 * own format: the network, its feature standardisation and the clamp) as the
 * network mass of ctx, exactly as bps_set_mass_net with those arguments.
 * BPS_EINVAL if blob (host, `bytes` long) is not in that format. */
bps_status bps_set_preconditioner(bps_ctx* ctx, const void* blob, size_t bytes);

/* The mass multipliers in use by chain `chain` (0 for a single context):
 * *n_mass_bins receives their number, scales (host double [64]) the values. */
bps_status bps_get_mass_scale(bps_ctx* ctx, int chain, int* n_mass_bins, double* scales);

/* ---- the mass-preconditioner network ----
 * A multilayer perceptron (ReLU hidden layers, linear output) that maps binned
 * features of a problem to per-bin log multipliers of the diagonal mass (for
 * bps_set_mass_scale).  The paper keeps the Fourier diagonal of Eq.
 * Mass_matrix and notes the mass changes efficiency only (Sec. 4.1.2); the
 * network is this library's way to choose better multipliers.  Matrix products
 * use BF16 operands with FP32 accumulation on the tensor cores; parameters and
 * Adam moments are FP32.  Parameters are one FP32 vector, layer by layer: W_l
 * [n_l][n_{l+1}] row-major, then b_l [n_{l+1}].  Loss: mean squared error. */
/* sizes[0..n_layers]: input, hidden..., output widths (each 1..512; 1..4 layers). */
bps_status bps_mlp_create(int n_layers, const int* sizes, void* cuda_stream, bps_mlp** out);
size_t bps_mlp_num_params(const bps_mlp* net);
bps_status bps_mlp_set_params(bps_mlp* net, const float* params);   /* host; resets Adam */
bps_status bps_mlp_get_params(bps_mlp* net, float* params);         /* host */
/* y_dev [batch][n_out] = network(x_dev [batch][n_in]) (device arrays). */
bps_status bps_mlp_forward(bps_mlp* net, int batch, const float* x_dev, float* y_dev);
/* Loss and parameter gradients for one batch; loss (host double) and grads
 * (host float [num_params]) may be NULL.  Keeps the gradients for bps_mlp_adam_step. */
bps_status bps_mlp_loss_grad(bps_mlp* net, int batch, const float* x_dev, const float* t_dev, double* loss,
                             float* grads);
/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected) with the last gradients. */
bps_status bps_mlp_adam_step(bps_mlp* net, float lr);
/* `steps` Adam steps on minibatches of `batch` rows drawn with replacement from
 * the n_examples rows of x_dev / t_dev (Philox key `seed`); last_loss (host, may
 * be NULL) receives the loss of the last minibatch. */
bps_status bps_mlp_train(bps_mlp* net, int n_examples, const float* x_dev, const float* t_dev, int batch,
                         int steps, float lr, uint64_t seed, double* last_loss);
/* Save net with its feature standardisation (host float [input width] each) and
 * log_clamp in the library format for bps_set_preconditioner.  blob NULL:
 * *bytes receives the size needed; else *bytes is the capacity of blob (host)
 * and receives the size written. */
bps_status bps_mlp_export(bps_mlp* net, const float* feat_mean, const float* feat_std, double log_clamp, void* blob,
                          size_t* bytes);
void bps_mlp_destroy(bps_mlp* net);

/* ---- building blocks of the path, for verification ---- */

/* Forward 3D transform of a real field (Eq. FFT, C_hat = 1):
 * real_dev float32 [N][N][N] -> spec_dev complex64 [N][N][N/2+1]. */
bps_status bps_fft_r2c(bps_ctx* ctx, const float* real_dev, float* spec_dev);
/* Inverse 3D transform (Eq. IFFT, C = 1/N^3): spec_dev -> real_dev. */
bps_status bps_fft_c2r(bps_ctx* ctx, const float* spec_dev, float* real_dev);

/* Force of the current state in Fourier space, grad_dev complex64
 * [N][N][N/2+1]: delta_k / lambda_k + FFT(a delta - c)_k (Eq.
 * Wiener_Posterior_force), k = 0 set to 0.  energies (host, may be NULL)
 * receives (prior term, likelihood term) of Eq. Wiener_Posterior_psi up to a
 * constant. */
bps_status bps_gradient(bps_ctx* ctx, float* grad_dev, double* energies);

/* n_words 64-bit Philox outputs for counter (block0 + i/4, iteration, stage,
 * sub), word i%4, into out_dev (uint64 device array). */
bps_status bps_philox_words(uint64_t seed, uint64_t iteration, uint64_t stage, uint64_t sub,
                            uint64_t block0, size_t n_words, uint64_t* out_dev, void* cuda_stream);

/* The momentum normals of one move: n float32 normals of stream
 * (seed, iteration, stage 1, sub 0), element i from block i/8. */
bps_status bps_voxel_normals(uint64_t seed, uint64_t iteration, size_t n, float* out_dev,
                             void* cuda_stream);

/* k-bin power without device allocation.  The paper has no counterpart: this
 * is a deployment variant of the sigma_m reduction behind bps_sample_power,
 * for callers that may not allocate device memory at all, neither directly nor
 * through this library (for example a host framework whose own pool must
 * account for every device byte, or a loop that cannot afford cudaMalloc's
 * implicit synchronisation).  It computes, for the half spectrum spec_dev
 * (complex64 [N][N][N/2+1], device), sigma_m = (V_cell/N^3) sum_{k in m} w_k
 * |spec_k|^2 into sigma_dev (n_bins doubles, device), with the bins of
 * bps_create and w_k the half-spectrum multiplicity; nothing is drawn and no
 * context is needed.  The caller passes input and output; the library keeps
 * its per-block partial sums in one file-scope device array of 1024 x 64
 * doubles (512 KiB), which every GPU that loads the library holds until the
 * process exits.  Limits: N even in 4..512, 1 <= n_bins <= 64, every bin
 * holding at least one wave vector of the grid (the bins of bps_create, checked
 * the same way), spec_dev and sigma_dev 8-byte aligned: BPS_EINVAL otherwise,
 * text in bps_last_error(NULL).  A CUDA error already pending in the calling
 * thread is reported as BPS_ECUDA and left pending; nothing is launched.  The
 * first call on each device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress) in the device's primary context and
 * caches it; make that first call before any stream capture.  The cache is not
 * renewed: calls after cudaDeviceReset of that device, or from a non-primary
 * context, are not supported.  No call allocates or frees anything.  All calls
 * share the array:
 * calls whose kernels overlap on the GPU (different streams, or other host
 * threads) race and must be serialised by the caller.  Work is queued on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream); the call does not
 * synchronise. */
bps_status bps_bin_power_noalloc(int grid_n, double box_len, int n_bins, const float* spec_dev,
                                 double* sigma_dev, void* cuda_stream);

/* ---- artificial surveys (Sec. 5; App. D; Eq. rel_bias) ----
 * Generated on the device, for fast sweeps over survey configurations; the
 * random numbers come from Philox4x64-10 with key `seed`, stage 8 for the field
 * and stage 9 for the counts, so any implementation of the same definitions
 * reproduces them.  Each call works on the single-chain context's grid (N, box,
 * n_sub of bps_create), queues on its stream and does not synchronise; the
 * context keeps one small device table for them until bps_destroy. */

/* True density field (Sec. 5): delta = IFFT(A_k FFT(xi)), A_k = sqrt(P_k /
 * V_cell) (forward transform unnormalised, inverse 1/N^3, so E|delta_k|^2 =
 * N^3 P_k / V_cell as in the prior of Eq. dens_prior), with xi the FP32 normals
 * of stream (seed, 0, 8, 0) laid out as in bps_voxel_normals.  P_n2 (host,
 * 3 (N/2)^2 + 1 doubles) is the power at every integer |n|^2 (P_n2[0] is
 * ignored: the k = 0 mode is zero); delta_dev float32 [N][N][N] (device).
 * BPS_EINVAL for a negative or non-finite P. */
bps_status bps_mock_field(bps_ctx* ctx, uint64_t seed, const double* P_n2, float* delta_dev);

/* Galaxy counts of every subsample l (Eq. data_model) from the true field
 * delta_dev and the response R_dev (float32 [n_sub][N][N][N], device), with
 * b[l], nbar[l] (host):
 *   noise 0: N ~ Poisson(lambda), lambda = (R Nbar) max(0, 1 + b delta), drawn by
 *     inversion of the Poisson distribution function in chunks of mean <= 32
 *     (their sum is Poisson with the summed mean), in FP64 operations that IEEE
 *     754 rounds exactly (e^-mu by halving, a degree-10 Taylor series and ten
 *     squarings); chunk j of voxel i reads word j % 4 of block
 *     (i, j / 4, 9, l).  A mean above 4096 gives the count 65536, which
 *     bps_set_data rejects.
 *   noise 1: the paper's Gaussian noise (Sec. 5, Eq. cov_mat_noise),
 *     N = Nbar R (1 + b delta) + sqrt(Nbar R) z, z the FP64 Box-Muller normal of
 *     words 0, 1 of block (i, 0, 9, l), rounded to the nearest integer (halves
 *     up) and clipped at 0, since counts are stored as integers.
 * counts_dev int32 [n_sub][N][N][N] (device). */
bps_status bps_mock_counts(bps_ctx* ctx, uint64_t seed, const float* delta_dev, const float* R_dev, const double* b,
                           const double* nbar, int noise, int32_t* counts_dev);

/* Survey response R^l_i = C_i f^l(r_i) (Sec. 5, the equation for R^l_i): the
 * completeness C is a spherical cap of sky fraction f_sky about axis[3]
 * (host; cos(theta) >= 1 - 2 f_sky, the SDSS mask itself is not available)
 * inside r <= box/2 about the box centre (the observer); f^l is the table
 * (host, [n_sub][n_r] doubles) of the radial selection at r_j = j (box/2) /
 * (n_r - 1), interpolated linearly.  All geometry in FP64 without fused
 * operations, so the zero pattern is exact.  R_dev float32 [n_sub][N][N][N]. */
bps_status bps_mock_response(bps_ctx* ctx, double f_sky, const double* axis, int n_r, const double* table,
                             float* R_dev);

/* Schechter luminosity function (App. D) and the apparent-magnitude limits of
 * a flux-limited survey (Sec. 5): Phi(M) dM = 0.4 ln10 Phi_* x^(alpha+1) e^-x dM,
 * x = 10^(0.4 (M_star - M)), magnitudes M - 5 log10 h. */
typedef struct {
  double M_star;    /* -20.44 in the paper */
  double alpha;     /* -1.05 */
  double m_bright;  /* 14.5 */
  double m_faint;   /* 17.77 */
  double omega_m;   /* flat LCDM for the luminosity distance (0.24) */
} bps_schechter;

/* Radial selection tables and mean numbers of n_sub absolute-magnitude bins
 * [M_edges[l], M_edges[l+1]] (host, increasing: brightest first), host code:
 *   table[l][j] = int_{M_lo(r_j)}^{M_hi(r_j)} Phi dM / int_{M_edges[l]}^{M_edges[l+1]} Phi dM
 * with r_j = j r_max / (n_r - 1) comoving (Mpc/h) and [M_lo, M_hi] the part of
 * the bin whose apparent magnitude m = M + 5 log10(D_L) + 25 lies within
 * [m_bright, m_faint], D_L = (1 + z) r (flat LCDM, no K-correction); and
 * nbar_rel[l] = int over the bin of Phi with Phi_* = 1 (Sec. 5: Nbar^l is this
 * integral times Phi_*; may be NULL).  Integrals by composite 16-point
 * Gauss-Legendre quadrature. */
bps_status bps_schechter_tables(const bps_schechter* s, int n_sub, const double* M_edges, double r_max, int n_r,
                                double* table, double* nbar_rel);

/* Luminosity-dependent bias, Eq. rel_bias: b_out[l] = b_star (a + b 10^(0.4
 * (M_star - M[l])) + c (M[l] - M_star)) (host arrays; the paper uses a = 0.895,
 * b = 0.105, c = -0.040, M_star = -20.83, b_star = 1.2). */
bps_status bps_bias_law(int n, const double* M, double b_star, double M_star, double a, double b, double c,
                        double* b_out);

/* Library version string and the text of the last error of ctx (or, when ctx
 * is NULL, of the calling thread's last failed call).  The text stays valid
 * until the next failure on ctx (or on the calling thread). */
const char* bps_version(void);
const char* bps_last_error(const bps_ctx* ctx);

/* Number of kernels this context has launched (for launch accounting). */
uint64_t bps_kernel_launches(const bps_ctx* ctx);

/* Per-kernel timing of the leapfrog passes of bps_hmc_step / bps_gibbs_iterate:
 * with enable = 1 the library records a CUDA event pair around every launch of
 * the four leapfrog kernels (0: x pass with kick/drift, 1: y inverse, 2: z pass
 * with the local force, 3: y forward) on the context's stream.  In
 * bps_gibbs_iterate a profiled iteration replays its own captured CUDA graph,
 * the iteration with event-record nodes around those kernels, and the times are
 * read after each replay (a host synchronisation per profiled iteration); the
 * kernels run as in an unprofiled replay, without host launch gaps.
 * bps_profile_read synchronises the stream and returns, per kernel kind, the
 * summed device milliseconds ms[4] and the launch counts n[4] since the last
 * read (then resets them).  Timing only; results are unchanged. */
bps_status bps_profile(bps_ctx* ctx, int enable);
bps_status bps_profile_read(bps_ctx* ctx, double* ms, uint64_t* n);

/* Running posterior moments on the device (the paper's posterior analysis,
 * Secs. 6.2 and 7, Figs. 6-11: ensemble mean and variance maps of the density
 * field, correlation matrices of P, b and Nbar).  With enable = 1 the sums are
 * reset and, from then on, every Gibbs iteration of bps_gibbs_iterate adds its
 * final sample: per voxel delta and delta^2 (FP64, the field transformed to real
 * space by one extra z pass) and the chain parameters x = (P_0..P_{n_bins-1},
 * b_0..b_{n_sub-1}, Nbar_0..Nbar_{n_sub-1}) and their products x_i x_j (FP64).
 * enable = 0 stops adding (the sums are kept).  Uses 16 N^3 + 8 (1 + D + D^2)
 * bytes of device memory, D = n_bins + 2 n_sub.  Single-chain contexts. */
bps_status bps_posterior_moments(bps_ctx* ctx, int enable);

/* The moments accumulated so far over n = *n_samples iterations: per voxel
 * mean_dev = S1 / n and var_dev = S2 / n - mean^2 (double [N][N][N], device;
 * population moments), param_mean [D] and param_cov [D][D] (host; population
 * covariance, the order of bps_posterior_moments).  Any output may be NULL.
 * BPS_ESTATE before bps_posterior_moments or before the first iteration. */
bps_status bps_posterior_read(bps_ctx* ctx, double* mean_dev, double* var_dev, double* param_mean,
                              double* param_cov, uint64_t* n_samples);

/* Self-test of failure detection.  Every device wait of the library (the bulk
 * tile copies of the z and fused y/z passes complete on shared-memory
 * mbarriers) is bounded: after 2 s the block gives up, records the timeout in
 * the chain's status word and exits, and the next call that reads the status
 * returns BPS_ETIMEOUT with the context still usable.  This call runs that
 * path on purpose: one block waits on an mbarrier for 16 bytes that no copy
 * will deliver (none is issued, so nothing is in flight when it gives up),
 * with the wait limited to limit_ns (1..1e9).  Returns BPS_ETIMEOUT when the
 * wait ran out as it must; the chain's state is untouched. */
bps_status bps_selftest_wait(bps_ctx* ctx, uint64_t limit_ns);

/* Line pairs per tile (4, 8 or 16) of the force z pass of ctx (the first
 * group of a batch).  Chosen when the context is created: the first context of
 * a (GPU model, grid, number of chains) kind times the three tile sizes on its
 * own buffers, once transforming every line (a full-sky survey) and once with
 * the line supports of a centred ball of radius 0.45 N, and keeps the smallest
 * total; the choice is cached for the process and
 * in the JSON file named by BPS_TUNE_CACHE (default $HOME/.cache/bps_tune.json),
 * so that later contexts and runs reuse it.  BPS_AUTOTUNE=0 keeps 8.  The tile
 * size changes only the grouping of the likelihood-energy partial sums. */
int bps_z_line_pairs(const bps_ctx* ctx);

/* Implementation of the leapfrog x pass in use by ctx (the first group of a
 * batch): 0 loads its tiles straight into registers; 1, 2, 3 stage them in
 * shared memory with tensor copies (W, delta and p; W and delta; W only); 4
 * streams the delta and p rows through a two-slot ring of quarter tiles filled
 * by tensor copies while W is transformed; 5 fills the same ring with 16-byte
 * asynchronous copies issued by every thread; 6 gives each warp its own rows of
 * the ring (no block barrier per quarter).  The seven give bit-identical
 * results.  Chosen when the context is created, like bps_z_line_pairs: the
 * first context of a (GPU model, grid, number of chains) kind times the seven
 * and keeps the fastest, cached with the z-pass choice; BPS_XTMA = 0..6 forces
 * one, BPS_AUTOTUNE=0 keeps 0. */
int bps_x_pass_variant(const bps_ctx* ctx);

void bps_destroy(bps_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BPS_H */
