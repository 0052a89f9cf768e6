// Scalar stages of the multiple-block scan, run on the device so that a Gibbs
// iteration needs no host round trip: step size and Metropolis decisions of the
// HMC moves (Sec. 4.1, Eq. acceptance_rule), the chi^2 draw of the power
// spectrum (Sec. 4.2), the normal bias draw (Sec. 3.5, App. B), the GIG draw of
// the normalisations (Sec. 3.6, App. A) and the HMC in ln P of the jump
// (Sec. 4.3, App. C).  All decisions are taken in FP64 from Philox4x64-10
// words at fixed counters.
#include <math.h>

#include "bps_internal.h"
#include "bps_passes.cuh"

namespace bps {

constexpr int MAX_ATTEMPTS = 64;

// the scalar arguments of chain `ch` of a batch (blockIdx.y)
__device__ __forceinline__ ScalarArgs chain_args(ScalarArgs a, int ch) {
  a.ds += ch;
  a.part += ch * a.cstride;
  return a;
}

// Deterministic sum of n partials (stride 1) by one block of 256 threads;
// the value is valid in thread 0.
__device__ double sum_partials(const double* p, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v += p[i];
  return block_sum<256>(v, sh);
}

// ------------------------------------------------------------------ HMC move
__global__ void k_move_begin(ScalarArgs a0) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  DevState* ds = a.ds;
  const int t = threadIdx.x;
  if (t == 0) {
    P4 r = philox(0, ds->iteration, ST_HMC, 0, ds->seed);
    ds->eps = a.eps_max * u52(r.w[0]);
    ds->u_acc = u52(r.w[1]);
  }
  if (t < MAXB) {
    if (t < a.n_bins) {
      // lambda_m = P_m / V_cell (Eq. dens_prior in Fourier space); M = 1/lambda + abar (Eq. Mass_matrix)
      const double il = ds->vc / ds->P[t];
      const double M = il + ds->abar;
      ds->inv_lambda[t] = (float)il;
      ds->inv_M[t] = (float)(1.0 / M);
      ds->sqrt_M[t] = (float)sqrt(M);
    } else {
      ds->inv_lambda[t] = 0.f;
      ds->inv_M[t] = 0.f;
      ds->sqrt_M[t] = 0.f;
    }
    const double sc = t < a.n_mass ? ds->mass_scale[t] : 1.0;
    ds->inv_ms[t] = (float)(1.0 / sc);
    ds->sqrt_ms[t] = (float)sqrt(sc);
  }
}

// H = (1/2N^3) sum w (|p|^2/M + |delta|^2/lambda) + (1/2) sum (a delta^2 - 2 c delta)
// The eight sums of a move, one block each (on different SMs: each sum is a
// chain of FP64 additions), into the chain state's scratch: K0, E0, L0, K1, E1,
// L1, G0, G1 (the kinetic, prior and likelihood energies at the start and the
// end, and the two force norms of the leapfrog energy identity).
__global__ void k_move_sums(ScalarArgs a0, int r_init, int r_lik0, int r_final, int r_lik1, int nx, int nz) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  const double h = 0.5 * a.inv_nv;
  const double* p = nullptr;
  int n = nx;
  double scale = h;
  switch (blockIdx.x) {
    case 0: p = a.part + r_init; break;
    case 1: p = a.part + r_init + a.stride; break;
    case 2: p = a.part + r_lik0; n = nz; scale = 1.0; break;
    case 3: p = a.part + r_final; break;
    case 4: p = a.part + r_final + a.stride; break;
    case 5: p = a.part + r_lik1; n = nz; scale = 1.0; break;
    case 6: p = a.part + r_init + 2 * a.stride; scale = a.inv_nv; break;
    default: p = a.part + r_final + 2 * a.stride; scale = a.inv_nv; break;
  }
  const double s = sum_partials(p, n, sh);
  if (threadIdx.x == 0) a.ds->scratch[blockIdx.x] = s * scale;
}

__global__ void k_move_end(ScalarArgs a0) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  DevState* ds = a.ds;
  if (threadIdx.x == 0) {
    const double K0 = ds->scratch[0], E0 = ds->scratch[1], L0 = ds->scratch[2];
    const double K1 = ds->scratch[3], E1 = ds->scratch[4], L1 = ds->scratch[5];
    const double G0 = ds->scratch[6], G1 = ds->scratch[7];
    const double H0 = K0 + E0 + L0, H1 = K1 + E1 + L1;
    // H(end) - H(start) of Eq. acceptance_rule.  The potential of the density
    // move (Eq. Wiener_Posterior_psi with fixed P, b, Nbar) is exactly quadratic
    // in delta, and for kick-drift-kick leapfrog on a quadratic potential the
    // energy change telescopes exactly: each step changes H by
    // (eps^2/8)(g_{n+1}^T M^-1 g_{n+1} - g_n^T M^-1 g_n), so over the whole
    // trajectory dH = (eps^2/8)(g_L^T M^-1 g_L - g_0^T M^-1 g_0).  Both norms are
    // O(N^3) and their difference is multiplied by eps^2/8, so the FP32 terms
    // carry ~1e-8 into dH, where the difference H1 - H0 of two ~1e7-sized
    // energies carries the FP32 error of the transformed field (~1e-3 at
    // 256^3).  eps is the FP32 step the passes applied.  H0 and H1 are kept
    // for the finiteness check and for inspection.
    const double e32 = (double)(float)ds->eps;
    const double dH = 0.125 * e32 * e32 * (G1 - G0);
    ds->H0 = H0;
    ds->H1 = H1;
    ds->dH = dH;
    ds->lik0 = L0;
    ds->lik1 = L1;
    int acc = 0;
    if (!isfinite(dH) || !isfinite(H0) || !isfinite(H1)) {
      ds->status |= ST_NONFINITE;
    } else {
      acc = log(ds->u_acc) < -dH;   // Eq. acceptance_rule, FP64
    }
    ds->accepted = acc;
    if (acc) {
      ds->cur = 1 - ds->cur;
      ds->n_accepted += 1;
    }
    ds->n_moves += 1;
  }
}

// ------------------------------------------------------------------ P draw
// Gamma(shape) by Marsaglia & Tsang (ACM TOMS 2000); attempt j of bin m reads
// Philox block (m, iteration, ST_POWER, j): words 0,1 -> normal, word 2 -> uniform;
// shape < 1 uses Gamma(shape + 1) U^(1/shape) with U from word 3 of attempt 0.
__device__ double gamma_mt(double shape, uint64_t seed, uint64_t it, int m, int* fail) {
  const bool boost = shape < 1.0;
  const double aa = boost ? shape + 1.0 : shape;
  const double d = aa - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  double val = d;
  bool ok = false;
  for (int j = 0; j < MAX_ATTEMPTS && !ok; ++j) {
    P4 r = philox((uint64_t)m, it, ST_POWER, (uint64_t)j, seed);
    const double z = normal64(r.w[0], r.w[1]);
    const double t = 1.0 + c * z;
    if (t <= 0.0) continue;
    const double v = t * t * t;
    const double u = u52(r.w[2]);
    if (log(u) < 0.5 * z * z + d - d * v + d * log(v)) {
      val = d * v;
      ok = true;
    }
  }
  if (!ok) *fail = 1;
  if (boost) {
    P4 r = philox((uint64_t)m, it, ST_POWER, 0, seed);
    val *= exp(log(u52(r.w[3])) / shape);
  }
  return val;
}

// block m: sigma_m = (V_cell/N^3) sum_{k in m} w |delta_k|^2; then (draw) P_m = sigma_m / x,
// x ~ chi^2_beta = 2 Gamma(beta/2), beta = n_m + 2 alpha - 2 (Sec. 4.2, Eq. XI_SQUARE)
__global__ void k_power(ScalarArgs a0, int region, int nx, int draw) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  DevState* ds = a.ds;
  const int m = blockIdx.x;
  const double s = sum_partials(a.part + region + (size_t)m * a.stride, nx, sh);
  if (threadIdx.x == 0) {
    const double sigma = s * ds->vc * a.inv_nv;
    ds->sigma[m] = sigma;
    if (draw) {
      const double beta = ds->nmodes[m] + 2.0 * a.alpha - 2.0;
      int fail = 0;
      const double g = gamma_mt(0.5 * beta, ds->seed, ds->iteration, m, &fail);
      if (fail || !(sigma > 0.0)) atomicOr(&ds->status, ST_DRAW_FAIL);
      else ds->P[m] = sigma / (2.0 * g);
    }
  }
}

// ------------------------------------------------------------------ GIG draw
// Density ~ x^(p-1) exp(-(A x + B/x)/2) (Eq. GIG_post).  With eta = sqrt(B/A),
// omega = sqrt(A B), y = x/eta (p >= 0) or eta/x (p < 0) has density
// h(y) ~ y^(lam-1) exp(-omega (y + 1/y)/2), lam = |p|; sampled by the
// ratio-of-uniforms method with mode shift (Kinderman & Monahan 1977), the
// bounding rectangle found by bisection, everything in log space about the mode.
__device__ double gig_logh(double y, double lam, double om, double m) {
  return (lam - 1.0) * log1p((y - m) / m) - 0.5 * om * (y - m) * (1.0 - 1.0 / (y * m));
}
__device__ double gig_dphi(double y, double lam, double om, double m) {
  return 1.0 / (y - m) + 0.5 * ((lam - 1.0) / y - 0.5 * om + 0.5 * om / (y * y));
}

// Root of gig_dphi in (lo, hi), found by the 32 lanes of a warp together:
// each round evaluates 32 interior points, keeps the one gap where the sign
// turns and shrinks the interval 33-fold (12 rounds reach FP64 resolution).
// `neg_right`: the right-hand side of the root is where gig_dphi < 0 (else
// where it is <= 0).  All lanes return the same value.
__device__ double warp_root(double lo, double hi, bool neg_right, double lam, double om, double m) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < 16; ++round) {
    const double w = (hi - lo) / 33.0;
    if (!(w > 0.0)) break;
    const double x = lo + w * (double)(lane + 1);
    const double d = gig_dphi(x, lam, om, m);
    const unsigned right = __ballot_sync(0xffffffffu, neg_right ? (d < 0.0) : !(d > 0.0));
    const int k = right ? __ffs(right) - 1 : 32;        // first point on the right-hand side
    const double nlo = lo + w * (double)k;
    const double nhi = k == 32 ? hi : lo + w * (double)(k + 1);
    if (!(nlo > lo || nhi < hi)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// Called by all 32 lanes of one warp (identical arguments); every lane returns
// the same draw.
__device__ double gig_draw(double p, double A, double B, uint64_t seed, uint64_t it, int l, int* fail) {
  const double lam = fabs(p);
  const double om = sqrt(A * B);
  const double eta = sqrt(B / A);
  const double q = lam - 1.0;
  const double sq = sqrt(q * q + om * om);
  const double m = q >= 0.0 ? (q + sq) / om : om / (sq - q);
  // upper extreme of (y - m) sqrt(h(y)/h(m))
  double step = m, hi = m + step;
  for (int i = 0; i < 200 && gig_dphi(hi, lam, om, m) > 0.0; ++i) {
    step *= 2.0;
    hi = m + step;
  }
  const double yp = warp_root(m, hi, false, lam, om, m);
  const double vp = (yp - m) * exp(0.5 * gig_logh(yp, lam, om, m));
  const double ym = warp_root(0.0, m, true, lam, om, m);
  const double vm = ym > 0.0 ? (ym - m) * exp(0.5 * gig_logh(ym, lam, om, m)) : -m;
  double y = m;
  bool ok = false;
  for (int j = 0; j < MAX_ATTEMPTS && !ok; ++j) {
    P4 r = philox((uint64_t)l, it, ST_NBAR, (uint64_t)j, seed);
    const double u = u52(r.w[0]);
    const double v = vm + (vp - vm) * u52(r.w[1]);
    const double yy = v / u + m;
    if (yy <= 0.0) continue;
    if (2.0 * log(u) <= gig_logh(yy, lam, om, m)) {
      y = yy;
      ok = true;
    }
  }
  if (!ok) *fail = 1;
  return p >= 0.0 ? eta * y : eta / y;
}

// block l: S1 = sum N delta, S2 = sum R delta, S3 = sum R delta^2; then
// b_l ~ N(D/C, 1/C), C = Nbar S3, D = S1 - Nbar S2 (Sec. 3.5, App. B; skipped for
// the fixed index) and Nbar_l ~ GIG(1 - N_obs/2, sum R + 2 b S2 + b^2 S3, sum N^2/R)
__global__ void k_bias_nbar(ScalarArgs a0, int region, int nz) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  DevState* ds = a.ds;
  const int l = blockIdx.x;
  if (l >= ds->nsub) return;
  double S[3];
  for (int q = 0; q < 3; ++q) S[q] = sum_partials(a.part + region + (size_t)(3 * l + q) * a.stride, nz, sh);
  // the sums are valid in thread 0: hand them to the first warp, which draws
  // together (the GIG bounds are found lane-parallel); lane 0 writes
  if (threadIdx.x == 0) {
    sh[0] = S[0];
    sh[1] = S[1];
    sh[2] = S[2];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    S[0] = sh[0];
    S[1] = sh[1];
    S[2] = sh[2];
    const bool lead = threadIdx.x == 0;
    const uint64_t it = ds->iteration;
    if (lead) {
      ds->sums[l][0] = S[0];
      ds->sums[l][1] = S[1];
      ds->sums[l][2] = S[2];
    }
    double b = ds->b[l];
    const double nb = ds->nbar[l];
    int fail = 0;
    if (l != a.fixed_bias) {
      const double C = nb * S[2];
      const double D = S[0] - nb * S[1];
      P4 r = philox((uint64_t)l, it, ST_BIAS, 0, ds->seed);
      const double z = normal64(r.w[0], r.w[1]);
      if (C > 0.0) b = D / C + z / sqrt(C);
      else fail = 1;
    }
    const double A = ds->sumR[l] + 2.0 * b * S[1] + b * b * S[2];
    const double p = 1.0 - 0.5 * ds->nobs[l];
    double x = nb;
    if (A > 0.0 && ds->sumB[l] > 0.0) x = gig_draw(p, A, ds->sumB[l], ds->seed, it, l, &fail);
    else fail = 1;
    if (lead) {
      if (fail || !isfinite(b) || !isfinite(x)) {
        atomicOr(&ds->status, ST_DRAW_FAIL);
      } else {
        ds->b[l] = b;
        ds->nbar[l] = x;
      }
    }
  }
}

__global__ void k_abar(ScalarArgs a0, int region, int nblk) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  const double s = sum_partials(a.part + region, nblk, sh);
  if (threadIdx.x == 0) a.ds->abar = s * a.inv_nv;
}

// ------------------------------------------------------------------ survey commit
// Activates a survey uploaded into data slot `slot`: sums the data kernel's
// per-block partials of each subsample (sum R, sum N^2/R, observed voxels,
// invalid voxels; 4 x nblk doubles per subsample) in a fixed order, and either
// writes the data constants of Secs. 3.5-3.6 and makes the slot active, or, for
// invalid data or a subsample without observed voxels, flags ST_BADDATA and
// keeps the previous slot.  One block per chain.
__global__ void k_commit_data(DevState* ds0, const double* part0, long long cstride, int nblk, int slot) {
  DevState* ds = ds0 + blockIdx.x;
  const double* part = part0 + blockIdx.x * cstride;
  __shared__ double s_v[MAXS][4];
  const int nsub = ds->nsub;
  // one warp per quantity (4 per subsample), lanes strided over the partials
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x >> 5; q < 4 * nsub; q += blockDim.x >> 5) {
    double v = 0.0;
    for (int i = lane; i < nblk; i += 32) v += part[(size_t)q * nblk + i];
    v = warp_sum(v);
    if (lane == 0) s_v[q >> 2][q & 3] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    for (int l = 0; l < nsub; ++l) ok = ok && s_v[l][3] == 0.0 && s_v[l][2] > 0.0;
    if (!ok) {
      atomicOr(&ds->status, ST_BADDATA);
    } else {
      for (int l = 0; l < nsub; ++l) {
        ds->sumR[l] = s_v[l][0];
        ds->sumB[l] = s_v[l][1];
        ds->nobs[l] = s_v[l][2];
      }
      ds->dslot = slot;
    }
  }
}

// ------------------------------------------------------------------ jump move
// HMC in theta = ln P with the whitened field fixed (Sec. 4.3, App. C).
// Mass mu_m = max(1, abar P_ref_m sigma_m / (4 V_cell P_m)): built from the
// whitened field and a fixed reference spectrum, never from the current P.
// reuse: the jump directly follows this iteration's HMC move and power draw, so
// after an accepted move the first gradient can take the move's last force.
__global__ void k_jump_begin(ScalarArgs a0, int reuse) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  DevState* ds = a.ds;
  const int m = threadIdx.x;
  const uint64_t it = ds->iteration;
  if (m == 0) {
    ds->jreuse = reuse && ds->accepted;
    P4 r = philox(0, it, ST_JUMP, 0, ds->seed);
    ds->jeps = a.jeps_max * u52(r.w[0]);
    ds->ju_acc = u52(r.w[1]);
    ds->jaccepted = 0;
  }
  if (m < MAXB) {
    if (m < a.n_bins) {
      const double mu = fmax(1.0, ds->abar * ds->P_ref[m] * ds->sigma[m] / (4.0 * ds->vc * ds->P[m]));
      P4 r = philox((uint64_t)m, it, ST_JUMP_MOM, 0, ds->seed);
      ds->mu[m] = mu;
      ds->rho[m] = sqrt(mu) * normal64(r.w[0], r.w[1]);
      ds->th[m] = log(ds->P[m]);
    }
    ds->js[m] = 1.f;
  }
}

// Leapfrog update of the jump's HMC in theta after a gradient evaluation (kind:
// J_FIRST half kick and drift with the starting energy, J_MID kick and drift,
// J_LAST half kick, final energy and Metropolis test).  Threads m < n_bins own
// bin m; every thread of the block takes part in the barriers.
__device__ void jump_update(const ScalarArgs& a, int kind, double* sh) {
  DevState* ds = a.ds;
  const int m = threadIdx.x;
  const double eps = ds->jeps;
  const bool act = m < a.n_bins;
  double kin = 0.0, pri = 0.0;
  double rho = act ? ds->rho[m] : 0.0, th = act ? ds->th[m] : 0.0;
  // written by the other blocks of this launch: read past L1
  const double mu = act ? ds->mu[m] : 1.0, g = act ? __ldcg(&ds->jgrad[m]) : 0.0;
  if (kind == J_FIRST && act) {
    kin = 0.5 * rho * rho / mu;
    pri = (a.alpha - 1.0) * th;
  }
  if (act) {
    const double ek = (kind == J_MID) ? eps : 0.5 * eps;
    rho -= ek * g;
    if (kind != J_LAST) th += eps * rho / mu;
  }
  if (kind == J_LAST && act) {
    kin = 0.5 * rho * rho / mu;
    pri = (a.alpha - 1.0) * th;
  }
  // 64-thread sums (two warps)
  double e = kin + pri;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  __syncthreads();
  if ((m & 31) == 0) sh[m >> 5] = e;
  __syncthreads();
  const double E = sh[0] + sh[1];   // bins live in the first two warps (n_bins <= 64)
  if (act) {
    ds->rho[m] = rho;
    ds->th[m] = th;
    ds->js[m] = (float)sqrt(exp(th) / ds->P[m]);
  }
  const double jlik = __ldcg(&ds->jlik);
  if (kind == J_FIRST && m == 0) ds->jH0 = E + jlik;
  if (kind == J_LAST) {
    __shared__ int s_acc;
    if (m == 0) {
      const double H1 = E + jlik;
      const double dH = H1 - ds->jH0;
      ds->jH1 = H1;
      ds->jdH = dH;
      int acc = 0;
      if (!isfinite(dH)) ds->status |= ST_NONFINITE;
      else acc = log(ds->ju_acc) < -dH;
      ds->jaccepted = acc;
      s_acc = acc;
    }
    __syncthreads();
    if (act && s_acc) ds->P[m] = exp(th);
  }
}


// One leapfrog step of the jump after its gradient evaluation, in one launch:
// blocks m < n_bins reduce the gradient d psi_J / d theta_m = (alpha - 1) +
// (1/2N^3) sum_{k in m} w Re(conj(g) delta), block n_bins (launched for J_FIRST
// and J_LAST only, whose update needs the energy) the likelihood energy at
// theta; the last block to finish (a counter in the chain state, which it
// resets) then applies the update of `kind`.
__global__ void k_jump_step(ScalarArgs a0, int r_grad, int nx, int r_lik, int r_lik_move, int nz, int kind) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  __shared__ int s_last;
  DevState* ds = a.ds;
  const int m = blockIdx.x;
  if (m < a.n_bins) {
    const double s = sum_partials(a.part + r_grad + (size_t)m * a.stride, nx, sh);
    if (threadIdx.x == 0) ds->jgrad[m] = (a.alpha - 1.0) + 0.5 * a.inv_nv * s;
  } else {
    // a reused force stage left its likelihood partials where the move's last one wrote them
    const double s = sum_partials(a.part + (ds->jreuse ? r_lik_move : r_lik), nz, sh);
    if (threadIdx.x == 0) ds->jlik = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ds->jdone, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    ds->jdone = 0;
    ds->jreuse = 0;               // only the first gradient can reuse the move's force
  }
  jump_update(a, kind, sh);
}

// ------------------------------------------------------------------ misc
__global__ void k_reduce_to(ScalarArgs a, int region, int nblk, double scale, double* out) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  const double s = sum_partials(a.part + region + (size_t)q * a.stride, nblk, sh);
  if (threadIdx.x == 0) out[q] = s * scale;
}

// chain record: P[n_bins], b[n_sub], nbar[n_sub], dH, accepted; slot rec_idx
// of chain (chain0 + blockIdx.y) in a buffer laid out [slot][chain][rec_len]
__global__ void k_record(ScalarArgs a0, double* rec0, int rec_len, long long iter_stride, int chain0) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  DevState* ds = a.ds;
  const int t = threadIdx.x;
  const int ns = ds->nsub;
  double* rec = rec0 + (long long)ds->rec_idx * iter_stride + (long long)(chain0 + blockIdx.y) * rec_len;
  if (t < a.n_bins) rec[t] = ds->P[t];
  if (t < ns) {
    rec[a.n_bins + t] = ds->b[t];
    rec[a.n_bins + ns + t] = ds->nbar[t];
  }
  if (t == 0) {
    rec[a.n_bins + 2 * ns] = ds->dH;
    rec[a.n_bins + 2 * ns + 1] = (double)ds->accepted;
  }
  __syncthreads();
  if (t == 0) ds->rec_idx += 1;
}

__global__ void k_advance(DevState* ds) { ds[blockIdx.x].iteration += 1; }

__global__ void k_reset_rec(DevState* ds) { ds[blockIdx.x].rec_idx = 0; }

__global__ void k_zero_dc(float2* spec) { spec[0] = make_float2(0.f, 0.f); }

// block j of chain blockIdx.y: sum of the per-tile partials of mass bin j
__global__ void k_mstat(ScalarArgs a0, int region, int nblk, int final_) {
  const ScalarArgs a = chain_args(a0, blockIdx.y);
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const double s = sum_partials(a.part + region + (size_t)j * a.stride, nblk, sh);
  if (threadIdx.x == 0) {
    if (final_) a.ds->mstat2[j] = s;
    else a.ds->mstat[j] += s;
  }
}

void launch_move_begin(const ScalarArgs& a, int nch, cudaStream_t s) { k_move_begin<<<dim3(1, nch), MAXB, 0, s>>>(a); }
void launch_move_end(const ScalarArgs& a, int r_init, int r_lik0, int r_final, int r_lik1, int nx, int nz, int nch,
                     cudaStream_t s) {
  k_move_sums<<<dim3(8, nch), 256, 0, s>>>(a, r_init, r_lik0, r_final, r_lik1, nx, nz);
  k_move_end<<<dim3(1, nch), 32, 0, s>>>(a);
}
void launch_power(const ScalarArgs& a, int region, int nx, int draw, int nch, cudaStream_t s) {
  k_power<<<dim3(a.n_bins, nch), 256, 0, s>>>(a, region, nx, draw);
}
void launch_bias_nbar(const ScalarArgs& a, int region, int nz, int nch, cudaStream_t s) {
  k_bias_nbar<<<dim3(a.max_sub, nch), 256, 0, s>>>(a, region, nz);
}
void launch_abar(const ScalarArgs& a, int region, int nblk, int nch, cudaStream_t s) {
  k_abar<<<dim3(1, nch), 256, 0, s>>>(a, region, nblk);
}
void launch_jump_begin(const ScalarArgs& a, int reuse, int nch, cudaStream_t s) {
  k_jump_begin<<<dim3(1, nch), MAXB, 0, s>>>(a, reuse);
}
void launch_jump_step(const ScalarArgs& a, int r_grad, int nx, int r_lik, int r_lik_move, int nz, int kind,
                      int nch, cudaStream_t s) {
  k_jump_step<<<dim3(a.n_bins + (kind == J_MID ? 0 : 1), nch), 256, 0, s>>>(a, r_grad, nx, r_lik, r_lik_move, nz,
                                                                          kind);
}
void launch_reduce_to(const ScalarArgs& a, int region, int nblk, int count, double scale, double* out_dev,
                      cudaStream_t s) {
  k_reduce_to<<<count, 256, 0, s>>>(a, region, nblk, scale, out_dev);
}
void launch_record(const ScalarArgs& a, double* rec_dev, int rec_len, long long iter_stride, int chain0, int nch,
                   cudaStream_t s) {
  k_record<<<dim3(1, nch), MAXB, 0, s>>>(a, rec_dev, rec_len, iter_stride, chain0);
}
void launch_advance(DevState* ds, int nch, cudaStream_t s) { k_advance<<<nch, 1, 0, s>>>(ds); }
void launch_commit_data(DevState* ds, const double* part, long long cstride, int nblk, int slot, int nch,
                        cudaStream_t s) {
  k_commit_data<<<nch, 1024, 0, s>>>(ds, part, cstride, nblk, slot);
}
void launch_reset_rec(DevState* ds, int nch, cudaStream_t s) { k_reset_rec<<<nch, 1, 0, s>>>(ds); }
void launch_zero_dc(float2* spec, cudaStream_t s) { k_zero_dc<<<1, 1, 0, s>>>(spec); }
void launch_mstat(const ScalarArgs& a, int region, int nblk, int n_mass, int final_, int nch, cudaStream_t s) {
  k_mstat<<<dim3(n_mass, nch), 256, 0, s>>>(a, region, nblk, final_);
}


// ------------------------------------------------------------------ posterior moments
// Running sums of the chain parameters of one chain (Secs. 6.2 and 7: the
// correlation matrices of P, b and Nbar), one FP64 accumulation per Gibbs
// iteration, in a fixed order.
__global__ void k_param_moments(ScalarArgs a, double* acc) {
  const DevState* ds = a.ds;
  const int nb = a.n_bins, ns = ds->nsub, D = nb + 2 * ns;
  __shared__ double x[MAXB + 2 * MAXS];
  for (int i = threadIdx.x; i < D; i += blockDim.x)
    x[i] = i < nb ? ds->P[i] : i < nb + ns ? ds->b[i - nb] : ds->nbar[i - nb - ns];
  __syncthreads();
  if (threadIdx.x == 0) acc[0] += 1.0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) acc[1 + i] += x[i];
  for (int q = threadIdx.x; q < D * D; q += blockDim.x) acc[1 + D + q] += x[q / D] * x[q % D];
}

// mean = S1 / n, var = S2 / n - mean^2 per voxel (population moments)
__global__ void k_moments_finish(const double* __restrict__ mom, long long nv, double n, double* mean, double* var) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    const double m = mom[i] / n;
    if (mean) mean[i] = m;
    if (var) var[i] = mom[nv + i] / n - m * m;
  }
}

void launch_moments_finish(const double* mom, long long nv, double n, double* mean, double* var, int blocks,
                           cudaStream_t s) {
  k_moments_finish<<<blocks, 256, 0, s>>>(mom, nv, n, mean, var);
}

void launch_param_moments(const ScalarArgs& a, double* acc, cudaStream_t s) {
  k_param_moments<<<1, 256, 0, s>>>(a, acc);
}

// ------------------------------------------------------------------ failure detection
// Self-test of the bounded device waits: one thread announces 16 bytes on a
// shared-memory mbarrier and waits for them, but no copy is ever issued, so the
// phase never completes.  The wait gives up after limit_ns and records the
// timeout in the chain's status word exactly as a field pass does when a tile
// copy does not land; nothing is in flight when the block exits.
__global__ void k_wait_probe(DevState* ds, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 16);
    if (!mbar_wait(&bar, 0, limit_ns)) atomicOr(&ds->status, (int)ST_TIMEOUT);
  }
}

void launch_wait_probe(DevState* ds, unsigned long long limit_ns, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(ds, limit_ns);
}

}  // namespace bps
