// Field-pass kernels of the sampler and their per-grid launch tables.
//
// HMC leapfrog step (Sec. 4.1.2, Eqs. HAMILTON1_a / HAMILTON2_a, kick-drift-kick)
// in four passes, each one HBM round trip of the half spectra it touches:
//   x pass  : ghat = FFT_x(W); p -= eps_k (delta/lambda + ghat); delta += eps p / M;
//             W = IFFT_x(delta)                         (reads W, delta, p; writes all three)
//   y pass  : W = IFFT_y(W)
//   z pass  : delta = C2R_z(W) / N^3; g = a delta - c; W = R2C_z(g)   (reads a, c)
//   y pass  : W = FFT_y(W)
// so the force of Eq. Wiener_Posterior_force costs one 3D C2R and one 3D R2C
// with the prior and the voxel-local likelihood fused into the passes.
#include "bps_internal.h"
#include "bps_passes.cuh"
#include "bps_tma.cuh"
#include <cudaTypedefs.h>

#include <type_traits>

namespace bps {

enum XMode {
  X_INIT = 0,   // momentum: p = sqrt(M) FFT_x(p); energies of p and delta; W = IFFT_x(delta)
  X_LEAP,       // kick (previous force) + drift + inverse x of the new delta
  X_FINAL,      // last half kick; kinetic and prior energies of the end point
  X_INV,        // dst = IFFT_x(src)
  X_FWD,        // dst = FFT_x(src)
  X_GRAD,       // dst = delta/lambda + FFT_x(W); prior energy
  X_JINV,       // W = IFFT_x(js_m delta)                (jump: field at theta)
  X_JGRAD,      // per-bin sum w Re(conj(FFT_x(W)) js_m delta)
  X_SCALE,      // delta *= js_m if the jump was accepted
  X_BINPOW,     // per-bin sum w |delta|^2
  X_MACC,       // acc += delta; per mass-bin sum w |delta|^2
  X_MMEAN,      // per mass-bin sum w |acc|^2
  X_WPOW,       // per-bin sum w |W|^2 (the power of whatever W holds)
  X_LEAPG       // X_LEAP of the first step, also reducing g^T M^-1 g of the force it applies
};

enum ZMode { Z_GRAD = 0, Z_NOISE, Z_R2C, Z_C2R, Z_SUMS };

// state buffer i without indexing the parameter array at run time
__device__ __forceinline__ float2* dsel(const Fields& fp, int i) { return i ? fp.dh[1] : fp.dh[0]; }

struct XArgs {
  int src_buf;   // staged input buffer (BUF_*), -1: the current state
  float2* dst;
  int first;
  int region;    // offset (doubles) of this launch's partial sums in Fields::part
};

struct ZArgs {
  const float2* src;
  float2* dst;
  const float* rin;
  float* rout;
  int region;
  uint64_t seed;
  // Z_C2R with mom: instead of writing delta, add delta and delta^2 to the
  // running sums mom[0..N^3) and mom[N^3..2 N^3) (FP64; posterior moments)
  double* mom = nullptr;
};

// ------------------------------------------------------------------ x pass helpers
// Tile schedule of the strided (x and y) passes: the NYQ tiles of the kz = N/2
// column come first.  Their accesses are one element per row (a quarter of each
// 32-byte sector is used), so a Nyquist tile runs several times longer than a
// regular one; scheduled last they formed a tail of a few SMs at the end of
// every pass, scheduled first they overlap with the regular tiles.
template <int N>
__device__ __forceinline__ int tile_id() {
  using C = Cfg<N>;
  const int id = blockIdx.x;
  return id < C::NYQ ? N * C::ZB + id : id - C::NYQ;
}

__device__ __forceinline__ const float2* buf_ptr(const Fields& fp, int b) {
  return b == BUF_D0 ? fp.dh[0] : b == BUF_D1 ? fp.dh[1] : b == BUF_PH ? fp.ph : fp.W;
}

#ifndef BPS_XPASS_MIN_BLOCKS
#define BPS_XPASS_MIN_BLOCKS 2
#endif
// the leapfrog x pass works through its column in BPS_XLEAP_CHUNKS parts, so
// that BPS_XLEAP_MIN_BLOCKS CTAs of 256 threads fit on an SM without spills
#ifndef BPS_XLEAP_MIN_BLOCKS
#define BPS_XLEAP_MIN_BLOCKS 3
#endif
#ifndef BPS_XLEAP_CHUNKS
#define BPS_XLEAP_CHUNKS 4
#endif
// the jump's inverse x pass and its gradient fit four CTAs per SM (64 registers)
// without spills
#ifndef BPS_XJINV_MIN_BLOCKS
#define BPS_XJINV_MIN_BLOCKS 4
#endif
#ifndef BPS_XJGRAD_MIN_BLOCKS
#define BPS_XJGRAD_MIN_BLOCKS 4
#endif
// the y passes fit four CTAs per SM (64 registers) without spills
#ifndef BPS_YPASS_MIN_BLOCKS
#define BPS_YPASS_MIN_BLOCKS 4
#endif

// ------------------------------------------------------------------ x pass
template <int N, int MODE>
__global__ void __launch_bounds__(Cfg<N>::NT, MODE == X_LEAP || MODE == X_LEAPG ? BPS_XLEAP_MIN_BLOCKS
                                              : MODE == X_JINV  ? BPS_XJINV_MIN_BLOCKS
                                              : MODE == X_JGRAD ? BPS_XJGRAD_MIN_BLOCKS
                                                                : BPS_XPASS_MIN_BLOCKS)
    k_xpass(Fields fp0, XArgs xa) {
  const Fields fp = at_chain(fp0, blockIdx.y);
  using C = Cfg<N>;
  constexpr int F = C::F, R1 = C::R1, R2 = C::R2, NT = C::NT, NW = NT / 32;
  constexpr bool BINNED = (MODE == X_JGRAD || MODE == X_BINPOW || MODE == X_MACC || MODE == X_MMEAN || MODE == X_WPOW);
  constexpr bool MASSBINS = (MODE == X_MACC || MODE == X_MMEAN);
  __shared__ float2 s_tw[N];
  __shared__ __align__(16) float2 s_ex[N * F];
  __shared__ int s_thr[MAXB], s_mthr[MAXB];
  __shared__ float s_il[MAXB], s_im[MAXB], s_sm[MAXB], s_ims[MAXB], s_sms[MAXB], s_js[MAXB];
  __shared__ double s_red[32];
  // per-warp bin sums as compensated FP32 pairs (sum, error): FP64 arithmetic is
  // scarce on this GPU, and each pair keeps the sum of the FP32 terms it was given
  // to about twice FP32 precision
  __shared__ float s_wh[BINNED ? NW : 1][MAXB], s_wl[BINNED ? NW : 1][MAXB];

  const int t = threadIdx.x;
  DevState* ds = fp.ds;
  if constexpr (MODE == X_SCALE) {
    if (!ds->jaccepted) return;   // uniform across the grid
  }
  if constexpr (MODE == X_JINV) {
    if (ds->jreuse) return;       // W already holds this force stage's input (uniform)
  }
  load_twiddles<N>(s_tw, fp.tw, t, NT);
  for (int i = t; i < MAXB; i += NT) {
    s_thr[i] = ds->thr[i];
    s_mthr[i] = ds->mthr[i];
    s_il[i] = ds->inv_lambda[i];
    s_im[i] = ds->inv_M[i];
    s_sm[i] = ds->sqrt_M[i];
    s_ims[i] = ds->inv_ms[i];
    s_sms[i] = ds->sqrt_ms[i];
    s_js[i] = ds->js[i];
    if constexpr (BINNED) {
      for (int w = 0; w < NW; ++w) {
        s_wh[w][i] = 0.f;
        s_wl[w][i] = 0.f;
      }
    }
  }
  __syncthreads();

  const Tile<N> T = tile_x<N>(tile_id<N>());
  const int f = t % F;
  const int ja = t / F;                       // row group of the spatial (x-) layout
  const int ky = T.ky0 + f * T.dky, kz = T.kz0 + f * T.dkz;
  const int ny = sgn_n<N>(ky);
  const int n2yz = ny * ny + kz * kz;
  const float wk = (kz == 0 || kz == C::H) ? 1.f : 2.f;
  const long long colo = T.base + (long long)f * T.cs;
  const int cur = ds->cur;
  const bool mm = fp.mass_mode != 0;
  const float scb = bin_scale(fp.n_bins, N), scm = bin_scale(fp.n_mass, N);

  float2 v[C::RMAX];
  auto mode_bin = [&](int k, float& il, float& im, float& sm) -> int {
    const int nx = sgn_n<N>(k);
    const int n2 = nx * nx + n2yz;
    const int m = bin_est(n2, s_thr, scb, fp.n_bins);
    if (m >= 0) {
      il = s_il[m];
      im = s_im[m];
      sm = s_sm[m];
      if (mm) {
        const int j = bin_est(n2, s_mthr, scm, fp.n_mass);
        im *= s_ims[j];
        sm *= s_sms[j];
      }
    } else {
      il = im = sm = 0.f;
    }
    return m;
  };

  // ---------------- modes that start from a spatial-x tile: forward transform
  if constexpr (MODE == X_INIT || MODE == X_LEAP || MODE == X_LEAPG || MODE == X_FINAL || MODE == X_FWD ||
                MODE == X_GRAD || MODE == X_JGRAD) {
    const float2* in = (MODE == X_INIT) ? fp.ph : (MODE == X_FWD) ? buf_ptr(fp, xa.src_buf) : fp.W;
    // X_FWD with no destination writes the current state buffer
    if (ja < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) v[b] = in[colo + (long long)(ja + R1 * b) * T.rs];
    }
    fft2<N, R1, R2, FWD, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  }
  const int jc = t / F;                       // row group of the Fourier (kx-) layout
  const bool act = jc < R2;

  if constexpr (MODE == X_FWD) {
    if (act) {
      float2* out = xa.dst ? xa.dst : dsel(fp, cur);
#pragma unroll
      for (int d = 0; d < R1; ++d) out[colo + (long long)(jc + R2 * d) * T.rs] = v[d];
    }
    return;
  }

  if constexpr (MODE == X_INIT) {
    // momentum p = sqrt(M_k) FFT(xi); kinetic energy (1/2N^3) sum w |p|^2 / M
    TwoSumAcc eK, eP;
    float2 x[R1];
    if (act) {
#pragma unroll
      for (int d = 0; d < R1; ++d) x[d] = dsel(fp, cur)[colo + (long long)(jc + R2 * d) * T.rs];
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const int k = jc + R2 * d;
        float il, im, sm;
        const int m = mode_bin(k, il, im, sm);
        float2 p = m >= 0 ? cscale(v[d], sm) : make_float2(0.f, 0.f);
        fp.ph[colo + (long long)k * T.rs] = p;
        eK.add(wk * (p.x * p.x + p.y * p.y) * im);
        float2 xx = m >= 0 ? x[d] : make_float2(0.f, 0.f);
        eP.add(wk * (xx.x * xx.x + xx.y * xx.y) * il);
        v[d] = xx;
      }
    }
    fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
    if (ja < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) fp.W[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
    }
    float* s_rf = reinterpret_cast<float*>(s_red);
    double sK = block_sum2<NT>(eK, s_rf);
    double sP = block_sum2<NT>(eP, s_rf);
    if (t == 0) {
      fp.part[xa.region + blockIdx.x] = sK;
      fp.part[xa.region + fp.part_stride + blockIdx.x] = sP;
    }
    return;
  }

  if constexpr (MODE == X_LEAP || MODE == X_LEAPG) {
    const bool first = MODE == X_LEAPG || xa.first;
    const float2* src = first ? dsel(fp, cur) : dsel(fp, 1 - cur);
    float2* dst = dsel(fp, 1 - cur);
    const float eps = (float)ds->eps;
    const float ek = first ? 0.5f * eps : eps;
    float eG = 0.f;   // X_LEAPG: sum w |g|^2 / M of the force at the start point
    // the column in parts: the loads of a part in flight together, at a
    // fraction of the registers of a whole column
    constexpr int HALF = R1 / BPS_XLEAP_CHUNKS > 0 ? R1 / BPS_XLEAP_CHUNKS : 1;
    if (act) {
#pragma unroll
      for (int h = 0; h < R1; h += HALF) {
      float2 x[HALF], p[HALF];
#pragma unroll
      for (int q = 0; q < HALF; ++q) {
        const long long idx = colo + (long long)(jc + R2 * (h + q)) * T.rs;
        x[q] = src[idx];
        p[q] = fp.ph[idx];
      }
#pragma unroll
      for (int q = 0; q < HALF; ++q) {
        const int d = h + q;
        const int k = jc + R2 * d;
        float il, im, sm;
        const int m = mode_bin(k, il, im, sm);
        float2 xx = x[q], pp = p[q];
        if (m >= 0) {
          const float gx = fmaf(xx.x, il, v[d].x), gy = fmaf(xx.y, il, v[d].y);
          if constexpr (MODE == X_LEAPG) eG += wk * (gx * gx + gy * gy) * im;
          pp.x = fmaf(-ek, gx, pp.x);
          pp.y = fmaf(-ek, gy, pp.y);
          const float s = eps * im;
          xx.x = fmaf(s, pp.x, xx.x);
          xx.y = fmaf(s, pp.y, xx.y);
        } else {
          xx = make_float2(0.f, 0.f);
          pp = make_float2(0.f, 0.f);
        }
        const long long idx = colo + (long long)k * T.rs;
        fp.ph[idx] = pp;
        dst[idx] = xx;
        v[d] = xx;
      }
      }
    }
    fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
    if (ja < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) fp.W[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
    }
    if constexpr (MODE == X_LEAPG) {
      const double sG = block_sum2<NT>(pair_of(eG), reinterpret_cast<float*>(s_red));
      if (t == 0) fp.part[xa.region + blockIdx.x] = sG;
    }
    return;
  }

  if constexpr (MODE == X_FINAL) {
    const float2* src = dsel(fp, 1 - cur);
    const float eps = (float)ds->eps;
    const float ek = 0.5f * eps;
    TwoSumAcc eK, eP;
    float eG = 0.f;   // sum w |g|^2 / M of the last force (the Delta H identity of k_move_end)
    float2 x[R1], p[R1];
    if (act) {
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const long long idx = colo + (long long)(jc + R2 * d) * T.rs;
        x[d] = src[idx];
        p[d] = fp.ph[idx];
      }
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const int k = jc + R2 * d;
        float il, im, sm;
        const int m = mode_bin(k, il, im, sm);
        if (m >= 0) {
          float2 xx = x[d], pp = p[d];
          const float gx = fmaf(xx.x, il, v[d].x), gy = fmaf(xx.y, il, v[d].y);
          eG += wk * (gx * gx + gy * gy) * im;
          pp.x = fmaf(-ek, gx, pp.x);
          pp.y = fmaf(-ek, gy, pp.y);
          eK.add(wk * (pp.x * pp.x + pp.y * pp.y) * im);
          eP.add(wk * (xx.x * xx.x + xx.y * xx.y) * il);
        }
      }
    }
    float* s_rf = reinterpret_cast<float*>(s_red);
    double sK = block_sum2<NT>(eK, s_rf);
    double sP = block_sum2<NT>(eP, s_rf);
    double sG = block_sum2<NT>(pair_of(eG), s_rf);
    if (t == 0) {
      fp.part[xa.region + blockIdx.x] = sK;
      fp.part[xa.region + fp.part_stride + blockIdx.x] = sP;
      fp.part[xa.region + 2 * fp.part_stride + blockIdx.x] = sG;
    }
    return;
  }

  if constexpr (MODE == X_GRAD) {
    TwoSumAcc eP;
    if (act) {
      float2 x[R1];
#pragma unroll
      for (int d = 0; d < R1; ++d) x[d] = dsel(fp, cur)[colo + (long long)(jc + R2 * d) * T.rs];
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const int k = jc + R2 * d;
        float il, im, sm;
        const int m = mode_bin(k, il, im, sm);
        float2 g = make_float2(0.f, 0.f);
        if (m >= 0) {
          g = make_float2(fmaf(x[d].x, il, v[d].x), fmaf(x[d].y, il, v[d].y));
          eP.add(wk * (x[d].x * x[d].x + x[d].y * x[d].y) * il);
        }
        xa.dst[colo + (long long)k * T.rs] = g;
      }
    }
    double sP = block_sum2<NT>(eP, reinterpret_cast<float*>(s_red));
    if (t == 0) fp.part[xa.region + blockIdx.x] = sP;
    return;
  }

  if constexpr (MODE == X_INV || MODE == X_JINV) {
    // X_INV with no source reads the current state buffer
    const float2* src = (MODE == X_INV && xa.src_buf >= 0) ? buf_ptr(fp, xa.src_buf) : dsel(fp, cur);
    if (act) {
#pragma unroll
      for (int d = 0; d < R1; ++d) v[d] = src[colo + (long long)(jc + R2 * d) * T.rs];
      if constexpr (MODE == X_JINV) {
        // the jump's field scale by bin, the bins read from the context's map
#pragma unroll
        for (int d = 0; d < R1; ++d) {
          const int m = bin_of_map(fp.pbin, colo + (long long)(jc + R2 * d) * T.rs);
          v[d] = m >= 0 ? cscale(v[d], s_js[m]) : make_float2(0.f, 0.f);
        }
      }
    }
    fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
    float2* out = (MODE == X_INV && xa.dst) ? xa.dst : fp.W;   // no destination: this chain's W
    if (ja < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) out[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
    }
    return;
  }

  if constexpr (MODE == X_SCALE) {
    if (act) {
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const long long idx = colo + (long long)(jc + R2 * d) * T.rs;
        const int m = bin_of_map(fp.pbin, idx);
        dsel(fp, cur)[idx] = m >= 0 ? cscale(dsel(fp, cur)[idx], s_js[m]) : make_float2(0.f, 0.f);
      }
    }
    return;
  }

  if constexpr (BINNED) {
    const int warp = t >> 5, lane = t & 31;
    // (1) every element's term into shared memory by (row kx, column f); the
    // bin factor s_m of the jump gradient is applied per bin at the end
    // column-major with a row stride of N + 2 floats: the writes (16 columns x 2
    // rows per warp) and the reads (32 lanes L rows apart) both avoid bank conflicts
    constexpr int SE = N + 2;
    float* s_e = reinterpret_cast<float*>(s_ex);   // F * SE floats, free after the transform
    if (act) {
      float2 xv[R1];
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const long long idx = colo + (long long)(jc + R2 * d) * T.rs;
        xv[d] = (MODE == X_MMEAN) ? fp.acc[idx] : (MODE == X_WPOW) ? fp.W[idx] : dsel(fp, cur)[idx];
      }
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const int k = jc + R2 * d;
        const float2 x = xv[d];
        if constexpr (MODE == X_MACC) {
          const long long idx = colo + (long long)k * T.rs;
          const float2 s0 = fp.acc[idx];
          fp.acc[idx] = make_float2(s0.x + x.x, s0.y + x.y);
        }
        float e;
        if constexpr (MODE == X_JGRAD) e = wk * (v[d].x * x.x + v[d].y * x.y);
        else e = wk * (x.x * x.x + x.y * x.y);
        s_e[f * SE + k] = e;
      }
    }
    __syncthreads();
    // (2) one warp per column.  Lane q takes |nx| in [q L, q L + L) (both rows
    // kx = |nx| and N - |nx|), in rising order, so its bins rise; consecutive
    // lanes follow each other.  A lane sums its elements into runs of equal
    // bin: a run that starts and ends inside the lane holds a bin no other lane
    // has and goes straight to the warp's bins; the lane's first and last runs
    // are combined across the warp by segmented sums (the first runs and the
    // last runs each form a bin-ordered sequence over the lanes).  Fixed order
    // throughout: the sums are deterministic.
    constexpr int HN = N / 2, L = (HN + 1 + 31) / 32;
    const int* thr = MASSBINS ? s_mthr : s_thr;
    const int nb = MASSBINS ? fp.n_mass : fp.n_bins;
    const float scl = MASSBINS ? scm : scb;
    float* wh = s_wh[warp];
    float* wl = s_wl[warp];
    for (int col = warp; col < F; col += NW) {
      const int nyc = sgn_n<N>(T.ky0 + col * T.dky), kzc = T.kz0 + col * T.dkz;
      const int n2c = nyc * nyc + kzc * kzc;
      const int a0 = lane * L, a1 = min(a0 + L, HN + 1);
      int mf = -1, ml = -1, mc = -1, nxt = 0x7fffffff;
      float vf = 0.f, vl = 0.f, vc = 0.f;   // FP32 runs; the warp's bins are compensated FP32 pairs
      bool first_done = false;
      for (int a = a0; a < a1; ++a) {
        const int n2 = a * a + n2c;
        if (n2 == 0) continue;                            // the DC mode is in no bin
        float val = s_e[col * SE + a];
        if (a != 0 && a != HN) val += s_e[col * SE + N - a];
        int m;
        if (mc < 0) {
          m = bin_est(n2, thr, scl, nb);
          nxt = m + 1 < nb ? thr[m + 1] : 0x7fffffff;
        } else {
          m = mc;
          while (n2 >= nxt) {
            ++m;
            nxt = m + 1 < nb ? thr[m + 1] : 0x7fffffff;
          }
        }
        if (m != mc) {
          if (mc >= 0) {                                  // close the current run
            if (!first_done) { mf = mc; vf = vc; first_done = true; }
            else two_sum_add(wh[mc], wl[mc], vc);       // a run inside this lane only
          }
          mc = m;
          vc = 0.f;
        }
        vc += val;
      }
      if (mc >= 0) {
        if (!first_done) { mf = mc; vf = vc; ml = mc; vl = 0.f; }
        else { ml = mc; vl = vc; }
      }
      // lanes without elements (beyond |nx| = N/2) carry the bin of their left
      // neighbours with nothing, which keeps both sequences bin-ordered
      __syncwarp();
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        float vv = pass == 0 ? vf : vl;
        int mm2 = pass == 0 ? mf : ml;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int pm = __shfl_up_sync(0xffffffffu, mm2, o);
          if (mm2 < 0 && lane >= o) mm2 = pm;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float pv = __shfl_down_sync(0xffffffffu, vv, o);
          const int pm = __shfl_down_sync(0xffffffffu, mm2, o);
          if (lane + o < 32 && pm == mm2) vv += pv;
        }
        const int prev = __shfl_up_sync(0xffffffffu, mm2, 1);
        if ((lane == 0 || prev != mm2) && mm2 >= 0) two_sum_add(wh[mm2], wl[mm2], vv);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int m = t; m < MAXB; m += NT) {
      TwoSumAcc acc;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        acc.add(s_wh[w][m]);
        acc.add(s_wl[w][m]);
      }
      double sum = acc.value();
      if constexpr (MODE == X_JGRAD) sum *= (double)s_js[m];
      fp.part[xa.region + m * fp.part_stride + blockIdx.x] = sum;
    }
    return;
  }
}

// ------------------------------------------------------------------ TMA-staged leapfrog x pass
// The leapfrog x pass (X_LEAP: FFT_x(W) -> force, kick, drift, IFFT_x -> W) with
// its three input tiles staged in shared memory before any arithmetic: for a
// regular tile one thread issues tensor copies of the W, delta and p tiles
// (N rows x F columns each; rows are kx, N ZP elements apart) on one mbarrier,
// so all of the tile's loads are in flight at once and no thread spends issue
// slots or registers on them; a Nyquist tile (columns are ky rows, one element
// per row) is loaded by the threads.  Stores go straight from registers.  The
// W tile lands in the buffer the transform exchanges through.
// SD, SP: the delta and p tiles are staged too (else read straight from HBM in
// the kick); staging all three holds 96 KB per block at 256^3, two blocks per SM.
template <int N, int SD, int SP>
struct XTma {
  using C = Cfg<N>;
  static constexpr int TILE = N * C::F;                    // complex elements of one tile
  static constexpr size_t SMEM = (1 + SD + SP) * (size_t)TILE * sizeof(float2);
  static constexpr int MIN_BLOCKS = SD + SP == 2 ? 2 : 3;
};

template <int N, int SD, int SP>
__global__ void __launch_bounds__(Cfg<N>::NT, (XTma<N, SD, SP>::MIN_BLOCKS))
    k_xleap_tma(Fields fp0, XArgs xa, const __grid_constant__ XMaps maps) {
  using XT = XTma<N, SD, SP>;
  const Fields fp = at_chain(fp0, blockIdx.y);
  using C = Cfg<N>;
  constexpr int F = C::F, R1 = C::R1, R2 = C::R2, NT = C::NT;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* s_ex = reinterpret_cast<float2*>(smem);          // W tile, then the transform's exchange
  float2* s_d = s_ex + XT::TILE;                            // delta tile [row][column] (SD)
  float2* s_p = s_d + (SD ? XT::TILE : 0);                  // p tile (SP)
  __shared__ float2 s_tw[N];
  __shared__ int s_thr[MAXB], s_mthr[MAXB];
  __shared__ float s_il[MAXB], s_im[MAXB], s_ims[MAXB];
  __shared__ __align__(8) uint64_t bar;
  const int t = threadIdx.x;
  DevState* ds = fp.ds;
  const int id = tile_id<N>();
  const Tile<N> T = tile_x<N>(id);
  const bool staged = id < N * C::ZB;
  const int cur = ds->cur;
  const int sbuf = xa.first ? cur : 1 - cur;
  if (staged && t == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_expect_tx(&bar, (uint32_t)XT::SMEM);
    const int kz0 = T.kz0, ky = T.ky0, ch = blockIdx.y;
    tma_load_4d(s_ex, &maps.W, kz0, ky, 0, ch, &bar);
    if constexpr (SD) tma_load_4d(s_d, sbuf ? &maps.d1 : &maps.d0, kz0, ky, 0, ch, &bar);
    if constexpr (SP) tma_load_4d(s_p, &maps.ph, kz0, ky, 0, ch, &bar);
  }
  load_twiddles<N>(s_tw, fp.tw, t, NT);
  for (int i = t; i < MAXB; i += NT) {
    s_thr[i] = ds->thr[i];
    s_mthr[i] = ds->mthr[i];
    s_il[i] = ds->inv_lambda[i];
    s_im[i] = ds->inv_M[i];
    s_ims[i] = ds->inv_ms[i];
  }
  const float2* src = dsel(fp, sbuf);
  if (!staged) {
    for (int i = t; i < XT::TILE; i += NT) {
      const int r = i / F, f = i % F;
      const long long g = T.base + (long long)r * T.rs + (long long)f * T.cs;
      s_ex[i] = fp.W[g];
      if constexpr (SD) s_d[i] = src[g];
      if constexpr (SP) s_p[i] = fp.ph[g];
    }
  }
  __syncthreads();
  if (staged) {
    bool ok = mbar_wait(&bar, 0);
    ok = __syncthreads_and(ok);
    if (!ok) {
      // record the timeout, then give the copies one more bounded wait so that
      // none is left writing into this block's shared memory when it exits
      if (t == 0) {
        atomicOr(&ds->status, (int)ST_TIMEOUT);
        mbar_wait(&bar, 0);
      }
      __syncthreads();
      return;
    }
  }
  const int f = t % F;
  const int ja = t / F;
  const int ky = T.ky0 + f * T.dky, kz = T.kz0 + f * T.dkz;
  const int ny = sgn_n<N>(ky);
  const int n2yz = ny * ny + kz * kz;
  const float wk = (kz == 0 || kz == C::H) ? 1.f : 2.f;
  (void)wk;
  const long long colo = T.base + (long long)f * T.cs;
  const bool mm = fp.mass_mode != 0;
  const float scb = bin_scale(fp.n_bins, N), scm = bin_scale(fp.n_mass, N);
  float2 v[C::RMAX];
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) v[b] = s_ex[(ja + R1 * b) * F + f];
  }
  __syncthreads();   // the exchange below overwrites the W tile
  fft2<N, R1, R2, FWD, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  const int jc = t / F;
  float2* dst = dsel(fp, 1 - cur);
  const float eps = (float)ds->eps;
  const float ek = xa.first ? 0.5f * eps : eps;
  if (jc < R2) {
#pragma unroll
    for (int d = 0; d < R1; ++d) {
      const int k = jc + R2 * d;
      const int nx = sgn_n<N>(k);
      const int n2 = nx * nx + n2yz;
      const int m = bin_est(n2, s_thr, scb, fp.n_bins);
      const long long gi = colo + (long long)k * T.rs;
      float2 xx = SD ? s_d[k * F + f] : src[gi];
      float2 pp = SP ? s_p[k * F + f] : fp.ph[gi];
      if (m >= 0) {
        const float il = s_il[m];
        float im = s_im[m];
        if (mm) im *= s_ims[bin_est(n2, s_mthr, scm, fp.n_mass)];
        const float gx = fmaf(xx.x, il, v[d].x), gy = fmaf(xx.y, il, v[d].y);
        pp.x = fmaf(-ek, gx, pp.x);
        pp.y = fmaf(-ek, gy, pp.y);
        const float sft = eps * im;
        xx.x = fmaf(sft, pp.x, xx.x);
        xx.y = fmaf(sft, pp.y, xx.y);
      } else {
        xx = make_float2(0.f, 0.f);
        pp = make_float2(0.f, 0.f);
      }
      const long long idx = colo + (long long)k * T.rs;
      fp.ph[idx] = pp;
      dst[idx] = xx;
      v[d] = xx;
    }
  }
  fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) fp.W[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
  }
}

// ------------------------------------------------------------------ x pass with a ring of quarters
// The leapfrog x pass (X_LEAP) with the delta and p rows it reads after the
// transform of W streamed through shared memory a quarter of the column at a
// time: the kick and drift work through the column in quarters (rows
// [q N/4, (q+1) N/4), the R1/4 elements of every thread), and a two-slot ring
// holds the delta and p rows of two quarters.  One thread issues the tensor
// copies of quarters 0 and 1 before W is loaded and transformed, and refills a
// slot with quarter q+2 as soon as every thread has read quarter q, so the
// kick reads shared memory while the next copies are in flight.  W is loaded
// straight into registers as in the direct pass; a Nyquist tile (one element
// per row, below the 16-byte copy width) reads delta and p directly.  32 KB of
// ring per block keeps three blocks per SM.  Every wait is bounded; a block
// whose copies do not arrive records the timeout, waits (bounded) for its
// copies in flight and returns.
template <int N>
struct XRing {
  using C = Cfg<N>;
  static constexpr int QR = N / 4;                          // rows of one quarter
  static constexpr int QT = QR * C::F;                      // complex elements of one quarter of one array
  // a tensor copy lands on a 128-byte boundary: each quarter array starts at a
  // multiple of QTP elements (QT rounded up to 128 bytes; 8^3 quarters are 64 bytes)
  static constexpr int QTP = (QT * (int)sizeof(float2) + 127) / 128 * 128 / (int)sizeof(float2);
  static constexpr uint32_t SLOT_BYTES = 2u * QT * sizeof(float2);   // bytes copied per slot (delta and p)
  static constexpr size_t SMEM = 4 * (size_t)QTP * sizeof(float2);
  static_assert(C::R1 % 4 == 0, "quarters of the column");
  static_assert(QTP * sizeof(float2) % 128 == 0, "copy destinations on 128-byte boundaries");
};

template <int N, bool TMA>
__global__ void __launch_bounds__(Cfg<N>::NT, BPS_XLEAP_MIN_BLOCKS)
    k_xleap_ring(Fields fp0, XArgs xa, const __grid_constant__ XMaps maps) {
  using XR = XRing<N>;
  const Fields fp = at_chain(fp0, blockIdx.y);
  using C = Cfg<N>;
  constexpr int F = C::F, R1 = C::R1, R2 = C::R2, NT = C::NT, HQ = R1 / 4;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* s_ring = reinterpret_cast<float2*>(smem);         // [slot][delta, p][QR rows][F], arrays QTP apart
  __shared__ float2 s_tw[N];
  __shared__ __align__(16) float2 s_ex[N * F];
  __shared__ int s_thr[MAXB], s_mthr[MAXB];
  __shared__ float s_il[MAXB], s_im[MAXB], s_ims[MAXB];
  __shared__ __align__(8) uint64_t bar[2];
  const int t = threadIdx.x;
  DevState* ds = fp.ds;
  const int id = tile_id<N>();
  const Tile<N> T = tile_x<N>(id);
  const bool staged = id < N * C::ZB;
  const int cur = ds->cur;
  const int sbuf = xa.first ? cur : 1 - cur;
  const CUtensorMap* dmap = sbuf ? &maps.d1q : &maps.d0q;
  const float2* src = dsel(fp, sbuf);
  // quarter q into slot q & 1: TMA, one thread issues two tensor copies on the
  // slot's barrier; else every thread issues 16-byte copies (two complex of one
  // row each, a warp covering four whole rows) in its own copy group
  auto issue = [&](int q) {
    float2* slot = s_ring + (size_t)(q & 1) * 2 * XR::QTP;
    if constexpr (TMA) {
      uint64_t* b = &bar[q & 1];
      mbar_expect_tx(b, XR::SLOT_BYTES);
      tma_load_4d(slot, dmap, T.kz0, T.ky0, q * XR::QR, blockIdx.y, b);
      tma_load_4d(slot + XR::QTP, &maps.phq, T.kz0, T.ky0, q * XR::QR, blockIdx.y, b);
    } else {
      constexpr int CH = XR::QT / 2;                        // 16-byte chunks of one array's quarter
      for (int c = t; c < 2 * CH; c += NT) {
        const int arr = c / CH, cc = c - arr * CH;
        const int row = cc / (F / 2), pair = cc - row * (F / 2);
        const float2* g = (arr ? fp.ph : src) + T.base + (long long)(q * XR::QR + row) * T.rs + 2 * pair;
        cp_async16(slot + arr * XR::QTP + row * F + 2 * pair, g);
      }
      cp_async_commit();
    }
  };
  if (staged) {
    if constexpr (TMA) {
      if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        issue(0);
        issue(1);
      }
    } else {
      issue(0);
      issue(1);
    }
  }
  load_twiddles<N>(s_tw, fp.tw, t, NT);
  for (int i = t; i < MAXB; i += NT) {
    s_thr[i] = ds->thr[i];
    s_mthr[i] = ds->mthr[i];
    s_il[i] = ds->inv_lambda[i];
    s_im[i] = ds->inv_M[i];
    s_ims[i] = ds->inv_ms[i];
  }
  __syncthreads();   // the transform reads the twiddles before its first barrier
  const int f = t % F;
  const int ja = t / F;
  const int ky = T.ky0 + f * T.dky, kz = T.kz0 + f * T.dkz;
  const int ny = sgn_n<N>(ky);
  const int n2yz = ny * ny + kz * kz;
  const long long colo = T.base + (long long)f * T.cs;
  const bool mm = fp.mass_mode != 0;
  const float scb = bin_scale(fp.n_bins, N), scm = bin_scale(fp.n_mass, N);
  float2* dst = dsel(fp, 1 - cur);
  float2 v[C::RMAX];
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) v[b] = fp.W[colo + (long long)(ja + R1 * b) * T.rs];
  }
  fft2<N, R1, R2, FWD, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  const int jc = t / F;
  const bool act = jc < R2;
  const float eps = (float)ds->eps;
  const float ek = xa.first ? 0.5f * eps : eps;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2* slot = s_ring + (size_t)(q & 1) * 2 * XR::QTP;
    if (staged && !TMA) {
      // this thread's copies of quarter q have landed (only quarter q + 1 may
      // still be in flight); the barrier makes every thread's copies visible
      if (q < 3) cp_async_wait<1>();
      else cp_async_wait<0>();
      __syncthreads();
    }
    if (staged && TMA) {
      // one thread polls the barrier (256 pollers flood the shared-memory
      // pipe); its acquire and the block barrier after it make the copied
      // rows visible to every thread
      bool ok = true;
      if (t == 0) ok = mbar_wait(&bar[q & 1], (uint32_t)(q >> 1));
      ok = __syncthreads_and(ok);
      if (!ok) {
        // record the timeout, then give the copies in flight one more bounded
        // wait so that none is left writing into this block's shared memory
        if (t == 0) {
          atomicOr(&ds->status, (int)ST_TIMEOUT);
          mbar_wait(&bar[q & 1], (uint32_t)(q >> 1));
          if (q + 1 < 4) mbar_wait(&bar[(q + 1) & 1], (uint32_t)((q + 1) >> 1));
        }
        __syncthreads();
        return;
      }
    }
    if (act) {
#pragma unroll
      for (int e = 0; e < HQ; ++e) {
        const int d = q * HQ + e;
        const int k = jc + R2 * d;
        const long long idx = colo + (long long)k * T.rs;
        const int r = jc + R2 * e;                          // row within the quarter
        float2 xx = staged ? slot[r * F + f] : src[idx];
        float2 pp = staged ? slot[XR::QTP + r * F + f] : fp.ph[idx];
        const int nx = sgn_n<N>(k);
        const int n2 = nx * nx + n2yz;
        const int m = bin_est(n2, s_thr, scb, fp.n_bins);
        if (m >= 0) {
          const float il = s_il[m];
          float im = s_im[m];
          if (mm) im *= s_ims[bin_est(n2, s_mthr, scm, fp.n_mass)];
          const float gx = fmaf(xx.x, il, v[d].x), gy = fmaf(xx.y, il, v[d].y);
          pp.x = fmaf(-ek, gx, pp.x);
          pp.y = fmaf(-ek, gy, pp.y);
          const float sft = eps * im;
          xx.x = fmaf(sft, pp.x, xx.x);
          xx.y = fmaf(sft, pp.y, xx.y);
        } else {
          xx = make_float2(0.f, 0.f);
          pp = make_float2(0.f, 0.f);
        }
        fp.ph[idx] = pp;
        dst[idx] = xx;
        v[d] = xx;
      }
    }
    if (staged && q + 2 < 4) {
      __syncthreads();                                      // every thread has read this slot
      if constexpr (TMA) {
        if (t == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(q + 2);
        }
      } else {
        issue(q + 2);
      }
    }
  }
  fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) fp.W[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
  }
}

// ------------------------------------------------------------------ y pass
template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::NT, BPS_YPASS_MIN_BLOCKS) k_ypass(Fields fp0, int buf) {
  const Fields fp = at_chain(fp0, blockIdx.y);
  if (buf == BUF_W && fp.ds->jreuse) return;   // force stage reused by the jump (uniform)
  using C = Cfg<N>;
  constexpr int F = C::F, R1 = C::R1, R2 = C::R2, NT = C::NT;
  __shared__ float2 s_tw[N];
  __shared__ __align__(16) float2 s_ex[N * F];
  const int t = threadIdx.x;
  const Tile<N> T = tile_y<N>(tile_id<N>());
  float2* data = const_cast<float2*>(buf_ptr(fp, buf));
  const int f = t % F, j = t / F;
  const long long colo = T.base + (long long)f * T.cs;
  float2 v[C::RMAX];
  if constexpr (DIR == FWD) {
    if (j < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) v[b] = data[colo + (long long)(j + R1 * b) * T.rs];
    }
  } else {
    if (j < R2) {
#pragma unroll
      for (int d = 0; d < R1; ++d) v[d] = data[colo + (long long)(j + R2 * d) * T.rs];
    }
  }
  load_twiddles<N>(s_tw, fp.tw, t, NT);
  __syncthreads();
  if constexpr (DIR == FWD) {
    fft2<N, R1, R2, FWD, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
    if (j < R2) {
#pragma unroll
      for (int d = 0; d < R1; ++d) data[colo + (long long)(j + R2 * d) * T.rs] = v[d];
    }
  } else {
    fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
    if (j < R1) {
#pragma unroll
      for (int b = 0; b < R2; ++b) data[colo + (long long)(j + R1 * b) * T.rs] = v[b];
    }
  }
}

// ------------------------------------------------------------------ z pass
// LP pairs of consecutive z lines per tile; line 2f is the real part and line
// 2f+1 the imaginary part of one complex transform of length N.  The lines of
// the tile are contiguous in HBM and arrive by bulk copies.
template <int N, int MODE, int LP = Cfg<N>::LP>
struct ZSmem {
  using C = Cfg<N>;
  static constexpr int LINES = 2 * LP;
  static constexpr size_t BUF = (size_t)LP * (N + C::RMAX) * sizeof(float2);
  static constexpr size_t OFF_BUF = 0;
  static constexpr size_t OFF_TW = BUF;
  static constexpr size_t OFF_RED = OFF_TW + (size_t)N * sizeof(float2);
  static constexpr size_t OFF_BAR = OFF_RED + 32 * sizeof(double);
  static constexpr size_t BYTES = OFF_BAR + sizeof(uint64_t);
  static_assert(BUF >= (size_t)LINES * C::ZP * sizeof(float2), "staging does not fit");
  static_assert(BUF >= (size_t)LINES * N * sizeof(float), "staging does not fit");
};

template <int N, int MODE, int LP = Cfg<N>::LP>
__global__ void __launch_bounds__(LP * Cfg<N>::RMAX) k_zpass(Fields fp0, ZArgs za) {
  const Fields fp = at_chain(fp0, blockIdx.y);
  using C = Cfg<N>;
  using L = ZSmem<N, MODE, LP>;
  constexpr int R1 = C::R1, R2 = C::R2, H = C::H, ZP = C::ZP, NTZ = LP * C::RMAX;
  constexpr int LINES = L::LINES;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* s_buf = reinterpret_cast<float2*>(smem + L::OFF_BUF);
  float2* s_tw = reinterpret_cast<float2*>(smem + L::OFF_TW);
  double* s_red = reinterpret_cast<double*>(smem + L::OFF_RED);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  const int t = threadIdx.x;
  DevState* ds = fp.ds;
  if constexpr (MODE == Z_GRAD) {
    if (ds->jreuse) return;       // force stage reused by the jump (uniform)
  }
  // Lines in decreasing x: the y passes visit the x planes upwards, so the planes
  // the z pass reads first are the ones the inverse y pass wrote last (still in
  // L2), and the forward y pass starts on the planes the z pass wrote last.
  const long long L0 = (long long)(gridDim.x - 1 - blockIdx.x) * LINES;
  constexpr bool STAGED = MODE != Z_NOISE;
  // Z_GRAD, Z_SUMS: support [lo, hi) of R on each line of the tile (whole lines
  // without support information).  Outside it R = 0, the counts are 0 and
  // a = c = 0, so g = 0 and every term of the sums vanishes there: both read a
  // and c (or the data) on the support only, and give a tile without support a
  // zero force, written without reading W, or zero sums.
  constexpr bool SUPPORT = MODE == Z_GRAD || MODE == Z_SUMS;
  __shared__ int s_lo[SUPPORT ? LINES : 1], s_hi[SUPPORT ? LINES : 1];
  const SurveyData sd = survey(fp);
  if constexpr (SUPPORT) {
    if (t < LINES) {
      if (sd.span) {
        const int2 sp = sd.span[L0 + t];
        s_lo[t] = N - sp.x;
        s_hi[t] = sp.y;
      } else {
        s_lo[t] = 0;
        s_hi[t] = N;
      }
    }
  }
  if constexpr (STAGED) {
    if (t == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if constexpr (SUPPORT) {
      bool any = false;
#pragma unroll
      for (int l = 0; l < LINES; ++l) any |= s_hi[l] > s_lo[l];
      if (!any) {
        if constexpr (MODE == Z_GRAD) {
          for (int i = t; i < LINES * (H + 1); i += NTZ) {
            const int l = i / (H + 1), k = i - l * (H + 1);
            fp.W[(L0 + l) * ZP + k] = make_float2(0.f, 0.f);
          }
          if (za.region >= 0 && t == 0) fp.part[za.region + blockIdx.x] = 0.0;
        } else {
          const int nsub = ds->nsub;
          for (int q = t; q < 3 * nsub; q += NTZ) fp.part[za.region + q * fp.part_stride + blockIdx.x] = 0.0;
        }
        return;
      }
    }
    if (t == 0) {
      if constexpr (MODE == Z_R2C) {
        constexpr uint32_t RB = LINES * N * sizeof(float);
        mbar_expect_tx(bar, RB);
        bulk_load(s_buf, za.rin + L0 * N, RB, bar);
      } else {
        const float2* src = (MODE == Z_C2R) ? za.src : fp.W;
        constexpr uint32_t SB = LINES * ZP * sizeof(float2);
        mbar_expect_tx(bar, SB);
        bulk_load(s_buf, src + L0 * ZP, SB, bar);
      }
    }
  }
  load_twiddles<N>(s_tw, fp.tw, t, NTZ);
  float2 v[C::RMAX];

  if constexpr (STAGED) {
    bool ok = mbar_wait(bar, 0);
    ok = __syncthreads_and(ok);
    if (!ok) {
      if (t == 0) atomicOr(&ds->status, ST_TIMEOUT);
      return;
    }
  }

  if constexpr (MODE == Z_GRAD || MODE == Z_C2R || MODE == Z_SUMS) {
    {
      const int f = t / R2, a = t % R2;
      if (f < LP) {
#pragma unroll
        for (int b = 0; b < R1; ++b) {
          const int k = a + R2 * b;
          float2 xa, xb;
          if (k <= H) {
            xa = s_buf[(2 * f) * ZP + k];
            xb = s_buf[(2 * f + 1) * ZP + k];
            if (k == 0 || k == H) { xa.y = 0.f; xb.y = 0.f; }
          } else {
            xa = cconj(s_buf[(2 * f) * ZP + N - k]);
            xb = cconj(s_buf[(2 * f + 1) * ZP + N - k]);
          }
          v[b] = make_float2(xa.x - xb.y, xa.y + xb.x);
        }
      }
    }
    __syncthreads();
    fft2<N, R2, R1, INV, MAP_ROW, LP, TwSquare<N>::value>(v, s_buf, s_tw, t);
  } else {
    float* sr = reinterpret_cast<float*>(s_buf);
    if constexpr (MODE == Z_NOISE) {
      const unsigned long long it = ds->iteration;
      const uint64_t key = ds->seed;
      const unsigned long long blk0 = (unsigned long long)(L0 * N) / 8;
      for (int q = t; q < LINES * N / 8; q += NTZ) {
        P4 r = philox(blk0 + q, it, ST_MOMENTUM, 0, key);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float u1, u2;
          u24pair(r.w[j], u1, u2);
          const float rad = sqrtf(-2.f * logf(u1));
          float sn, cs;
          sincospif(2.f * u2, &sn, &cs);
          sr[8 * q + 2 * j] = rad * cs;
          sr[8 * q + 2 * j + 1] = rad * sn;
        }
      }
      __syncthreads();
    }
    const int f = t / R1, c = t % R1;
    if (f < LP) {
#pragma unroll
      for (int d = 0; d < R2; ++d) {
        const int n = c + R1 * d;
        v[d] = make_float2(sr[(2 * f) * N + n], sr[(2 * f + 1) * N + n]);
      }
    }
    __syncthreads();
  }

  // here: thread (f = t / R1, c = t % R1), f < LP, holds y[c + R1 d], d < R2
  if constexpr (MODE == Z_GRAD || MODE == Z_C2R || MODE == Z_SUMS) {
    const int f = t / R1, c = t % R1;
    const long long la = (L0 + 2 * f) * N, lb = la + N;
    if constexpr (MODE == Z_C2R) {
      if (f < LP) {
        if (za.mom) {
          const long long nv3 = (long long)N * N * N;
#pragma unroll
          for (int d = 0; d < R2; ++d) {
            const int n = c + R1 * d;
            const double da = (double)(v[d].x * fp.inv_nv), db = (double)(v[d].y * fp.inv_nv);
            za.mom[la + n] += da;
            za.mom[lb + n] += db;
            za.mom[nv3 + la + n] += da * da;
            za.mom[nv3 + lb + n] += db * db;
          }
        } else {
#pragma unroll
          for (int d = 0; d < R2; ++d) {
            const int n = c + R1 * d;
            za.rout[la + n] = v[d].x * fp.inv_nv;
            za.rout[lb + n] = v[d].y * fp.inv_nv;
          }
        }
      }
      return;
    }
    if constexpr (MODE == Z_SUMS) {
      const long long nv = (long long)N * N * N;
      const int nsub = ds->nsub;
      const int loa = f < LP ? s_lo[2 * f] : 0, hia = f < LP ? s_hi[2 * f] : 0;
      const int lob = f < LP ? s_lo[2 * f + 1] : 0, hib = f < LP ? s_hi[2 * f + 1] : 0;
      // per-warp sums of all 3 nsub quantities as compensated FP32 pairs, then one
      // pass over the warps (the same additions, in the same order, as one block
      // sum per quantity)
      constexpr int NW = (NTZ + 31) / 32;
      __shared__ float s_ws[NW][3 * MAXS][2];   // compensated pairs
      const int lane = t & 31, w = t >> 5;
      for (int l = 0; l < nsub; ++l) {
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (f < LP) {
          const uint16_t* cn = sd.cnt + l * nv;
          const float* rr = sd.R + l * nv;
#pragma unroll
          for (int d = 0; d < R2; ++d) {
            const int n = c + R1 * d;
            const bool ina = n >= loa && n < hia, inb = n >= lob && n < hib;
            const float da = v[d].x * fp.inv_nv, db = v[d].y * fp.inv_nv;
            const float ra = ina ? rr[la + n] : 0.f, rb = inb ? rr[lb + n] : 0.f;
            const float na = ina ? (float)cn[la + n] : 0.f, nb = inb ? (float)cn[lb + n] : 0.f;
            s1 += na * da + nb * db;
            s2 += ra * da + rb * db;
            s3 += ra * da * da + rb * db * db;
          }
        }
        float c1 = 0.f, c2 = 0.f, c3 = 0.f;
        warp_sum2<NTZ>(s1, c1);
        warp_sum2<NTZ>(s2, c2);
        warp_sum2<NTZ>(s3, c3);
        if (lane == 0) {
          s_ws[w][3 * l + 0][0] = s1;
          s_ws[w][3 * l + 0][1] = c1;
          s_ws[w][3 * l + 1][0] = s2;
          s_ws[w][3 * l + 1][1] = c2;
          s_ws[w][3 * l + 2][0] = s3;
          s_ws[w][3 * l + 2][1] = c3;
        }
      }
      __syncthreads();
      for (int q = t; q < 3 * nsub; q += NTZ) {
        TwoSumAcc r;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          r.add(s_ws[i][q][0]);
          r.add(s_ws[i][q][1]);
        }
        fp.part[za.region + q * fp.part_stride + blockIdx.x] = r.value();
      }
      return;
    }
    // Z_GRAD: the local force g = a delta - c (Eq. Wiener_Posterior_force) and the
    // likelihood energy (1/2) sum (a delta^2 - 2 c delta).  a and c are read from
    // global memory on the support only (not staged: shared memory would cap the
    // resident tiles of this latency-bound pass).
    // the energy only where it is asked for (the last force evaluation of a
    // trajectory): the compensated sum costs issue slots this pass is short of
    TwoSumAcc e;
    const bool want_e = za.region >= 0;
    if (f < LP) {
      const int loa = s_lo[2 * f], hia = s_hi[2 * f], lob = s_lo[2 * f + 1], hib = s_hi[2 * f + 1];
#pragma unroll
      for (int d = 0; d < R2; ++d) {
        const int n = c + R1 * d;
        const bool ina = n >= loa && n < hia, inb = n >= lob && n < hib;
        const long long ga0 = (L0 + 2 * f) * N + n, gb0 = ga0 + N;
        const float aa = ina ? __ldg(fp.a + ga0) : 0.f, ca = ina ? __ldg(fp.c + ga0) : 0.f;
        const float ab = inb ? __ldg(fp.a + gb0) : 0.f, cb = inb ? __ldg(fp.c + gb0) : 0.f;
        const float da = v[d].x * fp.inv_nv, db = v[d].y * fp.inv_nv;
        const float ga = fmaf(aa, da, -ca), gb = fmaf(ab, db, -cb);
        if (want_e) {                           // a d^2 - 2 c d
          e.add(da * (ga - ca));
          e.add(db * (gb - cb));
        }
        v[d] = make_float2(ga, gb);
      }
    }
    if (want_e) {
      TwoSumAcc h;                 // halving is exact
      h.s = 0.5f * e.s;
      h.c = 0.5f * e.c;
      double s = block_sum2<NTZ>(h, reinterpret_cast<float*>(s_red));
      if (t == 0) fp.part[za.region + blockIdx.x] = s;
    }
  }

  // forward transform of the packed pair, then split into the two half spectra:
  // G_a[k] = (Y[k] + conj Y[N-k]) / 2 and G_b[k] = -i (Y[k] - conj Y[N-k]) / 2,
  // k <= N/2.  Thread (f, c) holds Y[c + R2 d], d < R1; Y[N - k] of its k =
  // c + R2 d sits in the same pair's thread R2 - c as element R1 - 1 - d (c > 0)
  // or in its own element (R1 - d) mod R1 (c = 0), so the split takes one
  // register shuffle per element instead of a pass through shared memory.
  fft2<N, R1, R2, FWD, MAP_ROW, LP, TwSquare<N>::value>(v, s_buf, s_tw, t);
  {
    static_assert(R1 % 2 == 0, "the split below covers k <= N/2 for even R1");
    constexpr unsigned MASK = NTZ >= 32 ? 0xffffffffu : ((1u << NTZ) - 1u);
    const int f = t / R2, c = t % R2;
    const int lane = t & 31;
    const int src = lane - c + (R2 - c) % R2;
    float2* dst = (MODE == Z_GRAD) ? fp.W : (MODE == Z_NOISE) ? fp.ph : za.dst;
    float2* da = dst + (L0 + 2 * f) * ZP;
    float2* db = da + ZP;
#pragma unroll
    for (int d = 0; d <= R1 / 2; ++d) {
      const float2 snd = v[R1 - 1 - d];
      float2 rcv;
      rcv.x = __shfl_sync(MASK, snd.x, src);
      rcv.y = __shfl_sync(MASK, snd.y, src);
      const int k = c + R2 * d;
      if (f < LP && k <= H) {
        const float2 yk = v[d];
        const float2 ym = cconj(c == 0 ? v[(R1 - d) % R1] : rcv);
        da[k] = make_float2(0.5f * (yk.x + ym.x), 0.5f * (yk.y + ym.y));
        db[k] = make_float2(0.5f * (yk.y - ym.y), -0.5f * (yk.x - ym.x));
      }
    }
  }
}

// ------------------------------------------------------------------ x pass with warp-private rings
// X_LEAP like k_xleap_ring, but each warp copies, waits for and reads only the
// delta and p rows its own threads use (16-byte cp.async copies into the same
// two-slot layout): the quarter loop has no block barrier, only the warp's own
// copy-group waits and warp barriers.  Nyquist tiles read delta and p directly.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::NT, BPS_XLEAP_MIN_BLOCKS)
    k_xleap_wring(Fields fp0, XArgs xa, const __grid_constant__ XMaps maps) {
  using XR = XRing<N>;
  const Fields fp = at_chain(fp0, blockIdx.y);
  using C = Cfg<N>;
  constexpr int F = C::F, R1 = C::R1, R2 = C::R2, NT = C::NT, HQ = R1 / 4;
  constexpr int JW = 32 / F;                                // row groups (jc values) per warp
  static_assert(32 % F == 0, "a warp covers whole row groups");
  (void)maps;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* s_ring = reinterpret_cast<float2*>(smem);         // [slot][delta, p][QR rows][F], arrays QTP apart
  __shared__ float2 s_tw[N];
  __shared__ __align__(16) float2 s_ex[N * F];
  __shared__ int s_thr[MAXB], s_mthr[MAXB];
  __shared__ float s_il[MAXB], s_im[MAXB], s_ims[MAXB];
  const int t = threadIdx.x, lane = t & 31;
  DevState* ds = fp.ds;
  const int id = tile_id<N>();
  const Tile<N> T = tile_x<N>(id);
  const bool staged = id < N * C::ZB;
  const int cur = ds->cur;
  const int sbuf = xa.first ? cur : 1 - cur;
  const float2* src = dsel(fp, sbuf);
  const int jw0 = (t / 32) * JW;                            // first row group of this warp
  // quarter q of this warp's rows into slot q & 1: rows jc + R2 e (jc of the
  // warp, e < HQ) of delta and p, two complex per 16-byte copy
  auto issue = [&](int q) {
    float2* slot = s_ring + (size_t)(q & 1) * 2 * XR::QTP;
    constexpr int PER_ARR = JW * HQ * (F / 2);
#pragma unroll
    for (int i = 0; i < 2 * PER_ARR / 32; ++i) {
      const int c = lane + 32 * i;
      const int arr = c / PER_ARR, cc = c - arr * PER_ARR;
      const int rl = cc / (F / 2), pair = cc - rl * (F / 2);
      const int jc = jw0 + rl % JW, e = rl / JW;
      if (jc < R2) {
        const int r = jc + R2 * e;
        const float2* g = (arr ? fp.ph : src) + T.base + (long long)(q * XR::QR + r) * T.rs + 2 * pair;
        cp_async16(slot + arr * XR::QTP + r * F + 2 * pair, g);
      }
    }
    cp_async_commit();
  };
  if (staged) {
    issue(0);
    issue(1);
  }
  load_twiddles<N>(s_tw, fp.tw, t, NT);
  for (int i = t; i < MAXB; i += NT) {
    s_thr[i] = ds->thr[i];
    s_mthr[i] = ds->mthr[i];
    s_il[i] = ds->inv_lambda[i];
    s_im[i] = ds->inv_M[i];
    s_ims[i] = ds->inv_ms[i];
  }
  __syncthreads();   // the transform reads the twiddles before its first barrier
  const int f = t % F;
  const int ja = t / F;
  const int ky = T.ky0 + f * T.dky, kz = T.kz0 + f * T.dkz;
  const int ny = sgn_n<N>(ky);
  const int n2yz = ny * ny + kz * kz;
  const long long colo = T.base + (long long)f * T.cs;
  const bool mm = fp.mass_mode != 0;
  const float scb = bin_scale(fp.n_bins, N), scm = bin_scale(fp.n_mass, N);
  float2* dst = dsel(fp, 1 - cur);
  float2 v[C::RMAX];
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) v[b] = fp.W[colo + (long long)(ja + R1 * b) * T.rs];
  }
  fft2<N, R1, R2, FWD, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  const int jc = t / F;
  const bool act = jc < R2;
  const float eps = (float)ds->eps;
  const float ek = xa.first ? 0.5f * eps : eps;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2* slot = s_ring + (size_t)(q & 1) * 2 * XR::QTP;
    if (staged) {
      // this lane's copies of quarter q have landed (only quarter q + 1 may still
      // be in flight); the warp barrier makes every lane's copies visible
      if (q < 3) cp_async_wait<1>();
      else cp_async_wait<0>();
      __syncwarp();
    }
    if (act) {
#pragma unroll
      for (int e = 0; e < HQ; ++e) {
        const int d = q * HQ + e;
        const int k = jc + R2 * d;
        const long long idx = colo + (long long)k * T.rs;
        const int r = jc + R2 * e;                          // row within the quarter
        float2 xx = staged ? slot[r * F + f] : src[idx];
        float2 pp = staged ? slot[XR::QTP + r * F + f] : fp.ph[idx];
        const int nx = sgn_n<N>(k);
        const int n2 = nx * nx + n2yz;
        const int m = bin_est(n2, s_thr, scb, fp.n_bins);
        if (m >= 0) {
          const float il = s_il[m];
          float im = s_im[m];
          if (mm) im *= s_ims[bin_est(n2, s_mthr, scm, fp.n_mass)];
          const float gx = fmaf(xx.x, il, v[d].x), gy = fmaf(xx.y, il, v[d].y);
          pp.x = fmaf(-ek, gx, pp.x);
          pp.y = fmaf(-ek, gy, pp.y);
          const float sft = eps * im;
          xx.x = fmaf(sft, pp.x, xx.x);
          xx.y = fmaf(sft, pp.y, xx.y);
        } else {
          xx = make_float2(0.f, 0.f);
          pp = make_float2(0.f, 0.f);
        }
        fp.ph[idx] = pp;
        dst[idx] = xx;
        v[d] = xx;
      }
    }
    if (staged && q + 2 < 4) {
      __syncwarp();                                         // every lane of the warp has read this slot
      issue(q + 2);
    }
  }
  fft2<N, R2, R1, INV, MAP_COL, F, TwSquare<N>::value>(v, s_ex, s_tw, t);
  if (ja < R1) {
#pragma unroll
    for (int b = 0; b < R2; ++b) fp.W[colo + (long long)(ja + R1 * b) * T.rs] = v[b];
  }
}

// ------------------------------------------------------------------ voxel kernels
// Kahan-compensated FP32 running sum (s, c); the sum is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// a_i = sum_l b_l^2 Nbar_l R^l_i,  c_i = sum_l b_l (N^l_i - Nbar_l R^l_i)  (Eq. Wiener_Posterior_force);
// the counts are zero wherever R = 0 (checked by set_data), so no mask is needed.
// With per-line supports only the voxels inside them are computed: outside,
// a = c = 0, which the data upload wrote once.
__global__ void __launch_bounds__(256) k_rebuild(Fields fp0, long long nv, int region) {
  const Fields fp = at_chain(fp0, blockIdx.y);
  __shared__ float s_a[MAXS], s_b[MAXS], s_bn[MAXS];
  __shared__ double s_red[32];
  DevState* ds = fp.ds;
  const int nsub = ds->nsub;
  if (threadIdx.x < nsub) {
    const double b = ds->b[threadIdx.x], nb = ds->nbar[threadIdx.x];
    s_a[threadIdx.x] = (float)(b * b * nb);
    s_b[threadIdx.x] = (float)b;
    s_bn[threadIdx.x] = (float)(b * nb);
  }
  __syncthreads();
  float acc = 0.f, comp = 0.f;   // FP32 with Kahan compensation per thread; FP64 across the block
  const SurveyData sd = survey(fp);
  // a and c of the four voxels of float4 group i
  auto group = [&](long long i) -> float {
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), Cc = A;
    for (int l = 0; l < nsub; ++l) {
      const float4 r = reinterpret_cast<const float4*>(sd.R + l * nv)[i];
      const ushort4 n = reinterpret_cast<const ushort4*>(sd.cnt + l * nv)[i];
      const float ka = s_a[l], kb = s_b[l], kbn = s_bn[l];
      A.x = fmaf(ka, r.x, A.x); A.y = fmaf(ka, r.y, A.y); A.z = fmaf(ka, r.z, A.z); A.w = fmaf(ka, r.w, A.w);
      Cc.x += kb * (float)n.x - kbn * r.x;
      Cc.y += kb * (float)n.y - kbn * r.y;
      Cc.z += kb * (float)n.z - kbn * r.z;
      Cc.w += kb * (float)n.w - kbn * r.w;
    }
    reinterpret_cast<float4*>(fp.a)[i] = A;
    reinterpret_cast<float4*>(fp.c)[i] = Cc;
    return (A.x + A.y) + (A.z + A.w);
  };
  if (sd.span) {
    // one warp per z line, its lanes over the line's support (multiples of 4 voxels)
    const int n_grid = fp.grid_n;
    const int lines = n_grid * n_grid, gpl = n_grid / 4;   // float4 groups per line
    const int lane = threadIdx.x & 31;
    for (int line = blockIdx.x * 8 + (threadIdx.x >> 5); line < lines; line += gridDim.x * 8) {
      const int2 sp = sd.span[line];
      const int g0 = (n_grid - sp.x) / 4, g1 = sp.y / 4;
      for (int g = g0 + lane; g < g1; g += 32) kahan_add(acc, comp, group((long long)line * gpl + g));
    }
  } else {
    const long long n4 = nv / 4;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n4; i += (long long)gridDim.x * 256)
      kahan_add(acc, comp, group(i));
  }
  TwoSumAcc k;                    // the Kahan sum acc - comp as a pair
  k.s = acc;
  k.c = -comp;
  double s = block_sum2<256>(k, reinterpret_cast<float*>(s_red));
  if (threadIdx.x == 0) fp.part[region + blockIdx.x] = s;
}

// Data check and compression: counts int32 -> uint16, R copied; per block the
// sums R, N^2/R, #(R>0) over R > 0 and the number of invalid voxels.  With
// cout = rout = NULL it only checks (data already in place).  Per
// thread the sums run in FP32 with Kahan compensation and the counts in
// integers (FP64 arithmetic is slow on this part); blocks combine in FP64.
//
// With `span` (grids with N a multiple of 32, so that a warp's 32 voxels lie on
// one z line) the kernel also widens each line's support [lo, hi) to the
// voxels with R > 0: a warp ballot, then two atomics by the warp's first lane.
// Since counts are zero where R = 0, a and c vanish outside the union of these
// supports over the subsamples.
template <typename CT>
__global__ void __launch_bounds__(256) k_data(const CT* cin, const float* rin, uint16_t* cout, float* rout,
                                              long long nv, double* part, int stride, int2* span, int n_grid) {
  __shared__ double s_red[32];
  float sR = 0.f, cR = 0.f, sB = 0.f, cB = 0.f;
  unsigned int no = 0, bad = 0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nv; i += (long long)gridDim.x * 256) {
    const float r = rin[i];
    const int n = (int)cin[i];
    const bool rok = (r >= 0.f) && isfinite(r);
    const bool nok = n >= 0 && n <= 65535;
    if (!rok || !nok || (r == 0.f && n > 0)) ++bad;
    if (span) {
      const unsigned m = __ballot_sync(0xffffffffu, rok && r > 0.f);
      if (m != 0u && (threadIdx.x & 31) == 0) {
        const int ii = (int)i;                 // < N^3 <= 512^3: 32-bit division
        const int line = ii / n_grid;
        const int z0 = ii - line * n_grid;
        const int lo = (z0 + __ffs((int)m) - 1) & ~3;
        const int hi = (z0 + 32 - __clz((int)m) + 3) & ~3;
        atomicMax(&span[line].x, n_grid - lo);
        atomicMax(&span[line].y, hi);
      }
    }
    if (cout) cout[i] = (uint16_t)(nok ? n : 0);
    if (rout) rout[i] = rok ? r : 0.f;
    if (rok && r > 0.f) {
      kahan_add(sR, cR, r);
      const float fn = (float)(nok ? n : 0);
      kahan_add(sB, cB, fn * fn / r);
      ++no;
    }
  }
  double v0 = block_sum<256>((double)sR - (double)cR, s_red);
  double v1 = block_sum<256>((double)sB - (double)cB, s_red);
  double v2 = block_sum<256>((double)no, s_red);
  double v3 = block_sum<256>((double)bad, s_red);
  if (threadIdx.x == 0) {
    part[0 * stride + blockIdx.x] = v0;
    part[1 * stride + blockIdx.x] = v1;
    part[2 * stride + blockIdx.x] = v2;
    part[3 * stride + blockIdx.x] = v3;
  }
}

// The same check, four consecutive voxels per thread (one 16-byte load of R,
// one 8- or 16-byte load of the counts, vector stores): every upload path of a
// survey (16-bit counts checked in place, 32-bit counts converted into the
// slot) sums in this one order, so they give the same data constants bit for
// bit.  A z line holds whole 4-voxel groups (N is a multiple of 4).  The line
// support is a warp minimum and maximum when a warp's 128 voxels lie on one z
// line (N a multiple of 128), else a pair of atomics per thread with data.
template <typename CT>
__global__ void __launch_bounds__(256, 4) k_data4(const CT* __restrict__ cin, const float* __restrict__ rin,
                                               uint16_t* cout, float* rout, long long nv, double* part, int stride,
                                               int2* span, int n_grid) {
  __shared__ double s_red[32];
  float sR = 0.f, cR = 0.f, sB = 0.f, cB = 0.f;
  unsigned int no = 0, bad = 0;
  const long long n4 = nv / 4;
  const int lane = threadIdx.x & 31;
  const bool warp_line = n_grid % 128 == 0;
  // DEPTH consecutive grid-stride groups are loaded before any is processed (more
  // loads in flight per thread); they are then processed in the order of the
  // plain grid-stride loop, so every sum sees its terms in the same order
  constexpr int DEPTH = sizeof(CT) == 2 ? 4 : 2;   // 16-bit counts leave room for four groups
  using CV = typename std::conditional<sizeof(CT) == 2, ushort4, int4>::type;
  const long long gstride = (long long)gridDim.x * 256;
  for (long long q0 = blockIdx.x * 256LL + threadIdx.x; q0 < n4; q0 += DEPTH * gstride) {
  CV cbuf[DEPTH];
  float4 rbuf[DEPTH];
#pragma unroll
  for (int u = 0; u < DEPTH; ++u) {
    const long long qu = q0 + u * gstride;
    if (qu < n4) {
      cbuf[u] = reinterpret_cast<const CV*>(cin)[qu];
      rbuf[u] = reinterpret_cast<const float4*>(rin)[qu];
    }
  }
#pragma unroll
  for (int u = 0; u < DEPTH; ++u) {
    const long long q = q0 + u * gstride;
    if (q >= n4) break;
    int c4[4];
    c4[0] = (int)cbuf[u].x; c4[1] = (int)cbuf[u].y; c4[2] = (int)cbuf[u].z; c4[3] = (int)cbuf[u].w;
    const float4 rr = rbuf[u];
    const float r4[4] = {rr.x, rr.y, rr.z, rr.w};
    unsigned short o4[4];
    float or4[4];
    int first = -1, last = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float r = r4[j];
      const int n = c4[j];
      const bool rok = (r >= 0.f) && isfinite(r);
      const bool nok = n >= 0 && n <= 65535;
      if (!rok || !nok || (r == 0.f && n > 0)) ++bad;
      o4[j] = (unsigned short)(nok ? n : 0);
      or4[j] = rok ? r : 0.f;
      if (rok && r > 0.f) {
        if (first < 0) first = j;
        last = j;
        kahan_add(sR, cR, r);
        const float fn = (float)(nok ? n : 0);
        kahan_add(sB, cB, fn * fn / r);
        ++no;
      }
    }
    if (cout) reinterpret_cast<ushort4*>(cout)[q] = make_ushort4(o4[0], o4[1], o4[2], o4[3]);
    if (rout) reinterpret_cast<float4*>(rout)[q] = make_float4(or4[0], or4[1], or4[2], or4[3]);
    if (span) {
      const int z0 = (int)((q * 4) % n_grid);
      const int line = (int)((q * 4) / n_grid);
      int lo = first >= 0 ? z0 + first : 0x7fffffff;
      int hi = last >= 0 ? z0 + last + 1 : -1;
      if (warp_line) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
          hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane != 0) hi = -1;
      }
      if (hi >= 0) {
        atomicMax(&span[line].x, n_grid - (lo & ~3));
        atomicMax(&span[line].y, (hi + 3) & ~3);
      }
    }
  }
  }
  double v0 = block_sum<256>((double)sR - (double)cR, s_red);
  double v1 = block_sum<256>((double)sB - (double)cB, s_red);
  double v2 = block_sum<256>((double)no, s_red);
  double v3 = block_sum<256>((double)bad, s_red);
  if (threadIdx.x == 0) {
    part[0 * stride + blockIdx.x] = v0;
    part[1 * stride + blockIdx.x] = v1;
    part[2 * stride + blockIdx.x] = v2;
    part[3 * stride + blockIdx.x] = v3;
  }
}

// the vectorised check applies to whole 4-voxel groups with aligned pointers
inline bool data4_ok(const void* cin, size_t csz, const void* rin, const void* cout, const void* rout, long long nv) {
  auto al = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
  return nv % 128 == 0 && al(cin, 4 * csz) && al(rin, 16) && al(cout, 8) && al(rout, 16);
}

__global__ void k_philox_words(uint64_t seed, uint64_t it, uint64_t stage, uint64_t sub, uint64_t blk0, size_t n,
                               uint64_t* out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i * 4 >= n) return;
  P4 r = philox(blk0 + i, it, stage, sub, seed);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (i * 4 + j < n) out[i * 4 + j] = r.w[j];
}

__global__ void k_voxel_normals(uint64_t seed, uint64_t it, size_t n, float* out) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q * 8 >= n) return;
  P4 r = philox(q, it, ST_MOMENTUM, 0, seed);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float u1, u2;
    u24pair(r.w[j], u1, u2);
    const float rad = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    if (q * 8 + 2 * j < n) out[q * 8 + 2 * j] = rad * cs;
    if (q * 8 + 2 * j + 1 < n) out[q * 8 + 2 * j + 1] = rad * sn;
  }
}

// ------------------------------------------------------------------ launch tables
template <int N>
struct Launch {
  using C = Cfg<N>;
  template <int M>
  static void x(const Fields& fp, const XArgs& xa, int nch, cudaStream_t s) {
    k_xpass<N, M><<<dim3(C::TILES, nch), C::NT, 0, s>>>(fp, xa);
  }
  template <int D>
  static void y(const Fields& fp, int buf, int nch, cudaStream_t s) {
    k_ypass<N, D><<<dim3(C::TILES, nch), C::NT, 0, s>>>(fp, buf);
  }
  template <int M, int LP = C::LP>
  static void z(const Fields& fp, const ZArgs& za, int nch, cudaStream_t s) {
    k_zpass<N, M, LP><<<dim3(N * N / (2 * LP), nch), LP * C::RMAX, ZSmem<N, M, LP>::BYTES, s>>>(fp, za);
  }
  template <int M, int LP = C::LP>
  static void zattr() {
    cudaFuncSetAttribute(k_zpass<N, M, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ZSmem<N, M, LP>::BYTES);
  }
  static void attrs() {
    zattr<Z_GRAD>(); zattr<Z_NOISE>(); zattr<Z_R2C>(); zattr<Z_C2R>(); zattr<Z_SUMS>();
    zattr<Z_GRAD, 4>(); zattr<Z_GRAD, 16>();
  }
};

template <int N>
static PassTable make_table() {
  using L = Launch<N>;
  using C = Cfg<N>;
  L::attrs();
  PassTable T;
  T.N = N;
  T.zp = C::ZP;
  T.F = C::F;
  T.x_tiles = C::TILES;
  T.z_tiles = C::ZTILES;
  T.x_init = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_INIT>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_leap = [](const Fields& f, int first, int n, cudaStream_t s) { L::template x<X_LEAP>(f, XArgs{-1, nullptr, first, -1}, n, s); };
  T.x_leapg = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_LEAPG>(f, XArgs{-1, nullptr, 1, region}, n, s); };
  T.x_final = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_FINAL>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_inv = [](const Fields& f, int src, float2* dst, int n, cudaStream_t s) { L::template x<X_INV>(f, XArgs{src, dst, 0, -1}, n, s); };
  T.x_fwd = [](const Fields& f, int src, float2* dst, int n, cudaStream_t s) { L::template x<X_FWD>(f, XArgs{src, dst, 0, -1}, n, s); };
  T.x_grad = [](const Fields& f, float2* dst, int region, int n, cudaStream_t s) { L::template x<X_GRAD>(f, XArgs{-1, dst, 0, region}, n, s); };
  T.x_jinv = [](const Fields& f, int n, cudaStream_t s) { L::template x<X_JINV>(f, XArgs{-1, nullptr, 0, -1}, n, s); };
  T.x_jgrad = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_JGRAD>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_scale = [](const Fields& f, int n, cudaStream_t s) { L::template x<X_SCALE>(f, XArgs{-1, nullptr, 0, -1}, n, s); };
  T.x_binpow = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_BINPOW>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_macc = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_MACC>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_mmean = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_MMEAN>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.x_wpow = [](const Fields& f, int region, int n, cudaStream_t s) { L::template x<X_WPOW>(f, XArgs{-1, nullptr, 0, region}, n, s); };
  T.y_fwd = [](const Fields& f, int buf, int n, cudaStream_t s) { L::template y<FWD>(f, buf, n, s); };
  T.y_inv = [](const Fields& f, int buf, int n, cudaStream_t s) { L::template y<INV>(f, buf, n, s); };
  T.z_grad = [](const Fields& f, int region, int n, cudaStream_t s) { L::template z<Z_GRAD>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, region, 0}, n, s); };
  // the force z pass at every tile size the autotuner chooses from
  T.z_grad_lp[0] = [](const Fields& f, int region, int n, cudaStream_t s) { L::template z<Z_GRAD, 4>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, region, 0}, n, s); };
  T.z_grad_lp[1] = [](const Fields& f, int region, int n, cudaStream_t s) { L::template z<Z_GRAD, 8>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, region, 0}, n, s); };
  T.z_grad_lp[2] = [](const Fields& f, int region, int n, cudaStream_t s) { L::template z<Z_GRAD, 16>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, region, 0}, n, s); };
  for (int i = 0; i < 3; ++i) T.z_lp_tiles[i] = N * N / (2 * (4 << i));
  T.z_noise = [](const Fields& f, int n, cudaStream_t s) { L::template z<Z_NOISE>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, -1, 0}, n, s); };
  T.z_r2c = [](const Fields& f, const float* rin, float2* dst, cudaStream_t s) { L::template z<Z_R2C>(f, ZArgs{nullptr, dst, rin, nullptr, -1, 0}, 1, s); };
  T.z_c2r = [](const Fields& f, const float2* src, float* rout, cudaStream_t s) { L::template z<Z_C2R>(f, ZArgs{src, nullptr, nullptr, rout, -1, 0}, 1, s); };
  T.z_mom = [](const Fields& f, double* mom, cudaStream_t s) { L::template z<Z_C2R>(f, ZArgs{f.W, nullptr, nullptr, nullptr, -1, 0, mom}, 1, s); };
  T.z_sums = [](const Fields& f, int region, int n, cudaStream_t s) { L::template z<Z_SUMS>(f, ZArgs{nullptr, nullptr, nullptr, nullptr, region, 0}, n, s); };
  return T;
}

// ---------------------------------------------------------------- TMA x pass: maps and launch
template <int N, int SD, int SP>
void launch_xleap_tma(const Fields& f, const XMaps& m, int first, int nch, cudaStream_t s) {
  k_xleap_tma<N, SD, SP><<<dim3(Cfg<N>::TILES, nch), Cfg<N>::NT, XTma<N, SD, SP>::SMEM, s>>>(
      f, XArgs{-1, nullptr, first, -1}, m);
}

template <int N, int SD, int SP>
XLeapTma xleap_entry() {
  if (cudaFuncSetAttribute(k_xleap_tma<N, SD, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)XTma<N, SD, SP>::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return launch_xleap_tma<N, SD, SP>;
}

template <int N, bool TMA>
void launch_xleap_ring(const Fields& f, const XMaps& m, int first, int nch, cudaStream_t s) {
  k_xleap_ring<N, TMA><<<dim3(Cfg<N>::TILES, nch), Cfg<N>::NT, XRing<N>::SMEM, s>>>(f, XArgs{-1, nullptr, first, -1},
                                                                                      m);
}

template <int N, bool TMA>
XLeapTma xleap_ring_entry() {
  if (cudaFuncSetAttribute(k_xleap_ring<N, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)XRing<N>::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return launch_xleap_ring<N, TMA>;
}

template <int N>
void launch_xleap_wring(const Fields& f, const XMaps& m, int first, int nch, cudaStream_t s) {
  k_xleap_wring<N><<<dim3(Cfg<N>::TILES, nch), Cfg<N>::NT, XRing<N>::SMEM, s>>>(f, XArgs{-1, nullptr, first, -1}, m);
}

template <int N>
XLeapTma xleap_wring_entry() {
  if (cudaFuncSetAttribute(k_xleap_wring<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XRing<N>::SMEM) !=
      cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return launch_xleap_wring<N>;
}

template <int N>
XLeapTma xleap_variant(int which) {
  switch (which) {
    case 1: return xleap_entry<N, 1, 1>();   // W, delta and p staged (two blocks per SM)
    case 2: return xleap_entry<N, 1, 0>();   // W and delta staged (three blocks per SM)
    case 3: return xleap_entry<N, 0, 0>();   // W staged (three blocks per SM)
    case 4: return xleap_ring_entry<N, true>();    // delta and p quarters through a ring filled by tensor copies
    case 5: return xleap_ring_entry<N, false>();   // the same ring filled by 16-byte copies of every thread
    case 6: return xleap_wring_entry<N>();          // warp-private rings, no block barrier per quarter
    default: return nullptr;
  }
}

XLeapTma xleap_tma(int N, int which) {
  switch (N) {
    case 8: return xleap_variant<8>(which);
    case 16: return xleap_variant<16>(which);
    case 32: return xleap_variant<32>(which);
    case 64: return xleap_variant<64>(which);
    case 96: return xleap_variant<96>(which);
    case 128: return xleap_variant<128>(which);
    case 256: return xleap_variant<256>(which);
    default: return nullptr;
  }
}

bool make_xmaps(const Fields& f, int N, int nch, XMaps* out) {
  out->ok = false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  const int ZP = ((N / 2 + 1) + 1) / 2 * 2;
  const int F = N / 2 < 16 ? N / 2 : 16;
  const unsigned long long plane = (unsigned long long)N * N * ZP;
  const unsigned long long cs = f.spec_stride > 0 ? (unsigned long long)f.spec_stride : plane;
  const cuuint64_t dims[4] = {(cuuint64_t)ZP, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)(nch > 0 ? nch : 1)};
  const cuuint64_t strides[3] = {(cuuint64_t)ZP * 8, (cuuint64_t)N * ZP * 8, cs * 8};
  const cuuint32_t box[4] = {(cuuint32_t)F, 1, (cuuint32_t)N, 1};
  const cuuint32_t boxq[4] = {(cuuint32_t)F, 1, (cuuint32_t)(N / 4), 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  float2* bufs[7] = {f.W, f.dh[0], f.dh[1], f.ph, f.dh[0], f.dh[1], f.ph};
  CUtensorMap* maps[7] = {&out->W, &out->d0, &out->d1, &out->ph, &out->d0q, &out->d1q, &out->phq};
  for (int i = 0; i < 7; ++i) {
    if (encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_INT64, 4, bufs[i], dims, strides, i < 4 ? box : boxq, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  out->ok = true;
  return true;
}

bool pass_table(int N, PassTable* out) {
  switch (N) {
    case 8: *out = make_table<8>(); return true;
    case 16: *out = make_table<16>(); return true;
    case 32: *out = make_table<32>(); return true;
    case 64: *out = make_table<64>(); return true;
    case 96: *out = make_table<96>(); return true;
    case 128: *out = make_table<128>(); return true;
    case 256: *out = make_table<256>(); return true;
    default: return false;
  }
}

void launch_rebuild(const Fields& fp, long long nv, int region, int blocks, int nch, cudaStream_t s) {
  k_rebuild<<<dim3(blocks, nch), 256, 0, s>>>(fp, nv, region);
}
void launch_data(const int32_t* cin, const float* rin, uint16_t* cout, float* rout, long long nv, double* part,
                 int stride, int blocks, int2* span, int n_grid, cudaStream_t s) {
  if (data4_ok(cin, sizeof(int32_t), rin, cout, rout, nv))
    k_data4<int32_t><<<blocks, 256, 0, s>>>(cin, rin, cout, rout, nv, part, stride, span, n_grid);
  else
    k_data<int32_t><<<blocks, 256, 0, s>>>(cin, rin, cout, rout, nv, part, stride, span, n_grid);
}
void launch_data16(const uint16_t* cin, const float* rin, uint16_t* cout, float* rout, long long nv, double* part,
                   int stride, int blocks, int2* span, int n_grid, cudaStream_t s) {
  if (data4_ok(cin, sizeof(uint16_t), rin, cout, rout, nv))
    k_data4<uint16_t><<<blocks, 256, 0, s>>>(cin, rin, cout, rout, nv, part, stride, span, n_grid);
  else
    k_data<uint16_t><<<blocks, 256, 0, s>>>(cin, rin, cout, rout, nv, part, stride, span, n_grid);
}
void launch_philox_words(uint64_t seed, uint64_t it, uint64_t stage, uint64_t sub, uint64_t blk0, size_t n,
                         uint64_t* out, cudaStream_t s) {
  size_t nb = (n + 3) / 4;
  k_philox_words<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(seed, it, stage, sub, blk0, n, out);
}
void launch_voxel_normals(uint64_t seed, uint64_t it, size_t n, float* out, cudaStream_t s) {
  size_t nb = (n + 7) / 8;
  k_voxel_normals<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(seed, it, n, out);
}

}  // namespace bps
