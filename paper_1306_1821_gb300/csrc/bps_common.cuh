// Shared device-side definitions of the bps CUDA library: complex helpers,
// the in-register DFT building blocks, the Philox4x64-10 generator, the
// device-resident chain state and the per-grid compile-time configuration.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bps.h"

namespace bps {

constexpr int MAXB = 64;   // maximum number of power-spectrum / mass bins
constexpr int MAXS = 16;   // maximum number of galaxy subsamples
constexpr int FWD = -1;    // exp(-2 pi i jk/N): forward transform (App. C.1, C_hat = 1)
constexpr int INV = +1;    // exp(+2 pi i jk/N): inverse transform (unnormalised here)

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by DIR * i  (DIR = -1: by -i, DIR = +1: by +i)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ------------------------------------------------- unit circle, 48ths of a turn
// cos(2 pi r / 48) for r = 0..12 (the first quadrant); every other 48th of a
// turn follows by quadrant symmetry, so the table is exactly symmetric.
__host__ __device__ constexpr double circ48_c(int r) {
  return r == 0 ? 1.0 : r == 1 ? 0.99144486137381038 : r == 2 ? 0.96592582628906831
       : r == 3 ? 0.92387953251128674 : r == 4 ? 0.86602540378443865 : r == 5 ? 0.79335334029123517
       : r == 6 ? 0.70710678118654752 : r == 7 ? 0.60876142900872066 : r == 8 ? 0.5
       : r == 9 ? 0.38268343236508977 : r == 10 ? 0.25881904510252074 : r == 11 ? 0.13052619222005159
       : 0.0;
}
// (cos, sin)(2 pi j / 48) for any integer j
__host__ __device__ constexpr double circ48_cos(int j) {
  int m = ((j % 48) + 48) % 48;
  int q = m / 12, r = m % 12;
  return q == 0 ? circ48_c(r) : q == 1 ? -circ48_c(12 - r) : q == 2 ? -circ48_c(r) : circ48_c(12 - r);
}
__host__ __device__ constexpr double circ48_sin(int j) { return circ48_cos(j - 12); }

// multiply v by W_R^(DIR * J) = exp(DIR * 2 pi i J / R), R | 48, J compile-time
template <int R, int J, int DIR>
__device__ __forceinline__ float2 twiddle_const(float2 v) {
  constexpr int j48 = ((J * (48 / R)) % 48 + 48) % 48;
  if constexpr (j48 == 0) {
    return v;
  } else if constexpr (j48 == 24) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (j48 == 12) {
    return mul_i<DIR>(v);
  } else if constexpr (j48 == 36) {
    return mul_i<-DIR>(v);
  } else {
    constexpr float c = (float)circ48_cos(j48);
    constexpr float s = (float)(DIR * circ48_sin(j48));
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// ------------------------------------------------- in-register DFTs, natural order
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<1, DIR> {
  __device__ __forceinline__ static void run(float2*) {}
};
template <int DIR>
struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <int DIR>
struct Dft<3, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float h = 0.86602540378443865f;  // sin(2 pi / 3)
    float2 t = cadd(v[1], v[2]);
    float2 u = csub(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 r = mul_i<DIR>(make_float2(h * u.x, h * u.y));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};
template <int DIR>
struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
    float2 s1 = cadd(v[1], v[3]), d1 = csub(v[1], v[3]);
    float2 r = mul_i<DIR>(d1);
    v[0] = cadd(s0, s1);
    v[2] = csub(s0, s1);
    v[1] = cadd(d0, r);
    v[3] = csub(d0, r);
  }
};

// R = A * B in one thread: X[c + B d] = sum_a W_R^(a c) W_A^(a d) sum_b x[a + A b] W_B^(b c)
template <int R, int A, int DIR>
struct DftSplit {
  static constexpr int B = R / A;
  template <int a, int c>
  __device__ __forceinline__ static void tw_row(float2* t) {
    if constexpr (c < B) {
      t[a * B + c] = twiddle_const<R, a * c, DIR>(t[a * B + c]);
      tw_row<a, c + 1>(t);
    }
  }
  template <int a>
  __device__ __forceinline__ static void stage_a(const float2* v, float2* t) {
    if constexpr (a < A) {
      float2 s[B];
#pragma unroll
      for (int b = 0; b < B; ++b) s[b] = v[a + A * b];
      Dft<B, DIR>::run(s);
#pragma unroll
      for (int c = 0; c < B; ++c) t[a * B + c] = s[c];
      tw_row<a, 0>(t);
      stage_a<a + 1>(v, t);
    }
  }
  __device__ __forceinline__ static void run(float2* v) {
    float2 t[R];
    stage_a<0>(v, t);
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float2 s[A];
#pragma unroll
      for (int a = 0; a < A; ++a) s[a] = t[a * B + c];
      Dft<A, DIR>::run(s);
#pragma unroll
      for (int d = 0; d < A; ++d) v[c + B * d] = s[d];
    }
  }
};
template <int DIR> struct Dft<6, DIR> { __device__ __forceinline__ static void run(float2* v) { DftSplit<6, 2, DIR>::run(v); } };
template <int DIR> struct Dft<8, DIR> { __device__ __forceinline__ static void run(float2* v) { DftSplit<8, 2, DIR>::run(v); } };
template <int DIR> struct Dft<12, DIR> { __device__ __forceinline__ static void run(float2* v) { DftSplit<12, 4, DIR>::run(v); } };
template <int DIR> struct Dft<16, DIR> { __device__ __forceinline__ static void run(float2* v) { DftSplit<16, 4, DIR>::run(v); } };

// ------------------------------------------------- grid configuration
// A transform of length N is split N = R1 * R2 across threads (two register
// DFTs and one shared-memory exchange).  ZP is the padded half-spectrum row
// (N/2 + 1 complex rounded up to an even count: 16-byte aligned rows).
template <int N>
struct Grid;
template <> struct Grid<8>   { static constexpr int R1 = 4,  R2 = 2;  };
template <> struct Grid<16>  { static constexpr int R1 = 4,  R2 = 4;  };
template <> struct Grid<32>  { static constexpr int R1 = 8,  R2 = 4;  };
template <> struct Grid<64>  { static constexpr int R1 = 8,  R2 = 8;  };
template <> struct Grid<96>  { static constexpr int R1 = 12, R2 = 8;  };
template <> struct Grid<128> { static constexpr int R1 = 16, R2 = 8;  };
template <> struct Grid<256> { static constexpr int R1 = 16, R2 = 16; };

#ifndef BPS_ZPAIRS
#define BPS_ZPAIRS 8
#endif

template <int N>
struct Cfg {
  static constexpr int R1 = Grid<N>::R1;
  static constexpr int R2 = Grid<N>::R2;
  static constexpr int RMAX = R1 > R2 ? R1 : R2;
  static constexpr int H = N / 2;                      // Nyquist index
  static constexpr int ZP = ((H + 1) + 1) / 2 * 2;     // padded row length (complex)
  static constexpr int F = H < 16 ? H : 16;            // tile columns
  static constexpr int NT = F * RMAX < 32 ? 32 : F * RMAX;  // threads per strided tile
  static constexpr int LP = BPS_ZPAIRS;                // line pairs per contiguous-axis tile
  static constexpr int NTZ = LP * RMAX;                // threads per contiguous-axis tile
  static constexpr int ZB = H / F;                     // regular column blocks per row
  static constexpr int NYQ = N / F;                    // Nyquist tiles per pass
  static constexpr int TILES = N * ZB + NYQ;           // tiles of one strided pass
  static constexpr int ZTILES = N * N / (2 * LP);
  static_assert(R1 * R2 == N, "bad split");
  static_assert(H % F == 0, "bad tile");
};

// ------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror & Shaw (SC'11): 4 x 64-bit counter, 2 x 64-bit key,
// ten rounds of two 64x64 -> 128-bit multiplies with the key bumped by the
// Weyl constants.  Counter layout: (element block, iteration, stage, sub).
struct P4 { uint64_t w[4]; };

__host__ __device__ __forceinline__ void mulhilo64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
  lo = a * b;
  hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  lo = (uint64_t)p;
  hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ __forceinline__ P4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t key) {
  uint64_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, k0 = key, k1 = 0;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(0xD2E7470EE14C6C93ULL, x0, hi0, lo0);
    mulhilo64(0xCA5A826395121157ULL, x2, hi1, lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  P4 r;
  r.w[0] = x0; r.w[1] = x1; r.w[2] = x2; r.w[3] = x3;
  return r;
}

enum Stage : uint64_t {
  ST_MOMENTUM = 1, ST_HMC = 2, ST_POWER = 3, ST_BIAS = 4, ST_NBAR = 5, ST_JUMP_MOM = 6, ST_JUMP = 7
};

// exact FP64 uniform in (0,1): ((w >> 12) + 1/2) 2^-52
__host__ __device__ __forceinline__ double u52(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 0x1p-52;
}
// FP64 standard normal, Box-Muller cosine branch
__device__ __forceinline__ double normal64(uint64_t a, uint64_t b) {
  return sqrt(-2.0 * log(u52(a))) * cospi(2.0 * u52(b));
}
// The FP32 uniform pair of one word, fl32(fl32(h) 2^-32 + 2^-33) for each half.
__device__ __forceinline__ void u24pair(uint64_t w, float& u1, float& u2) {
  u1 = __fadd_rn(__fmul_rn(__uint2float_rn((uint32_t)w), 0x1p-32f), 0x1p-33f);
  u2 = __fadd_rn(__fmul_rn(__uint2float_rn((uint32_t)(w >> 32)), 0x1p-32f), 0x1p-33f);
}

// ------------------------------------------------- device-resident chain state
// One instance per context, in device memory; every kernel of a Gibbs
// iteration reads its parameters from here, so an iteration needs no host
// round trip and can be captured in a CUDA graph.
struct DevState {
  // chain (Sec. 3.2): power spectrum bins, biases, normalisations
  double P[MAXB], b[MAXS], nbar[MAXS], P_ref[MAXB];
  // data constants per subsample: sum R, sum N^2/R, number of observed voxels
  double sumR[MAXS], sumB[MAXS], nobs[MAXS];
  double abar;                       // voxel mean of a = sum_l b_l^2 Nbar_l R^l
  // HMC move
  double eps, u_acc, H0, H1, dH;
  int accepted, cur, status, pad0;
  // jump move
  double th[MAXB], rho[MAXB], mu[MAXB], jscale[MAXB], jgrad[MAXB];
  double jeps, ju_acc, jH0, jH1, jdH, jlik;
  int jaccepted;
  int jdone;                         // blocks of the running jump step that finished (k_jump_step)
  // 1 while the jump's first gradient can reuse the force of the HMC move just
  // accepted (W and the likelihood partials of its last force evaluation are
  // those of the current field): its force stage is skipped
  int jreuse, pad1;
  // reductions handed between kernels
  double sigma[MAXB], sums[MAXS][3];
  double lik0, lik1;
  double nmodes[MAXB];               // full-grid mode count n_m of each bin
  double mass_scale[MAXB];           // per mass-bin multipliers of the diagonal mass
  float wfeat[MAXB];                 // ln of the window power per P bin (network mass features)
  // per-bin FP32 tables used inside the field passes
  float inv_lambda[MAXB], inv_M[MAXB], sqrt_M[MAXB];
  float inv_ms[MAXB], sqrt_ms[MAXB]; // 1/s_j and sqrt(s_j) of the mass scales
  float js[MAXB];                    // jump field scale sqrt(exp(theta_m) / P_m)
  int thr[MAXB];                     // smallest |n|^2 of each P bin
  int mthr[MAXB];                    // smallest |n|^2 of each mass-scale bin
  double scratch[8];                 // small results handed to the host
  double mstat[MAXB], mstat2[MAXB];  // posterior statistics per mass bin (bps_mass_stats)
  // per-chain constants (chains of one batch share the kernels, not these)
  double vc;                         // cell volume V_cell
  unsigned long long seed;           // Philox key
  int nsub;                          // galaxy subsamples of this chain
  int rec_idx;                       // next slot of the chain record buffer
  int dslot;                         // active survey-data slot (Fields::data_slot)
  int pad2;
  unsigned long long iteration;
  unsigned long long n_moves, n_accepted;
};

enum StatusBits : int { ST_OK = 0, ST_NONFINITE = 1, ST_DRAW_FAIL = 2, ST_BADDATA = 8 };

}  // namespace bps
