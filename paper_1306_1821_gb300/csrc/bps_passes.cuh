// Field passes of the sampler: each pass moves one axis of the 3D transform
// through shared memory and fuses the pointwise work of the method into it.
//
// Layout in HBM: real fields [N][N][N] float32, x slowest; half spectra
// [N][N][ZP] complex64 with ZP = N/2+1 rounded up to an even count (16-byte
// aligned rows; the pad column is never read as data).  A 3D transform is three
// passes:  z (contiguous lines, real <-> half spectrum, two real lines packed in
// one complex line), y (stride ZP) and x (stride N*ZP).  The strided passes
// work on tiles of F adjacent columns by all N rows; the Nyquist column
// kz = N/2 has its own tiles whose F columns are adjacent rows of the other
// transverse axis.
//
// One transform of length N = R1*R2 is split across threads: a register DFT of
// one factor, a twiddle by W_N^(j c), one exchange through shared memory, a
// register DFT of the other factor.  Global loads and stores of every pass go
// straight between registers and HBM in the order a warp reads contiguously.
#pragma once
#include "bps_common.cuh"

namespace bps {

// ------------------------------------------------------------ pass arguments
struct Fields {
  float2* dh[2];          // state double buffer (DevState::cur selects the current one)
  float2* ph;             // momentum half spectrum
  float2* W;              // work half spectrum
  float2* acc;            // running sum of the state (posterior statistics), or NULL
  float* a;               // local curvature  a = sum_l b_l^2 Nbar_l R^l
  float* c;               // local drive      c = sum_l b_l (N^l - Nbar_l R^l)
  const uint16_t* cnt;    // counts [n_sub][N^3]
  const float* R;         // response [n_sub][N^3]
  // Support of a and c along each z line (x, y): span[x N + y] = (N - lo, hi),
  // lo and hi multiples of 4, a = c = 0 outside [lo, hi) (empty when hi <= lo).
  // NULL: dense (no support information).
  const int2* span;
  int n_sub;
  DevState* ds;
  double* part;           // per-block partial sums (FP64)
  int part_stride;        // doubles between consecutive quantities of one region
  const float2* tw;       // W_N^j = exp(-2 pi i j / N), j < N (FP64-rounded)
  // k bin of every mode, in the half-spectrum layout (255: the DC mode, the pad
  // column); the same for every chain of a batch group (one grid, one bin layout)
  const uint8_t* pbin;
  int grid_n;             // N
  float inv_nv;           // 1 / N^3
  int mass_mode;
  int n_bins, n_mass;     // entries of the P-bin and mass-bin threshold tables
  int n_sm;               // streaming multiprocessors
  // chains of one batch: chain j's buffers sit at j times these strides
  long long spec_stride;  // complex elements per half spectrum
  long long real_stride;  // voxels per real field
  long long data_stride;  // elements per chain of counts / response (max subsamples x voxels)
  long long part_cstride; // doubles of partial sums per chain
  long long span_stride;  // lines per chain (N^2)
  // Two survey-data slots (counts, R, spans), so that the next survey can be
  // uploaded while the kernels read the current one; slot s of counts and R
  // starts s * data_slot elements, of the spans s * span_slot lines, after the
  // pointers above.  DevState::dslot selects the active slot of each chain.
  long long data_slot, span_slot;
};

// The survey data of the chain's active slot.
struct SurveyData {
  const uint16_t* cnt;
  const float* R;
  const int2* span;       // NULL: dense
};
__device__ __forceinline__ SurveyData survey(const Fields& fp) {
  const long long s = fp.ds->dslot;
  return {fp.cnt + s * fp.data_slot, fp.R + s * fp.data_slot, fp.span ? fp.span + s * fp.span_slot : nullptr};
}

// The fields of chain `ch` of a batch (blockIdx.y of the field passes).
__host__ __device__ __forceinline__ Fields at_chain(Fields f, int ch) {
  f.dh[0] += ch * f.spec_stride;
  f.dh[1] += ch * f.spec_stride;
  f.ph += ch * f.spec_stride;
  f.W += ch * f.spec_stride;
  if (f.acc) f.acc += ch * f.spec_stride;
  f.a += ch * f.real_stride;
  f.c += ch * f.real_stride;
  f.cnt += ch * f.data_stride;
  f.R += ch * f.data_stride;
  if (f.span) f.span += ch * f.span_stride;
  f.ds += ch;
  f.part += ch * f.part_cstride;
  return f;
}

enum { MAP_COL = 0, MAP_ROW = 1 };

template <int MAP, int A, int B, int F>
__device__ __forceinline__ int exidx(int f, int a, int c) {
  if constexpr (MAP == MAP_COL) return (c * A + a) * F + f;
  else return f * (B * (A + 1)) + c * (A + 1) + a;
}

// Transform of length N = A*B over F independent columns.
// In : thread (f, j<A) holds v[b] = x[j + A b], b < B.
// Out: thread (f, j<B) holds v[d] = X[j + B d], d < A.
// MAP_COL: f = t % F, j = t / F.   MAP_ROW: f = t / (A or B), j = t % (A or B).
// tw: W_N^j at entry j, or (TW2, a square split A = B) W_N^(j c) at entry
// c A + j, where the lanes j of one twiddle read hit consecutive entries instead
// of entries c apart (load_twiddles).
template <int N, int A, int B, int DIR, int MAP, int F, bool TW2 = false>
__device__ __forceinline__ void fft2(float2* v, float2* ex, const float2* tw, int t) {
  static_assert(!TW2 || A == B, "the two-dimensional twiddle table is for square splits");
  int f, j;
  if constexpr (MAP == MAP_COL) { f = t % F; j = t / F; } else { f = t / A; j = t % A; }
  if (j < A && f < F) {
    Dft<B, DIR>::run(v);
#pragma unroll
    for (int c = 1; c < B; ++c) {
      float2 w = TW2 ? tw[c * A + j] : tw[j * c];
      if constexpr (DIR == INV) w.y = -w.y;
      v[c] = cmul(v[c], w);
    }
#pragma unroll
    for (int c = 0; c < B; ++c) ex[exidx<MAP, A, B, F>(f, j, c)] = v[c];
  }
  __syncthreads();
  if constexpr (MAP == MAP_COL) { f = t % F; j = t / F; } else { f = t / B; j = t % B; }
  if (j < B && f < F) {
#pragma unroll
    for (int a = 0; a < A; ++a) v[a] = ex[exidx<MAP, A, B, F>(f, a, j)];
    Dft<A, DIR>::run(v);
  }
  __syncthreads();
}

// The shared-memory twiddle table of the field passes in the layout their fft2
// calls read (TwSquare<N>: two-dimensional for a square split).
template <int N>
struct TwSquare {
  static constexpr bool value = Cfg<N>::R1 == Cfg<N>::R2;
};
template <int N>
__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* tw, int t, int nt) {
  constexpr int R = Cfg<N>::R1;
  for (int i = t; i < N; i += nt) s_tw[i] = TwSquare<N>::value ? tw[(i / R) * (i % R)] : tw[i];
}

// ------------------------------------------------------------ tile geometry
// Strided pass over axis X (rows = kx) or Y (rows = ky).
template <int N>
struct Tile {
  long long base, rs, cs;   // element (row r, column f) at base + r*rs + f*cs
  int ky0, kz0, kx0;        // transverse coordinates of column 0
  int dky, dkz, dkx;        // increments per column
};

template <int N>
__device__ __forceinline__ Tile<N> tile_x(int id) {
  using C = Cfg<N>;
  Tile<N> T;
  T.rs = (long long)N * C::ZP;
  T.kx0 = 0; T.dkx = 0;
  if (id < N * C::ZB) {
    int y = id / C::ZB, zb = id % C::ZB;
    T.base = (long long)y * C::ZP + zb * C::F; T.cs = 1;
    T.ky0 = y; T.dky = 0; T.kz0 = zb * C::F; T.dkz = 1;
  } else {
    int yb = id - N * C::ZB;
    T.base = (long long)yb * C::F * C::ZP + C::H; T.cs = C::ZP;
    T.ky0 = yb * C::F; T.dky = 1; T.kz0 = C::H; T.dkz = 0;
  }
  return T;
}

template <int N>
__device__ __forceinline__ Tile<N> tile_y(int id) {
  using C = Cfg<N>;
  Tile<N> T;
  T.rs = C::ZP;
  T.ky0 = 0; T.dky = 0;
  if (id < N * C::ZB) {
    int x = id / C::ZB, zb = id % C::ZB;
    T.base = (long long)x * N * C::ZP + zb * C::F; T.cs = 1;
    T.kx0 = x; T.dkx = 0; T.kz0 = zb * C::F; T.dkz = 1;
  } else {
    int xb = id - N * C::ZB;
    T.base = (long long)xb * C::F * N * C::ZP + C::H; T.cs = (long long)N * C::ZP;
    T.kx0 = xb * C::F; T.dkx = 1; T.kz0 = C::H; T.dkz = 0;
  }
  return T;
}

template <int N>
__device__ __forceinline__ int sgn_n(int k) { return k <= N / 2 ? k : k - N; }

// Bin of |n|^2 from the table of each bin's smallest |n|^2 (padded with INT_MAX
// to 64 entries); -1 for the DC mode.
__device__ __forceinline__ int bin_of(int n2, const int* thr) {
  if (n2 == 0) return -1;
  int lo = 0;
#pragma unroll
  for (int s = 32; s > 0; s >>= 1)
    if (thr[lo + s] <= n2) lo += s;
  return lo;
}

// The same bin from an FP32 estimate floor(sqrt(n2) * nb / (sqrt(3) N / 2)),
// which is never more than one bin off for N <= 512 and nb <= 64 (checked
// exhaustively on the host by the test suite), corrected against the exact
// integer thresholds: two independent table reads instead of six dependent ones.
__device__ __forceinline__ int bin_of_map(const uint8_t* pbin, long long idx) {
  const int b = __ldg(pbin + idx);
  return b == 255 ? -1 : b;
}

__device__ __forceinline__ float bin_scale(int nb, int N) { return (float)nb / (0.8660254f * (float)N); }
__device__ __forceinline__ int bin_est(int n2, const int* thr, float scale, int nb) {
  if (n2 == 0) return -1;
  int m = min(nb - 1, (int)(sqrtf((float)n2) * scale));
  const int lo = thr[m];
  const int hi = m + 1 < nb ? thr[m + 1] : 0x7fffffff;
  if (n2 >= hi) ++m;
  else if (n2 < lo) --m;
  return m;
}

// ------------------------------------------------------------ reductions
// Per-thread FP32 running sum that keeps the rounding error of every addition
// (Knuth's TwoSum, error-free for round-to-nearest: s + c carries the exact sum
// of the terms up to the last compensation add).  The Hamiltonian terms of a
// 256^3 grid are summed over 10^7 modes; with plain FP32 partials of 16-32
// terms each partial rounds at ~1e-7 of itself and the sum over all partials
// loses ~1e-3 in absolute energy, the size of the Delta H tolerance.  The
// intrinsics keep the compiler from contracting or reordering the steps.
struct TwoSumAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// The TwoSumAcc step on a pair (s, c) held elsewhere (e.g. in shared memory).
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
  s = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum; result valid in thread 0.  sh: >= 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < (NT + 31) / 32; ++i) r += sh[i];
  }
  return r;
}

// Sum of the compensated pairs (s, c) of the lanes of this warp that exist in a
// block of NT threads, by TwoSum steps in FP32 only: the total pair is in lane 0.
// FP64 arithmetic is scarce on this GPU; a pair carries the sum to about twice
// FP32 precision.  Shuffles name only the lanes that exist (a block need not
// fill its last warp), and a lane adds only values from lanes that exist.
template <int NT>
__device__ __forceinline__ void warp_sum2(float& s, float& c) {
  const int lane = threadIdx.x & 31;
  const int nl = NT % 32 == 0 ? 32 : min(32, NT - (int)(threadIdx.x & ~31u));
  const unsigned mask = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(mask, s, o), c2 = __shfl_down_sync(mask, c, o);
    if (lane + o < nl) {
      const float t = __fadd_rn(s, s2);
      const float z = __fsub_rn(t, s);
      const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
      s = t;
      c = __fadd_rn(c, __fadd_rn(c2, err));
    }
  }
}

// Deterministic block sum of per-thread compensated pairs; the FP64 result is
// valid in thread 0 (one conversion there).  sh: >= 2 * ceil(NT / 32) floats.
template <int NT>
__device__ __forceinline__ double block_sum2(TwoSumAcc a, float* sh) {
  float s = a.s, c = a.c;
  warp_sum2<NT>(s, c);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[2 * w] = s;
    sh[2 * w + 1] = c;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    TwoSumAcc t;
#pragma unroll
    for (int i = 0; i < (NT + 31) / 32; ++i) {
      t.add(sh[2 * i]);
      t.add(sh[2 * i + 1]);
    }
    r = t.value();
  }
  return r;
}
__device__ __forceinline__ TwoSumAcc pair_of(float x) {
  TwoSumAcc a;
  a.s = x;
  return a;
}

// Per-bin accumulation for one element per thread of a column tile: within
// each group of G consecutive lanes (one tile row) the bin is monotone along
// the lanes, so lanes of one bin are contiguous; a segmented shuffle sum gives
// the segment total to its first lane, which adds it to the warp's own bins.
// Groups of one warp add in a fixed order: the result is deterministic.
template <int G>
__device__ __forceinline__ void bin_accumulate(float v, int m, double* wbins) {
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    float pv = __shfl_down_sync(0xffffffffu, v, o);
    int pm = __shfl_down_sync(0xffffffffu, m, o);
    if (gl + o < G && pm == m) v += pv;
  }
  int prev = __shfl_up_sync(0xffffffffu, m, 1);
  bool head = (gl == 0) || (prev != m);
#pragma unroll
  for (int g = 0; g < 32 / G; ++g) {
    if (lane / G == g && head && m >= 0) wbins[m] += (double)v;
    __syncwarp();
  }
}

}  // namespace bps
