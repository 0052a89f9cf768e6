// Fused y^-1 / z / y stage of the force evaluation (Eq. Wiener_Posterior_force):
// one CTA (or one thread-block cluster) per x plane of the work spectrum
// W(x, ky, kz).
//
// The three separate passes (inverse y transform, z pass with C2R, local force
// and R2C, forward y transform) each read and write all of W: 6 S_c + 2 S_r of
// HBM traffic.  Here a plane (N rows ky, ZP columns kz) is held in shared
// memory, split over a cluster of CL CTAs when it does not fit one (CTA r
// holds rows [r M, (r+1) M), M = N / CL), and is read and written once:
// 2 S_c + 2 S_r.
//
// With CL > 1 the y transforms are split radix-CL across the cluster (App. C.1
// transform, length N = CL * M):
//   inverse: out[CL m + r] = IFFT_M(b_r)[m],
//            b_r[i] = e^{+2 pi i i r / N} sum_h in[i + M h] e^{+2 pi i h r / CL}
//   forward: out[i + M r] = sum_r' e^{-2 pi i i r' / N} e^{-2 pi i r r' / CL} F_r'[i],
//            F_r' = FFT_M of the rows y = CL m + r' held by CTA r'
// so CTA r combines the CL row blocks of the cluster through distributed
// shared memory, transforms its block along y (length M), and then holds the
// complete z lines y = CL m + r, on which the z work runs locally.  The table
// below builds the single-CTA form (CL = 1) for grids whose plane fits, where
// it is faster than the three passes; the 256^3 plane would need a cluster, and
// the cluster form measured slower than the passes there.
#include <cooperative_groups.h>

#include "bps_internal.h"
#include "bps_passes.cuh"

namespace cg = cooperative_groups;

namespace bps {
namespace {

template <int N, int CL>
struct YZ {
  static constexpr int M = N / CL;                       // rows per CTA
  static constexpr int ZP = Cfg<N>::ZP, H = N / 2;
  static constexpr int LP = 16;                          // z line pairs per round
  static constexpr int R1 = Cfg<N>::R1, R2 = Cfg<N>::R2, RMAX = Cfg<N>::RMAX;      // z transform split
  static constexpr int NT = LP * RMAX;                   // threads
  static constexpr int MR1 = Cfg<M>::R1, MR2 = Cfg<M>::R2, MRMAX = Cfg<M>::RMAX;   // y transform split
  static constexpr int FC = NT / MRMAX;                  // columns per y-transform round
  static constexpr int GROUPS = (ZP + FC - 1) / FC;
  static constexpr int ROUNDS = M / (2 * LP);            // z rounds
  static constexpr int E = M * ZP;                       // elements of the block
  static constexpr int CHUNK = (E + 2 * NT - 1) / (2 * NT);   // per-thread elements per combine chunk
  static constexpr size_t BLK = (size_t)E * sizeof(float2);
  static constexpr size_t EXC = (size_t)M * FC * sizeof(float2);
  static constexpr size_t EXZ = (size_t)LP * (N + RMAX) * sizeof(float2);
  static constexpr size_t EX = EXC > EXZ ? EXC : EXZ;
  static constexpr size_t OFF_EX = BLK;
  static constexpr size_t OFF_TWN = OFF_EX + EX;
  static constexpr size_t OFF_TWM = OFF_TWN + (size_t)N * sizeof(float2);
  static constexpr size_t OFF_RED = OFF_TWM + (size_t)M * sizeof(float2);
  static constexpr size_t OFF_SPAN = OFF_RED + 32 * sizeof(double);      // lo[M], hi[M]
  static constexpr size_t OFF_BAR = OFF_SPAN + (size_t)2 * M * sizeof(int);
  static constexpr size_t BYTES = OFF_BAR + sizeof(uint64_t);
  static_assert(N % CL == 0 && M % (2 * LP) == 0, "bad cluster split");
  static_assert(NT % MRMAX == 0, "bad column split");
  static_assert(EX >= (size_t)LP * N * sizeof(float2), "split buffer does not fit");
  static_assert(BLK % 16 == 0, "bulk copy size");
};

// v * exp(DIR 2 pi i k / CL), CL in {1, 2, 4}
template <int CL, int DIR>
__device__ __forceinline__ float2 root_cl(float2 v, int k) {
  k %= CL;
  if (k == 0) return v;
  if (CL == 2 || k == 2) return make_float2(-v.x, -v.y);
  return k == 1 ? mul_i<DIR>(v) : mul_i<-DIR>(v);
}

template <int N, int CL>
__global__ void __launch_bounds__(YZ<N, CL>::NT, 2) k_yzpass(Fields fp0, int region) {
  using Y = YZ<N, CL>;
  constexpr int M = Y::M, ZP = Y::ZP, H = Y::H, NT = Y::NT, FC = Y::FC, LP = Y::LP;
  constexpr int R1 = Y::R1, R2 = Y::R2, MR1 = Y::MR1, MR2 = Y::MR2;
  const Fields fp = at_chain(fp0, blockIdx.y);
  extern __shared__ __align__(128) unsigned char smem[];
  float2* blk = reinterpret_cast<float2*>(smem);
  float2* ex = reinterpret_cast<float2*>(smem + Y::OFF_EX);
  float2* twN = reinterpret_cast<float2*>(smem + Y::OFF_TWN);
  float2* twM = reinterpret_cast<float2*>(smem + Y::OFF_TWM);
  double* red = reinterpret_cast<double*>(smem + Y::OFF_RED);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Y::OFF_BAR);
  int* s_lo = reinterpret_cast<int*>(smem + Y::OFF_SPAN);
  int* s_hi = s_lo + M;
  const int t = threadIdx.x;
  const int r = CL > 1 ? (int)(blockIdx.x % CL) : 0;     // rank in the cluster (cluster along x)
  const int plane = (int)blockIdx.x / CL;
  DevState* ds = fp.ds;
  if (ds->jreuse) return;         // force stage reused by the jump (uniform)
  float2* Wp = fp.W + (long long)plane * N * ZP;

  // ---- supports [lo, hi) of a and c on the z lines of this CTA (local row i is
  // y = CL i + r); outside them g = 0
  bool mine = false;
  const int2* span = survey(fp).span;
  for (int i = t; i < M; i += NT) {
    int lo = 0, hi = N;
    if (span) {
      const int2 sp = span[(long long)plane * N + CL * i + r];
      lo = N - sp.x;
      hi = sp.y;
    }
    s_lo[i] = lo;
    s_hi[i] = hi;
    mine |= hi > lo;
  }
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  const bool any_support = __syncthreads_or(mine);
  if constexpr (CL == 1) {
    // a plane without support has g = 0 on every line: a zero force, W not read
    if (!any_support) {
      for (int e = t; e < Y::E; e += NT)
        if (e % ZP <= H) Wp[e] = make_float2(0.f, 0.f);
      if (region >= 0 && t == 0) fp.part[region + blockIdx.x] = 0.0;
      return;
    }
  }

  // ---- own rows ky in [r M, (r + 1) M): one bulk copy
  if (t == 0) {
    mbar_expect_tx(bar, (uint32_t)Y::BLK);
    bulk_load(blk, Wp + (long long)r * M * ZP, (uint32_t)Y::BLK, bar);
  }
  for (int i = t; i < N; i += NT) twN[i] = fp.tw[i];
  for (int i = t; i < M; i += NT) twM[i] = fp.tw[i * CL];
  bool ok = mbar_wait(bar, 0);
  ok = __syncthreads_and(ok);
  if (!ok && t == 0) atomicOr(&ds->status, ST_TIMEOUT);
  // no early return below: every CTA of the cluster must reach every cluster barrier

  // ---- radix-CL combination of the cluster's row blocks (inverse sign)
  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                                      // every block has landed
    const float2* peer[CL];
#pragma unroll
    for (int h = 0; h < CL; ++h) peer[h] = cluster.map_shared_rank(blk, h);
#pragma unroll
    for (int chunk = 0; chunk < 2; ++chunk) {
      float2 acc[Y::CHUNK];
#pragma unroll
      for (int q = 0; q < Y::CHUNK; ++q) {
        const int e = t + NT * (chunk * Y::CHUNK + q);
        float2 s = make_float2(0.f, 0.f);
        if (e < Y::E) {
#pragma unroll
          for (int h = 0; h < CL; ++h) s = cadd(s, root_cl<CL, INV>(peer[h][e], h * r));
          float2 w = twN[(e / ZP) * r];
          w.y = -w.y;                                    // e^{+2 pi i i r / N}
          s = cmul(s, w);
        }
        acc[q] = s;
      }
      cluster.sync();                                    // all reads of this chunk are done
#pragma unroll
      for (int q = 0; q < Y::CHUNK; ++q) {
        const int e = t + NT * (chunk * Y::CHUNK + q);
        if (e < Y::E) blk[e] = acc[q];
      }
    }
    __syncthreads();
  }

  // ---- inverse y transform of length M on every column of the block
  for (int g = 0; g < Y::GROUPS; ++g) {
    const int col = g * FC + t % FC, j = t / FC;
    const bool cv = col < ZP;
    float2 v[Y::MRMAX];
    if (j < MR2) {
#pragma unroll
      for (int d = 0; d < MR1; ++d) v[d] = cv ? blk[(j + MR2 * d) * ZP + col] : make_float2(0.f, 0.f);
    }
    fft2<M, MR2, MR1, INV, MAP_COL, FC>(v, ex, twM, t);
    if (j < MR1 && cv) {
#pragma unroll
      for (int b = 0; b < MR2; ++b) blk[(j + MR1 * b) * ZP + col] = v[b];
    }
  }
  __syncthreads();

  // ---- z lines: local row i is y = CL i + r.  C2R (two lines per complex
  // transform), g = a delta - c and (1/2) sum (a delta^2 - 2 c delta), R2C.
  double eacc = 0.0;
  for (int q = 0; q < Y::ROUNDS; ++q) {
    const int i0 = q * 2 * LP;
    bool round_support = false;
#pragma unroll
    for (int l = 0; l < 2 * LP; ++l) round_support |= s_hi[i0 + l] > s_lo[i0 + l];
    if (!round_support) {
      // every line of the round has g = 0: zero rows, no transforms
      for (int i = t; i < 2 * LP * (H + 1); i += NT) {
        const int l = i / (H + 1), k = i - l * (H + 1);
        blk[(i0 + l) * ZP + k] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      continue;
    }
    float2 v[Y::RMAX];
    {
      const int f = t / R2, a = t % R2;
      if (f < LP) {
        const float2* ra = blk + (i0 + 2 * f) * ZP;
        const float2* rb = ra + ZP;
#pragma unroll
        for (int b = 0; b < R1; ++b) {
          const int k = a + R2 * b;
          float2 xa, xb;
          if (k <= H) {
            xa = ra[k];
            xb = rb[k];
            if (k == 0 || k == H) { xa.y = 0.f; xb.y = 0.f; }
          } else {
            xa = cconj(ra[N - k]);
            xb = cconj(rb[N - k]);
          }
          v[b] = make_float2(xa.x - xb.y, xa.y + xb.x);
        }
      }
    }
    fft2<N, R2, R1, INV, MAP_ROW, LP>(v, ex, twN, t);
    TwoSumAcc e;   // compensated: see TwoSumAcc
    {
      const int f = t / R1, c = t % R1;
      if (f < LP) {
        const long long la = ((long long)plane * N + (long long)CL * (i0 + 2 * f) + r) * N;
        const long long lb = la + (long long)CL * N;
        const float* pa = fp.a;
        const float* pc = fp.c;
        const int loa = s_lo[i0 + 2 * f], hia = s_hi[i0 + 2 * f];
        const int lob = s_lo[i0 + 2 * f + 1], hib = s_hi[i0 + 2 * f + 1];
#pragma unroll
        for (int d = 0; d < R2; ++d) {
          const int n = c + R1 * d;
          const bool ina = n >= loa && n < hia, inb = n >= lob && n < hib;
          const float aa = ina ? pa[la + n] : 0.f, ca = ina ? pc[la + n] : 0.f;
          const float ab = inb ? pa[lb + n] : 0.f, cb = inb ? pc[lb + n] : 0.f;
          const float da = v[d].x * fp.inv_nv, db = v[d].y * fp.inv_nv;
          const float ga = fmaf(aa, da, -ca), gb = fmaf(ab, db, -cb);
          if (region >= 0) {                             // a d^2 - 2 c d
            e.add(da * (ga - ca));
            e.add(db * (gb - cb));
          }
          v[d] = make_float2(ga, gb);
        }
      }
    }
    eacc += e.value();
    fft2<N, R1, R2, FWD, MAP_ROW, LP>(v, ex, twN, t);
    {
      const int f = t / R2, c = t % R2;
      if (f < LP) {
#pragma unroll
        for (int d = 0; d < R1; ++d) ex[f * N + c + R2 * d] = v[d];
      }
    }
    __syncthreads();
    for (int i = t; i < 2 * LP * (H + 1); i += NT) {
      const int l = i / (H + 1), k = i - l * (H + 1);
      const int f = l >> 1;
      const float2 yk = ex[f * N + k];
      const float2 ym = cconj(ex[f * N + (k == 0 ? 0 : N - k)]);
      float2 g;
      if ((l & 1) == 0) g = make_float2(0.5f * (yk.x + ym.x), 0.5f * (yk.y + ym.y));
      else g = make_float2(0.5f * (yk.y - ym.y), -0.5f * (yk.x - ym.x));
      blk[(i0 + l) * ZP + k] = g;
    }
    __syncthreads();
  }
  if (region >= 0) {
    const double s = block_sum<NT>(0.5 * eacc, red);
    if (t == 0) fp.part[region + blockIdx.x] = s;
  }

  // ---- forward y transform of length M on every column of the block
  for (int g = 0; g < Y::GROUPS; ++g) {
    const int col = g * FC + t % FC, j = t / FC;
    const bool cv = col < ZP;
    float2 v[Y::MRMAX];
    if (j < MR1) {
#pragma unroll
      for (int b = 0; b < MR2; ++b) v[b] = cv ? blk[(j + MR1 * b) * ZP + col] : make_float2(0.f, 0.f);
    }
    fft2<M, MR1, MR2, FWD, MAP_COL, FC>(v, ex, twM, t);
    if (j < MR2 && cv) {
#pragma unroll
      for (int d = 0; d < MR1; ++d) blk[(j + MR2 * d) * ZP + col] = v[d];
    }
  }
  __syncthreads();

  // ---- radix-CL combination (forward sign) into rows ky = i + M r of W
  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                                      // every F_r' is complete
    const float2* peer[CL];
#pragma unroll
    for (int h = 0; h < CL; ++h) peer[h] = cluster.map_shared_rank(blk, h);
    float2* out = Wp + (long long)r * M * ZP;
    for (int e = t; e < Y::E; e += NT) {
      const int i = e / ZP, kz = e - i * ZP;
      if (kz > H) continue;
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int h = 0; h < CL; ++h) s = cadd(s, root_cl<CL, FWD>(cmul(peer[h][e], twN[i * h]), r * h));
      out[e] = s;
    }
    cluster.sync();                                      // peers are done reading this block
  } else {
    for (int e = t; e < Y::E; e += NT) {
      const int kz = e % ZP;
      if (kz <= H) Wp[e] = blk[e];
    }
  }
}

template <int N, int CL>
void launch_yz(const Fields& f, int region, int nch, cudaStream_t s) {
  using Y = YZ<N, CL>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(N * CL, nch);
  cfg.blockDim = dim3(Y::NT);
  cfg.dynamicSmemBytes = Y::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_yzpass<N, CL>, f, region);
}

template <int N, int CL>
bool set_yz(YzEntry* out) {
  if (cudaFuncSetAttribute(k_yzpass<N, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YZ<N, CL>::BYTES) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  out->run = launch_yz<N, CL>;
  out->tiles = N * CL;
  return true;
}

}  // namespace

bool yz_table(int N, YzEntry* out) {
  switch (N) {
    case 32: return set_yz<32, 1>(out);
    case 64: return set_yz<64, 1>(out);
    case 96: return set_yz<96, 1>(out);
    case 128: return set_yz<128, 1>(out);
    default: return false;
  }
}

}  // namespace bps
