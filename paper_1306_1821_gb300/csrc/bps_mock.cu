// Artificial surveys on the device (Sec. 5 of the paper; App. D; Eq. rel_bias):
// the true density field, the galaxy counts of every subsample (Poisson, or
// the paper's Gaussian noise), the survey response of a spherical cap times a
// tabulated radial selection, and on the host the Schechter selection tables,
// the mean numbers per magnitude bin and the luminosity-dependent bias.
//
// Every FP64 step that decides an integer (a count, whether a voxel is
// inside the survey) is written with round-to-nearest intrinsics in a fixed
// order, without contraction into fused multiply-adds, so the results are the
// ones any IEEE 754 implementation of the same definition gives from the same
// inputs.  The ABI is declared and documented in include/bps.h.
#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>

#include "bps_internal.h"
#include "bps_passes.cuh"

namespace bps {
namespace {

constexpr uint64_t ST_MOCK_FIELD = 8, ST_MOCK_COUNTS = 9;
constexpr double CHUNK_MEAN = 32.0;    // largest mean of one inversion chunk
constexpr double LAMBDA_MAX = 4096.0;  // larger means give the out-of-range count 65536
constexpr int MAX_STEPS = 200;         // bound of one chunk's inversion search

// normals of stream (seed, 0, ST_MOCK_FIELD, 0): element i from block i/8, the
// FP32 Box-Muller pair of word (i % 8)/2, cosine branch for even i
__global__ void k_mock_normals(uint64_t seed, size_t n, float* out) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q * 8 >= n) return;
  P4 r = philox(q, 0, ST_MOCK_FIELD, 0, seed);
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

// W[ix][iy][iz] *= A[|n|^2] (padded half spectrum, rows of zp)
__global__ void k_mock_amp(float2* W, int N, int zp, const double* amp) {
  const long long H1 = N / 2 + 1, total = (long long)N * N * H1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(i % H1);
    const long long row = i / H1;
    const int iy = (int)(row % N), ix = (int)(row / N);
    const int nx = ix <= N / 2 ? ix : ix - N, ny = iy <= N / 2 ? iy : iy - N;
    const float a = (float)amp[nx * nx + ny * ny + iz * iz];
    float2& v = W[row * zp + iz];
    v.x *= a;
    v.y *= a;
  }
}

struct Coef {
  double c[11];   // 1/j!, j = 0..10
};

// e^-mu for 0 <= mu <= 32: mu 2^-10 (exact), Taylor series of e^-x to degree
// 10 by Horner's rule, then ten squarings (IEEE-exact operations only)
__device__ __forceinline__ double exp_neg(double mu, const Coef& k) {
  const double y = -__dmul_rn(mu, 0x1p-10);
  double s = k.c[10];
#pragma unroll
  for (int j = 9; j >= 0; --j) s = __dadd_rn(__dmul_rn(s, y), k.c[j]);
#pragma unroll
  for (int q = 0; q < 10; ++q) s = __dmul_rn(s, s);
  return s;
}

struct MockSub {
  double b[MAXS], nbar[MAXS];
};

// counts of subsample blockIdx.y: noise 0 Poisson(lambda) by chunked CDF
// inversion, lambda = (R Nbar) max(0, 1 + b delta); noise 1 the Gaussian
// noise model, round((R Nbar)(1 + b delta) + sqrt(R Nbar) z) clipped at 0
__global__ void k_mock_counts(const float* __restrict__ delta, const float* __restrict__ R, long long nv,
                              MockSub sub, Coef coef, int noise, uint64_t seed, int32_t* out) {
  const int l = blockIdx.y;
  const double b = sub.b[l], nbar = sub.nbar[l];
  const float* Rl = R + (long long)l * nv;
  int32_t* ol = out + (long long)l * nv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)delta[i];
    const double rn = __dmul_rn((double)Rl[i], nbar);
    double t = __dadd_rn(1.0, __dmul_rn(b, d));
    if (noise == 0) {
      t = fmax(0.0, t);
      const double lam = __dmul_rn(rn, t);
      if (!(lam <= LAMBDA_MAX)) {
        ol[i] = 65536;
        continue;
      }
      const double K = ceil(__ddiv_rn(lam, CHUNK_MEAN));
      const double mu = K > 0.0 ? __ddiv_rn(lam, K) : 0.0;
      const double e = exp_neg(mu, coef);
      int total = 0;
      const int nk = (int)K;
      P4 r{};
      for (int j = 0; j < nk; ++j) {
        if ((j & 3) == 0) r = philox((uint64_t)i, (uint64_t)(j >> 2), ST_MOCK_COUNTS, (uint64_t)l, seed);
        const double u = u52(r.w[j & 3]);
        double p = e, F = e;
        int k = 0;
        while (u > F && k < MAX_STEPS) {
          ++k;
          p = __ddiv_rn(__dmul_rn(p, mu), (double)k);
          F = __dadd_rn(F, p);
        }
        total += k;
      }
      ol[i] = total;
    } else {
      const double m = __dmul_rn(rn, t);
      const P4 r = philox((uint64_t)i, 0, ST_MOCK_COUNTS, (uint64_t)l, seed);
      const double u1 = u52(r.w[0]), u2 = u52(r.w[1]);
      const double z = sqrt(-2.0 * log(u1)) * cos(__dmul_rn(2.0 * 3.141592653589793, u2));
      const double x = __dadd_rn(m, __dmul_rn(__dsqrt_rn(rn), z));
      const double c = floor(__dadd_rn(x, 0.5));
      ol[i] = rn > 0.0 ? (int32_t)fmax(c, 0.0) : 0;
    }
  }
}

struct RespArgs {
  int N, n_r, n_sub;
  double dx, half_box, thr_cos, r_max;
  double ax, ay, az;   // axis as given; normalised in the kernel
};

// R[l][i] = [cos(theta_i) >= 1 - 2 f_sky and r_i <= r_max] * table_l(r_i),
// the table sampled at r_j = j r_max / (n_r - 1) and interpolated linearly
__global__ void k_mock_response(RespArgs a, const double* __restrict__ table, float* __restrict__ R) {
  const long long nv = (long long)a.N * a.N * a.N;
  const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.ax, a.ax), __dmul_rn(a.ay, a.ay)),
                                          __dmul_rn(a.az, a.az)));
  const double ux = __ddiv_rn(a.ax, nrm), uy = __ddiv_rn(a.ay, nrm), uz = __ddiv_rn(a.az, nrm);
  const double nr1 = (double)(a.n_r - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv;
       i += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(i % a.N);
    const int iy = (int)((i / a.N) % a.N);
    const int ix = (int)(i / ((long long)a.N * a.N));
    const double x = __dsub_rn(__dmul_rn((double)ix + 0.5, a.dx), a.half_box);
    const double y = __dsub_rn(__dmul_rn((double)iy + 0.5, a.dx), a.half_box);
    const double z = __dsub_rn(__dmul_rn((double)iz + 0.5, a.dx), a.half_box);
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    const double proj = __dadd_rn(__dadd_rn(__dmul_rn(ux, x), __dmul_rn(uy, y)), __dmul_rn(uz, z));
    const double cos_t = r > 0.0 ? __ddiv_rn(proj, r) : 1.0;
    const bool inside = cos_t >= a.thr_cos && r <= a.r_max;
    const double t = fmin(__dmul_rn(__ddiv_rn(r, a.r_max), nr1), nr1);
    const int j = (int)fmin(floor(t), nr1 - 1.0);
    const double w = __dsub_rn(t, (double)j);
    const double omw = __dsub_rn(1.0, w);
    for (int l = 0; l < a.n_sub; ++l) {
      const double* tl = table + (long long)l * a.n_r;
      const double f = __dadd_rn(__dmul_rn(tl[j], omw), __dmul_rn(tl[j + 1], w));
      R[(long long)l * nv + i] = inside ? __double2float_rn(f) : 0.f;
    }
  }
}

// ---------------------------------------------------------------- host: Schechter tables
// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from
// the usual cosine starting points)
struct Gauss {
  static constexpr int n = 16;
  double x[n], w[n];
  Gauss() {
    for (int i = 0; i < (n + 1) / 2; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
          const double p3 = p2;
          p2 = p1;
          p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        const double dz = p1 / pp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = -z;
      x[n - 1 - i] = z;
      w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
  }
  // composite rule over [a, b] with pieces no wider than h
  template <class F>
  double integrate(F f, double a, double b, double h) const {
    if (!(b > a)) return 0.0;
    const int m = std::max(1, (int)std::ceil((b - a) / h));
    const double step = (b - a) / m;
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
      const double c = a + (k + 0.5) * step, hw = 0.5 * step;
      for (int i = 0; i < n; ++i) s += hw * w[i] * f(c + hw * x[i]);
    }
    return s;
  }
};

struct Schechter {
  double M_star, alpha, m_bright, m_faint, omega_m;
  const Gauss& g;
  double phi(double M) const {
    const double x = std::pow(10.0, 0.4 * (M_star - M));
    return 0.4 * std::log(10.0) * std::pow(x, alpha + 1.0) * std::exp(-x);
  }
  double integral(double lo, double hi) const {
    return g.integrate([this](double M) { return phi(M); }, lo, hi, 0.05);
  }
  double hubble(double z) const { return std::sqrt(omega_m * (1.0 + z) * (1.0 + z) * (1.0 + z) + 1.0 - omega_m); }
  double comoving(double z) const {
    return 2997.92458 * g.integrate([this](double t) { return 1.0 / hubble(t); }, 0.0, z, 0.01);
  }
  double redshift(double r) const {   // Newton on D_C(z) = r
    double z = r / 2997.92458;
    for (int it = 0; it < 30; ++it) {
      const double dz = (comoving(z) - r) * hubble(z) / 2997.92458;
      z -= dz;
      if (std::fabs(dz) < 1e-15 * (1.0 + z)) break;
    }
    return z;
  }
};

}  // namespace
}  // namespace bps

using namespace bps;

extern "C" {

bps_status bps_schechter_tables(const bps_schechter* s, int n_sub, const double* M_edges, double r_max, int n_r,
                                double* table, double* nbar_rel) {
  if (!s || !M_edges || !table || n_sub < 1 || n_sub > MAXS || n_r < 2 || !(r_max > 0.0)) {
    set_last_error("bps_schechter_tables: bad arguments");
    return BPS_EINVAL;
  }
  for (int l = 0; l < n_sub; ++l)
    if (!(M_edges[l + 1] > M_edges[l])) {
      set_last_error("bps_schechter_tables: magnitude edges must increase (brightest first)");
      return BPS_EINVAL;
    }
  if (!(s->omega_m > 0.0 && s->omega_m <= 1.0) || !(s->m_faint > s->m_bright)) {
    set_last_error("bps_schechter_tables: need 0 < omega_m <= 1 and m_faint > m_bright");
    return BPS_EINVAL;
  }
  static const Gauss g;
  const Schechter sc{s->M_star, s->alpha, s->m_bright, s->m_faint, s->omega_m, g};
  // distance moduli of the sample radii (shared by all subsamples)
  std::vector<double> mu(n_r, 0.0);
  for (int j = 1; j < n_r; ++j) {
    const double r = j * (r_max / (n_r - 1));
    mu[j] = 5.0 * std::log10((1.0 + sc.redshift(r)) * r) + 25.0;
  }
  for (int l = 0; l < n_sub; ++l) {
    const double norm = sc.integral(M_edges[l], M_edges[l + 1]);
    if (nbar_rel) nbar_rel[l] = norm;
    table[(size_t)l * n_r] = 0.0;
    for (int j = 1; j < n_r; ++j) {
      const double lo = std::max(M_edges[l], s->m_bright - mu[j]);
      const double hi = std::min(M_edges[l + 1], s->m_faint - mu[j]);
      table[(size_t)l * n_r + j] = hi > lo ? sc.integral(lo, hi) / norm : 0.0;
    }
  }
  return BPS_OK;
}

bps_status bps_bias_law(int n, const double* M, double b_star, double M_star, double a, double b, double c,
                        double* b_out) {
  if (n < 0 || (n > 0 && (!M || !b_out))) {
    set_last_error("bps_bias_law: bad arguments");
    return BPS_EINVAL;
  }
  for (int l = 0; l < n; ++l) b_out[l] = b_star * (a + b * std::pow(10.0, 0.4 * (M_star - M[l])) + c * (M[l] - M_star));
  return BPS_OK;
}

}  // extern "C"

// ---- context-bound mock calls (they use the context's transforms and buffers)
namespace bps {

bps_status mock_field(const MockView& v, uint64_t seed, const double* P_n2, float* delta_dev) {
  const int N = v.N;
  const size_t nt = (size_t)3 * (N / 2) * (N / 2) + 1;
  const double vc = std::pow(v.box / N, 3);
  std::vector<double> amp(nt);
  amp[0] = 0.0;
  for (size_t i = 1; i < nt; ++i) {
    if (!(P_n2[i] >= 0.0) || !std::isfinite(P_n2[i])) {
      set_last_error("bps_mock_field: the spectrum must be finite and non-negative");
      return BPS_EINVAL;
    }
    amp[i] = std::sqrt(P_n2[i] / vc);
  }
  double* damp = nullptr;
  bps_status st = v.get_scratch(nt * sizeof(double), (void**)&damp);
  if (st != BPS_OK) return st;
  cudaStream_t s = v.stream;
  if (cudaMemcpyAsync(damp, amp.data(), nt * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_last_error("bps_mock_field: copy of the amplitude table failed");
    return BPS_ECUDA;
  }
  const size_t nv = (size_t)N * N * N;
  k_mock_normals<<<(unsigned)((nv / 8 + 255) / 256), 256, 0, s>>>(seed, nv, delta_dev);
  v.pt->z_r2c(*v.f, delta_dev, v.f->W, s);
  v.pt->y_fwd(*v.f, BUF_W, 1, s);
  v.pt->x_fwd(*v.f, BUF_W, v.f->W, 1, s);
  k_mock_amp<<<v.n_sm * 8, 256, 0, s>>>(v.f->W, N, v.zp, damp);
  v.pt->x_inv(*v.f, BUF_W, v.f->W, 1, s);
  v.pt->y_inv(*v.f, BUF_W, 1, s);
  v.pt->z_c2r(*v.f, v.f->W, delta_dev, s);
  *v.launches += 8;
  if (cudaGetLastError() != cudaSuccess) {
    set_last_error("bps_mock_field: kernel launch failed");
    return BPS_ECUDA;
  }
  return BPS_OK;
}

bps_status mock_counts(const MockView& v, uint64_t seed, const float* delta_dev, const float* R_dev, const double* b,
                       const double* nbar, int noise, int32_t* counts_dev) {
  MockSub sub{};
  for (int l = 0; l < v.n_sub; ++l) {
    if (!std::isfinite(b[l]) || !(nbar[l] >= 0.0) || !std::isfinite(nbar[l])) {
      set_last_error("bps_mock_counts: b must be finite and nbar non-negative");
      return BPS_EINVAL;
    }
    sub.b[l] = b[l];
    sub.nbar[l] = nbar[l];
  }
  Coef coef;
  double fact = 1.0;
  for (int j = 0; j <= 10; ++j) {
    if (j > 0) fact *= j;
    coef.c[j] = 1.0 / fact;
  }
  const long long nv = (long long)v.N * v.N * v.N;
  k_mock_counts<<<dim3(v.n_sm * 8, v.n_sub), 256, 0, v.stream>>>(delta_dev, R_dev, nv, sub, coef, noise, seed,
                                                                  counts_dev);
  *v.launches += 1;
  if (cudaGetLastError() != cudaSuccess) {
    set_last_error("bps_mock_counts: kernel launch failed");
    return BPS_ECUDA;
  }
  return BPS_OK;
}

bps_status mock_response(const MockView& v, double f_sky, const double* axis, int n_r, const double* table,
                         float* R_dev) {
  if (!(f_sky > 0.0 && f_sky <= 1.0) || n_r < 2 || n_r > (1 << 20) || !axis ||
      !(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2] > 0.0)) {
    set_last_error("bps_mock_response: need 0 < f_sky <= 1, 2 <= n_r <= 2^20 and a nonzero axis");
    return BPS_EINVAL;
  }
  const size_t tn = (size_t)v.n_sub * n_r;
  for (size_t i = 0; i < tn; ++i)
    if (!(table[i] >= 0.0) || !std::isfinite(table[i])) {
      set_last_error("bps_mock_response: the selection table must be finite and non-negative");
      return BPS_EINVAL;
    }
  double* dt = nullptr;
  bps_status st = v.get_scratch(tn * sizeof(double), (void**)&dt);
  if (st != BPS_OK) return st;
  if (cudaMemcpyAsync(dt, table, tn * sizeof(double), cudaMemcpyHostToDevice, v.stream) != cudaSuccess) {
    set_last_error("bps_mock_response: copy of the selection table failed");
    return BPS_ECUDA;
  }
  RespArgs a;
  a.N = v.N;
  a.n_r = n_r;
  a.n_sub = v.n_sub;
  a.dx = v.box / v.N;
  a.half_box = v.box / 2.0;
  a.thr_cos = 1.0 - 2.0 * f_sky;
  a.r_max = v.box / 2.0;
  a.ax = axis[0];
  a.ay = axis[1];
  a.az = axis[2];
  k_mock_response<<<v.n_sm * 8, 256, 0, v.stream>>>(a, dt, R_dev);
  *v.launches += 1;
  if (cudaGetLastError() != cudaSuccess) {
    set_last_error("bps_mock_response: kernel launch failed");
    return BPS_ECUDA;
  }
  return BPS_OK;
}

}  // namespace bps
