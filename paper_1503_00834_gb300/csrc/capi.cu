// C-ABI of the spectral-difference library (declared in include/chorus.h): mesh handle, background
// preparation, seeded initial state, residual, SSP-RK3 stepping and FP64 reductions.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "chorus.h"
#include "closure.h"
#include "internal.h"
#include "mesh_builder.h"
#include "mesh_state.h"
#include "sd_tables.h"

using namespace chorus;


namespace {

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

template <class R>
MeshArg<R> mesh_arg(const chorus_mesh_s* m);
template <>
MeshArg<double> mesh_arg<double>(const chorus_mesh_s* m) {
  return MeshArg<double>{(int)m->E, m->d_nbr,   m->d_code, m->d_Sf64,
                         m->d_invJ64, m->d_x64, m->kr_active ? m->d_kr64 : nullptr};
}
template <>
MeshArg<float> mesh_arg<float>(const chorus_mesh_s* m) {
  return MeshArg<float>{(int)m->E, m->d_nbr,   m->d_code, m->d_Sf32,
                        m->d_invJ32, m->d_x32, m->kr_active ? m->d_kr32 : nullptr};
}

template <class R>
PhysArg<R> phys_arg(const chorus_params& P, double r_inner, double r_outer) {
  PhysArg<R> a{};
  const double gamma = P.gamma;
  // polytrope of Eqs. 25-27; p_c from hydrostatic balance dp/dr = -rho GM / r^2 (Eq. 20)
  const double beta = r_inner / r_outer, d = r_outer - r_inner, n = P.poly_n;
  const double chi_o = (beta + 1.0) / (beta * std::exp(P.N_rho / n) + 1.0);
  const double c = (2.0 * chi_o - beta - 1.0) / (1.0 - beta);
  const double alpha = (1.0 + beta) * (1.0 - chi_o) / ((1.0 - beta) * (1.0 - beta));
  const double p_c = P.GM * P.rho_c / ((n + 1.0) * alpha * d);
  const double T_c = p_c / (P.R_gas * P.rho_c);
  const double T_top = std::isnan(P.T_top) ? T_c * (c + alpha * d / r_outer) : P.T_top;
  a.gamma = (R)gamma;
  a.gm1 = (R)(gamma - 1.0);
  a.Rgas = (R)P.R_gas;
  a.CpR = (R)(gamma / (gamma - 1.0));
  a.kappa = (R)P.kappa;
  a.kappa_r = (R)P.kappa_r;
  a.nu = (R)P.nu;
  a.GM = (R)P.GM;
  a.twoOmega = (R)(2.0 * P.Omega);
  a.T_top = (R)T_top;
  a.bottom_flux = (R)P.bottom_flux;
  a.chi_c = c;
  a.chi_ad = alpha * d;
  a.rho_c = P.rho_c;
  a.p_c = p_c;
  a.poly_n = n;
  return a;
}

bool params_ok(const chorus_params* P) {
  return P && P->gamma > 1.0 && P->R_gas > 0 && P->GM > 0 && P->nu >= 0 && P->kappa >= 0 &&
         (P->kappa_r >= 0 || P->kappa_r1 != 0.0 || P->kappa_r2 != 0.0) && std::isfinite(P->kappa_r1) &&
         std::isfinite(P->kappa_r2) &&
         P->poly_n > 0 && P->N_rho > 0 && P->rho_c > 0 && std::isfinite(P->Omega) && std::isfinite(P->bottom_flux);
}

chorus_status cu(cudaError_t e) { return e == cudaSuccess ? CHORUS_OK : CHORUS_ECUDA; }

#define CHK(x)                                   \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return CHORUS_ECUDA;  \
  } while (0)

// ---------------------------------------------------------------- small kernels

// polytrope at rest at the solution points (FP64)
__global__ void k_background(int64_t n_pts, int N3, const double* __restrict__ x, PhysArg<double> ph,
                             double* __restrict__ Q0) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_pts) return;
  const int64_t e = g / N3, pt = g % N3;
  const double x0 = x[(e * 3 + 0) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
  const double r = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
  const double chi = ph.chi_c + ph.chi_ad / r;
  const double rho = ph.rho_c * pow(chi, ph.poly_n);
  const double p = ph.p_c * pow(chi, ph.poly_n + 1.0);
  double* Qe = Q0 + e * 5 * N3;
  Qe[pt] = rho;
  Qe[N3 + pt] = 0.0;
  Qe[2 * N3 + pt] = 0.0;
  Qe[3 * N3 + pt] = 0.0;
  Qe[4 * N3 + pt] = p / (double)ph.gm1;
}

// background at rest from a radial table (uniform grid from r0 with spacing h): cubic Lagrange
// interpolation on the four nodes around the point's radius
__global__ void k_background_table(int64_t n_pts, int N3, const double* __restrict__ x, double r0, double h,
                                   int64_t n_tab, const double* __restrict__ rho_t, const double* __restrict__ p_t,
                                   double gm1, double* __restrict__ Q0) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_pts) return;
  const int64_t e = g / N3, pt = g % N3;
  const double x0 = x[(e * 3 + 0) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
  const double t = (sqrt(x0 * x0 + x1 * x1 + x2 * x2) - r0) / h;
  int64_t j = (int64_t)floor(t) - 1;
  j = j < 0 ? 0 : (j > n_tab - 4 ? n_tab - 4 : j);
  const double s = t - (double)j;
  const double w[4] = {-(s - 1.0) * (s - 2.0) * (s - 3.0) / 6.0, s * (s - 2.0) * (s - 3.0) / 2.0,
                       -s * (s - 1.0) * (s - 3.0) / 2.0, s * (s - 1.0) * (s - 2.0) / 6.0};
  double rho = 0.0, p = 0.0;
  for (int i = 0; i < 4; ++i) {
    rho += w[i] * rho_t[j + i];
    p += w[i] * p_t[j + i];
  }
  double* Qe = Q0 + e * 5 * N3;
  Qe[pt] = rho;
  Qe[N3 + pt] = 0.0;
  Qe[2 * N3 + pt] = 0.0;
  Qe[3 * N3 + pt] = 0.0;
  Qe[4 * N3 + pt] = p / gm1;
}

// radiative diffusivity kappa_r(r) = a0 + a1 r + a2 r^2 at the flux points, as the interpolant (Eq. 17)
// of its solution-point values along each line; layout [E][3 d][N+1 f][N*N line] like the metrics
__global__ void k_kr_table(int64_t E, int N, const double* __restrict__ x, OpsArg<double> ops, double a0, double a1,
                           double a2, double* __restrict__ kr64, float* __restrict__ kr32) {
  const int N2 = N * N, N3 = N2 * N, per = 3 * (N + 1) * N2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= E * per) return;
  const int64_t e = g / per;
  const int rem = (int)(g % per), D = rem / ((N + 1) * N2), f = (rem % ((N + 1) * N2)) / N2, ln = rem % N2;
  const int a = ln % N, b = ln / N;
  double v = 0.0;
  for (int s = 0; s < N; ++s) {
    const int i = D == 0 ? s : a, j = D == 0 ? a : (D == 1 ? s : b), k = D == 2 ? s : b;
    const int pt = i + N * j + N2 * k;
    const double x0 = x[(e * 3 + 0) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
    const double r = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    v += ops.I[f][s] * (a0 + (a1 + a2 * r) * r);
  }
  kr64[g] = v;
  kr32[g] = (float)v;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// seeded entropy perturbation: rho = rho0 exp(-A xi), p and u unchanged (Section 4)
__global__ void k_init(int64_t n_pts, int N3, const double* __restrict__ Q0, uint64_t seed, double amp, int fp32,
                       double* __restrict__ q64, float* __restrict__ q32) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_pts) return;
  const int64_t e = g / N3, pt = g % N3;
  const uint64_t z = splitmix64(seed ^ (uint64_t)g);
  const double xi = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
  const double rho0 = Q0[e * 5 * N3 + pt];
  if (fp32) {
    float* qe = q32 + e * 5 * N3;
    qe[pt] = (float)(rho0 * expm1(-amp * xi));
    for (int v = 1; v < 5; ++v) qe[v * N3 + pt] = 0.0f;
  } else {
    double* qe = q64 + e * 5 * N3;
    qe[pt] = rho0 * exp(-amp * xi);
    for (int v = 1; v < 4; ++v) qe[v * N3 + pt] = 0.0;
    qe[4 * N3 + pt] = Q0[e * 5 * N3 + 4 * N3 + pt];
  }
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// background tables of the perturbation form from the FP64 background state and its traces (rho0,
// E0 and the lifted grad rho0 in the tables' point order, bg_point)
__global__ void k_bg_tables(int64_t E, int N, const double* __restrict__ Q0, const double* __restrict__ T,
                            const double* __restrict__ grho0, float* __restrict__ bg, float* __restrict__ bgT,
                            float* __restrict__ grho0_f) {
  const int N2 = N * N, N3 = N2 * N;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < E * N3) {
    const int64_t e = g / N3, pt = g % N3;
    const int bp = bg_point(N, (int)pt);
    bg[(e * 2) * N3 + bp] = (float)Q0[(e * 5) * N3 + pt];
    bg[(e * 2 + 1) * N3 + bp] = (float)Q0[(e * 5 + 4) * N3 + pt];
    for (int n = 0; n < 3; ++n) grho0_f[(e * 3 + n) * N3 + bp] = (float)grho0[(e * 3 + n) * N3 + pt];
  }
  if (g < E * 6 * N2) {
    const int64_t ef = g / N2, t = g % N2;
    bgT[(ef * 2) * N2 + t] = (float)T[(ef * 5) * N2 + t];
    bgT[(ef * 2 + 1) * N2 + t] = (float)T[(ef * 5 + 4) * N2 + t];
  }
}

// deterministic two-level FP64 reduction: per-block partial sums of
// (mass, energy, kinetic, Lx, Ly, Lz), then one block sums the partials in a fixed order
template <class R>
__global__ void k_reduce_partial(int64_t n_pts, int N3, const R* __restrict__ q, const double* __restrict__ Q0,
                                 const double* __restrict__ wJ, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_pts; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / N3, pt = g % N3;
    double Q[5];
    for (int v = 0; v < 5; ++v) {
      Q[v] = (double)q[(e * 5 + v) * N3 + pt];
      if (Q0) Q[v] += Q0[(e * 5 + v) * N3 + pt];
    }
    const double w = wJ[g];
    const double x0 = x[(e * 3) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
    acc[0] += w * Q[0];
    acc[1] += w * Q[4];
    acc[2] += w * 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) / Q[0];
    acc[3] += w * (x1 * Q[3] - x2 * Q[2]);
    acc[4] += w * (x2 * Q[1] - x0 * Q[3]);
    acc[5] += w * (x0 * Q[2] - x1 * Q[1]);
  }
  for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; ++c) part[blockIdx.x * 6 + c] = sh[c][0];
}

__global__ void k_reduce_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x < 6) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * 6 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// angular momentum L = sum w x cross m and moments of inertia I_i = sum w rho (|x|^2 - x_i^2)
// (Section 6, Eq. 32), per-block partial sums in FP64
template <class R>
__global__ void k_am_partial(int64_t n_pts, int N3, const R* __restrict__ q, const double* __restrict__ Q0,
                             const double* __restrict__ wJ, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_pts; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / N3, pt = g % N3;
    double rho = (double)q[(e * 5) * N3 + pt];
    if (Q0) rho += Q0[(e * 5) * N3 + pt];
    const double m0 = (double)q[(e * 5 + 1) * N3 + pt], m1 = (double)q[(e * 5 + 2) * N3 + pt],
                 m2 = (double)q[(e * 5 + 3) * N3 + pt];  // background momentum is zero
    const double w = wJ[g];
    const double x0 = x[(e * 3) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
    acc[0] += w * (x1 * m2 - x2 * m1);
    acc[1] += w * (x2 * m0 - x0 * m2);
    acc[2] += w * (x0 * m1 - x1 * m0);
    acc[3] += w * rho * (x1 * x1 + x2 * x2);
    acc[4] += w * rho * (x0 * x0 + x2 * x2);
    acc[5] += w * rho * (x0 * x0 + x1 * x1);
  }
  for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; ++c) part[blockIdx.x * 6 + c] = sh[c][0];
}

// out[0..5] = (L, I) summed in a fixed order, out[6..8] = delta Omega = L / I (Eq. 33)
__global__ void k_am_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
      for (int c = 0; c < 6; ++c) s[c] += part[b * 6 + c];
    for (int c = 0; c < 6; ++c) out[c] = s[c];
    for (int c = 0; c < 3; ++c) out[6 + c] = s[3 + c] > 0.0 ? s[c] / s[3 + c] : 0.0;
  }
}

// velocity update of Eq. 34 (u -= delta Omega x r), density and pressure kept
template <class R>
__global__ void k_am_update(int64_t n_pts, int N3, R* __restrict__ q, const double* __restrict__ Q0,
                            const double* __restrict__ x, const double* __restrict__ dO) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_pts) return;
  const int64_t e = g / N3, pt = g % N3;
  double rho = (double)q[(e * 5) * N3 + pt];
  if (Q0) rho += Q0[(e * 5) * N3 + pt];
  const double x0 = x[(e * 3) * N3 + pt], x1 = x[(e * 3 + 1) * N3 + pt], x2 = x[(e * 3 + 2) * N3 + pt];
  const double w0 = dO[0], w1 = dO[1], w2 = dO[2];
  const double c0 = w1 * x2 - w2 * x1, c1 = w2 * x0 - w0 * x2, c2 = w0 * x1 - w1 * x0;  // delta Omega x r
  double m[3], mn[3];
  for (int a = 0; a < 3; ++a) m[a] = (double)q[(e * 5 + 1 + a) * N3 + pt];
  mn[0] = m[0] - rho * c0;
  mn[1] = m[1] - rho * c1;
  mn[2] = m[2] - rho * c2;
  const double dke = 0.5 * ((mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) - (m[0] * m[0] + m[1] * m[1] + m[2] * m[2])) / rho;
  for (int a = 0; a < 3; ++a) q[(e * 5 + 1 + a) * N3 + pt] = (R)mn[a];
  q[(e * 5 + 4) * N3 + pt] = (R)((double)q[(e * 5 + 4) * N3 + pt] + dke);
}

constexpr int kRedBlocks = 1024;

// Arithmetic-rate probe for rooflines: every thread runs kChains independent FMA chains of `iters`
// steps (x = x a + b) and stores their sum so that nothing is dead code.
constexpr int kChains = 8;
template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a, T b, T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <class R>
void fill_ops(const Tables1D& T, OpsArg<R>* o) {
  std::memset(o, 0, sizeof(*o));
  const int N = T.N;
  for (int f = 0; f <= N; ++f)
    for (int s = 0; s < N; ++s) o->I[f][s] = (R)T.I[f * N + s];
  for (int s = 0; s < N; ++s)
    for (int f = 0; f <= N; ++f) {
      o->D[s][f] = (R)T.D[s * (N + 1) + f];
      o->Lfs[s][f] = (R)T.Lfs[s * (N + 1) + f];
    }
  for (int i = 0; i < N; ++i)
    for (int s = 0; s < N; ++s) o->Dsol[i][s] = (R)T.Dsol[i * N + s];
  for (int s = 0; s < N; ++s) o->w[s] = (R)T.w[s];
}

void free_background(chorus_mesh_s* m) {
  dev_free(m->d_Q0);
  dev_free(m->d_bg);
  dev_free(m->d_grho0);
  dev_free(m->d_bgT);
  dev_free(m->d_R0);
  m->d_Q0 = nullptr;
  m->d_bg = m->d_grho0 = m->d_bgT = m->d_R0 = nullptr;
  m->prepared = false;
}

cudaEvent_t take_event(chorus_mesh_s* m) {
  if (!m->pool.empty()) {
    cudaEvent_t e = m->pool.back();
    m->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void release_records(chorus_mesh_s* m) {
  for (auto& r : m->recs) {
    m->pool.push_back(r.a);
    m->pool.push_back(r.b);
  }
  m->recs.clear();
}

// Runs one launch; with timing enabled, brackets it with events on the stream.
template <class Fn>
cudaError_t timed(chorus_mesh_s* m, int cls, cudaStream_t st, Fn&& fn) {
  if (!m->timing) return fn();
  cudaEvent_t a = take_event(m), b = take_event(m);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, st);
  if (e == cudaSuccess) e = fn();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  m->recs.push_back({cls, a, b});
  return e;
}

void free_mesh(chorus_mesh_s* m) {
  for (cudaEvent_t& e : m->copy_ev)
    if (e) cudaEventDestroy(e);
  if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
  dev_free(m->closure_buf);
  release_records(m);
  for (cudaEvent_t e : m->pool) cudaEventDestroy(e);
  m->pool.clear();
  free_background(m);
  dev_free(m->d_nbr);
  dev_free(m->d_code);
  dev_free(m->d_Sf64);
  dev_free(m->d_invJ64);
  dev_free(m->d_x64);
  dev_free(m->d_wJ);
  dev_free(m->d_Sf32);
  dev_free(m->d_invJ32);
  dev_free(m->d_x32);
  dev_free(m->d_kr64);
  dev_free(m->d_kr32);
  dev_free(m->d_err);
  dev_free(m->d_red);
  dev_free(m->d_faces);
  delete m;
}

size_t ws_words(const chorus_mesh_s* m) {
  const size_t N = m->N, E = m->E;
  const size_t N2 = N * N, N3 = N2 * N;
  // stage buffer + two trace buffers + viscous normal-flux traces + two more stage buffers (RK(5,4))
  // + the gradient record handed from the gradient kernel to the residual kernel + the common face
  // fluxes of every face point
  return 3 * E * 5 * N3 + 2 * E * 6 * 5 * N2 + E * 6 * 4 * N2 + E * 12 * N3 + E * 6 * 5 * N2;
}

template <class R>
struct Ws {
  R* s;
  R* Ta;
  R* Tb;
  R* Tv;
  R* A;
  R* B;
  R* G;
  R* Fc;
};

template <class R>
Ws<R> split_ws(const chorus_mesh_s* m, void* w) {
  const size_t N = m->N, E = m->E;
  const size_t N2 = N * N, N3 = N2 * N;
  R* p = (R*)w;
  Ws<R> r;
  r.s = p;
  r.Ta = r.s + E * 5 * N3;
  r.Tb = r.Ta + E * 6 * 5 * N2;
  r.Tv = r.Tb + E * 6 * 5 * N2;
  r.A = r.Tv + E * 6 * 4 * N2;
  r.B = r.A + E * 5 * N3;
  r.G = r.B + E * 5 * N3;
  r.Fc = r.G + E * 12 * N3;
  return r;
}

BgArg bg_arg(const chorus_mesh_s* m) {
  return BgArg{m->d_bg, m->d_grho0, m->d_bgT, m->well_balanced ? nullptr : m->d_R0};
}

bool same_params(const chorus_params& a, const chorus_params& b) {
  const double* x = &a.gamma;
  const double* y = &b.gamma;
  for (size_t i = 0; i < sizeof(chorus_params) / sizeof(double); ++i)
    if (!(x[i] == y[i] || (std::isnan(x[i]) && std::isnan(y[i])))) return false;
  return true;
}

inline dim3 grid1(int64_t n, int bs = 256) { return dim3((unsigned)((n + bs - 1) / bs)); }

// Report a pending device-side error flag once: CHORUS_ETIMEOUT if set (then cleared), else OK.
chorus_status take_flag(chorus_mesh_s* m) {
  unsigned err = 0;
  CHK(cudaMemcpy(&err, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (err == 0) return CHORUS_OK;
  CHK(cudaMemset(m->d_err, 0, sizeof(unsigned)));
  return CHORUS_ETIMEOUT;
}

// Build (or refresh) the radiative-diffusivity table when the params vary kappa_r with radius.
// may_alloc false: a missing table is not allocated (CHORUS_EINVAL instead); refreshing an existing
// one for other coefficients allocates nothing.
chorus_status ensure_kr(chorus_mesh_s* m, const chorus_params& P, cudaStream_t st, bool may_alloc = true) {
  const bool active = P.kappa_r1 != 0.0 || P.kappa_r2 != 0.0;
  if (!active) {
    m->kr_active = false;
    return CHORUS_OK;
  }
  auto kr_at = [&](double r) { return P.kappa_r + (P.kappa_r1 + P.kappa_r2 * r) * r; };
  if (!(kr_at(m->r_inner) >= 0.0) || !(kr_at(m->r_outer) >= 0.0)) return CHORUS_EINVAL;
  if (m->kr_active && m->kr_coef[0] == P.kappa_r && m->kr_coef[1] == P.kappa_r1 && m->kr_coef[2] == P.kappa_r2)
    return CHORUS_OK;
  const int64_t nF = m->E * 3 * (m->N + 1) * m->N * m->N;
  if (!m->d_kr64 && !may_alloc) return CHORUS_EINVAL;
  if (!m->d_kr64 && (dev_alloc(&m->d_kr64, (size_t)nF) != cudaSuccess || dev_alloc(&m->d_kr32, (size_t)nF) != cudaSuccess))
    return CHORUS_ENOMEM;
  k_kr_table<<<grid1(nF), 256, 0, st>>>(m->E, m->N, m->d_x64, m->ops64, P.kappa_r, P.kappa_r1, P.kappa_r2, m->d_kr64,
                                        m->d_kr32);
  if (cudaGetLastError() != cudaSuccess) return CHORUS_ECUDA;
  m->kr_coef[0] = P.kappa_r;
  m->kr_coef[1] = P.kappa_r1;
  m->kr_coef[2] = P.kappa_r2;
  m->kr_active = true;
  return CHORUS_OK;
}

LaunchSet launchers_for(int p, int tile) {
  switch (p) {
    case 2: return launchers_p2(tile);
    case 3: return launchers_p3(tile);
    case 4: return launchers_p4(tile);
    default: return launchers_p5(tile);
  }
}

}  // namespace

extern "C" {

const char* chorus_strerror(chorus_status s) {
  switch (s) {
    case CHORUS_OK: return "ok";
    case CHORUS_EINVAL: return "invalid argument";
    case CHORUS_ENOMEM: return "out of memory";
    case CHORUS_ECUDA: return "CUDA error";
    case CHORUS_EMESH: return "invalid mesh";
    case CHORUS_ENAN: return "non-finite value";
    case CHORUS_ETIMEOUT: return "device wait timed out";
    case CHORUS_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

chorus_status chorus_mesh_create(int64_t n_nodes, const double* node_xyz, int64_t n_elem, const int64_t* hex20, int p,
                                 double r_inner, double r_outer, int metric_mode, void* stream, chorus_mesh* out) {
  if (!out) return CHORUS_EINVAL;
  *out = nullptr;
  if (p < 2 || p > 5) return CHORUS_EUNSUPPORTED;
  chorus_mesh_s* m = new (std::nothrow) chorus_mesh_s();
  if (!m) return CHORUS_ENOMEM;
  m->p = p;
  m->N = p + 1;
  m->E = n_elem;
  m->r_inner = r_inner;
  m->r_outer = r_outer;
  m->tab = make_tables(m->N);
  const char* why = "";
  const int rc = build_mesh(n_nodes, node_xyz, n_elem, hex20, p, r_inner, r_outer, metric_mode, m->tab, &m->host, &why);
  if (rc != 0) {
    delete m;
    return (chorus_status)rc;
  }
  m->L = launchers_for(p, 0);
  fill_ops(m->tab, &m->ops64);
  fill_ops(m->tab, &m->ops32);
  const int N = m->N, N2 = N * N, N3 = N2 * N;
  const size_t E = (size_t)n_elem;
  const size_t nS = E * 9 * (N + 1) * N2, nP = E * N3;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> wJ(nP), invJ(nP);
  for (size_t e = 0; e < E; ++e)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          const size_t g = e * N3 + i + N * j + N2 * k;
          wJ[g] = m->tab.w[i] * m->tab.w[j] * m->tab.w[k] * m->host.detJ[g];
          invJ[g] = 1.0 / m->host.detJ[g];
        }
  std::vector<float> f32(nS);
  bool ok = dev_alloc(&m->d_nbr, E * 6) == cudaSuccess && dev_alloc(&m->d_code, E * 6) == cudaSuccess &&
            dev_alloc(&m->d_Sf64, nS) == cudaSuccess && dev_alloc(&m->d_invJ64, nP) == cudaSuccess &&
            dev_alloc(&m->d_x64, 3 * nP) == cudaSuccess && dev_alloc(&m->d_wJ, nP) == cudaSuccess &&
            dev_alloc(&m->d_Sf32, nS) == cudaSuccess && dev_alloc(&m->d_invJ32, nP) == cudaSuccess &&
            dev_alloc(&m->d_x32, 3 * nP) == cudaSuccess && dev_alloc(&m->d_err, 4) == cudaSuccess &&
            dev_alloc(&m->d_red, (size_t)kRedBlocks * 6 + 16) == cudaSuccess;
  if (!ok) {
    free_mesh(m);
    return CHORUS_ENOMEM;
  }
  // the face kernel's work list: interior faces from their lower-numbered element, then wall faces
  std::vector<int2> faces;
  faces.reserve((size_t)(m->host.n_interior_faces + m->host.n_wall_faces));
  for (size_t e = 0; e < E; ++e)
    for (int F = 0; F < 6; ++F)
      if (m->host.nbr[e * 6 + F] > (int)e) faces.push_back(make_int2((int)e, F));
  m->n_ifaces = (int)faces.size();
  for (size_t e = 0; e < E; ++e)
    for (int F = 0; F < 6; ++F)
      if (m->host.nbr[e * 6 + F] < 0) faces.push_back(make_int2((int)e, F));
  m->n_wfaces = (int)faces.size() - m->n_ifaces;
  if (!faces.empty() && dev_alloc(&m->d_faces, faces.size()) != cudaSuccess) {
    free_mesh(m);
    return CHORUS_ENOMEM;
  }
  cudaError_t ce = cudaSuccess;
  auto up = [&](void* d, const void* h, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // host buffers are reused below
  };
  up(m->d_nbr, m->host.nbr.data(), E * 6 * sizeof(int));
  up(m->d_code, m->host.code.data(), E * 6 * sizeof(int));
  up(m->d_Sf64, m->host.Sf.data(), nS * sizeof(double));
  up(m->d_invJ64, invJ.data(), nP * sizeof(double));
  up(m->d_x64, m->host.x.data(), 3 * nP * sizeof(double));
  up(m->d_wJ, wJ.data(), nP * sizeof(double));
  if (!faces.empty()) up(m->d_faces, faces.data(), faces.size() * sizeof(int2));
  for (size_t i = 0; i < nS; ++i) f32[i] = (float)m->host.Sf[i];
  up(m->d_Sf32, f32.data(), nS * sizeof(float));
  for (size_t i = 0; i < nP; ++i) f32[i] = (float)invJ[i];
  up(m->d_invJ32, f32.data(), nP * sizeof(float));
  for (size_t i = 0; i < 3 * nP; ++i) f32[i] = (float)m->host.x[i];
  up(m->d_x32, f32.data(), 3 * nP * sizeof(float));
  if (ce == cudaSuccess) ce = cudaMemsetAsync(m->d_err, 0, 4 * sizeof(unsigned), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    free_mesh(m);
    return CHORUS_ECUDA;
  }
  // the host keeps only what chorus_mesh_info needs
  m->host.Sf.clear();
  m->host.Sf.shrink_to_fit();
  *out = m;
  return CHORUS_OK;
}

chorus_status chorus_mesh_destroy(chorus_mesh m) {
  if (!m) return CHORUS_EINVAL;
  cudaDeviceSynchronize();
  free_mesh(m);
  return CHORUS_OK;
}

chorus_status chorus_mesh_info(chorus_mesh m, int64_t* n_dof, int64_t* n_faces, double* h_min, double* volume) {
  if (!m) return CHORUS_EINVAL;
  if (n_dof) *n_dof = m->E * m->N * m->N * m->N;
  if (n_faces) *n_faces = m->host.n_interior_faces + m->host.n_wall_faces;
  if (h_min) *h_min = m->host.h_min;
  if (volume) *volume = m->host.volume;
  return CHORUS_OK;
}

size_t chorus_rk_workspace_bytes(chorus_mesh m, chorus_precision prec) {
  if (!m) return 0;
  return ws_words(m) * (prec == CHORUS_FP64 ? sizeof(double) : sizeof(float)) + 256;
}

}  // extern "C"

namespace {

// Background preparation: Q0 from the polytrope (tab == nullptr) or from a radial table of
// rho_0, p_0 on a uniform grid over [r_inner, r_outer]; then its FP64 residual, lifted density
// gradient and the FP32 tables of the perturbation form.
chorus_status prepare_background(chorus_mesh_s* m, const chorus_params* P, int64_t n_tab, double r0, double r1,
                                 const double* rho_tab, const double* p_tab, cudaStream_t st) {
  const chorus_status ks = ensure_kr(m, *P, st);
  if (ks != CHORUS_OK) return ks;
  free_background(m);
  const int N = m->N, N2 = N * N, N3 = N2 * N;
  const size_t E = m->E, nP = E * N3, nT = E * 6 * 5 * N2;
  if (dev_alloc(&m->d_Q0, 5 * nP) || dev_alloc(&m->d_bg, 2 * nP) || dev_alloc(&m->d_grho0, 3 * nP) ||
      dev_alloc(&m->d_bgT, E * 6 * 2 * N2) || dev_alloc(&m->d_R0, 5 * nP)) {
    free_background(m);
    return CHORUS_ENOMEM;
  }
  double *T = nullptr, *Tv = nullptr, *R0 = nullptr, *gr = nullptr, *tab = nullptr, *G = nullptr, *Fc = nullptr;
  if (dev_alloc(&T, nT) || dev_alloc(&Tv, E * 6 * 4 * N2) || dev_alloc(&R0, 5 * nP) || dev_alloc(&gr, 3 * nP) ||
      dev_alloc(&G, (size_t)kG * nP) || dev_alloc(&Fc, nT) || (rho_tab && dev_alloc(&tab, 2 * (size_t)n_tab))) {
    dev_free(T); dev_free(Tv); dev_free(R0); dev_free(gr); dev_free(tab); dev_free(G); dev_free(Fc);
    free_background(m);
    return CHORUS_ENOMEM;
  }
  const PhysArg<double> ph = phys_arg<double>(*P, m->r_inner, m->r_outer);
  const MeshArg<double> ma = mesh_arg<double>(m);
  cudaError_t ce = cudaSuccess;
  if (rho_tab) {
    ce = cudaMemcpyAsync(tab, rho_tab, n_tab * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(tab + n_tab, p_tab, n_tab * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) {
      const double h = (r1 - r0) / (double)(n_tab - 1);
      k_background_table<<<grid1(nP), 256, 0, st>>>((int64_t)nP, N3, m->d_x64, r0, h, n_tab, tab, tab + n_tab,
                                                     P->gamma - 1.0, m->d_Q0);
      ce = cudaGetLastError();
    }
  } else {
    k_background<<<grid1(nP), 256, 0, st>>>((int64_t)nP, N3, m->d_x64, ph, m->d_Q0);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = m->L.trace64(ma, m->ops64, m->d_Q0, T, st);
  if (ce == cudaSuccess) ce = m->L.grad64(ma, m->ops64, ph, m->d_Q0, T, Tv, gr, G, Fc, m->d_err, st);
  if (ce == cudaSuccess) ce = m->L.face64(ma, ph, m->d_faces, m->n_ifaces, m->n_wfaces, T, Tv, Fc, st);
  if (ce == cudaSuccess)
    ce = m->L.resid64(ma, m->ops64, ph, m->d_Q0, T, Tv, G, Fc, R0, nullptr, RkCoef<double>{}, 0.0, kModeResidual,
                      m->d_err, st);
  if (ce == cudaSuccess) {
    k_d2f<<<grid1(5 * nP), 256, 0, st>>>((int64_t)(5 * nP), R0, m->d_R0);
    k_bg_tables<<<grid1(std::max(nP, E * 6 * N2)), 256, 0, st>>>((int64_t)E, N, m->d_Q0, T, gr, m->d_bg, m->d_bgT,
                                                                 m->d_grho0);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  dev_free(T); dev_free(Tv); dev_free(R0); dev_free(gr); dev_free(tab); dev_free(G); dev_free(Fc);
  if (ce != cudaSuccess) {
    free_background(m);
    return CHORUS_ECUDA;
  }
  m->prep = *P;
  m->prepared = true;
  return CHORUS_OK;
}

// Right-hand side of the almost-flux-balance equations (Section 4.3) for y = (rho_0, p_0).
struct AfbRhs {
  PhysArg<double> ph;
  double Tc, Cp, L, kappa, kappa_r, kappa_r1, kappa_r2, gamma, GM;
  void operator()(double r, const double y[2], double dy[2]) const {
    const double chi = ph.chi_c + ph.chi_ad / r;
    const double rho_a = ph.rho_c * std::pow(chi, ph.poly_n);
    const double T_a = Tc * chi, dT_a = -Tc * ph.chi_ad / (r * r);
    // the thermal balance integrated once with outward luminosity L (superadiabatic: Gamma < 0)
    const double kr = kappa_r + (kappa_r1 + kappa_r2 * r) * r;
    const double Gamma = -(L / (4.0 * kPi * r * r) + rho_a * Cp * kr * dT_a) / (rho_a * T_a * kappa);
    const double g = GM / (r * r);
    dy[0] = -y[0] * (Gamma / Cp + g * y[0] / (gamma * y[1]));
    dy[1] = -y[0] * g;
  }
  static constexpr double kPi = 3.14159265358979323846;
};

// classical fourth-order Runge-Kutta step of size h
void rk4(const AfbRhs& f, double r, double h, double y[2]) {
  double k1[2], k2[2], k3[2], k4[2], t[2];
  f(r, y, k1);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * h * k1[i];
  f(r + 0.5 * h, t, k2);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * h * k2[i];
  f(r + 0.5 * h, t, k3);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + h * k3[i];
  f(r + h, t, k4);
  for (int i = 0; i < 2; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

}  // namespace

extern "C" {

chorus_status chorus_prepare(chorus_mesh m, const chorus_params* P, void* stream) {
  if (!m || !params_ok(P)) return CHORUS_EINVAL;
  if (m->prepared && same_params(m->prep, *P)) return CHORUS_OK;  // keeps a tabulated background too
  return prepare_background(m, P, 0, 0.0, 0.0, nullptr, nullptr, (cudaStream_t)stream);
}

chorus_status chorus_prepare_profile(chorus_mesh m, const chorus_params* P, int64_t n, double r0, double r1,
                                     const double* rho0, const double* p0, void* stream) {
  if (!m || !params_ok(P) || n < 4 || !rho0 || !p0 || !(r0 > 0.0) || !(r1 > r0)) return CHORUS_EINVAL;
  for (int64_t j = 0; j < n; ++j)
    if (!(rho0[j] > 0.0) || !(p0[j] > 0.0) || !std::isfinite(rho0[j]) || !std::isfinite(p0[j])) return CHORUS_EINVAL;
  return prepare_background(m, P, n, r0, r1, rho0, p0, (cudaStream_t)stream);
}

chorus_status chorus_afb_profile(const chorus_params* P, double r_inner, double r_outer, double r0, double r1,
                                 int64_t n, double* rho0, double* p0) {
  if (!params_ok(P) || !(P->kappa > 0.0) || !(r_inner > 0.0) || !(r_outer > r_inner) || !(r0 > 0.0) || !(r1 > r0) ||
      n < 2 || !rho0 || !p0)
    return CHORUS_EINVAL;
  AfbRhs f;
  f.ph = phys_arg<double>(*P, r_inner, r_outer);
  f.Tc = f.ph.p_c / (P->R_gas * f.ph.rho_c);
  f.Cp = P->gamma * P->R_gas / (P->gamma - 1.0);
  f.L = 4.0 * AfbRhs::kPi * r_inner * r_inner * P->bottom_flux;
  f.kappa = P->kappa;
  f.kappa_r = P->kappa_r;
  f.kappa_r1 = P->kappa_r1;
  f.kappa_r2 = P->kappa_r2;
  f.gamma = P->gamma;
  f.GM = P->GM;
  // grid r_j = r0 + j h; integrate from the middle radius r_m of the shell through the grid points on
  // each side of it in order, with kSub RK4 substeps per grid interval (partial first interval)
  const double h = (r1 - r0) / (double)(n - 1);
  const double rm = 0.5 * (r_inner + r_outer);
  const double chi = f.ph.chi_c + f.ph.chi_ad / rm;
  constexpr int kSub = 16;
  int64_t first_up = 0;  // first grid point with r_j >= r_m
  while (first_up < n && r0 + (double)first_up * h < rm) ++first_up;
  for (int dir = -1; dir <= 1; dir += 2) {
    double y[2] = {f.ph.rho_c * std::pow(chi, f.ph.poly_n), f.ph.p_c * std::pow(chi, f.ph.poly_n + 1.0)};
    double r = rm;
    for (int64_t j = dir > 0 ? first_up : first_up - 1; dir > 0 ? j < n : j >= 0; j += dir) {
      const double rj = r0 + (double)j * h;
      const double span = rj - r;
      const int sub = (int)std::ceil(std::fabs(span) / h * kSub - 1e-9);
      for (int s = 0; s < sub; ++s) rk4(f, r + span * s / sub, span / sub, y);
      r = rj;
      if (!(y[0] > 0.0) || !(y[1] > 0.0) || !std::isfinite(y[0]) || !std::isfinite(y[1])) return CHORUS_ENAN;
      rho0[j] = y[0];
      p0[j] = y[1];
    }
  }
  return CHORUS_OK;
}

chorus_status chorus_state_init(chorus_mesh m, const chorus_params* P, uint64_t seed, double amp,
                                chorus_precision prec, void* Q, void* stream) {
  if (!m || !Q || !params_ok(P) || !(amp >= 0.0 && amp < 1.0) || (prec != CHORUS_FP64 && prec != CHORUS_FP32_PERT))
    return CHORUS_EINVAL;
  chorus_status s = chorus_prepare(m, P, stream);
  if (s != CHORUS_OK) return s;
  const int64_t nP = m->E * m->N * m->N * m->N;
  cudaStream_t st = (cudaStream_t)stream;
  k_init<<<grid1(nP), 256, 0, st>>>(nP, m->N * m->N * m->N, m->d_Q0, seed, amp, prec == CHORUS_FP32_PERT,
                                     (double*)Q, (float*)Q);
  return cu(cudaGetLastError());
}

chorus_status chorus_residual(chorus_mesh m, const chorus_params* P, chorus_precision prec, const void* Q, void* R,
                              void* workspace, void* stream) {
  if (!m || !Q || !R || !workspace || !params_ok(P)) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CHORUS_FP64) {
    const chorus_status ks = ensure_kr(m, *P, st);
    if (ks != CHORUS_OK) return ks;
    const PhysArg<double> ph = phys_arg<double>(*P, m->r_inner, m->r_outer);
    const MeshArg<double> ma = mesh_arg<double>(m);
    Ws<double> w = split_ws<double>(m, workspace);
    CHK(timed(m, 0, st, [&] { return m->L.trace64(ma, m->ops64, (const double*)Q, w.Ta, st); }));
    CHK(timed(m, 1, st, [&] {
      return m->L.grad64(ma, m->ops64, ph, (const double*)Q, w.Ta, w.Tv, nullptr, w.G, w.Fc, m->d_err, st);
    }));
    CHK(timed(m, 3, st, [&] { return m->L.face64(ma, ph, m->d_faces, m->n_ifaces, m->n_wfaces, w.Ta, w.Tv, w.Fc, st); }));
    RkCoef<double> rc{};
    if (m->closure) {
      if (!m->prepared) return CHORUS_EINVAL;  // the network reads q' = Q - Q0
      CHK(mlp_elements_tc(0, m->closure, Q, m->d_Q0, m->closure_buf, m->E, 0, m->d_err, st));
      rc.radd = (const double*)m->closure_buf;
    }
    CHK(timed(m, 2, st, [&] {
      return m->L.resid64(ma, m->ops64, ph, (const double*)Q, w.Ta, w.Tv, w.G, w.Fc, (double*)R, nullptr, rc, 0.0,
                          kModeResidual, m->d_err, st);
    }));
    return CHORUS_OK;
  }
  if (prec != CHORUS_FP32_PERT) return CHORUS_EINVAL;
  if (!m->prepared || !same_params(m->prep, *P)) return CHORUS_EINVAL;
  const chorus_status ks = ensure_kr(m, *P, st);
  if (ks != CHORUS_OK) return ks;
  const PhysArg<float> ph = phys_arg<float>(*P, m->r_inner, m->r_outer);
  const MeshArg<float> ma = mesh_arg<float>(m);
  Ws<float> w = split_ws<float>(m, workspace);
  const BgArg bg = bg_arg(m);
  CHK(timed(m, 0, st, [&] { return m->L.trace32(ma, m->ops32, (const float*)Q, w.Ta, st); }));
  CHK(timed(m, 1, st, [&] {
    return m->L.grad32(ma, m->ops32, ph, bg, (const float*)Q, w.Ta, w.Tv, w.G, w.Fc, m->d_err, st);
  }));
  CHK(timed(m, 3, st, [&] { return m->L.face32(ma, ph, bg, m->d_faces, m->n_ifaces, m->n_wfaces, w.Ta, w.Tv, w.Fc, st); }));
  RkCoef<float> rc{};
  if (m->closure) {
    CHK(mlp_elements_tc(1, m->closure, Q, nullptr, m->closure_buf, m->E, 0, m->d_err, st));
    rc.radd = (const float*)m->closure_buf;
  }
  CHK(timed(m, 2, st, [&] {
    return m->L.resid32(ma, m->ops32, ph, bg, (const float*)Q, w.Ta, w.Tv, w.G, w.Fc, (float*)R, nullptr, rc, 0.0f,
                        kModeResidual, m->d_err, st);
  }));
  return CHORUS_OK;
}

}  // extern "C"

namespace chorus {

// SSP-RK3 (Shu-Osher) and SSP-RK(5,4) (Spiteri-Ruuth) stage lists
const std::vector<Stage>& stages_of(int scheme) {
  static const std::vector<Stage> rk3 = {
      {0, 1, 0, 0.0, 1.0, 1.0, -1, -1, 0, 0, 0},
      {1, 1, 0, 0.75, 0.25, 0.25, -1, -1, 0, 0, 0},
      {1, 0, 0, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, -1, -1, 0, 0, 0},
  };
  static const std::vector<Stage> rk54 = {
      {0, 1, 0, 0.0, 1.0, 0.391752226571890, -1, -1, 0, 0, 0},
      {1, 2, 0, 0.444370493651235, 0.555629506348765, 0.368410593050371, -1, -1, 0, 0, 0},
      {2, 1, 0, 0.620101851488403, 0.379898148511597, 0.251891774271694, -1, -1, 0, 0, 0},
      {1, 1, 0, 0.178079954393132, 0.821920045606868, 0.544974750228521, 2, 3, 0.517231671970585,
       0.096059710526147, 0.063692468666290},
      {1, 0, 3, 1.0, 0.386708617503269, 0.226007483236906, -1, -1, 0, 0, 0},
  };
  return scheme == 1 ? rk54 : rk3;
}

}  // namespace chorus

namespace {

template <class R, class Grad, class Face, class Resid, class Trace>
chorus_status run_rk(chorus_mesh_s* m, R* u, const Ws<R>& w, double dt, int64_t n_steps, int scheme, cudaStream_t st,
                     Grad grad, Face face, Resid resid, Trace trace) {
  R* buf[4] = {u, w.s, w.A, w.B};
  R *Tc = w.Ta, *Tn = w.Tb;
  CHK(timed(m, 0, st, [&] { return trace(u, Tc); }));
  const auto& stg = stages_of(scheme);
  for (int64_t n = 0; n < n_steps; ++n)
    for (const Stage& g : stg) {
      RkCoef<R> c{buf[g.un], (R)g.a, (R)g.b, (R)g.c, g.un2 >= 0 ? buf[g.un2] : nullptr,
                  g.out2 >= 0 ? buf[g.out2] : nullptr, (R)g.a2, (R)g.b2, (R)g.c2, nullptr};
      if (m->closure) {
        CHK(mlp_elements_tc(sizeof(R) == 8 ? 0 : 1, m->closure, buf[g.src], sizeof(R) == 8 ? m->d_Q0 : nullptr,
                            m->closure_buf, m->E, 0, m->d_err, st));
        c.radd = (const R*)m->closure_buf;
      }
      CHK(timed(m, 1, st, [&] { return grad(buf[g.src], Tc); }));
      CHK(timed(m, 3, st, [&] { return face(Tc); }));
      CHK(timed(m, 2, st, [&] { return resid(buf[g.src], Tc, buf[g.dst], Tn, c); }));
      std::swap(Tc, Tn);
    }
  return CHORUS_OK;
}

// Element chunks of chorus_rk_step_host (FP32): the copy in with the traces, the last stage's residual
// with the copy out.
constexpr int kHostChunks = 8;

// The residual kernel's per-element arguments shifted to elements [e0, e0 + ne): with the face kernel
// the residual kernel reads no neighbour data (the common face fluxes are in each element's own face
// numbering), so a range of elements is a mesh of its own for it.
MeshArg<float> mesh_range(MeshArg<float> a, int64_t e0, int64_t ne, int N) {
  const int64_t N2 = N * N, N3 = N2 * N;
  a.E = (int)ne;
  a.nbr += e0 * 6;
  a.code += e0 * 6;
  a.Sf += e0 * 9 * (N + 1) * N2;
  a.invJ += e0 * N3;
  a.x += e0 * 3 * N3;
  if (a.kr) a.kr += e0 * 3 * (N + 1) * N2;
  return a;
}
BgArg bg_range(BgArg b, int64_t e0, int N) {
  const int64_t N2 = N * N, N3 = N2 * N;
  b.bg += e0 * 2 * N3;
  b.grho0 += e0 * 3 * N3;
  b.bgT += e0 * 12 * N2;
  if (b.R0) b.R0 += e0 * 5 * N3;
  return b;
}

// chorus_rk_step_host, FP32 perturbation form: the state is copied in in kHostChunks element ranges
// on the mesh's copy stream, each range's traces computed as soon as it has arrived; the last stage's
// residual runs on the same ranges, and each range's new state is copied to the host while the next
// range is computed.  Synchronises.
chorus_status rk_step_host_fp32(chorus_mesh_s* m, const chorus_params& P, float* Qh, float* Qd, void* workspace,
                                double dt, int64_t n_steps, cudaStream_t st) {
  if (!m->prepared || !same_params(m->prep, P)) return CHORUS_EINVAL;
  const chorus_status ks = ensure_kr(m, P, st);
  if (ks != CHORUS_OK) return ks;
  if (!m->copy_stream) {
    CHK(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : m->copy_ev) CHK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  static_assert(2 * kHostChunks + 2 <= (int)(sizeof(m->copy_ev) / sizeof(cudaEvent_t)), "events per chunk");
  cudaEvent_t* ev_in = m->copy_ev + kHostChunks + 1;  // [kHostChunks + 1]: the start, then one per range in
  auto range = [&](int k, int64_t* e0, int64_t* ne) {
    *e0 = m->E * k / kHostChunks;
    *ne = m->E * (k + 1) / kHostChunks - *e0;
  };
  const PhysArg<float> ph = phys_arg<float>(P, m->r_inner, m->r_outer);
  const MeshArg<float> ma = mesh_arg<float>(m);
  const BgArg bg = bg_arg(m);
  Ws<float> w = split_ws<float>(m, workspace);
  const int N = m->N;
  const int64_t N2 = N * N, N3 = N2 * N;
  const int64_t last = n_steps * (int64_t)stages_of(0).size();
  int64_t stage = 0;
  bool copied = false;  // the chunks of the last stage copied the state out
  const chorus_status s = run_rk<float>(
      m, Qd, w, dt, n_steps, 0, st,
      [&](const float* q, const float* T) {
        return m->L.grad32(ma, m->ops32, ph, bg, q, T, w.Tv, w.G, w.Fc, m->d_err, st);
      },
      [&](const float* T) { return m->L.face32(ma, ph, bg, m->d_faces, m->n_ifaces, m->n_wfaces, T, w.Tv, w.Fc, st); },
      [&](const float* q, const float* T, float* dst, float* Tn, const RkCoef<float>& c) -> cudaError_t {
        if (++stage < last || dst != Qd)
          return m->L.resid32(ma, m->ops32, ph, bg, q, T, w.Tv, w.G, w.Fc, dst, Tn, c, (float)dt, kModeRK, m->d_err, st);
        for (int k = 0; k < kHostChunks; ++k) {
          int64_t e0, ne;
          range(k, &e0, &ne);
          if (ne == 0) continue;
          RkCoef<float> ck = c;
          const int64_t o5 = e0 * 5 * N3;
          ck.un = c.un ? c.un + o5 : nullptr;
          ck.un2 = c.un2 ? c.un2 + o5 : nullptr;
          ck.out2 = c.out2 ? c.out2 + o5 : nullptr;
          ck.radd = c.radd ? c.radd + o5 : nullptr;
          cudaError_t e = m->L.resid32(mesh_range(ma, e0, ne, N), m->ops32, ph, bg_range(bg, e0, N), q + o5, T + e0 * 30 * N2,
                                       w.Tv + e0 * 24 * N2, w.G + e0 * 12 * N3, w.Fc + e0 * 30 * N2, dst + o5,
                                       Tn + e0 * 30 * N2, ck, (float)dt, kModeRK, m->d_err, st);
          if (e == cudaSuccess) e = cudaEventRecord(m->copy_ev[k], st);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(m->copy_stream, m->copy_ev[k], 0);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(Qh + o5, dst + o5, ne * 5 * N3 * sizeof(float), cudaMemcpyDeviceToHost, m->copy_stream);
          if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventRecord(m->copy_ev[kHostChunks], m->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, m->copy_ev[kHostChunks], 0);
        copied = e == cudaSuccess;
        return e;
      },
      [&](const float* q, float* T) -> cudaError_t {
        // the copy in, range by range on the copy stream (after the caller's earlier work on st), and
        // each range's traces once it has arrived
        cudaError_t e = cudaEventRecord(ev_in[kHostChunks], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->copy_stream, ev_in[kHostChunks], 0);
        for (int k = 0; k < kHostChunks && e == cudaSuccess; ++k) {
          int64_t e0, ne;
          range(k, &e0, &ne);
          if (ne == 0) continue;
          const int64_t o5 = e0 * 5 * N3;
          e = cudaMemcpyAsync(Qd + o5, Qh + o5, ne * 5 * N3 * sizeof(float), cudaMemcpyHostToDevice, m->copy_stream);
          if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], m->copy_stream);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in[k], 0);
          if (e == cudaSuccess) e = m->L.trace32(mesh_range(ma, e0, ne, N), m->ops32, q + o5, T + e0 * 30 * N2, st);
        }
        return e;
      });
  if (s != CHORUS_OK) return s;
  if (!copied)  // a scheme whose last stage does not write the caller's state: one copy after it
    CHK(cudaMemcpyAsync(Qh, Qd, (size_t)m->E * 5 * N3 * sizeof(float), cudaMemcpyDeviceToHost, st));
  CHK(cudaStreamSynchronize(st));
  return CHORUS_OK;
}

}  // namespace

extern "C" {

chorus_status chorus_rk_step_scheme(chorus_mesh m, const chorus_params* P, chorus_precision prec, int scheme, void* Q,
                                    void* workspace, double dt, int64_t n_steps, void* stream) {
  if (!m || !Q || !workspace || !params_ok(P) || !(dt > 0.0) || !std::isfinite(dt) || n_steps < 0 ||
      (scheme != 0 && scheme != 1))
    return CHORUS_EINVAL;
  if (n_steps == 0) return CHORUS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CHORUS_FP64) {
    if (m->closure && !m->prepared) return CHORUS_EINVAL;  // the network reads q' = Q - Q0
    const chorus_status ks = ensure_kr(m, *P, st);
    if (ks != CHORUS_OK) return ks;
    const PhysArg<double> ph = phys_arg<double>(*P, m->r_inner, m->r_outer);
    const MeshArg<double> ma = mesh_arg<double>(m);
    Ws<double> w = split_ws<double>(m, workspace);
    return run_rk<double>(
        m, (double*)Q, w, dt, n_steps, scheme, st,
        [&](const double* q, const double* T) {
          return m->L.grad64(ma, m->ops64, ph, q, T, w.Tv, nullptr, w.G, w.Fc, m->d_err, st);
        },
        [&](const double* T) { return m->L.face64(ma, ph, m->d_faces, m->n_ifaces, m->n_wfaces, T, w.Tv, w.Fc, st); },
        [&](const double* q, const double* T, double* dst, double* Tn, const RkCoef<double>& c) {
          return m->L.resid64(ma, m->ops64, ph, q, T, w.Tv, w.G, w.Fc, dst, Tn, c, dt, kModeRK, m->d_err, st);
        },
        [&](const double* q, double* T) { return m->L.trace64(ma, m->ops64, q, T, st); });
  }
  if (prec != CHORUS_FP32_PERT) return CHORUS_EINVAL;
  if (!m->prepared || !same_params(m->prep, *P)) return CHORUS_EINVAL;
  const chorus_status ks = ensure_kr(m, *P, st);
  if (ks != CHORUS_OK) return ks;
  const PhysArg<float> ph = phys_arg<float>(*P, m->r_inner, m->r_outer);
  const MeshArg<float> ma = mesh_arg<float>(m);
  const BgArg bg = bg_arg(m);
  Ws<float> w = split_ws<float>(m, workspace);
  return run_rk<float>(
      m, (float*)Q, w, dt, n_steps, scheme, st,
      [&](const float* q, const float* T) {
        return m->L.grad32(ma, m->ops32, ph, bg, q, T, w.Tv, w.G, w.Fc, m->d_err, st);
      },
      [&](const float* T) { return m->L.face32(ma, ph, bg, m->d_faces, m->n_ifaces, m->n_wfaces, T, w.Tv, w.Fc, st); },
      [&](const float* q, const float* T, float* dst, float* Tn, const RkCoef<float>& c) {
        return m->L.resid32(ma, m->ops32, ph, bg, q, T, w.Tv, w.G, w.Fc, dst, Tn, c, (float)dt, kModeRK, m->d_err, st);
      },
      [&](const float* q, float* T) { return m->L.trace32(ma, m->ops32, q, T, st); });
}

chorus_status chorus_rk_step(chorus_mesh m, const chorus_params* P, chorus_precision prec, void* Q, void* workspace,
                             double dt, int64_t n_steps, void* stream) {
  return chorus_rk_step_scheme(m, P, prec, 0, Q, workspace, dt, n_steps, stream);
}

chorus_status chorus_rk_step_host(chorus_mesh m, const chorus_params* P, chorus_precision prec, void* Q_host,
                                  void* Q_dev, void* workspace, double dt, int64_t n_steps, void* stream) {
  if (!m || !Q_host || !Q_dev || (prec != CHORUS_FP64 && prec != CHORUS_FP32_PERT)) return CHORUS_EINVAL;
  const size_t bytes = (size_t)m->E * 5 * m->N * m->N * m->N * (prec == CHORUS_FP64 ? sizeof(double) : sizeof(float));
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CHORUS_FP32_PERT && n_steps > 0 && P && workspace && dt > 0.0 && std::isfinite(dt)) {
    // copies in element chunks overlapping the first traces and the last stage's residual
    // (synchronises)
    return rk_step_host_fp32(m, *P, (float*)Q_host, (float*)Q_dev, workspace, dt, n_steps, st);
  }
  CHK(cudaMemcpyAsync(Q_dev, Q_host, bytes, cudaMemcpyHostToDevice, st));
  const chorus_status s = chorus_rk_step_scheme(m, P, prec, 0, Q_dev, workspace, dt, n_steps, stream);
  if (s != CHORUS_OK) return s;
  CHK(cudaMemcpyAsync(Q_host, Q_dev, bytes, cudaMemcpyDeviceToHost, st));
  CHK(cudaStreamSynchronize(st));
  return CHORUS_OK;
}

chorus_status chorus_reduce(chorus_mesh m, const chorus_params* P, chorus_precision prec, const void* Q, double* out,
                            void* stream) {
  if (!m || !Q || !out) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int N3 = m->N * m->N * m->N;
  const int64_t nP = m->E * N3;
  if (prec == CHORUS_FP64) {
    k_reduce_partial<double><<<kRedBlocks, 256, 0, st>>>(nP, N3, (const double*)Q, nullptr, m->d_wJ, m->d_x64, m->d_red);
  } else if (prec == CHORUS_FP32_PERT) {
    if (!P || !m->prepared || !same_params(m->prep, *P)) return CHORUS_EINVAL;
    k_reduce_partial<float><<<kRedBlocks, 256, 0, st>>>(nP, N3, (const float*)Q, m->d_Q0, m->d_wJ, m->d_x64, m->d_red);
  } else {
    return CHORUS_EINVAL;
  }
  k_reduce_final<<<1, 32, 0, st>>>(kRedBlocks, m->d_red, m->d_red + kRedBlocks * 6);
  CHK(cudaGetLastError());
  double r[6];
  CHK(cudaMemcpyAsync(r, m->d_red + kRedBlocks * 6, sizeof(r), cudaMemcpyDeviceToHost, st));
  CHK(cudaStreamSynchronize(st));
  out[0] = r[0];
  out[1] = r[1];
  out[2] = r[2];
  out[3] = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(out[i])) return CHORUS_ENAN;
  return take_flag(m);
}

chorus_status chorus_am_correct(chorus_mesh m, const chorus_params* P, chorus_precision prec, void* Q,
                                double* domega, void* stream) {
  if (!m || !Q) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int N3 = m->N * m->N * m->N;
  const int64_t nP = m->E * N3;
  double* out = m->d_red + kRedBlocks * 6;
  if (prec == CHORUS_FP64) {
    k_am_partial<double><<<kRedBlocks, 256, 0, st>>>(nP, N3, (const double*)Q, nullptr, m->d_wJ, m->d_x64, m->d_red);
    k_am_final<<<1, 32, 0, st>>>(kRedBlocks, m->d_red, out);
    k_am_update<double><<<grid1(nP), 256, 0, st>>>(nP, N3, (double*)Q, nullptr, m->d_x64, out + 6);
  } else if (prec == CHORUS_FP32_PERT) {
    if (!P || !m->prepared || !same_params(m->prep, *P)) return CHORUS_EINVAL;
    k_am_partial<float><<<kRedBlocks, 256, 0, st>>>(nP, N3, (const float*)Q, m->d_Q0, m->d_wJ, m->d_x64, m->d_red);
    k_am_final<<<1, 32, 0, st>>>(kRedBlocks, m->d_red, out);
    k_am_update<float><<<grid1(nP), 256, 0, st>>>(nP, N3, (float*)Q, m->d_Q0, m->d_x64, out + 6);
  } else {
    return CHORUS_EINVAL;
  }
  CHK(cudaGetLastError());
  if (domega) {
    CHK(cudaMemcpyAsync(domega, out + 6, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CHK(cudaStreamSynchronize(st));
  }
  return CHORUS_OK;
}

size_t chorus_closure_bytes(void) { return closure_record_bytes(); }

chorus_status chorus_closure_set_scales(void* weights, const float* in_scale, const float* out_scale, void* stream) {
  if (!weights || !in_scale || !out_scale) return CHORUS_EINVAL;
  for (int v = 0; v < 5; ++v)
    if (!(in_scale[v] > 0.f) || !(out_scale[v] > 0.f)) return CHORUS_EINVAL;
  float s[10];
  for (int v = 0; v < 5; ++v) {
    s[v] = in_scale[v];
    s[5 + v] = out_scale[v];
  }
  cudaStream_t st = (cudaStream_t)stream;
  CHK(cudaMemcpyAsync((unsigned char*)weights + ClosureLayout::oin, s, sizeof(s), cudaMemcpyHostToDevice, st));
  CHK(cudaStreamSynchronize(st));
  return CHORUS_OK;
}

chorus_status chorus_closure_init(void* weights, uint64_t seed, const float* in_scale, const float* out_scale,
                                  void* stream) {
  if (!weights || !in_scale || !out_scale) return CHORUS_EINVAL;
  for (int v = 0; v < 5; ++v)
    if (!(in_scale[v] > 0.f) || !(out_scale[v] > 0.f)) return CHORUS_EINVAL;
  const std::vector<unsigned char> rec = init_record(seed, in_scale, out_scale);
  cudaStream_t st = (cudaStream_t)stream;
  CHK(cudaMemcpyAsync(weights, rec.data(), rec.size(), cudaMemcpyHostToDevice, st));
  CHK(cudaStreamSynchronize(st));
  return CHORUS_OK;
}

chorus_status chorus_project(chorus_mesh fine, chorus_mesh coarse, chorus_precision prec, int kind, const void* Qf,
                             void* Qc, void* stream) {
  if (!fine || !coarse || !Qf || !Qc || fine->E != coarse->E || (kind != 0 && kind != 1) ||
      (prec != CHORUS_FP64 && prec != CHORUS_FP32_PERT))
    return CHORUS_EINVAL;
  const double *add = nullptr, *sub = nullptr;
  if (kind == 0 && prec == CHORUS_FP32_PERT) {
    if (!fine->prepared || !coarse->prepared || !same_params(fine->prep, coarse->prep)) return CHORUS_EINVAL;
    add = fine->d_Q0;
    sub = coarse->d_Q0;
  }
  return cu(launch_project(fine->E, fine->N, coarse->N, prec == CHORUS_FP64 ? 0 : 1, Qf, Qc, add, sub, 5,
                           (cudaStream_t)stream));
}

chorus_status chorus_closure_forward(const void* weights, const float* X, float* Y, int64_t n, void* stream) {
  if (!weights || !X || !Y || n < 0) return CHORUS_EINVAL;
  if (n == 0) return CHORUS_OK;
  return cu(mlp_forward(weights, X, Y, n, (cudaStream_t)stream));
}

chorus_status chorus_closure_forward_tc(const void* weights, const float* X, float* Y, int64_t n, void* stream) {
  if (!weights || !X || !Y || n < 0) return CHORUS_EINVAL;
  if (n == 0) return CHORUS_OK;
  return cu(mlp_forward_tc(weights, X, Y, n, nullptr, (cudaStream_t)stream));
}

chorus_status chorus_closure_grad(const void* weights, const float* X, const float* Y, int64_t n, float* grad,
                                  double* loss, void* stream) {
  if (!weights || !X || !Y || !grad || n <= 0) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double* dl = nullptr;
  CHK(cudaMallocAsync((void**)&dl, sizeof(double), st));
  CHK(cudaMemsetAsync(dl, 0, sizeof(double), st));
  CHK(cudaMemsetAsync(grad, 0, ClosureLayout::n_params * sizeof(float), st));
  cudaError_t e = mlp_backward(weights, X, Y, n, 0, n, grad, dl, st);
  double h = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dl, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(dl, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (loss) *loss = h;
  return cu(e);
}

chorus_status chorus_closure_make_pairs(chorus_mesh coarse, chorus_precision prec, const void* weights, const void* Qc,
                                        const void* PRf, const void* Rc, float* X, float* Y, void* stream) {
  if (!coarse || coarse->p != 2 || !weights || !Qc || !PRf || !Rc || !X || !Y) return CHORUS_EINVAL;
  if (prec == CHORUS_FP64 && !coarse->prepared) return CHORUS_EINVAL;
  return cu(make_pairs(prec == CHORUS_FP64 ? 0 : 1, weights, Qc, prec == CHORUS_FP64 ? coarse->d_Q0 : nullptr, PRf,
                       Rc, X, Y, coarse->E, (cudaStream_t)stream));
}

chorus_status chorus_closure_train(const float* X, const float* Y, int64_t n_pairs, void* weights,
                                   const chorus_train_cfg* cfg, double* losses, void* stream) {
  if (!X || !Y || !weights || !cfg || n_pairs <= 0 || cfg->epochs <= 0 || cfg->batch <= 0 || !(cfg->lr > 0))
    return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t np = ClosureLayout::n_params;
  float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
  double* dl = nullptr;
  if (dev_alloc(&master, np) || dev_alloc(&m1, np) || dev_alloc(&m2, np) || dev_alloc(&grad, np) ||
      dev_alloc(&dl, 1)) {
    dev_free(master); dev_free(m1); dev_free(m2); dev_free(grad); dev_free(dl);
    return CHORUS_ENOMEM;
  }
  cudaError_t e = load_master(weights, master, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m1, 0, np * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m2, 0, np * sizeof(float), st);
  int64_t t = 0;
  for (int64_t ep = 0; ep < cfg->epochs && e == cudaSuccess; ++ep) {
    e = cudaMemsetAsync(dl, 0, sizeof(double), st);
    for (int64_t b0 = 0; b0 < n_pairs && e == cudaSuccess; b0 += cfg->batch) {
      const int64_t rows = std::min<int64_t>(cfg->batch, n_pairs - b0);
      e = cudaMemsetAsync(grad, 0, np * sizeof(float), st);
      if (e == cudaSuccess) e = mlp_backward(weights, X, Y, n_pairs, b0, rows, grad, dl, st);
      if (e == cudaSuccess)
        e = adam(master, m1, m2, grad, weights, (float)cfg->lr, (float)cfg->beta1, (float)cfg->beta2, (float)cfg->eps,
                 ++t, st);
    }
    if (losses && e == cudaSuccess) {
      double h = 0.0;
      e = cudaMemcpyAsync(&h, dl, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      // each batch added its mean loss; report the mean over batches
      losses[ep] = h / (double)((n_pairs + cfg->batch - 1) / cfg->batch);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(master); dev_free(m1); dev_free(m2); dev_free(grad); dev_free(dl);
  return cu(e);
}

chorus_status chorus_closure_apply(chorus_mesh coarse, chorus_precision prec, const void* weights, const void* Q,
                                   void* R, void* stream) {
  if (!coarse || coarse->p != 2 || !weights || !Q || !R) return CHORUS_EINVAL;
  if (prec == CHORUS_FP64 && !coarse->prepared) return CHORUS_EINVAL;
  return cu(mlp_elements_tc(prec == CHORUS_FP64 ? 0 : 1, weights, Q, prec == CHORUS_FP64 ? coarse->d_Q0 : nullptr,
                            R, coarse->E, 1, coarse->d_err, (cudaStream_t)stream));
}

chorus_status chorus_set_well_balanced(chorus_mesh m, int enable) {
  if (!m) return CHORUS_EINVAL;
  m->well_balanced = enable != 0;
  return CHORUS_OK;
}

chorus_status chorus_closure_attach(chorus_mesh coarse, const void* weights) {
  if (!coarse) return CHORUS_EINVAL;
  if (weights == nullptr) {
    coarse->closure = nullptr;
    return CHORUS_OK;
  }
  if (coarse->p != 2) return CHORUS_EINVAL;
  if (!coarse->closure_buf) {
    if (dev_alloc((double**)&coarse->closure_buf, (size_t)coarse->E * 5 * 27)) return CHORUS_ENOMEM;
  }
  coarse->closure = weights;
  return CHORUS_OK;
}

chorus_status chorus_timing_enable(chorus_mesh m, int enable) {
  if (!m) return CHORUS_EINVAL;
  m->timing = enable != 0;
  return CHORUS_OK;
}

chorus_status chorus_timing_read(chorus_mesh m, void* stream, double* ms, int64_t* counts) {
  if (!m || !ms || !counts) return CHORUS_EINVAL;
  CHK(cudaStreamSynchronize((cudaStream_t)stream));
  for (int c = 0; c < 4; ++c) {
    ms[c] = 0.0;
    counts[c] = 0;
  }
  cudaError_t e = cudaSuccess;
  for (auto& r : m->recs) {
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (r.cls >= 0 && r.cls < 4) {
      ms[r.cls] += t;
      counts[r.cls] += 1;
    }
  }
  release_records(m);
  return cu(e);
}

chorus_status chorus_check(chorus_mesh m, void* stream) {
  if (!m) return CHORUS_EINVAL;
  CHK(cudaStreamSynchronize((cudaStream_t)stream));
  return take_flag(m);
}

chorus_status chorus_set_wait_limit(chorus_mesh m, int64_t polls) {
  if (!m || polls >= (int64_t)0xFFFFFFFFu) return CHORUS_EINVAL;
  const unsigned v = polls < 0 ? 0u : (unsigned)polls + 1u;  // device encoding: 0 default, k + 1 = k polls
  CHK(cudaMemcpy(m->d_err + 1, &v, sizeof(v), cudaMemcpyHostToDevice));
  return CHORUS_OK;
}

chorus_status chorus_stable_dt_rule(int p, double h_min, double r_inner, double r_outer, const chorus_params* P,
                                    double* dt) {
  if (!dt || !params_ok(P) || p < 2 || p > 5 || !(h_min > 0.0) || !(r_inner > 0.0) || !(r_outer > r_inner))
    return CHORUS_EINVAL;
  // largest sound speed of the polytrope at rest (Eqs. 25-27): at the inner wall, where chi and T peak
  const PhysArg<double> ph = phys_arg<double>(*P, r_inner, r_outer);
  const double T_i = ph.p_c / (P->R_gas * ph.rho_c) * (ph.chi_c + ph.chi_ad / r_inner);
  const double c_max = std::sqrt(P->gamma * P->R_gas * T_i);
  const double k = 2.0 * p + 1.0;
  double d = 0.25 * h_min / (k * c_max);
  const double diff = std::max(P->nu, P->kappa);
  if (diff > 0.0) d = std::min(d, 0.25 * h_min * h_min / (k * k * diff));
  if (!(d > 0.0) || !std::isfinite(d)) return CHORUS_ENAN;
  *dt = d;
  return CHORUS_OK;
}

chorus_status chorus_fma_rate(int prec, void* stream, double* flops_per_s) {
  if (!flops_per_s || (prec != CHORUS_FP64 && prec != CHORUS_FP32_PERT)) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CHK(cudaGetDevice(&dev));
  CHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const size_t n = (size_t)blocks * threads;
  void* out = nullptr;
  CHK(cudaMallocAsync(&out, n * 8, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  auto run = [&](int iters) -> cudaError_t {
    if (prec == CHORUS_FP64)
      k_fma_rate<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, (double*)out);
    else
      k_fma_rate<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)out);
    return cudaGetLastError();
  };
  // size the timed launch to about 20 ms from a short one, then time it
  int iters = 64;
  float ms = 0.f;
  for (int pass = 0; pass < 3 && ce == cudaSuccess; ++pass) {
    ce = cudaEventRecord(e0, st);
    if (ce == cudaSuccess) ce = run(iters);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess && pass < 2) {
      const double scale = 20.0 / std::max(ms, 1e-3f);
      iters = (int)std::min(std::max(iters * scale, 64.0), 1e8);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (ce != cudaSuccess) return CHORUS_ECUDA;
  CHK(cudaStreamSynchronize(st));
  *flops_per_s = 2.0 * kChains * 16.0 * (double)iters * (double)n / (ms * 1e-3);
  return CHORUS_OK;
}

chorus_status chorus_stable_dt(chorus_mesh m, const chorus_params* P, double* dt) {
  if (!m) return CHORUS_EINVAL;
  return chorus_stable_dt_rule(m->p, m->host.h_min, m->r_inner, m->r_outer, P, dt);
}

}  // extern "C"

// ---------------------------------------------------------------- residual without allocation
//
// chorus_residual needs a caller-allocated workspace for the face traces.  Some callers cannot
// allocate device memory at the point where they want a residual, so this variant keeps its
// scratch in one file-scope device array of fixed size instead.  The array exists once per GPU
// that loads this library and stays allocated until the process exits.  Its device address is
// looked up once per device (cudaGetSymbolAddress, with that device current) on the first call;
// the host-side symbol is only a stand-in and is never handed to a kernel.
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (set up on first use per device).
chorus_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return CHORUS_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CHORUS_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CHORUS_OK;
}

}  // namespace

extern "C" chorus_status chorus_residual_noalloc(chorus_mesh m, const chorus_params* P, chorus_precision prec,
                                                 const void* Q, void* R, void* stream) {
  if (!m || !Q || !R || !params_ok(P)) return CHORUS_EINVAL;
  if (prec != CHORUS_FP64 && prec != CHORUS_FP32_PERT) return CHORUS_EINVAL;
  const size_t N2 = (size_t)m->N * m->N, E = (size_t)m->E;
  const size_t word = prec == CHORUS_FP64 ? sizeof(double) : sizeof(float);
  const size_t N3 = N2 * (size_t)m->N;
  const size_t nT = E * 6 * 5 * N2, nTv = E * 6 * 4 * N2, nG = E * kG * N3;
  if ((2 * nT + nTv + nG) * word > kNoAllocScratchBytes) return CHORUS_EINVAL;  // mesh too large for the scratch
  if (prec == CHORUS_FP32_PERT && (!m->prepared || !same_params(m->prep, *P))) return CHORUS_EINVAL;
  // the attached closure's output buffer was allocated by chorus_closure_attach; FP64 reads Q0
  if (m->closure && prec == CHORUS_FP64 && !m->prepared) return CHORUS_EINVAL;
  void* scratch = nullptr;
  chorus_status s = noalloc_scratch(&scratch);
  if (s != CHORUS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // a radial kappa_r(r) needs its flux-point table, built (allocated) by chorus_prepare or a call
  // with a workspace; here a missing table is an error, not an allocation
  const chorus_status ks = ensure_kr(m, *P, st, false);
  if (ks != CHORUS_OK) return ks;
  if (prec == CHORUS_FP64) {
    const PhysArg<double> ph = phys_arg<double>(*P, m->r_inner, m->r_outer);
    const MeshArg<double> ma = mesh_arg<double>(m);
    double* T = (double*)scratch;
    double* Tv = T + nT;
    double* G = Tv + nTv;
    double* Fc = G + nG;
    RkCoef<double> rc{};
    if (m->closure) {
      CHK(mlp_elements_tc(0, m->closure, Q, m->d_Q0, m->closure_buf, m->E, 0, m->d_err, st));
      rc.radd = (const double*)m->closure_buf;
    }
    CHK(m->L.trace64(ma, m->ops64, (const double*)Q, T, st));
    CHK(m->L.grad64(ma, m->ops64, ph, (const double*)Q, T, Tv, nullptr, G, Fc, m->d_err, st));
    CHK(m->L.face64(ma, ph, m->d_faces, m->n_ifaces, m->n_wfaces, T, Tv, Fc, st));
    CHK(m->L.resid64(ma, m->ops64, ph, (const double*)Q, T, Tv, G, Fc, (double*)R, nullptr, rc, 0.0, kModeResidual,
                     m->d_err, st));
    return CHORUS_OK;
  }
  const PhysArg<float> ph = phys_arg<float>(*P, m->r_inner, m->r_outer);
  const MeshArg<float> ma = mesh_arg<float>(m);
  const BgArg bg = bg_arg(m);
  float* T = (float*)scratch;
  float* Tv = T + nT;
  float* G = Tv + nTv;
  float* Fc = G + nG;
  RkCoef<float> rc{};
  if (m->closure) {
    CHK(mlp_elements_tc(1, m->closure, Q, nullptr, m->closure_buf, m->E, 0, m->d_err, st));
    rc.radd = (const float*)m->closure_buf;
  }
  CHK(m->L.trace32(ma, m->ops32, (const float*)Q, T, st));
  CHK(m->L.grad32(ma, m->ops32, ph, bg, (const float*)Q, T, Tv, G, Fc, m->d_err, st));
  CHK(m->L.face32(ma, ph, bg, m->d_faces, m->n_ifaces, m->n_wfaces, T, Tv, Fc, st));
  CHK(m->L.resid32(ma, m->ops32, ph, bg, (const float*)Q, T, Tv, G, Fc, (float*)R, nullptr, rc, 0.0f, kModeResidual,
                   m->d_err, st));
  return CHORUS_OK;
}

// ---------------------------------------------------------------- calls of the batched-shell layer

namespace chorus {

chorus_status mesh_init_range(chorus_mesh_s* m, uint64_t seed, double amp, float* Q, int64_t e0, int64_t ne,
                              cudaStream_t st) {
  if (!m || !Q || !m->prepared || e0 < 0 || ne < 0 || e0 + ne > m->E || !(amp >= 0.0 && amp < 1.0))
    return CHORUS_EINVAL;
  if (ne == 0) return CHORUS_OK;
  const int N3 = m->N * m->N * m->N;
  const int64_t nP = ne * N3;
  const size_t off = (size_t)e0 * 5 * N3;
  k_init<<<grid1(nP), 256, 0, st>>>(nP, N3, m->d_Q0 + off, seed, amp, 1, nullptr, Q + off);
  return cu(cudaGetLastError());
}

chorus_status mesh_reduce_range(chorus_mesh_s* m, const float* Q, int64_t e0, int64_t ne, double out[4],
                                cudaStream_t st) {
  if (!m || !Q || !out || !m->prepared || e0 < 0 || ne < 0 || e0 + ne > m->E) return CHORUS_EINVAL;
  const int N3 = m->N * m->N * m->N;
  const int64_t nP = ne * N3;
  const size_t off5 = (size_t)e0 * 5 * N3, off1 = (size_t)e0 * N3;
  k_reduce_partial<float><<<kRedBlocks, 256, 0, st>>>(nP, N3, Q + off5, m->d_Q0 + off5, m->d_wJ + off1,
                                                      m->d_x64 + 3 * off1, m->d_red);
  k_reduce_final<<<1, 32, 0, st>>>(kRedBlocks, m->d_red, m->d_red + kRedBlocks * 6);
  CHK(cudaGetLastError());
  double r[6];
  CHK(cudaMemcpyAsync(r, m->d_red + kRedBlocks * 6, sizeof(r), cudaMemcpyDeviceToHost, st));
  CHK(cudaStreamSynchronize(st));
  out[0] = r[0];
  out[1] = r[1];
  out[2] = r[2];
  out[3] = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(out[i])) return CHORUS_ENAN;
  return CHORUS_OK;
}

int mesh_set_tile(chorus_mesh_s* m, int tile) {
  if (!m || tile < 0 || tile >= kTiles) return -1;
  m->L = launchers_for(m->p, tile);
  m->tile = tile;
  return m->L.epb32;
}

chorus_status mesh_stage_ptrs(chorus_mesh_s* m, const chorus_params& P, float* u, void* ws, StagePtrs* out) {
  if (!m || !u || !ws || !out || !m->prepared || !same_params(m->prep, P)) return CHORUS_EINVAL;
  const Ws<float> w = split_ws<float>(m, ws);
  out->m = mesh_arg<float>(m);
  out->ops = m->ops32;
  out->ph = phys_arg<float>(P, m->r_inner, m->r_outer);
  out->bg = bg_arg(m);
  out->buf[0] = u;
  out->buf[1] = w.s;
  out->buf[2] = w.A;
  out->buf[3] = w.B;
  out->Ta = w.Ta;
  out->Tb = w.Tb;
  out->Tv = w.Tv;
  out->G = w.G;
  out->Fc = w.Fc;
  out->faces = m->d_faces;
  out->nf = m->n_ifaces;
  out->nw = m->n_wfaces;
  out->err = m->d_err;
  return CHORUS_OK;
}

}  // namespace chorus
