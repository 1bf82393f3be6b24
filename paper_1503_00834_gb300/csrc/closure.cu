// Learned subgrid closure for coarse-order runs: per-element order projection, a small MLP
// (135 -> 128 -> 128 -> 135, SiLU, BF16 weights, FP32 accumulation) with forward, backward and Adam
// kernels, and its use inside the residual / RK path.  The paper names subgrid-scale modelling as
// future work (Section 8); the network and its training data are defined by the workload.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "chorus.h"
#include "closure.h"
#include "internal.h"
#include "sd_tables.h"

namespace chorus {

// ------------------------------------------------------------------ record layout

size_t closure_record_bytes() { return (size_t)ClosureLayout::total_bytes; }

// ------------------------------------------------------------------ projection matrix (host)

// 1D L2 projection from Nf to Nc solution points on [0,1] (reference cube, unweighted):
// P = M_c^{-1} B with M_c[a][b] = int h^c_a h^c_b, B[a][s] = int h^c_a h^f_s (Gauss-Legendre).
std::vector<double> projection_matrix(int Nf, int Nc) {
  const Tables1D tf = make_tables(Nf), tc = make_tables(Nc);
  const int G = Nf + Nc;
  const double pi = 3.14159265358979323846;
  std::vector<double> gx(G), gw(G);
  for (int k = 1; k <= G; ++k) {
    double t = std::cos(pi * (k - 0.25) / (G + 0.5));
    for (int it = 0; it < 100; ++it) {
      double v, d;
      legendre(G, t, &v, &d);
      const double dt = v / d;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double v, d;
    legendre(G, t, &v, &d);
    gx[k - 1] = 0.5 * (t + 1.0);
    gw[k - 1] = 1.0 / ((1.0 - t * t) * d * d);
  }
  std::vector<double> M(Nc * Nc, 0.0), B(Nc * Nf, 0.0);
  for (int g = 0; g < G; ++g) {
    for (int a = 0; a < Nc; ++a) {
      const double ha = lag(tc.Xs, a, gx[g]);
      for (int b = 0; b < Nc; ++b) M[a * Nc + b] += gw[g] * ha * lag(tc.Xs, b, gx[g]);
      for (int s = 0; s < Nf; ++s) B[a * Nf + s] += gw[g] * ha * lag(tf.Xs, s, gx[g]);
    }
  }
  // solve M P = B by Gauss-Jordan elimination with partial pivoting
  for (int c = 0; c < Nc; ++c) {
    int piv = c;
    for (int r = c + 1; r < Nc; ++r)
      if (std::fabs(M[r * Nc + c]) > std::fabs(M[piv * Nc + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < Nc; ++k) std::swap(M[c * Nc + k], M[piv * Nc + k]);
      for (int k = 0; k < Nf; ++k) std::swap(B[c * Nf + k], B[piv * Nf + k]);
    }
    const double d = M[c * Nc + c];
    for (int k = 0; k < Nc; ++k) M[c * Nc + k] /= d;
    for (int k = 0; k < Nf; ++k) B[c * Nf + k] /= d;
    for (int r = 0; r < Nc; ++r) {
      if (r == c) continue;
      const double f = M[r * Nc + c];
      for (int k = 0; k < Nc; ++k) M[r * Nc + k] -= f * M[c * Nc + k];
      for (int k = 0; k < Nf; ++k) B[r * Nf + k] -= f * B[c * Nf + k];
    }
  }
  return B;
}

// ------------------------------------------------------------------ projection kernel

struct ProjArg {
  double P[kMaxN][kMaxN];  // [Nc][Nf]
  int Nf, Nc;
};

// Qc[e] = Pi(Qf[e]) along the three axes; `add_f`/`sub_c` add the fine background before and
// subtract the coarse one after (perturbation storage), all in FP64.
template <class R>
__global__ void k_project(int64_t E, ProjArg pa, const R* __restrict__ Qf, R* __restrict__ Qc,
                          const double* __restrict__ add_f, const double* __restrict__ sub_c, int nvar) {
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  const int Nf = pa.Nf, Nc = pa.Nc;
  const int N3f = Nf * Nf * Nf, N3c = Nc * Nc * Nc;
  __shared__ double a[kMaxN * kMaxN * kMaxN], b[kMaxN * kMaxN * kMaxN], c[kMaxN * kMaxN * kMaxN];
  for (int v = 0; v < nvar; ++v) {
    for (int i = threadIdx.x; i < N3f; i += blockDim.x) {
      double x = (double)Qf[(e * nvar + v) * N3f + i];
      if (add_f) x += add_f[(e * nvar + v) * N3f + i];
      a[i] = x;
    }
    __syncthreads();
    // along i: b[k][j][ci] = sum_s P[ci][s] a[k][j][s]
    for (int t = threadIdx.x; t < Nf * Nf * Nc; t += blockDim.x) {
      const int ci = t % Nc, kj = t / Nc;
      double s = 0;
      for (int q = 0; q < Nf; ++q) s += pa.P[ci][q] * a[kj * Nf + q];
      b[kj * Nc + ci] = s;
    }
    __syncthreads();
    // along j: c[k][cj][ci]
    for (int t = threadIdx.x; t < Nf * Nc * Nc; t += blockDim.x) {
      const int ci = t % Nc, cj = (t / Nc) % Nc, k = t / (Nc * Nc);
      double s = 0;
      for (int q = 0; q < Nf; ++q) s += pa.P[cj][q] * b[(k * Nf + q) * Nc + ci];
      c[(k * Nc + cj) * Nc + ci] = s;
    }
    __syncthreads();
    // along k
    for (int t = threadIdx.x; t < N3c; t += blockDim.x) {
      const int ij = t % (Nc * Nc), ck = t / (Nc * Nc);
      double s = 0;
      for (int q = 0; q < Nf; ++q) s += pa.P[ck][q] * c[q * Nc * Nc + ij];
      if (sub_c) s -= sub_c[(e * nvar + v) * N3c + t];
      Qc[(e * nvar + v) * N3c + t] = (R)s;
    }
    __syncthreads();
  }
}

ProjArg proj_arg(int Nf, int Nc) {
  ProjArg pa{};
  pa.Nf = Nf;
  pa.Nc = Nc;
  const std::vector<double> P = projection_matrix(Nf, Nc);
  for (int a = 0; a < Nc; ++a)
    for (int s = 0; s < Nf; ++s) pa.P[a][s] = P[a * Nf + s];
  return pa;
}

cudaError_t launch_project(int64_t E, int Nf, int Nc, int prec, const void* Qf, void* Qc, const double* add_f,
                           const double* sub_c, int nvar, cudaStream_t st) {
  const ProjArg pa = proj_arg(Nf, Nc);
  if (prec == 0)
    k_project<double><<<(unsigned)E, 128, 0, st>>>(E, pa, (const double*)Qf, (double*)Qc, add_f, sub_c, nvar);
  else
    k_project<float><<<(unsigned)E, 128, 0, st>>>(E, pa, (const float*)Qf, (float*)Qc, add_f, sub_c, nvar);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ network kernels

namespace {

constexpr int NI = ClosureLayout::NI, NH = ClosureLayout::NH, NO = ClosureLayout::NO;
constexpr int TB = 32;           // samples per CTA
constexpr int kThreads = 256;    // 8 warps: lane = sample row, warp = column group
constexpr int SX = NI + 2;       // odd row strides avoid bank conflicts across the 32 rows
constexpr int SH = NH + 1;

struct Rec {
  const __nv_bfloat16* W1;
  const __nv_bfloat16* W2;
  const __nv_bfloat16* W3;
  const float* b1;
  const float* b2;
  const float* b3;
  const float* in_scale;
  const float* out_scale;
};

__host__ __device__ inline Rec rec_of(const void* w) {
  const unsigned char* p = (const unsigned char*)w;
  Rec r;
  r.W1 = (const __nv_bfloat16*)(p + ClosureLayout::oW1);
  r.W2 = (const __nv_bfloat16*)(p + ClosureLayout::oW2);
  r.W3 = (const __nv_bfloat16*)(p + ClosureLayout::oW3);
  r.b1 = (const float*)(p + ClosureLayout::ob1);
  r.b2 = (const float*)(p + ClosureLayout::ob2);
  r.b3 = (const float*)(p + ClosureLayout::ob3);
  r.in_scale = (const float*)(p + ClosureLayout::oin);
  r.out_scale = (const float*)(p + ClosureLayout::oout);
  return r;
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_g(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// out[r][c] = bias[c] + sum_k A[r][k] W[c][k] for the CTA's rows; W (bf16, [n_out][K]) staged in
// shared memory; thread = (row, column group).
__device__ __forceinline__ void dense(const float* A, int lda, int K, const __nv_bfloat16* Wg, const float* bias,
                                      int n_out, __nv_bfloat16* sW, float* out, int ldo, int rows) {
  for (int i = threadIdx.x; i < n_out * K; i += blockDim.x) sW[i] = Wg[i];
  __syncthreads();
  const int r = threadIdx.x % 32, grp = threadIdx.x / 32;
  const int per = (n_out + 7) / 8;
  const int c0 = grp * per;
  if (r < rows) {
    for (int c = c0; c < min(c0 + per, n_out); ++c) {
      float acc = bias[c];
      const __nv_bfloat16* w = sW + c * K;
      for (int k = 0; k < K; ++k) acc += A[r * lda + k] * __bfloat162float(w[k]);
      out[r * ldo + c] = acc;
    }
  }
  __syncthreads();
}

// forward pass of TB samples; keeps the pre-activations z1, z2 and the output y in shared memory
struct FwdSmem {
  float X[TB * SX];
  float z1[TB * SH];
  float z2[TB * SH];
  float h[TB * SH];
  float y[TB * SX];
  __nv_bfloat16 W[NO * NH > NH * NI ? NO * NH : NH * NI];
};

__device__ void forward_tile(const Rec& w, FwdSmem& s, int rows) {
  dense(s.X, SX, NI, w.W1, w.b1, NH, s.W, s.z1, SH, rows);
  for (int i = threadIdx.x; i < TB * NH; i += blockDim.x) s.h[(i / NH) * SH + i % NH] = silu_f(s.z1[(i / NH) * SH + i % NH]);
  __syncthreads();
  dense(s.h, SH, NH, w.W2, w.b2, NH, s.W, s.z2, SH, rows);
  for (int i = threadIdx.x; i < TB * NH; i += blockDim.x) s.h[(i / NH) * SH + i % NH] = silu_f(s.z2[(i / NH) * SH + i % NH]);
  __syncthreads();
  dense(s.h, SH, NH, w.W3, w.b3, NO, s.W, s.y, SX, rows);
}

}  // namespace

// Y = MLP(X) for n samples ([n][135] FP32, row-major).
__global__ void k_mlp_forward(const void* weights, const float* __restrict__ X, float* __restrict__ Y, int64_t n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smraw);
  const Rec w = rec_of(weights);
  const int64_t r0 = (int64_t)blockIdx.x * TB;
  const int rows = (int)((n - r0) < TB ? (n - r0) : TB);
  for (int i = threadIdx.x; i < TB * NI; i += blockDim.x) {
    const int r = i / NI, k = i % NI;
    s.X[r * SX + k] = r < rows ? X[(r0 + r) * NI + k] : 0.f;
  }
  __syncthreads();
  forward_tile(w, s, rows);
  for (int i = threadIdx.x; i < rows * NO; i += blockDim.x) Y[(r0 + i / NO) * NO + i % NO] = s.y[(i / NO) * SX + i % NO];
}

// Training pairs: X = q'_c / in_scale, Y = (P R_f - R_c) / out_scale per element.
template <class R>
__global__ void k_make_pairs(const void* weights, const R* __restrict__ Qc, const double* __restrict__ Q0,
                             const R* __restrict__ PRf, const R* __restrict__ Rc, float* __restrict__ X,
                             float* __restrict__ Y, int64_t E) {
  const Rec w = rec_of(weights);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= E * NI) return;
  const int v = (int)(i % NI) / 27;
  double q = (double)Qc[i];
  if (Q0) q -= Q0[i];
  X[i] = (float)(q / (double)w.in_scale[v]);
  Y[i] = (float)(((double)PRf[i] - (double)Rc[i]) / (double)w.out_scale[v]);
}

// Gradient of L = sum (y - t)^2 / (2 n_total) over the CTA's samples, accumulated into
// grad (FP32, layout of ClosureLayout::master) with atomics; loss partial into *loss.
__global__ void k_mlp_backward(const void* weights, const float* __restrict__ X, const float* __restrict__ T,
                               int64_t n, int64_t row0, int64_t rows_total, float* __restrict__ grad,
                               double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smraw);
  float* h1 = reinterpret_cast<float*>(smraw + sizeof(FwdSmem));  // [TB][SH]
  const Rec w = rec_of(weights);
  const int64_t r0 = row0 + (int64_t)blockIdx.x * TB;
  const int64_t left = row0 + rows_total - r0;
  const int rows = (int)(left < 0 ? 0 : (left < TB ? left : TB));
  for (int i = threadIdx.x; i < TB * NI; i += blockDim.x) {
    const int r = i / NI, k = i % NI;
    s.X[r * SX + k] = r < rows ? X[(r0 + r) * NI + k] : 0.f;
  }
  __syncthreads();
  forward_tile(w, s, rows);
  // h1 = silu(z1), h2 = silu(z2) (s.h holds h2 after the forward pass)
  for (int i = threadIdx.x; i < TB * NH; i += blockDim.x) h1[(i / NH) * SH + i % NH] = silu_f(s.z1[(i / NH) * SH + i % NH]);
  // dY = (y - t) / n_total, loss partial
  const double inv_n = 1.0 / ((double)rows_total * NO);
  double lp = 0.0;
  for (int i = threadIdx.x; i < TB * NO; i += blockDim.x) {
    const int r = i / NO, k = i % NO;
    float d = 0.f;
    if (r < rows) {
      const float diff = s.y[r * SX + k] - T[(r0 + r) * NO + k];
      lp += 0.5 * (double)diff * diff;
      d = (float)(diff * inv_n);
    }
    s.y[r * SX + k] = d;  // y now holds dY
  }
  atomicAdd(loss, lp * inv_n);
  __syncthreads();
  float* gW1 = grad + ClosureLayout::mW1;
  float* gW2 = grad + ClosureLayout::mW2;
  float* gW3 = grad + ClosureLayout::mW3;
  float* gb1 = grad + ClosureLayout::mb1;
  float* gb2 = grad + ClosureLayout::mb2;
  float* gb3 = grad + ClosureLayout::mb3;
  // dW3[c][k] = sum_r dY[r][c] h2[r][k];  db3[c] = sum_r dY[r][c]
  for (int i = threadIdx.x; i < NO * NH; i += blockDim.x) {
    const int c = i / NH, k = i % NH;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += s.y[r * SX + c] * s.h[r * SH + k];
    atomicAdd(gW3 + i, acc);
  }
  for (int c = threadIdx.x; c < NO; c += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += s.y[r * SX + c];
    atomicAdd(gb3 + c, acc);
  }
  // dz2[r][k] = (sum_c dY[r][c] W3[c][k]) silu'(z2[r][k])  -> stored in z2
  for (int i = threadIdx.x; i < NO * NH; i += blockDim.x) s.W[i] = w.W3[i];
  __syncthreads();
  for (int i = threadIdx.x; i < TB * NH; i += blockDim.x) {
    const int r = i / NH, k = i % NH;
    float acc = 0.f;
    for (int c = 0; c < NO; ++c) acc += s.y[r * SX + c] * __bfloat162float(s.W[c * NH + k]);
    s.z2[r * SH + k] = r < rows ? acc * silu_g(s.z2[r * SH + k]) : 0.f;
  }
  __syncthreads();
  // dW2[c][k] = sum_r dz2[r][c] h1[r][k]
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
    const int c = i / NH, k = i % NH;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += s.z2[r * SH + c] * h1[r * SH + k];
    atomicAdd(gW2 + i, acc);
  }
  for (int c = threadIdx.x; c < NH; c += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += s.z2[r * SH + c];
    atomicAdd(gb2 + c, acc);
  }
  // dz1[r][k] = (sum_c dz2[r][c] W2[c][k]) silu'(z1[r][k])  -> stored in z1
  __syncthreads();
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) s.W[i] = w.W2[i];
  __syncthreads();
  for (int i = threadIdx.x; i < TB * NH; i += blockDim.x) {
    const int r = i / NH, k = i % NH;
    float acc = 0.f;
    for (int c = 0; c < NH; ++c) acc += s.z2[r * SH + c] * __bfloat162float(s.W[c * NH + k]);
    h1[r * SH + k] = r < rows ? acc * silu_g(s.z1[r * SH + k]) : 0.f;  // h1 now holds dz1
  }
  __syncthreads();
  // dW1[c][k] = sum_r dz1[r][c] X[r][k]
  for (int i = threadIdx.x; i < NH * NI; i += blockDim.x) {
    const int c = i / NI, k = i % NI;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += h1[r * SH + c] * s.X[r * SX + k];
    atomicAdd(gW1 + i, acc);
  }
  for (int c = threadIdx.x; c < NH; c += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += h1[r * SH + c];
    atomicAdd(gb1 + c, acc);
  }
}

// Adam update of the FP32 master parameters; writes the BF16 weights and FP32 biases of the record.
__global__ void k_adam(float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ grad, void* weights, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ClosureLayout::n_params) return;
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float b = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = b;
  const float p = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  master[i] = p;
  closure_store_param(weights, i, p);
}

// master <- record (BF16 weights widened, FP32 biases)
__global__ void k_load_master(const void* weights, float* __restrict__ master) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ClosureLayout::n_params) return;
  master[i] = closure_load_param(weights, i);
}

size_t mlp_smem_bytes(bool backward) {
  return sizeof(FwdSmem) + (backward ? sizeof(float) * TB * SH : 0);
}

template __global__ void k_make_pairs<float>(const void*, const float*, const double*, const float*, const float*,
                                             float*, float*, int64_t);
template __global__ void k_make_pairs<double>(const void*, const double*, const double*, const double*,
                                              const double*, float*, float*, int64_t);

cudaError_t mlp_forward(const void* weights, const float* X, float* Y, int64_t n, cudaStream_t st) {
  const size_t sm = mlp_smem_bytes(false);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mlp_forward<<<(unsigned)((n + TB - 1) / TB), kThreads, sm, st>>>(weights, X, Y, n);
  return cudaGetLastError();
}

cudaError_t mlp_backward(const void* weights, const float* X, const float* T, int64_t n, int64_t row0, int64_t rows,
                         float* grad, double* loss, cudaStream_t st) {
  const size_t sm = mlp_smem_bytes(true);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mlp_backward<<<(unsigned)((rows + TB - 1) / TB), kThreads, sm, st>>>(weights, X, T, n, row0, rows, grad, loss);
  return cudaGetLastError();
}

cudaError_t make_pairs(int prec, const void* weights, const void* Qc, const double* Q0, const void* PRf,
                       const void* Rc, float* X, float* Y, int64_t E, cudaStream_t st) {
  const int64_t n = E * NI;
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (prec == 0)
    k_make_pairs<double><<<nb, 256, 0, st>>>(weights, (const double*)Qc, Q0, (const double*)PRf, (const double*)Rc, X,
                                             Y, E);
  else
    k_make_pairs<float><<<nb, 256, 0, st>>>(weights, (const float*)Qc, Q0, (const float*)PRf, (const float*)Rc, X, Y,
                                            E);
  return cudaGetLastError();
}

cudaError_t adam(float* master, float* m1, float* m2, const float* grad, void* weights, float lr, float b1, float b2,
                 float eps, int64_t t, cudaStream_t st) {
  const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
  k_adam<<<(ClosureLayout::n_params + 255) / 256, 256, 0, st>>>(master, m1, m2, grad, weights, lr, b1, b2, eps, c1,
                                                                c2);
  return cudaGetLastError();
}

cudaError_t load_master(const void* weights, float* master, cudaStream_t st) {
  k_load_master<<<(ClosureLayout::n_params + 255) / 256, 256, 0, st>>>(weights, master);
  return cudaGetLastError();
}

// Seeded host initialisation of a record: uniform weights scaled by sqrt(3 / fan_in) (output layer
// by 0.1), zero biases, given input and output scales.
std::vector<unsigned char> init_record(uint64_t seed, const float* in_scale, const float* out_scale) {
  std::vector<unsigned char> rec(ClosureLayout::total_bytes, 0);
  std::mt19937_64 gen(seed);
  std::uniform_real_distribution<double> uni(-1.0, 1.0);
  auto fill = [&](size_t off, int n_out, int n_in, double scale) {
    __nv_bfloat16* w = (__nv_bfloat16*)(rec.data() + off);
    const double lim = scale * std::sqrt(3.0 / n_in);
    for (int i = 0; i < n_out * n_in; ++i) w[i] = __float2bfloat16_rn((float)(lim * uni(gen)));
  };
  fill(ClosureLayout::oW1, NH, NI, 1.0);
  fill(ClosureLayout::oW2, NH, NH, 1.0);
  fill(ClosureLayout::oW3, NO, NH, 0.1);
  std::memcpy(rec.data() + ClosureLayout::oin, in_scale, 5 * sizeof(float));
  std::memcpy(rec.data() + ClosureLayout::oout, out_scale, 5 * sizeof(float));
  return rec;
}

}  // namespace chorus
