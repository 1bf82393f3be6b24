// Internal structures shared by the C-ABI layer and the per-order kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace chorus {

constexpr int kMaxN = 6;
// entries of the gradient record per solution point: grad rho (3), trace-free strain (6), grad p (3)
constexpr int kG = 12;

// 1D operators for one order, passed to kernels by value (parameter bank).
template <class R>
struct OpsArg {
  R I[kMaxN + 1][kMaxN];     // h_s(Xf_f)
  R D[kMaxN][kMaxN + 1];     // l'_f(X_s)
  R Dsol[kMaxN][kMaxN];      // D I
  R Lfs[kMaxN][kMaxN + 1];   // l_a(X_s)
  R w[kMaxN];                // quadrature weights
};

// Physical constants derived from chorus_params (nondimensional).
template <class R>
struct PhysArg {
  R gamma, gm1, Rgas, CpR;   // CpR = C_p / R_gas
  R kappa, kappa_r, nu;
  R GM, twoOmega;
  R T_top, bottom_flux;
  // polytrope (Eqs. 25-27): chi = c + alpha d / r, rho_a = rho_c chi^n, p_a = p_c chi^(n+1)
  double chi_c, chi_ad, rho_c, p_c, poly_n;
};

// Mesh data on the device for one precision.
template <class R>
struct MeshArg {
  int E;
  const int* nbr;    // [E][6] neighbour element, -1 inner wall, -2 outer wall
  const int* code;   // [E][6] neighbour local face * 8 + orientation bits
  const R* Sf;       // [E][3 d][3 n][N+1 f][N*N line]  S^d_n = |J| d xi_d / d x_n at the d-flux points
  const R* invJ;     // [E][N^3] 1/|J| at the solution points
  const R* x;        // [E][3][N^3] solution-point coordinates
  const R* kr;       // [E][3 d][N+1 f][N*N line] radiative diffusivity at the d-flux points, or null:
                     // the constant kappa_r
};

// Background tables of the perturbation path (float, from FP64 computations).
struct BgArg {
  const float* bg;     // [E][2][N^3]     rho0, E0
  const float* grho0;  // [E][3][N^3]     lifted background density gradient
  const float* bgT;    // [E][6][2][N^2]  rho0, E0 on the face points
  const float* R0;     // [E][5][N^3]     FP64 residual of the background, rounded (null: left out)
};

// Point order of the FP32 background tables rho0, E0 and the lifted grad rho0: at N = 4 they are
// stored in the kernels' XOR-swizzled shared-memory order (point (i,j,k) at i + 4((j^k)&3) + 16k),
// so that the bulk copies land them conflict-free for the line sweeps of every direction; at other
// orders in the state's linear order i + N j + N^2 k.
constexpr bool kBgSwizzle = true;
__host__ __device__ inline constexpr bool bg_swizzle(int N) { return kBgSwizzle && N == 4; }
__host__ __device__ inline int bg_point(int N, int pt) {
  if (!bg_swizzle(N)) return pt;
  const int i = pt % 4, j = (pt / 4) % 4, k = pt / 16;
  return i + 4 * ((j ^ k) & 3) + 16 * k;
}

enum ResidMode { kModeResidual = 0, kModeRK = 1 };

// Stage combination of the RK update fused into the residual kernel:
//   out  = a un  + b q + c dt R
//   out2 = a2 un2 + b2 q + c2 dt R   (when out2 != nullptr)
// where R includes `radd` (an additive residual correction, e.g. the learned closure) when non-null.
template <class R>
struct RkCoef {
  const R* un;
  R a, b, c;
  const R* un2;
  R* out2;
  R a2, b2, c2;
  const R* radd;
};

// Per-order launchers (defined in kern_p<N>.cu).  All return cudaGetLastError().
struct LaunchSet {
  cudaError_t (*trace64)(const MeshArg<double>&, const OpsArg<double>&, const double* q, double* T, cudaStream_t);
  // G: gradient record [E][12][N^3] written by grad (when non-null) and read by resid (required:
  // resid returns cudaErrorInvalidValue without it).  Fc: common face fluxes F~ [E][6][5][N^2], written
  // by face (interior and wall faces) and read by resid (required).
  cudaError_t (*grad64)(const MeshArg<double>&, const OpsArg<double>&, const PhysArg<double>&, const double* q,
                        const double* T, double* Tv, double* grad_rho_out, double* G, double* Fc, unsigned* err,
                        cudaStream_t);
  // faces: n_faces interior faces (from their lower element), then n_walls wall faces
  cudaError_t (*face64)(const MeshArg<double>&, const PhysArg<double>&, const int2* faces, int n_faces, int n_walls,
                        const double* T, const double* Tv, double* Fc, cudaStream_t);
  cudaError_t (*resid64)(const MeshArg<double>&, const OpsArg<double>&, const PhysArg<double>&, const double* q,
                         const double* T, const double* Tv, const double* G, const double* Fc, double* out,
                         double* T_out, const RkCoef<double>& rk, double dt, int mode, unsigned* err, cudaStream_t);
  cudaError_t (*trace32)(const MeshArg<float>&, const OpsArg<float>&, const float* q, float* T, cudaStream_t);
  cudaError_t (*grad32)(const MeshArg<float>&, const OpsArg<float>&, const PhysArg<float>&, const BgArg&,
                        const float* q, const float* T, float* Tv, float* G, float* Fc, unsigned* err, cudaStream_t);
  cudaError_t (*face32)(const MeshArg<float>&, const PhysArg<float>&, const BgArg&, const int2* faces, int n_faces,
                        int n_walls, const float* T, const float* Tv, float* Fc, cudaStream_t);
  cudaError_t (*resid32)(const MeshArg<float>&, const OpsArg<float>&, const PhysArg<float>&, const BgArg&,
                         const float* q, const float* T, const float* Tv, const float* G, const float* Fc, float* out,
                         float* T_out, const RkCoef<float>& rk, float dt, int mode, unsigned* err, cudaStream_t);
  int epb32;  // elements per CTA of the FP32 kernels
};

// Each order is built with kTiles tile shapes of its FP32 kernels (elements per CTA); tile 0 is
// the default, the others are candidates for the batched-shell autotuner.  FP64 kernels have one.
constexpr int kTiles = 2;
LaunchSet launchers_p2(int tile);
LaunchSet launchers_p3(int tile);
LaunchSet launchers_p4(int tile);
LaunchSet launchers_p5(int tile);

}  // namespace chorus
