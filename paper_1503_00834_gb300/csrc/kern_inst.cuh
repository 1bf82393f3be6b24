// Launchers of the residual kernels for one order N, for the FP64 total-state form and the FP32
// perturbation form.  Each kern_p<p>.cu instantiates this header once.
#pragma once
#include "sd_kernels.cuh"

namespace chorus {

// EPB32R: elements per CTA of the FP32 residual kernel (by default those of the FP32 lifting kernel;
// the two kernels share no shared-memory layout, only the per-element arrays in global memory).
template <int N, int EPB64, int EPB32, int EPB32R = EPB32>
struct Inst {
  using L64 = Launch<N, false, double, EPB64>;
  using L32 = Launch<N, true, float, EPB32>;
  using L32R = Launch<N, true, float, EPB32R>;

  static cudaError_t trace64(const MeshArg<double>& m, const OpsArg<double>& ops, const double* q, double* T,
                             cudaStream_t st) {
    return L64::trace(m, ops, q, T, st);
  }
  static cudaError_t trace32(const MeshArg<float>& m, const OpsArg<float>& ops, const float* q, float* T,
                             cudaStream_t st) {
    return L32::trace(m, ops, q, T, st);
  }
  static cudaError_t grad64(const MeshArg<double>& m, const OpsArg<double>& ops, const PhysArg<double>& ph,
                            const double* q, const double* T, double* Tv, double* grad_rho_out, double* G,
                            double* Fc, unsigned* err, cudaStream_t st) {
    KArgs<double> A{};
    A.m = m; A.ops = ops; A.ph = ph; A.q = q; A.T = T; A.Tv_out = Tv; A.grad_rho_out = grad_rho_out; A.err = err;
    A.G_out = G; A.Fc_out = Fc;
    return L64::grad(A, st);
  }
  static cudaError_t grad32(const MeshArg<float>& m, const OpsArg<float>& ops, const PhysArg<float>& ph,
                            const BgArg& bg, const float* q, const float* T, float* Tv, float* G, float* Fc,
                            unsigned* err, cudaStream_t st) {
    KArgs<float> A{};
    A.m = m; A.ops = ops; A.ph = ph; A.bg = bg; A.q = q; A.T = T; A.Tv_out = Tv; A.err = err;
    A.G_out = G; A.Fc_out = Fc;
    return L32::grad(A, st);
  }
  static cudaError_t face64(const MeshArg<double>& m, const PhysArg<double>& ph, const int2* faces, int nf, int nw,
                            const double* T, const double* Tv, double* Fc, cudaStream_t st) {
    KArgs<double> A{};
    A.m = m; A.ph = ph; A.T = T; A.Tv = Tv; A.Fc_out = Fc;
    return L64::face(A, faces, nf, nw, st);
  }
  static cudaError_t face32(const MeshArg<float>& m, const PhysArg<float>& ph, const BgArg& bg, const int2* faces,
                            int nf, int nw, const float* T, const float* Tv, float* Fc, cudaStream_t st) {
    KArgs<float> A{};
    A.m = m; A.ph = ph; A.bg = bg; A.T = T; A.Tv = Tv; A.Fc_out = Fc;
    return L32::face(A, faces, nf, nw, st);
  }
  template <class R>
  static void set_rk(KArgs<R>& A, const RkCoef<R>& rk) {
    A.un = rk.un; A.a = rk.a; A.b = rk.b; A.c = rk.c;
    A.un2 = rk.un2; A.out2 = rk.out2; A.a2 = rk.a2; A.b2 = rk.b2; A.c2 = rk.c2; A.radd = rk.radd;
  }
  static cudaError_t resid64(const MeshArg<double>& m, const OpsArg<double>& ops, const PhysArg<double>& ph,
                             const double* q, const double* T, const double* Tv, const double* G, const double* Fc,
                             double* out, double* T_out, const RkCoef<double>& rk, double dt, int mode, unsigned* err,
                             cudaStream_t st) {
    KArgs<double> A{};
    A.m = m; A.ops = ops; A.ph = ph; A.q = q; A.T = T; A.Tv = Tv; A.out = out; A.T_out = T_out; A.G_in = G;
    A.Fc = Fc;
    set_rk(A, rk);
    A.dt = dt; A.err = err;
    return mode == kModeRK ? L64::template resid<kModeRK>(A, st) : L64::template resid<kModeResidual>(A, st);
  }
  static cudaError_t resid32(const MeshArg<float>& m, const OpsArg<float>& ops, const PhysArg<float>& ph,
                             const BgArg& bg, const float* q, const float* T, const float* Tv, const float* G,
                             const float* Fc, float* out, float* T_out, const RkCoef<float>& rk, float dt, int mode,
                             unsigned* err, cudaStream_t st) {
    KArgs<float> A{};
    A.m = m; A.ops = ops; A.ph = ph; A.bg = bg; A.q = q; A.T = T; A.Tv = Tv; A.out = out; A.T_out = T_out;
    A.G_in = G; A.Fc = Fc;
    set_rk(A, rk);
    A.dt = dt; A.err = err;
    return mode == kModeRK ? L32R::template resid<kModeRK>(A, st) : L32R::template resid<kModeResidual>(A, st);
  }
  static LaunchSet set() {
    return LaunchSet{trace64, grad64, face64, resid64, trace32, grad32, face32, resid32, EPB32};
  }
};

}  // namespace chorus
