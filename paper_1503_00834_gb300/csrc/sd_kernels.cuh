// Spectral-difference residual kernels for one order N = p + 1 (paper Sections 3 and 5).
//
// One CTA processes EPB elements; each element is handled by N*N threads, thread `ln` owning the
// line (t1, t2) = (ln % N, ln / N) of every direction (xi-line (j,k), eta-line (i,k), zeta-line
// (i,j)).  A thread therefore does the whole 1D work of its line - interpolation to the N+1 flux
// points (Eq. 17), fluxes, face common fluxes at the two end points, derivative back to the N
// solution points (Eq. 18) - in registers; shared memory carries the element data between the
// three directional sweeps.  The element's state block is staged into shared memory with a 1D
// bulk TMA copy (cp.async.bulk + mbarrier) when it is 16-byte aligned.
//
// Two physics forms share the kernels:
//   PERT = false, R = double : Q is the total conserved state; plain fluxes.
//   PERT = true,  R = float  : Q is q' = Q - Q0 about the polytrope at rest; every nonlinear
//                              term is written as an exact algebraic difference F(Q0+q') - F(Q0)
//                              so that FP32 rounding is relative to the perturbation, and the
//                              FP64 background residual R(Q0) is added at the end.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace chorus {

// ------------------------------------------------------------------ async-copy helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// 1D bulk copy global -> shared, completion signalled on the mbarrier (byte count).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait on phase 0 of the barrier.  Returns false (and sets *err) if the limit ran out.
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar, unsigned* err) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.b32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  if (err) atomicOr(err, 1u);
  return false;
}

// ------------------------------------------------------------------ index helpers

// point index of position s along line `ln` of direction d
template <int N>
__device__ __forceinline__ int pt_of(int d, int ln, int s) {
  const int t1 = ln % N, t2 = ln / N;
  if (d == 0) return s + N * t1 + N * N * t2;
  if (d == 1) return t1 + N * s + N * N * t2;
  return t1 + N * t2 + N * N * s;
}

// neighbour face-point index of own face point t under the orientation bits (swap, flip1, flip2)
template <int N>
__device__ __forceinline__ int map_face_pt(int t, int orient) {
  const int t1 = t % N, t2 = t / N;
  int a = (orient & 4) ? t2 : t1;
  int b = (orient & 4) ? t1 : t2;
  if (orient & 2) a = N - 1 - a;
  if (orient & 1) b = N - 1 - b;
  return a + N * b;
}

// ------------------------------------------------------------------ point physics

template <class R>
struct Pt {
  R rho;    // total density
  R rhop;   // the form's density variable (rho or rho')
  R u[3];   // velocity
  R p;      // the form's pressure variable (p or p')
  R ptot;   // total pressure
  R Etot;   // total energy
};

template <bool PERT, class R>
__device__ __forceinline__ Pt<R> point_state(const R q[5], R rho0, R E0, const PhysArg<R>& ph) {
  Pt<R> s;
  s.rhop = q[0];
  s.rho = PERT ? rho0 + q[0] : q[0];
  const R ir = R(1) / s.rho;
  s.u[0] = q[1] * ir;
  s.u[1] = q[2] * ir;
  s.u[2] = q[3] * ir;
  const R ke = R(0.5) * (q[1] * s.u[0] + q[2] * s.u[1] + q[3] * s.u[2]);
  s.p = ph.gm1 * (q[4] - ke);
  if (PERT) {
    s.ptot = ph.gm1 * E0 + s.p;
    s.Etot = E0 + q[4];
  } else {
    s.ptot = s.p;
    s.Etot = q[4];
  }
  return s;
}

// s . (F, G, H)_inv (Eq. 6); in the perturbation form the difference from the background.
template <class R>
__device__ __forceinline__ void flux_inv(const R q[5], const Pt<R>& st, const R s[3], R F[5]) {
  const R Vn = st.u[0] * s[0] + st.u[1] * s[1] + st.u[2] * s[2];
  F[0] = q[1] * s[0] + q[2] * s[1] + q[3] * s[2];
  F[1] = q[1] * Vn + st.p * s[0];
  F[2] = q[2] * Vn + st.p * s[1];
  F[3] = q[3] * Vn + st.p * s[2];
  F[4] = Vn * (st.Etot + st.ptot);
}

// s . (F, G, H)_v (Eqs. 7-9; energy entry u.tau - f as in Eq. 3).
// g: the form's grad rho [0..2], grad u [3 + 3a + b] = d u_a / d x_b, the form's grad p [12..14].
// gr0: background density gradient (perturbation form only).
template <bool PERT, class R>
__device__ __forceinline__ void flux_visc(const Pt<R>& st, const R g[15], const R gr0[3], R rho0, R p0,
                                          const R s[3], const PhysArg<R>& ph, R Fv[5]) {
  const R mu = st.rho * ph.nu;
  const R div = g[3] + g[7] + g[11];
  R ts[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R acc = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) acc += (g[3 + 3 * a + b] + g[3 + 3 * b + a]) * s[b];
    ts[a] = mu * (acc - R(2.0 / 3.0) * div * s[a]);
  }
  const R pr = st.ptot / st.rho;
  R dpr = R(0);
  if (PERT) dpr = (st.p * rho0 - p0 * st.rhop) / (st.rho * rho0);  // p/rho - p0/rho0
  R fs = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    R A = pr * g[b];
    if (PERT) A += dpr * gr0[b];
    const R fb = -ph.CpR * (ph.kappa * (g[12 + b] / ph.gamma - A) + ph.kappa_r * (g[12 + b] - A));
    fs += fb * s[b];
  }
  Fv[0] = R(0);
  Fv[1] = ts[0];
  Fv[2] = ts[1];
  Fv[3] = ts[2];
  Fv[4] = st.u[0] * ts[0] + st.u[1] * ts[1] + st.u[2] * ts[2] - fs;
}

// primitive gradients from conserved ones: gq[3 v + n] = d q_v / d x_n
template <bool PERT, class R>
__device__ __forceinline__ void grad_prim(const Pt<R>& st, const R gq[15], const R gr0[3], const PhysArg<R>& ph,
                                          R g[15]) {
  R grt[3];
#pragma unroll
  for (int n = 0; n < 3; ++n) {
    grt[n] = PERT ? gr0[n] + gq[n] : gq[n];
    g[n] = gq[n];
  }
  const R ir = R(1) / st.rho;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int n = 0; n < 3; ++n) g[3 + 3 * a + n] = (gq[3 * (1 + a) + n] - st.u[a] * grt[n]) * ir;
  const R ke = R(0.5) * (st.u[0] * st.u[0] + st.u[1] * st.u[1] + st.u[2] * st.u[2]);
#pragma unroll
  for (int n = 0; n < 3; ++n)
    g[12 + n] = ph.gm1 * (gq[12 + n] - (st.u[0] * gq[3 + n] + st.u[1] * gq[6 + n] + st.u[2] * gq[9 + n]) +
                          ke * grt[n]);
}

template <bool PERT, class R>
__device__ __forceinline__ void rusanov(const R qL[5], const Pt<R>& sL, R rho0L, R E0L, const R qR[5],
                                        const Pt<R>& sR, R rho0R, R E0R, const R n[3], const PhysArg<R>& ph,
                                        R F[5]) {
  R FL[5], FR[5];
  flux_inv(qL, sL, n, FL);
  flux_inv(qR, sR, n, FR);
  const R cL = sqrt(ph.gamma * sL.ptot / sL.rho);
  const R cR = sqrt(ph.gamma * sR.ptot / sR.rho);
  const R vL = fabs(sL.u[0] * n[0] + sL.u[1] * n[1] + sL.u[2] * n[2]) + cL;
  const R vR = fabs(sR.u[0] * n[0] + sR.u[1] * n[1] + sR.u[2] * n[2]) + cR;
  const R lam = vL > vR ? vL : vR;
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * lam * (qR[v] - qL[v]);
  if (PERT) {
    const R c0L = sqrt(ph.gamma * ph.gm1 * E0L / rho0L);
    const R c0R = sqrt(ph.gamma * ph.gm1 * E0R / rho0R);
    const R lam0 = c0L > c0R ? c0L : c0R;
    F[0] -= R(0.5) * (lam - lam0) * (rho0R - rho0L);
    F[4] -= R(0.5) * (lam - lam0) * (E0R - E0L);
  }
}

// ------------------------------------------------------------------ shared layouts

template <int N, bool PERT, class R, int EPB>
struct Layout {
  static constexpr int N2 = N * N, N3 = N * N * N;
  // per-element sizes in R words
  static constexpr int SQ = 5 * N3;
  static constexpr int SG = 15 * N3;
  static constexpr int SDIV = 5 * N3;
  static constexpr int ST = 6 * 5 * N2;
  static constexpr int STV = 6 * 4 * N2;
  static constexpr int SBG = PERT ? 2 * N3 : 0;
  static constexpr int SGR0 = PERT ? 3 * N3 : 0;
  static constexpr int STBG = PERT ? 6 * 2 * N2 : 0;
  // offsets of the per-CTA arrays (arrays of EPB element blocks), kept 16-byte aligned
  static constexpr int al(int x) { return (x + (16 / (int)sizeof(R)) - 1) / (16 / (int)sizeof(R)) * (16 / (int)sizeof(R)); }
  static constexpr int oQ = 0;
  static constexpr int oBG = oQ + al(EPB * SQ);
  static constexpr int oGR0 = oBG + al(EPB * SBG);
  static constexpr int oG = oGR0 + al(EPB * SGR0);
  static constexpr int oT = oG + al(EPB * SG);
  static constexpr int oTBG = oT + al(EPB * ST);
  static constexpr int oTV = oTBG + al(EPB * STBG);
  static constexpr int oDIV = oTV + al(EPB * STV);
  static constexpr int total_grad = oTV;  // grad kernel needs no Tv / div
  static constexpr int total_resid = oDIV + al(EPB * SDIV);
};

// Copy `count` R words from global to shared: one bulk TMA copy when aligned, else a cooperative
// plain copy.  Returns whether the TMA path was used (the caller then waits on the barrier).
template <class R>
__device__ __forceinline__ bool stage(R* dst, const R* src, int count, uint64_t* bar, bool issue_tma) {
  const uint32_t bytes = (uint32_t)count * sizeof(R);
  const bool tma = issue_tma && (((uintptr_t)src & 15u) == 0) && ((bytes & 15u) == 0) && bytes > 0;
  if (!tma) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
  }
  return tma;
}

// ------------------------------------------------------------------ kernel arguments

template <class R>
struct KArgs {
  MeshArg<R> m;
  OpsArg<R> ops;
  PhysArg<R> ph;
  BgArg bg;            // perturbation form only
  const R* q;          // state (form variables)
  const R* T;          // own-face traces of q, [E][6][5][N2]
  const R* Tv;         // one-sided normal viscous fluxes [E][6][4][N2] (resid kernel input)
  R* Tv_out;           // grad kernel output
  R* grad_rho_out;     // optional grad kernel output: lifted d rho / d x_n [E][3][N3]
  R* out;              // residual or new state
  R* T_out;            // traces of the new state (RK mode)
  const R* un;         // u^n for the RK combination
  R a, b, dt;          // out = a un + b (q + dt R)
  unsigned* err;
};

// ------------------------------------------------------------------ trace kernel

template <int N, class R, int EPB>
__global__ void __launch_bounds__(EPB * N * N) k_trace(const MeshArg<R> m, const OpsArg<R> ops, const R* __restrict__ q,
                                                      R* __restrict__ T) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int e = blockIdx.x * EPB + el;
  if (el >= EPB || e >= m.E) return;
  const R* qe = q + (size_t)e * 5 * N3;
  R* Te = T + (size_t)e * 6 * 5 * N2;
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R lo = R(0), hi = R(0);
#pragma unroll
      for (int s = 0; s < N; ++s) {
        const R val = qe[v * N3 + pt_of<N>(d, ln, s)];
        lo += ops.I[0][s] * val;
        hi += ops.I[N][s] * val;
      }
      Te[((2 * d) * 5 + v) * N2 + ln] = lo;
      Te[((2 * d + 1) * 5 + v) * N2 + ln] = hi;
    }
}

// ------------------------------------------------------------------ shared lifting phase

// Stages the element data, gathers the neighbour traces and computes the lifted primitive
// gradients g[15][N3] of every element of the CTA into shared memory (BR1-like averaging,
// conserved-variable lifting, chain rule with grad xi = S / |J|).
template <int N, bool PERT, class R, int EPB, bool RESID>
__device__ __forceinline__ void lift_phase(const KArgs<R>& A, R* sm, uint64_t* bar, int el, int ln, int e,
                                           bool active, int ne) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N2 = N * N, N3 = N * N * N;
  const int e0 = blockIdx.x * EPB;
  R* sq = sm + L::oQ;
  R* sbg = sm + L::oBG;
  R* sgr0 = sm + L::oGR0;
  R* sg = sm + L::oG;
  R* sT = sm + L::oT;
  R* sTbg = sm + L::oTBG;
  R* sTv = sm + L::oTV;

  // ---- stage the element blocks (bulk TMA when aligned)
  const bool full = (ne == EPB);
  bool t0 = stage(sq, A.q + (size_t)e0 * 5 * N3, ne * 5 * N3, bar, full);
  bool t1 = false, t2 = false;
  if (PERT) {
    t1 = stage(sbg, (const R*)A.bg.bg + (size_t)e0 * 2 * N3, ne * 2 * N3, bar, full);
    t2 = stage(sgr0, (const R*)A.bg.grho0 + (size_t)e0 * 3 * N3, ne * 3 * N3, bar, full);
  }
  if (threadIdx.x == 0 && (t0 || t1 || t2)) {
    uint32_t bytes = (t0 ? ne * 5 * N3 : 0) * sizeof(R);
    if (PERT) bytes += ((t1 ? ne * 2 * N3 : 0) + (t2 ? ne * 3 * N3 : 0)) * sizeof(R);
    mbar_expect_tx(bar, bytes);
    if (t0) bulk_g2s(sq, A.q + (size_t)e0 * 5 * N3, ne * 5 * N3 * sizeof(R), bar);
    if (PERT && t1) bulk_g2s(sbg, (const R*)A.bg.bg + (size_t)e0 * 2 * N3, ne * 2 * N3 * sizeof(R), bar);
    if (PERT && t2) bulk_g2s(sgr0, (const R*)A.bg.grho0 + (size_t)e0 * 3 * N3, ne * 3 * N3 * sizeof(R), bar);
  }

  // ---- gather neighbour face data (overlaps the bulk copy) and clear the gradient accumulator
  if (active) {
#pragma unroll 1
    for (int F = 0; F < 6; ++F) {
      const int nb = A.m.nbr[e * 6 + F];
      if (nb >= 0) {
        const int c = A.m.code[e * 6 + F];
        const int tp = map_face_pt<N>(ln, c & 7);
        const size_t base = (size_t)nb * 6 + (c >> 3);
#pragma unroll
        for (int v = 0; v < 5; ++v) sT[(el * 6 + F) * 5 * N2 + v * N2 + ln] = A.T[base * 5 * N2 + v * N2 + tp];
        if (RESID) {
#pragma unroll
          for (int v = 0; v < 4; ++v) sTv[(el * 6 + F) * 4 * N2 + v * N2 + ln] = A.Tv[base * 4 * N2 + v * N2 + tp];
          if (PERT) {
#pragma unroll
            for (int v = 0; v < 2; ++v)
              sTbg[(el * 6 + F) * 2 * N2 + v * N2 + ln] = (R)A.bg.bgT[base * 2 * N2 + v * N2 + tp];
          }
        }
      }
    }
  }
  for (int i = threadIdx.x; i < EPB * 15 * N3; i += blockDim.x) sg[i] = R(0);
  if (t0 || t1 || t2) mbar_wait0(bar, A.err);
  __syncthreads();

  // ---- lifting, one direction at a time
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    if (active) {
      R qv[5][N];
      R r0[N], E0l[N];
#pragma unroll
      for (int s = 0; s < N; ++s) {
        const int pt = pt_of<N>(d, ln, s);
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v][s] = sq[el * 5 * N3 + v * N3 + pt];
        if (PERT) {
          r0[s] = sbg[el * 2 * N3 + pt];
          E0l[s] = sbg[el * 2 * N3 + N3 + pt];
        } else {
          r0[s] = R(0);
          E0l[s] = R(0);
        }
      }
      R S[3][N + 1];
      const R* Sl = A.m.Sf + ((size_t)e * 3 + d) * 3 * (N + 1) * N2;
#pragma unroll
      for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int f = 0; f <= N; ++f) S[n][f] = Sl[(n * (N + 1) + f) * N2 + ln];
      // common state at both ends
      R dq[5][2];  // q_c - q_own at end 0 and end N
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int f = side ? N : 0;
        const int F = 2 * d + side;
        R qe[5];
        R rho0e = R(0), E0e = R(0);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          R acc = R(0);
#pragma unroll
          for (int s = 0; s < N; ++s) acc += A.ops.I[f][s] * qv[v][s];
          qe[v] = acc;
        }
        if (PERT) {
#pragma unroll
          for (int s = 0; s < N; ++s) {
            rho0e += A.ops.I[f][s] * r0[s];
            E0e += A.ops.I[f][s] * E0l[s];
          }
        }
        const int nb = A.m.nbr[e * 6 + F];
        if (nb >= 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v)
            dq[v][side] = R(0.5) * (sT[(el * 6 + F) * 5 * N2 + v * N2 + ln] - qe[v]);
        } else {
          // wall common state: zero normal velocity, interior density, interior pressure (inner
          // wall) or p = R rho T_top (outer wall)
          const R sg_ = side ? R(1) : R(-1);
          const R mag = sqrt(S[0][f] * S[0][f] + S[1][f] * S[1][f] + S[2][f] * S[2][f]);
          const R nh[3] = {sg_ * S[0][f] / mag, sg_ * S[1][f] / mag, sg_ * S[2][f] / mag};
          const Pt<R> st = point_state<PERT>(qe, rho0e, E0e, A.ph);
          const R mn = qe[1] * nh[0] + qe[2] * nh[1] + qe[3] * nh[2];
          R mc[3] = {qe[1] - mn * nh[0], qe[2] - mn * nh[1], qe[3] - mn * nh[2]};
          R pc;
          if (nb == -2) pc = A.ph.Rgas * st.rhop * A.ph.T_top;  // the form's density times R T_top
          else pc = st.p;
          const R Ec = pc / A.ph.gm1 + R(0.5) * (mc[0] * mc[0] + mc[1] * mc[1] + mc[2] * mc[2]) / st.rho;
          dq[0][side] = R(0);
          dq[1][side] = mc[0] - qe[1];
          dq[2][side] = mc[1] - qe[2];
          dq[3][side] = mc[2] - qe[3];
          dq[4][side] = Ec - qe[4];
        }
      }
      // grad xi_d at the line's solution points
      R gx[3][N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const R ij = A.m.invJ[(size_t)e * N3 + pt_of<N>(d, ln, i)];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          R acc = R(0);
#pragma unroll
          for (int f = 0; f <= N; ++f) acc += A.ops.Lfs[i][f] * S[n][f];
          gx[n][i] = acc * ij;
        }
      }
      // d q / d xi_d = Dsol q + D[:,0] (q_c0 - q_0) + D[:,N] (q_cN - q_N), then accumulate grad q
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int pt = pt_of<N>(d, ln, i);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          R acc = A.ops.D[i][0] * dq[v][0] + A.ops.D[i][N] * dq[v][1];
#pragma unroll
          for (int s = 0; s < N; ++s) acc += A.ops.Dsol[i][s] * qv[v][s];
#pragma unroll
          for (int n = 0; n < 3; ++n) sg[el * 15 * N3 + (3 * v + n) * N3 + pt] += acc * gx[n][i];
        }
      }
    }
    __syncthreads();
  }

  // ---- optional raw density-gradient output, then conversion to primitive gradients
  if (active) {
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      const int pt = N * ln + i;
      if (A.grad_rho_out) {
#pragma unroll
        for (int n = 0; n < 3; ++n) A.grad_rho_out[((size_t)e * 3 + n) * N3 + pt] = sg[el * 15 * N3 + n * N3 + pt];
      }
      R q[5], gq[15], gr0[3], g[15];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = sq[el * 5 * N3 + v * N3 + pt];
#pragma unroll
      for (int c = 0; c < 15; ++c) gq[c] = sg[el * 15 * N3 + c * N3 + pt];
      R rho0 = R(0), E0 = R(0);
      if (PERT) {
        rho0 = sbg[el * 2 * N3 + pt];
        E0 = sbg[el * 2 * N3 + N3 + pt];
#pragma unroll
        for (int n = 0; n < 3; ++n) gr0[n] = sgr0[el * 3 * N3 + n * N3 + pt];
      } else {
        gr0[0] = gr0[1] = gr0[2] = R(0);
      }
      const Pt<R> st = point_state<PERT>(q, rho0, E0, A.ph);
      grad_prim<PERT>(st, gq, gr0, A.ph, g);
#pragma unroll
      for (int c = 0; c < 15; ++c) sg[el * 15 * N3 + c * N3 + pt] = g[c];
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ gradient kernel

// Lifted gradients, then the one-sided normal viscous flux F_v . n_out on every face point,
// written for the neighbours: Tv[e][F][0..2] = tau n, Tv[e][F][3] = u.tau n - f.n.
template <int N, bool PERT, class R, int EPB>
__global__ void __launch_bounds__(EPB * N * N) k_grad(const KArgs<R> A) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  R* sm = reinterpret_cast<R*>(smem_raw);
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int e0 = blockIdx.x * EPB;
  const int ne = min(EPB, A.m.E - e0);
  const int e = e0 + el;
  const bool active = el < ne;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  lift_phase<N, PERT, R, EPB, false>(A, sm, &bar, el, ln, e, active, ne);
  if (!active || A.Tv_out == nullptr) return;
  const R* sq = sm + L::oQ;
  const R* sbg = sm + L::oBG;
  const R* sgr0 = sm + L::oGR0;
  const R* sg = sm + L::oG;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const R* Sl = A.m.Sf + ((size_t)e * 3 + d) * 3 * (N + 1) * N2;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const int f = side ? N : 0;
      R qf[5] = {R(0), R(0), R(0), R(0), R(0)}, gf[15], gr0f[3] = {R(0), R(0), R(0)};
      R rho0f = R(0), E0f = R(0);
#pragma unroll
      for (int c = 0; c < 15; ++c) gf[c] = R(0);
#pragma unroll
      for (int s = 0; s < N; ++s) {
        const int pt = pt_of<N>(d, ln, s);
        const R w = A.ops.I[f][s];
#pragma unroll
        for (int v = 0; v < 5; ++v) qf[v] += w * sq[el * 5 * N3 + v * N3 + pt];
#pragma unroll
        for (int c = 0; c < 15; ++c) gf[c] += w * sg[el * 15 * N3 + c * N3 + pt];
        if (PERT) {
          rho0f += w * sbg[el * 2 * N3 + pt];
          E0f += w * sbg[el * 2 * N3 + N3 + pt];
#pragma unroll
          for (int n = 0; n < 3; ++n) gr0f[n] += w * sgr0[el * 3 * N3 + n * N3 + pt];
        }
      }
      R s3[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) s3[n] = Sl[(n * (N + 1) + f) * N2 + ln];
      const R sgn = side ? R(1) : R(-1);
      const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
      const R nh[3] = {sgn * s3[0] / mag, sgn * s3[1] / mag, sgn * s3[2] / mag};
      const Pt<R> st = point_state<PERT>(qf, rho0f, E0f, A.ph);
      R Fv[5];
      flux_visc<PERT>(st, gf, gr0f, rho0f, A.ph.gm1 * E0f, nh, A.ph, Fv);
      const int F = 2 * d + side;
      R* o = A.Tv_out + ((size_t)e * 6 + F) * 4 * N2;
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v * N2 + ln] = Fv[1 + v];
    }
  }
}

// ------------------------------------------------------------------ residual kernel

template <int N, bool PERT, class R, int EPB, int MODE>
__global__ void __launch_bounds__(EPB * N * N) k_resid(const KArgs<R> A) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  R* sm = reinterpret_cast<R*>(smem_raw);
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int e0 = blockIdx.x * EPB;
  const int ne = min(EPB, A.m.E - e0);
  const int e = e0 + el;
  const bool active = el < ne;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  lift_phase<N, PERT, R, EPB, true>(A, sm, &bar, el, ln, e, active, ne);
  R* sq = sm + L::oQ;
  const R* sbg = sm + L::oBG;
  const R* sgr0 = sm + L::oGR0;
  const R* sg = sm + L::oG;
  const R* sT = sm + L::oT;
  const R* sTbg = sm + L::oTBG;
  const R* sTv = sm + L::oTV;
  R* sdiv = sm + L::oDIV;
  const PhysArg<R>& ph = A.ph;

  // ---- flux sweeps: transformed fluxes at the flux points, common fluxes at the two ends,
  //      derivative back to the solution points (Eqs. 12, 17, 18)
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    if (active) {
      R acc[5][N];
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int i = 0; i < N; ++i) acc[v][i] = R(0);
      const R* Sl = A.m.Sf + ((size_t)e * 3 + d) * 3 * (N + 1) * N2;
#pragma unroll
      for (int f = 0; f <= N; ++f) {
        R qf[5], gf[15], gr0f[3] = {R(0), R(0), R(0)};
        R rho0f = R(0), E0f = R(0);
#pragma unroll
        for (int v = 0; v < 5; ++v) qf[v] = R(0);
#pragma unroll
        for (int c = 0; c < 15; ++c) gf[c] = R(0);
#pragma unroll
        for (int s = 0; s < N; ++s) {
          const int pt = pt_of<N>(d, ln, s);
          const R w = A.ops.I[f][s];
#pragma unroll
          for (int v = 0; v < 5; ++v) qf[v] += w * sq[el * 5 * N3 + v * N3 + pt];
#pragma unroll
          for (int c = 0; c < 15; ++c) gf[c] += w * sg[el * 15 * N3 + c * N3 + pt];
          if (PERT) {
            rho0f += w * sbg[el * 2 * N3 + pt];
            E0f += w * sbg[el * 2 * N3 + N3 + pt];
#pragma unroll
            for (int n = 0; n < 3; ++n) gr0f[n] += w * sgr0[el * 3 * N3 + n * N3 + pt];
          }
        }
        R s3[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) s3[n] = Sl[(n * (N + 1) + f) * N2 + ln];
        const Pt<R> st = point_state<PERT>(qf, rho0f, E0f, ph);
        const R p0f = ph.gm1 * E0f;
        R Ft[5];
        if (f > 0 && f < N) {
          R Fi[5], Fv[5];
          flux_inv(qf, st, s3, Fi);
          flux_visc<PERT>(st, gf, gr0f, rho0f, p0f, s3, ph, Fv);
#pragma unroll
          for (int v = 0; v < 5; ++v) Ft[v] = Fi[v] - Fv[v];
        } else {
          const int side = (f == N);
          const int F = 2 * d + side;
          const R sgn = side ? R(1) : R(-1);
          const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
          const R nh[3] = {sgn * s3[0] / mag, sgn * s3[1] / mag, sgn * s3[2] / mag};
          const int nb = A.m.nbr[e * 6 + F];
          R Fh[5];
          if (nb >= 0) {
            R qR[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) qR[v] = sT[(el * 6 + F) * 5 * N2 + v * N2 + ln];
            R rho0R = R(0), E0R = R(0);
            if (PERT) {
              rho0R = sTbg[(el * 6 + F) * 2 * N2 + ln];
              E0R = sTbg[(el * 6 + F) * 2 * N2 + N2 + ln];
            }
            const Pt<R> sR = point_state<PERT>(qR, rho0R, E0R, ph);
            rusanov<PERT>(qf, st, rho0f, E0f, qR, sR, rho0R, E0R, nh, ph, Fh);
            R Fv[5];
            flux_visc<PERT>(st, gf, gr0f, rho0f, p0f, nh, ph, Fv);
#pragma unroll
            for (int v = 1; v < 5; ++v)  // neighbour stored F_v . n_out(neighbour) = -F_v . n
              Fh[v] -= R(0.5) * (Fv[v] - sTv[(el * 6 + F) * 4 * N2 + (v - 1) * N2 + ln]);
          } else {
            // walls (Section 5): exact inviscid flux (0, p n, 0); normal traction only;
            // energy: f.n from the lifted gradient with T = T_top (outer) or the prescribed flux (inner)
            const R mu = st.rho * ph.nu;
            const R div = gf[3] + gf[7] + gf[11];
            R trac = R(0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b) {
                R t = mu * (gf[3 + 3 * a + b] + gf[3 + 3 * b + a]);
                if (a == b) t -= mu * R(2.0 / 3.0) * div;
                trac += nh[a] * t * nh[b];
              }
            Fh[0] = R(0);
#pragma unroll
            for (int a = 0; a < 3; ++a) Fh[1 + a] = (st.p - trac) * nh[a];
            if (nb == -2) {
              const R RT = ph.Rgas * ph.T_top;
              R fn = R(0);
#pragma unroll
              for (int b = 0; b < 3; ++b)
                fn += -ph.CpR * (ph.kappa * (gf[12 + b] / ph.gamma - RT * gf[b]) + ph.kappa_r * (gf[12 + b] - RT * gf[b])) *
                      nh[b];
              Fh[4] = fn;
            } else {
              Fh[4] = PERT ? R(0) : -ph.bottom_flux;
            }
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) Ft[v] = sgn * mag * Fh[v];
        }
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
          for (int i = 0; i < N; ++i) acc[v][i] += A.ops.D[i][f] * Ft[v];
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int pt = pt_of<N>(d, ln, i);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (d == 0) sdiv[el * 5 * N3 + v * N3 + pt] = acc[v][i];
          else sdiv[el * 5 * N3 + v * N3 + pt] += acc[v][i];
        }
      }
    }
    __syncthreads();
  }

  // ---- residual dQ/dt = -div/|J| - M (Eqs. 4, 11), sources of Eqs. 2-3, and the RK combination
  if (active) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pt = N * ln + i;
      const size_t gi = (size_t)e * N3 + pt;
      R q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = sq[el * 5 * N3 + v * N3 + pt];
      const R x0 = A.m.x[((size_t)e * 3 + 0) * N3 + pt];
      const R x1 = A.m.x[((size_t)e * 3 + 1) * N3 + pt];
      const R x2 = A.m.x[((size_t)e * 3 + 2) * N3 + pt];
      const R r2 = x0 * x0 + x1 * x1 + x2 * x2;
      const R gr = ph.GM / (r2 * sqrt(r2));  // g = gr * x points outward (the source uses -rho g_vec)
      const R g3[3] = {gr * x0, gr * x1, gr * x2};
      R M[5];
      M[0] = R(0);
      M[1] = q[0] * g3[0] - ph.twoOmega * q[2];
      M[2] = q[0] * g3[1] + ph.twoOmega * q[1];
      M[3] = q[0] * g3[2];
      M[4] = q[1] * g3[0] + q[2] * g3[1] + q[3] * g3[2];
      const R ij = A.m.invJ[gi];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        R Rv = -sdiv[el * 5 * N3 + v * N3 + pt] * ij - M[v];
        if (PERT) Rv += (R)A.bg.R0[((size_t)e * 5 + v) * N3 + pt];
        const size_t oi = ((size_t)e * 5 + v) * N3 + pt;
        if (MODE == kModeResidual) {
          A.out[oi] = Rv;
        } else {
          const R nv = A.a * A.un[oi] + A.b * (q[v] + A.dt * Rv);
          A.out[oi] = nv;
          sq[el * 5 * N3 + v * N3 + pt] = nv;
        }
      }
    }
  }
  if (MODE == kModeRK) {
    __syncthreads();
    if (active && A.T_out) {
#pragma unroll 1
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          R lo = R(0), hi = R(0);
#pragma unroll
          for (int s = 0; s < N; ++s) {
            const R val = sq[el * 5 * N3 + v * N3 + pt_of<N>(d, ln, s)];
            lo += A.ops.I[0][s] * val;
            hi += A.ops.I[N][s] * val;
          }
          A.T_out[((size_t)e * 6 + 2 * d) * 5 * N2 + v * N2 + ln] = lo;
          A.T_out[((size_t)e * 6 + 2 * d + 1) * 5 * N2 + v * N2 + ln] = hi;
        }
    }
  }
}

// ------------------------------------------------------------------ launch helpers

template <int N, bool PERT, class R, int EPB>
struct Launch {
  using L = Layout<N, PERT, R, EPB>;
  static constexpr int threads = EPB * N * N;
  static int blocks(int E) { return (E + EPB - 1) / EPB; }

  static cudaError_t trace(const MeshArg<R>& m, const OpsArg<R>& ops, const R* q, R* T, cudaStream_t st) {
    if (m.E == 0) return cudaSuccess;
    k_trace<N, R, EPB><<<blocks(m.E), threads, 0, st>>>(m, ops, q, T);
    return cudaGetLastError();
  }
  static cudaError_t grad(const KArgs<R>& A, cudaStream_t st) {
    if (A.m.E == 0) return cudaSuccess;
    const size_t sm = (size_t)L::total_grad * sizeof(R);
    cudaError_t e = cudaFuncSetAttribute(k_grad<N, PERT, R, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_grad<N, PERT, R, EPB><<<blocks(A.m.E), threads, sm, st>>>(A);
    return cudaGetLastError();
  }
  template <int MODE>
  static cudaError_t resid(const KArgs<R>& A, cudaStream_t st) {
    if (A.m.E == 0) return cudaSuccess;
    const size_t sm = (size_t)L::total_resid * sizeof(R);
    cudaError_t e =
        cudaFuncSetAttribute(k_resid<N, PERT, R, EPB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_resid<N, PERT, R, EPB, MODE><<<blocks(A.m.E), threads, sm, st>>>(A);
    return cudaGetLastError();
  }
};

}  // namespace chorus
