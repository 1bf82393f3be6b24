// Device helpers of the spectral-difference kernels: bulk-copy / mbarrier primitives, index
// helpers and the point physics (paper Section 2 Eqs. 5-9, Section 3 Rusanov flux).
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

// 1D bulk copy shared -> global (bulk-group completion).  The shared data must have been written
// before a fence.proxy.async by the writing threads and a barrier.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have read their shared-memory source (before the CTA exits).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until the committed bulk stores have completed their writes to global memory.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Polls of a bounded mbarrier wait when the mesh sets no limit of its own (about a second with the
// back-off below).
constexpr uint32_t kDefaultWaitPolls = 1u << 24;

// Bounded wait for the completion of the barrier's phase of the given parity (0 for a barrier's first
// use): at most `polls` polls.  Returns false if they ran out.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity, uint32_t polls) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.b32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ bool mbar_try0(uint64_t* bar, uint32_t polls) { return mbar_try(bar, 0u, polls); }

// The device control block of a mesh: err[0] error flags, err[1] the wait limit (0: the default,
// k + 1: k polls).  Returns the number of polls of a kernel's staging waits.
__device__ __forceinline__ uint32_t wait_polls(const unsigned* err) {
  if (err == nullptr) return kDefaultWaitPolls;
  const uint32_t lim = *(const volatile unsigned*)(err + 1);
  return lim == 0u ? kDefaultWaitPolls : lim - 1u;
}

// Bounded wait for the bulk copies of a staging barrier.  If `polls` run out, sets bit 0 of *err
// and waits once more (default limit) for the copies still in flight, so that no copy writes into
// the shared memory of a CTA that has given up; returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err, uint32_t polls) {
  if (mbar_try(bar, parity, polls)) return true;
  if (err) atomicOr(err, 1u);
  mbar_try(bar, parity, kDefaultWaitPolls);
  return false;
}
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar, unsigned* err, uint32_t polls) {
  return mbar_wait(bar, 0u, err, polls);
}

// ------------------------------------------------------------------ division

// Quotients of the point physics.  FP64: the correctly rounded quotient.  FP32 (the perturbation
// form, whose tolerance is relative 1e-5): with kFastDivF32 the approximate quotient __fdividef
// (reciprocal and product, error of a few ulp for divisors of normal magnitude) instead of the
// correctly rounded division sequence.
constexpr bool kFastDivF32 = true;

template <class R>
__device__ __forceinline__ R qdiv(R a, R b) {
  if constexpr (sizeof(R) == 4 && kFastDivF32) return __fdividef(a, b);
  else return a / b;
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
  const R ir = qdiv(R(1), s.rho);
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

// Gradient record of a point, 12 entries: g[0..2] the form's grad rho, g[3..8] the trace-free
// strain sigma = grad u + grad u^T - 2/3 (div u) I as (xx, yy, zz, xy, yz, zx), g[9..11] the form's
// grad p.  tau = mu sigma (Eq. 9).

template <class R>
__device__ __forceinline__ R sig(const R g[kG], int a, int b) {
  if (a == b) return g[3 + a];
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? g[6] : g[8]) : g[7];
}

// s . (F, G, H)_v (Eqs. 7-9; energy entry u.tau - f as in Eq. 3).
// gr0: background density gradient (perturbation form only).
template <bool PERT, class R>
__device__ __forceinline__ void flux_visc(const Pt<R>& st, const R g[kG], const R gr0[3], R rho0, R p0,
                                          const R s[3], const PhysArg<R>& ph, R kr, R Fv[5]) {
  const R mu = st.rho * ph.nu;
  R ts[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) ts[a] = mu * (sig(g, a, 0) * s[0] + sig(g, a, 1) * s[1] + sig(g, a, 2) * s[2]);
  const R pr = qdiv(st.ptot, st.rho);
  R dpr = R(0);
  if (PERT) dpr = qdiv(st.p * rho0 - p0 * st.rhop, st.rho * rho0);  // p/rho - p0/rho0
  R fs = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    R A = pr * g[b];
    if (PERT) A += dpr * gr0[b];
    const R fb = -ph.CpR * (ph.kappa * (qdiv(g[9 + b], ph.gamma) - A) + kr * (g[9 + b] - A));
    fs += fb * s[b];
  }
  Fv[0] = R(0);
  Fv[1] = ts[0];
  Fv[2] = ts[1];
  Fv[3] = ts[2];
  Fv[4] = st.u[0] * ts[0] + st.u[1] * ts[1] + st.u[2] * ts[2] - fs;
}

// primitive gradient record from conserved gradients gq[3 v + n] = d q_v / d x_n:
//   grad u_a = (grad m_a - u_a grad rho) / rho,  grad p = (gamma-1)(grad E - u.grad m + |u|^2/2 grad rho)
template <bool PERT, class R>
__device__ __forceinline__ void grad_prim(const Pt<R>& st, const R gq[15], const R gr0[3], const PhysArg<R>& ph,
                                          R g[kG]) {
  R grt[3];
#pragma unroll
  for (int n = 0; n < 3; ++n) {
    grt[n] = PERT ? gr0[n] + gq[n] : gq[n];
    g[n] = gq[n];
  }
  const R ir = qdiv(R(1), st.rho);
  R gu[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int n = 0; n < 3; ++n) gu[a][n] = (gq[3 * (1 + a) + n] - st.u[a] * grt[n]) * ir;
  const R div = gu[0][0] + gu[1][1] + gu[2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) g[3 + a] = R(2) * gu[a][a] - R(2.0 / 3.0) * div;
  g[6] = gu[0][1] + gu[1][0];
  g[7] = gu[1][2] + gu[2][1];
  g[8] = gu[0][2] + gu[2][0];
  const R ke = R(0.5) * (st.u[0] * st.u[0] + st.u[1] * st.u[1] + st.u[2] * st.u[2]);
#pragma unroll
  for (int n = 0; n < 3; ++n)
    g[9 + n] = ph.gm1 * (gq[12 + n] - (st.u[0] * gq[3 + n] + st.u[1] * gq[6 + n] + st.u[2] * gq[9 + n]) +
                         ke * grt[n]);
}

template <bool PERT, class R>
__device__ __forceinline__ void rusanov(const R qL[5], const Pt<R>& sL, R rho0L, R E0L, const R qR[5],
                                        const Pt<R>& sR, R rho0R, R E0R, const R n[3], const PhysArg<R>& ph,
                                        R F[5]) {
  R FL[5], FR[5];
  flux_inv(qL, sL, n, FL);
  flux_inv(qR, sR, n, FR);
  const R cL = sqrt(qdiv(ph.gamma * sL.ptot, sL.rho));
  const R cR = sqrt(qdiv(ph.gamma * sR.ptot, sR.rho));
  const R vL = fabs(sL.u[0] * n[0] + sL.u[1] * n[1] + sL.u[2] * n[2]) + cL;
  const R vR = fabs(sR.u[0] * n[0] + sR.u[1] * n[1] + sR.u[2] * n[2]) + cR;
  const R lam = vL > vR ? vL : vR;
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * lam * (qR[v] - qL[v]);
  if (PERT) {
    const R c0L = sqrt(qdiv(ph.gamma * ph.gm1 * E0L, rho0L));
    const R c0R = sqrt(qdiv(ph.gamma * ph.gm1 * E0R, rho0R));
    const R lam0 = c0L > c0R ? c0L : c0R;
    F[0] -= R(0.5) * (lam - lam0) * (rho0R - rho0L);
    F[4] -= R(0.5) * (lam - lam0) * (E0R - E0L);
  }
}
}  // namespace chorus
