// Spectral-difference residual kernels for one order N = p + 1 (paper Sections 3 and 5).
//
// One CTA processes EPB elements; each element is handled by N*N threads, thread `ln` owning the
// line (a, b) = (ln % N, ln / N) of every direction (xi-line (j,k), eta-line (i,k), zeta-line
// (i,j)).  A thread does the whole 1D work of its line in registers: interpolation to the N+1
// flux points (Eq. 17), fluxes, the common fluxes at the two end points, and the derivative back
// to the N solution points (Eq. 18).  Shared memory links the three directional sweeps.
//
// Shared memory per element: the staged state (bulk TMA copy per element block, linear layout),
// the background tables (perturbation form), the lifted gradients and the divergence accumulator.
// Element blocks are padded so that the two elements of a warp at p = 3 use opposite halves of the
// banks, and for N = 4 in FP32 the computed arrays are XOR-swizzled so that xi-, eta- and
// zeta-line accesses are conflict free.  Neighbour face data are gathered from global memory
// straight into registers when a sweep needs them.
#pragma once
#include <type_traits>

#include "sd_device.cuh"

namespace chorus {

// ------------------------------------------------------------------ layout helpers

// Count of R words padded to a multiple of 16 bytes whose byte size is 64 mod 128.
template <class R>
constexpr int pad_stride(int count) {
  int bytes = (count * (int)sizeof(R) + 15) / 16 * 16;
  const int r = bytes % 128;
  bytes += (64 - r + 128) % 128;
  return bytes / (int)sizeof(R);
}

// Shared-memory index of solution point (i,j,k) within one component array of the computed arrays.
template <int N, class R>
__device__ __forceinline__ int sidx(int i, int j, int k) {
  if (N == 4 && sizeof(R) == 4) return i + 4 * ((j ^ k) & 3) + 16 * k;
  return i + N * j + N * N * k;
}

// (i,j,k) of position s on line ln of direction D
template <int N, int D>
__device__ __forceinline__ void line_ijk(int ln, int s, int& i, int& j, int& k) {
  const int a = ln % N, b = ln / N;
  if (D == 0) {
    i = s; j = a; k = b;
  } else if (D == 1) {
    i = a; j = s; k = b;
  } else {
    i = a; j = b; k = s;
  }
}

template <int N, int D>
__device__ __forceinline__ int line_pt(int ln, int s) {
  int i, j, k;
  line_ijk<N, D>(ln, s, i, j, k);
  return i + N * j + N * N * k;
}

template <int N, int D, class R>
__device__ __forceinline__ int line_sidx(int ln, int s) {
  int i, j, k;
  line_ijk<N, D>(ln, s, i, j, k);
  return sidx<N, R>(i, j, k);
}

// Residual-kernel option (FP32 perturbation form): whether the background line data are staged in
// shared memory (else read through L1 per flux point).
constexpr bool kResidBgShared = true;
// Whether the xi-line sweeps at N = 4 (FP32) read a line of the gradient record as one 16-byte
// shared-memory load per component (the swizzled layout keeps a xi-line's 4 points contiguous).
constexpr bool kVecGradLoad = true;

// Resident CTAs asked of the compiler (the register cap), from timings on the shells of every order:
// the kernels ask for a number of warps per SM whatever their CTA size, 12 for the residual kernel
// (~168 registers a thread) and 16 for the lifting kernel at N = 3, 4 (128), 12 at N = 5, 6.  Smaller
// CTAs at the same warp count measured faster where their lanes stay full: the residual kernel at
// p = 3 in four-element CTAs, six per SM (8 % faster than eight-element CTAs, three per SM), at p = 2
// in seven-element ones (4.6 % faster than fourteen), at p = 5 in two-element ones, four per SM (5 %
// faster than four-element CTAs, two per SM; the lifting kernel 3 %); at p = 4 the 25-thread
// elements fill four warps only five to a CTA (two-element CTAs ran 14 % slower).  Shared memory
// allows these counts at every order.  Also per order: whether the flux sweep holds the line's
// gradient record in registers (else it reads it from shared memory per flux point).
template <int N, int EPB>
__host__ __device__ constexpr int warps_per_cta() { return (EPB * N * N + 31) / 32; }
template <int N, int EPB>
__host__ __device__ constexpr int resid_min_blocks() { return 12 / warps_per_cta<N, EPB>(); }
template <int N, int EPB>
__host__ __device__ constexpr int grad_min_blocks() { return (N <= 4 ? 16 : 12) / warps_per_cta<N, EPB>(); }
template <int N>
__host__ __device__ constexpr bool reg_grad_lines() { return N <= 4; }

// Whether direction 0 of the N = 4 residual sweep visits its end points first, their neighbour data
// loaded with the staging (3 % slower: off); and how many flux points ahead the sweep loads the
// metrics at N = 4 and N = 5 (1 or 2: two is 1.4 % faster at N = 4, 0.6 % slower at N = 5; the
// other orders, 1: two spill there).
constexpr bool kEndFirstD0 = false;
constexpr int kS3AheadN4 = 2;
constexpr int kS3AheadN5 = 1;
template <int N>
__host__ __device__ constexpr int s3_ahead() { return N == 4 ? kS3AheadN4 : N == 5 ? kS3AheadN5 : 1; }

// Whether the residual kernel stages each direction's metric block S^D_n (3 x (N+1) x N^2 words per
// element, contiguous in global memory) in shared memory by bulk copies, double-buffered across the
// three sweeps (direction 0 with the element blocks, 1 during sweep 0, 2 during sweep 1), instead of
// loading the metrics of each flux point from global memory ahead of use.
constexpr bool kStageMetricsN4 = true;
template <int N, class R>
__host__ __device__ constexpr bool stage_metrics() { return sizeof(R) == 4 && N == 4 && kStageMetricsN4; }

// Face-kernel mode: the common flux of every interior face point is computed once by k_face (Rusanov
// + averaged viscous, from both sides' traces) and of every wall face point by the lifting kernel
// (which holds the face gradients), both written as F~ in each element's own face numbering; the
// residual kernel's sweeps then evaluate fluxes at the interior flux points only and take the two
// end points' F~ from that array (one coalesced read per face) instead of gathering neighbour data.
constexpr bool kFaceKernel = true;

// The lifting kernel's viscous face pass reads each line component from shared memory once and keeps
// only its values at the two end points (2 x 22 live values) instead of holding the whole line data
// (22 x N values) through both end points, and evaluates the two end points with the side loop
// unrolled.  Timed per order: the lifting kernel 8 % faster at N = 4, 12 % at N = 6 (its spills
// gone), 2 % at N = 5; at N = 3 2.5 % slower.
template <int N>
__host__ __device__ constexpr bool face_ends() { return N >= 4; }

// Whether the lifting kernel stages each element's six (neighbour, face code) pairs in shared memory
// with its element blocks, so that the later directions' neighbour loads need no index load first.
constexpr bool kGradNbShared = true;

// Lifting order: false = directions 0, 1, 2 and a separate pass that forms the gradient record;
// true = directions 1, 2, 0 with the record formed in the last sweep.
constexpr bool kLiftFused = true;

// Lifting with raw partial derivatives (with the fused order only): the first two sweeps store, per
// point, their five derivatives d q_v / d xi_D and the three components of grad xi_D (8 words, no
// read-modify-write), and the last sweep forms the conserved gradients from them and its own:
// 44 shared-memory accesses per point instead of 72 for the 15 accumulated components.
constexpr bool kLiftRaw = true;
template <int N, class R>
__host__ __device__ constexpr bool lift_raw() { return kLiftRaw && kLiftFused && sizeof(R) == 4 && N == 4; }
// Direction order of the raw-derivative lifting: xi, eta, zeta (the xi sweep stores its raw slot as
// 16-byte vectors, conflict-free in the swizzled layout, and the record is formed in the zeta sweep,
// whose scalar accesses are conflict-free in both the swizzled and the linear layout); otherwise
// eta, zeta, xi as in the accumulated lifting.
constexpr bool kLiftXiFirst = true;
template <int N, class R>
__host__ __device__ constexpr int lift_dir_at(int k) {
  return (lift_raw<N, R>() && kLiftXiFirst) ? k : (k == 0 ? 1 : k == 1 ? 2 : 0);
}

// Whether the lifting kernel writes the gradient record with bulk stores from shared memory (timed
// per order: 1-4 % faster at N = 3, 4, 6, 3 % slower at N = 5).
template <int N>
__host__ __device__ constexpr bool grad_bulk_store() { return N != 5; }

// RES: the residual kernel's layout (it reads the 12-entry gradient record instead of lifting, so the
// gradient array holds kG components; the lifting kernel needs 15).
template <int N, bool PERT, class R, int EPB, bool RES = false>
struct Layout {
  static constexpr int N2 = N * N, N3 = N * N * N;
  static constexpr bool bgShared = PERT && (!RES || kResidBgShared);
  static constexpr int SQ = pad_stride<R>(5 * N3);
  static constexpr int SBG = bgShared ? pad_stride<R>(2 * N3) : 0;
  static constexpr int SGR0 = bgShared ? pad_stride<R>(3 * N3) : 0;
  static constexpr int SG = pad_stride<R>((RES ? kG : (lift_raw<N, R>() ? 16 : 15)) * N3);
  static constexpr int SDIV = pad_stride<R>(5 * N3);
  // staged metric blocks of one direction (residual kernel, when stage_metrics)
  static constexpr bool SM = RES && stage_metrics<N, R>();
  // staged flux points per line and the first of them: all N + 1 (one 960-byte copy per element and
  // direction at N = 4); staging only the interior points 1..N-1 that the face-kernel mode visits
  // took three copies per element and direction and made the residual kernel 8 % slower
  static constexpr int SFP = N + 1;
  static constexpr int SF0 = 0;
  static constexpr int SSF = SM ? 3 * SFP * N2 : 0;
  // interpolation I[f][s] and derivative D[i][f] tables, indexed at run time by rolled loops
  static constexpr int TAB = pad_stride<R>(2 * (N + 1) * N);
  static constexpr int oTAB = 0;
  static constexpr int oQ = oTAB + TAB;
  static constexpr int oBG = oQ + EPB * SQ;
  static constexpr int oGR0 = oBG + EPB * SBG;
  static constexpr int oG = oGR0 + EPB * SGR0;
  static constexpr int oDIV = oG + EPB * SG;
  static constexpr int total_grad = oDIV;
  static constexpr int oSF0 = oDIV + EPB * SDIV;
  static constexpr int oSF1 = oSF0 + EPB * SSF;
  static constexpr int total_resid = oSF1 + EPB * SSF;
  // per-element bulk copies need 16-byte element blocks in global memory
  static constexpr bool tmaQ = (5 * N3 * sizeof(R)) % 16 == 0;
  static constexpr bool tmaBG = (2 * N3 * sizeof(R)) % 16 == 0 && (3 * N3 * sizeof(R)) % 16 == 0;
};

// Copy the operator tables into shared memory (static indices only; thread 0).
template <int N, class R>
__device__ __forceinline__ void fill_tables(const OpsArg<R>& ops, R* tab) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f <= N; ++f)
#pragma unroll
      for (int s = 0; s < N; ++s) tab[f * N + s] = ops.I[f][s];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int f = 0; f <= N; ++f) tab[(N + 1) * N + i * (N + 1) + f] = ops.D[i][f];
  }
}

// Load the N values of one component along line ln of direction D from a linear element array.
template <int N, int D, class R>
__device__ __forceinline__ void load_line_lin(const R* __restrict__ base, int ln, R out[N]) {
  if (D == 0 && N == 4 && sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(base + 4 * ln);
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) out[s] = base[line_pt<N, D>(ln, s)];
  }
}

// Load the N values of one background table component (rho0, E0 or a component of the lifted
// grad rho0) along line ln of direction D, in the tables' point order (bg_point).
template <int N, int D, class R>
__device__ __forceinline__ void load_line_bg(const R* __restrict__ base, int ln, R out[N]) {
  if constexpr (bg_swizzle(N) && sizeof(R) == 4) {
    if constexpr (D == 0) {
      const float4 v = *reinterpret_cast<const float4*>(base + line_sidx<N, 0, R>(ln, 0));
      out[0] = v.x;
      out[1] = v.y;
      out[2] = v.z;
      out[3] = v.w;
    } else {
#pragma unroll
      for (int s = 0; s < N; ++s) out[s] = base[line_sidx<N, D, R>(ln, s)];
    }
  } else {
    load_line_lin<N, D>(base, ln, out);
  }
}

// Index of position s along line ln of direction D in the background tables' point order.
template <int N, int D, class R>
__device__ __forceinline__ int line_bg(int ln, int s) {
  if constexpr (bg_swizzle(N) && sizeof(R) == 4) return line_sidx<N, D, R>(ln, s);
  else return line_pt<N, D>(ln, s);
}

// Load the kG components of the gradient record along line ln of direction D from the shared array.
template <int N, int D, class R>
__device__ __forceinline__ void load_grad_lines(const R* sg, int ln, R (&gv)[kG][N]) {
  constexpr int N3 = N * N * N;
  if constexpr (D == 0 && N == 4 && sizeof(R) == 4 && kVecGradLoad) {
    const int s0 = line_sidx<N, 0, R>(ln, 0);
#pragma unroll
    for (int c = 0; c < kG; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(sg + c * N3 + s0);
      gv[c][0] = v.x;
      gv[c][1] = v.y;
      gv[c][2] = v.z;
      gv[c][3] = v.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const int si = line_sidx<N, D, R>(ln, s);
#pragma unroll
      for (int c = 0; c < kG; ++c) gv[c][s] = sg[c * N3 + si];
    }
  }
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
  R* G_out;            // optional grad kernel output: the gradient record [E][kG][N3] (shared layout)
  const R* G_in;       // resid kernel input: that record
  R* out;              // residual or new state
  R* T_out;            // traces of the new state (RK mode)
  const R* un;         // first extra state of the RK combination
  R a, b, c, dt;       // out = a un + b q + c dt R
  const R* un2;        // optional second output: out2 = a2 un2 + b2 q + c2 dt R
  R* out2;
  R a2, b2, c2;
  const R* radd;       // optional additive residual correction [E][5][N3]
  R* Fc_out;           // grad kernel output (face-kernel mode): wall common fluxes F~ [E][6][5][N2]
  const R* Fc;         // resid kernel input (face-kernel mode): common fluxes F~ of every face point
  unsigned* err;
};

// neighbour data of one face point
template <class R>
struct NbFace {
  int kind;  // >= 0 interior, -1 inner wall, -2 outer wall
  R q[5];
  R tv[4];
  R r0, E0;
};

// Where the neighbour's face block of face F of element e sits: bf = neighbour * 6 + its face (or the
// wall code -1 / -2), tp = the neighbour's face-point index of own face point ln.
struct NbIdx {
  int bf, tp;
};

// Where the neighbour data of own face point ln sit, from the face's (neighbour, face code) pair.
template <int N>
__device__ __forceinline__ NbIdx nb_index_of(int k, int c, int ln) {
  NbIdx x;
  x.bf = k >= 0 ? k * 6 + (c >> 3) : k;
  x.tp = k >= 0 ? map_face_pt<N>(ln, c & 7) : 0;
  return x;
}

template <int N, class R>
__device__ __forceinline__ NbIdx nb_index(const KArgs<R>& A, int e, int F, int ln) {
  // both words issued together (a wall's code entry is read and ignored)
  const int k = __ldg(A.m.nbr + e * 6 + F);
  const int c = __ldg(A.m.code + e * 6 + F);
  return nb_index_of<N>(k, c, ln);
}

template <int N, bool PERT, bool WANT_TV, class R>
__device__ __forceinline__ NbFace<R> load_nb_at(const KArgs<R>& A, NbIdx x) {
  constexpr int N2 = N * N;
  NbFace<R> f;
  f.kind = x.bf;
  if (x.bf >= 0) {
    const size_t base = (size_t)x.bf;
    const int tp = x.tp;
#pragma unroll
    for (int v = 0; v < 5; ++v) f.q[v] = __ldg(A.T + (base * 5 + v) * N2 + tp);
    if (WANT_TV) {
#pragma unroll
      for (int v = 0; v < 4; ++v) f.tv[v] = __ldg(A.Tv + (base * 4 + v) * N2 + tp);
      if (PERT) {
        f.r0 = (R)__ldg(A.bg.bgT + (base * 2) * N2 + tp);
        f.E0 = (R)__ldg(A.bg.bgT + (base * 2 + 1) * N2 + tp);
      }
    }
  }
  return f;
}

template <int N, bool PERT, bool WANT_TV, class R>
__device__ __forceinline__ NbFace<R> load_nb(const KArgs<R>& A, int e, int F, int ln) {
  return load_nb_at<N, PERT, WANT_TV>(A, nb_index<N>(A, e, F, ln));
}

// Global-memory inputs of one direction sweep, loaded ahead of their use so that their latency
// overlaps the preceding work (the sweeps otherwise stall on them once per flux point).
template <int N, class R>
struct LiftPre {
  R S[3][N + 1];  // S^D_n at the N+1 flux points of the line
  R ij[N];        // 1/|J| at the line's solution points
  NbFace<R> nb[2];
};

// Members only some orders use (unused members of the struct cost registers at the others).
template <class R, bool X>
struct FluxPreExtra {
  R s3b[3];         // S^D_n at the second flux point the sweep visits (metrics two points ahead)
  NbFace<R> nb[2];  // the end points' neighbour data (sweeps that visit the end points first)
};
template <class R>
struct FluxPreExtra<R, false> {};

template <class R, bool X>
struct FluxPre : FluxPreExtra<R, X> {
  R s3[3];       // S^D_n at the first flux point the sweep visits
  NbIdx nbi[2];  // where the neighbour data of the two end points sit (modes 1, 2)
};

// snb: the element's six (neighbour, face code) pairs in shared memory, or null (read them from the
// mesh tables).
template <int N, bool PERT, class R, int D>
__device__ __forceinline__ void lift_prefetch(const KArgs<R>& A, int e, int ln, LiftPre<N, R>& p,
                                              const int* snb = nullptr) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const R* Sl = A.m.Sf + ((size_t)e * 3 + D) * 3 * (N + 1) * N2;
#pragma unroll
  for (int n = 0; n < 3; ++n)
#pragma unroll
    for (int f = 0; f <= N; ++f) p.S[n][f] = __ldg(Sl + (n * (N + 1) + f) * N2 + ln);
#pragma unroll
  for (int i = 0; i < N; ++i) p.ij[i] = __ldg(A.m.invJ + (size_t)e * N3 + line_pt<N, D>(ln, i));
  if (snb != nullptr) {
    p.nb[0] = load_nb_at<N, PERT, false>(A, nb_index_of<N>(snb[4 * D], snb[4 * D + 1], ln));
    p.nb[1] = load_nb_at<N, PERT, false>(A, nb_index_of<N>(snb[4 * D + 2], snb[4 * D + 3], ln));
  } else {
    p.nb[0] = load_nb<N, PERT, false>(A, e, 2 * D, ln);
    p.nb[1] = load_nb<N, PERT, false>(A, e, 2 * D + 1, ln);
  }
}

// How the flux sweep gets the neighbour data of its two end points: 0 = index and data loaded at
// the end point; 1 = index (neighbour, face, orientation) loaded with the sweep's first metrics, data
// at the end point; 2 = as 1, and the data of each end point issued one flux point ahead; 3 = the
// element's six (neighbour, face code) pairs staged in shared memory with the state, data loaded at
// the end point.  Timed per order: 3 is fastest at N = 3, 4, 6 (2 spills at N = 4 and is 2 % slower
// at N = 3, 6); 2 is 0.9 % faster at N = 5.
template <int N>
__host__ __device__ constexpr int flux_nb_mode() { return (N == 4 || N == 3 || N == 6) ? 3 : 2; }

// Sweeps whose end points come first: direction 0 at N = 4 (mode 3), whose neighbour data are loaded
// while the kernel waits for its staged element blocks.
template <int N, int D>
__host__ __device__ constexpr bool end_first() {
  return kEndFirstD0 && D == 0 && flux_nb_mode<N>() == 3;
}

// The flux point a sweep visits at step it: 1, ..., N, 0, or (end points first) N, 0, 1, ..., N - 1.
template <int N, bool EF>
__device__ __forceinline__ int flux_order(int it) {
  if (EF) return it == 0 ? N : it - 1;
  return it < N ? it + 1 : 0;
}

template <int N, bool PERT, class R, int D, bool X>
__device__ __forceinline__ void flux_prefetch(const KArgs<R>& A, int e, int ln, FluxPre<R, X>& p) {
  constexpr int N2 = N * N;
  constexpr bool EF = end_first<N, D>();
  const R* Sl = A.m.Sf + ((size_t)e * 3 + D) * 3 * (N + 1) * N2;
  if constexpr (!stage_metrics<N, R>()) {
#pragma unroll
    for (int n = 0; n < 3; ++n) p.s3[n] = __ldg(Sl + (n * (N + 1) + flux_order<N, EF>(0)) * N2 + ln);
  }
  if constexpr (!stage_metrics<N, R>() && s3_ahead<N>() == 2) {
#pragma unroll
    for (int n = 0; n < 3; ++n) p.s3b[n] = __ldg(Sl + (n * (N + 1) + flux_order<N, EF>(1)) * N2 + ln);
  }
  if (!kFaceKernel && (flux_nb_mode<N>() == 1 || flux_nb_mode<N>() == 2)) {
    p.nbi[0] = nb_index<N>(A, e, 2 * D, ln);
    p.nbi[1] = nb_index<N>(A, e, 2 * D + 1, ln);
  }
  if constexpr (EF) {
    p.nb[0] = load_nb<N, PERT, true>(A, e, 2 * D, ln);
    p.nb[1] = load_nb<N, PERT, true>(A, e, 2 * D + 1, ln);
  }
}

// Radiative diffusivity at flux point f of line ln (direction D): from the mesh's flux-point table
// (the interpolant of its solution-point values) when a profile is active, else the constant.  KR
// false compiles the lookup out (the FP32 kernels are built both ways).
template <int N, int D, bool KR, class R>
__device__ __forceinline__ R kr_at(const KArgs<R>& A, int e, int ln, int f) {
  if constexpr (!KR) return A.ph.kappa_r;
  if (A.m.kr == nullptr) return A.ph.kappa_r;
  return __ldg(A.m.kr + (((size_t)e * 3 + D) * (N + 1) + f) * (N * N) + ln);
}

// ------------------------------------------------------------------ trace kernel

// Traces of tile `tile` (elements tile * EPB ...), one thread per (element, line); threads beyond
// EPB * N^2 idle.
template <int N, class R, int EPB>
__device__ __forceinline__ void trace_tile(const MeshArg<R>& m, const OpsArg<R>& ops, const R* __restrict__ q,
                                           R* __restrict__ T, int64_t tile) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int64_t e = tile * EPB + el;
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
        const int pt = d == 0 ? line_pt<N, 0>(ln, s) : (d == 1 ? line_pt<N, 1>(ln, s) : line_pt<N, 2>(ln, s));
        const R val = qe[v * N3 + pt];
        lo += ops.I[0][s] * val;
        hi += ops.I[N][s] * val;
      }
      Te[((2 * d) * 5 + v) * N2 + ln] = lo;
      Te[((2 * d + 1) * 5 + v) * N2 + ln] = hi;
    }
}

template <int N, class R, int EPB>
__global__ void __launch_bounds__(EPB * N * N) k_trace(const MeshArg<R> m, const OpsArg<R> ops, const R* __restrict__ q,
                                                      R* __restrict__ T) {
  trace_tile<N, R, EPB>(m, ops, q, T, blockIdx.x);
}

// ------------------------------------------------------------------ staging

// Bulk copy of element e's direction-d metrics S^d_n at the staged flux points (L::SF0 ..
// L::SF0 + L::SFP - 1) into `dst` as [n][staged point][line]: one copy when all points are staged,
// else one per component n.
template <int N, class R, class L>
__device__ __forceinline__ void stage_metric_block(const R* Sf, int64_t e, int d, R* dst, uint64_t* bar) {
  constexpr int N2 = N * N;
  const R* src = Sf + ((size_t)e * 3 + d) * 3 * (N + 1) * N2;
  if constexpr (L::SFP == N + 1) {
    bulk_g2s(dst, src, 3 * (N + 1) * N2 * sizeof(R), bar);
  } else {
#pragma unroll
    for (int n = 0; n < 3; ++n)
      bulk_g2s(dst + n * L::SFP * N2, src + (n * (N + 1) + L::SF0) * N2, L::SFP * N2 * sizeof(R), bar);
  }
}

// Stages the elements e0 .. e0 + ne - 1.  `between` runs after the copies are issued and before the
// wait (it issues the first sweep's global loads so that both latencies overlap).  The copies
// complete the phase of `bar` whose parity is `parity` (flipped here whenever the barrier was used).
// Returns false, the same in every thread of the CTA, when the bounded wait for the copies ran out
// (the flag is set in *A.err and the copies in flight have been waited for): the caller then skips
// its computation and every global store.
template <int N, bool PERT, class R, int EPB, bool RES, class Between>
__device__ __forceinline__ bool stage_elements(const KArgs<R>& A, R* sm, uint64_t* bar, uint32_t& parity, int e0, int ne,
                                               Between&& between) {
  using L = Layout<N, PERT, R, EPB, RES>;
  constexpr int N3 = N * N * N;
  const bool tq = L::tmaQ && (((uintptr_t)A.q & 15u) == 0);
  const bool tb = L::bgShared && L::tmaBG && (((uintptr_t)A.bg.bg & 15u) == 0) && (((uintptr_t)A.bg.grho0 & 15u) == 0);
  const bool tg = A.G_in != nullptr && ((kG * N3 * sizeof(R)) % 16 == 0) && (((uintptr_t)A.G_in & 15u) == 0);
  if (A.G_in != nullptr && !tg) {
    for (int i = threadIdx.x; i < ne * kG * N3; i += blockDim.x)
      sm[L::oG + (i / (kG * N3)) * L::SG + i % (kG * N3)] = A.G_in[(size_t)e0 * kG * N3 + i];
  }
  const bool any_bulk = tq || tb || tg || L::SM;
  if (threadIdx.x == 0 && any_bulk) {
    uint32_t bytes = 0;
    if (tq) bytes += ne * 5 * N3 * sizeof(R);
    if (tb) bytes += ne * 5 * N3 * sizeof(R);
    if (tg) bytes += ne * kG * N3 * sizeof(R);
    if (L::SM) bytes += ne * L::SSF * sizeof(R);
    mbar_expect_tx(bar, bytes);
    if constexpr (L::SM) {
      for (int el = 0; el < ne; ++el) stage_metric_block<N, R, L>(A.m.Sf, e0 + el, 0, sm + L::oSF0 + el * L::SSF, bar);
    }
    for (int el = 0; el < ne; ++el) {
      if (tg) bulk_g2s(sm + L::oG + el * L::SG, A.G_in + (size_t)(e0 + el) * kG * N3, kG * N3 * sizeof(R), bar);
      if (tq) bulk_g2s(sm + L::oQ + el * L::SQ, A.q + (size_t)(e0 + el) * 5 * N3, 5 * N3 * sizeof(R), bar);
      if (tb) {
        bulk_g2s(sm + L::oBG + el * L::SBG, (const R*)A.bg.bg + (size_t)(e0 + el) * 2 * N3, 2 * N3 * sizeof(R), bar);
        bulk_g2s(sm + L::oGR0 + el * L::SGR0, (const R*)A.bg.grho0 + (size_t)(e0 + el) * 3 * N3, 3 * N3 * sizeof(R),
                 bar);
      }
    }
  }
  if (!tq) {
    for (int i = threadIdx.x; i < ne * 5 * N3; i += blockDim.x)
      sm[L::oQ + (i / (5 * N3)) * L::SQ + i % (5 * N3)] = A.q[(size_t)e0 * 5 * N3 + i];
  }
  if (L::bgShared && !tb) {
    for (int i = threadIdx.x; i < ne * 2 * N3; i += blockDim.x)
      sm[L::oBG + (i / (2 * N3)) * L::SBG + i % (2 * N3)] = (R)A.bg.bg[(size_t)e0 * 2 * N3 + i];
    for (int i = threadIdx.x; i < ne * 3 * N3; i += blockDim.x)
      sm[L::oGR0 + (i / (3 * N3)) * L::SGR0 + i % (3 * N3)] = (R)A.bg.grho0[(size_t)e0 * 3 * N3 + i];
  }
  const uint32_t polls = wait_polls(A.err);
  between();
  bool ok = true;
  if (any_bulk) {
    ok = mbar_wait(bar, parity, A.err, polls);
    parity ^= 1u;
  }
  return __syncthreads_and(ok) != 0;
}

// ------------------------------------------------------------------ lifting, one direction

// d q / d xi_D along the thread's D-line with common face values (BR1-like averaging, Section 3;
// walls Section 5), times grad xi_D = S^D / |J|, accumulated into the gradient array.
// FIRST: the sweep stores its contribution (no partial sums yet).  LAST: the sweep adds the partial
// sums of the other two directions and turns the complete conserved gradients of its line's points
// into the gradient record in place (its line's points are touched by no other thread in this phase).
template <int N, bool PERT, class R, int EPB, int D, bool FIRST, bool LAST>
__device__ __forceinline__ void lift_dir(const KArgs<R>& A, R* sm, int el, int ln, int e, const LiftPre<N, R>& pre) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N3 = N * N * N;
  const R* sq = sm + L::oQ + el * L::SQ;
  const R* sbg = sm + L::oBG + el * L::SBG;
  R* sg = sm + L::oG + el * L::SG;
  const PhysArg<R>& ph = A.ph;

  R qv[5][N];
#pragma unroll
  for (int v = 0; v < 5; ++v) load_line_lin<N, D>(sq + v * N3, ln, qv[v]);
  R r0[N], E0l[N];
  if (PERT) {
    load_line_bg<N, D>(sbg, ln, r0);
    load_line_bg<N, D>(sbg + N3, ln, E0l);
  }
  const auto& S = pre.S;

  R dq[5][2];  // common state minus own trace at the two ends
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int f = side ? N : 0;
    const NbFace<R>& nb = pre.nb[side];
    R qe[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R acc = R(0);
#pragma unroll
      for (int s = 0; s < N; ++s) acc += A.ops.I[f][s] * qv[v][s];
      qe[v] = acc;
    }
    if (nb.kind >= 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) dq[v][side] = R(0.5) * (nb.q[v] - qe[v]);
    } else {
      R rho0e = R(0), E0e = R(0);
      if (PERT) {
#pragma unroll
        for (int s = 0; s < N; ++s) {
          rho0e += A.ops.I[f][s] * r0[s];
          E0e += A.ops.I[f][s] * E0l[s];
        }
      }
      // wall common state: zero normal velocity, interior density, interior pressure (inner wall)
      // or p = R rho T_top (outer wall)
      const R sg_ = side ? R(1) : R(-1);
      const R mag = sqrt(S[0][f] * S[0][f] + S[1][f] * S[1][f] + S[2][f] * S[2][f]);
      const R im = qdiv(sg_, mag);
      const R nh[3] = {im * S[0][f], im * S[1][f], im * S[2][f]};
      const Pt<R> st = point_state<PERT>(qe, rho0e, E0e, ph);
      const R mn = qe[1] * nh[0] + qe[2] * nh[1] + qe[3] * nh[2];
      const R mc[3] = {qe[1] - mn * nh[0], qe[2] - mn * nh[1], qe[3] - mn * nh[2]};
      const R pc = nb.kind == -2 ? ph.Rgas * st.rhop * ph.T_top : st.p;
      const R Ec = qdiv(pc, ph.gm1) + qdiv(R(0.5) * (mc[0] * mc[0] + mc[1] * mc[1] + mc[2] * mc[2]), st.rho);
      dq[0][side] = R(0);
      dq[1][side] = mc[0] - qe[1];
      dq[2][side] = mc[1] - qe[2];
      dq[3][side] = mc[2] - qe[3];
      dq[4][side] = Ec - qe[4];
    }
  }
  // xi sweep at N = 4 (FP32, raw lifting, not last): the raw slot leaves as one 16-byte store per
  // component, the line's four points being contiguous in the swizzled layout
  constexpr bool RAWVEC = lift_raw<N, R>() && !LAST && D == 0;
  R rawv[RAWVEC ? 8 : 1][RAWVEC ? N : 1];
  R g0[LAST && PERT ? 3 : 1][N];
  if constexpr (LAST && PERT) {
    const R* sgr0 = sm + L::oGR0 + el * L::SGR0;
#pragma unroll
    for (int n = 0; n < 3; ++n) load_line_bg<N, D>(sgr0 + n * N3, ln, g0[n]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const R ij = pre.ij[i];
    R gx[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      R acc = R(0);
#pragma unroll
      for (int f = 0; f <= N; ++f) acc += A.ops.Lfs[i][f] * S[n][f];
      gx[n] = acc * ij;
    }
    const int si = line_sidx<N, D, R>(ln, i);
    R gq[LAST ? 15 : 1];
    constexpr bool RAW = lift_raw<N, R>();
    R dvv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R dv = A.ops.D[i][0] * dq[v][0] + A.ops.D[i][N] * dq[v][1];
#pragma unroll
      for (int s = 0; s < N; ++s) dv += A.ops.Dsol[i][s] * qv[v][s];
      dvv[v] = dv;
      if constexpr (!RAW) {
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          R* p = sg + (3 * v + n) * N3 + si;
          if constexpr (LAST) gq[3 * v + n] = *p + dv * gx[n];
          else if constexpr (FIRST) *p = dv * gx[n];
          else *p += dv * gx[n];
        }
      }
    }
    if constexpr (RAW && !LAST && RAWVEC) {
#pragma unroll
      for (int v = 0; v < 5; ++v) rawv[v][i] = dvv[v];
#pragma unroll
      for (int n = 0; n < 3; ++n) rawv[5 + n][i] = gx[n];
    } else if constexpr (RAW && !LAST) {
      // slot 0 (first sweep) or 1: the five derivatives, then grad xi_D
      constexpr int o = FIRST ? 0 : 8;
#pragma unroll
      for (int v = 0; v < 5; ++v) sg[(o + v) * N3 + si] = dvv[v];
#pragma unroll
      for (int n = 0; n < 3; ++n) sg[(o + 5 + n) * N3 + si] = gx[n];
    }
    if constexpr (RAW && LAST) {
      R raw[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) raw[c] = sg[c * N3 + si];
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int n = 0; n < 3; ++n)
          gq[3 * v + n] = dvv[v] * gx[n] + raw[v] * raw[5 + n] + raw[8 + v] * raw[13 + n];
    }
    if constexpr (LAST) {
      if (A.grad_rho_out) {
        const int pt = line_pt<N, D>(ln, i);
#pragma unroll
        for (int n = 0; n < 3; ++n) A.grad_rho_out[((size_t)e * 3 + n) * N3 + pt] = gq[n];
      }
      R q[5], gr0[3], g[kG];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = qv[v][i];
#pragma unroll
      for (int n = 0; n < 3; ++n) gr0[n] = PERT ? g0[PERT ? n : 0][i] : R(0);
      const Pt<R> st = point_state<PERT>(q, PERT ? r0[i] : R(0), PERT ? E0l[i] : R(0), A.ph);
      grad_prim<PERT>(st, gq, gr0, A.ph, g);
#pragma unroll
      for (int c = 0; c < kG; ++c) sg[c * N3 + si] = g[c];
    }
  }
  if constexpr (RAWVEC) {
    constexpr int o = FIRST ? 0 : 8;
    const int s0 = line_sidx<N, 0, R>(ln, 0);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      *reinterpret_cast<float4*>(sg + (o + c) * N3 + s0) = make_float4(rawv[c][0], rawv[c][1], rawv[c][2], rawv[c][3]);
  }
}

// Lifting of every element of the CTA; afterwards the first kG component arrays of the gradient
// array hold the gradient record (grad rho, trace-free strain, grad p) of the form's variables.
// `pre` holds the first direction's prefetch on entry (direction 1 with kLiftFused, else 0); each
// later direction's loads are issued before the barrier that precedes it.
template <int N, bool PERT, class R, int EPB>
__device__ __forceinline__ void lift_all(const KArgs<R>& A, R* sm, int el, int ln, int e, bool active,
                                         LiftPre<N, R>& pre, const int* snb) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N3 = N * N * N;
  if constexpr (kLiftFused) {
    // three directions (lift_dir_at), the last of which also forms the record (see lift_dir)
    constexpr int d0 = lift_dir_at<N, R>(0), d1 = lift_dir_at<N, R>(1), d2 = lift_dir_at<N, R>(2);
    if (active) {
      lift_dir<N, PERT, R, EPB, d0, true, false>(A, sm, el, ln, e, pre);
      lift_prefetch<N, PERT, R, d1>(A, e, ln, pre, snb);
    }
    __syncthreads();
    if (active) {
      lift_dir<N, PERT, R, EPB, d1, false, false>(A, sm, el, ln, e, pre);
      lift_prefetch<N, PERT, R, d2>(A, e, ln, pre, snb);
    }
    __syncthreads();
    if (active) lift_dir<N, PERT, R, EPB, d2, false, true>(A, sm, el, ln, e, pre);
    if (grad_bulk_store<N>()) fence_async_smem();  // the record may leave by bulk store after the barrier
    __syncthreads();
    return;
  }
  if (active) {
    lift_dir<N, PERT, R, EPB, 0, true, false>(A, sm, el, ln, e, pre);
    lift_prefetch<N, PERT, R, 1>(A, e, ln, pre, snb);
  }
  __syncthreads();
  if (active) {
    lift_dir<N, PERT, R, EPB, 1, false, false>(A, sm, el, ln, e, pre);
    lift_prefetch<N, PERT, R, 2>(A, e, ln, pre, snb);
  }
  __syncthreads();
  if (active) lift_dir<N, PERT, R, EPB, 2, false, false>(A, sm, el, ln, e, pre);
  __syncthreads();
  if (active) {
    const R* sq = sm + L::oQ + el * L::SQ;
    const R* sbg = sm + L::oBG + el * L::SBG;
    const R* sgr0 = sm + L::oGR0 + el * L::SGR0;
    R* sg = sm + L::oG + el * L::SG;
    R qv[5][N], r0[N], E0l[N], g0[3][N];
#pragma unroll
    for (int v = 0; v < 5; ++v) load_line_lin<N, 0>(sq + v * N3, ln, qv[v]);
    if (PERT) {
      load_line_bg<N, 0>(sbg, ln, r0);
      load_line_bg<N, 0>(sbg + N3, ln, E0l);
#pragma unroll
      for (int n = 0; n < 3; ++n) load_line_bg<N, 0>(sgr0 + n * N3, ln, g0[n]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int si = line_sidx<N, 0, R>(ln, i);
      R q[5], gq[15], gr0[3], g[kG];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = qv[v][i];
#pragma unroll
      for (int c = 0; c < 15; ++c) gq[c] = sg[c * N3 + si];
      if (A.grad_rho_out) {
        const int pt = line_pt<N, 0>(ln, i);
#pragma unroll
        for (int n = 0; n < 3; ++n) A.grad_rho_out[((size_t)e * 3 + n) * N3 + pt] = gq[n];
      }
#pragma unroll
      for (int n = 0; n < 3; ++n) gr0[n] = PERT ? g0[n][i] : R(0);
      const Pt<R> st = point_state<PERT>(q, PERT ? r0[i] : R(0), PERT ? E0l[i] : R(0), A.ph);
      grad_prim<PERT>(st, gq, gr0, A.ph, g);
#pragma unroll
      for (int c = 0; c < kG; ++c) sg[c * N3 + si] = g[c];
    }
  }
  if (grad_bulk_store<N>()) fence_async_smem();  // the record may leave by bulk store after the barrier
  __syncthreads();
}

// Interpolated state, background and gradients of line ln at flux point f of direction D.
template <int N, bool PERT, class R>
struct FluxPointData {
  R q[5], g[kG], gr0[3], r0, E0;
};

// ------------------------------------------------------------------ wall flux

// Conductive energy flux f.n through the outer wall with the temperature imposed there (Section 5):
// T = T_top in f = -kappa rho T grad S - kappa_r rho C_p grad T written in rho and p.
template <class R>
__device__ __forceinline__ R wall_conduction(const R g[kG], const R nh[3], R krf, const PhysArg<R>& ph) {
  const R RT = ph.Rgas * ph.T_top;
  R fn = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b)
    fn += -ph.CpR * (ph.kappa * (qdiv(g[9 + b], ph.gamma) - RT * g[b]) + krf * (g[9 + b] - RT * g[b])) * nh[b];
  return fn;
}

// Common flux F_n through a wall face point (Section 5): exact inviscid flux (0, p n, 0); viscous
// momentum flux = the normal traction only; energy: f.n from the gradient with T = T_top (outer wall,
// kind -2) or the prescribed flux (inner wall; in the perturbation form the background residual
// carries it).  g: the gradient record at the point; nh: the unit outward normal.
template <bool PERT, class R>
__device__ __forceinline__ void wall_flux(const Pt<R>& st, const R g[kG], const R nh[3], int kind, R krf,
                                          const PhysArg<R>& ph, R Fh[5]) {
  const R mu = st.rho * ph.nu;
  R trac = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) trac += nh[a] * mu * sig(g, a, b) * nh[b];
  Fh[0] = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) Fh[1 + a] = (st.p - trac) * nh[a];
  if (kind == -2) {
    Fh[4] = wall_conduction(g, nh, krf, ph);
  } else {
    Fh[4] = PERT ? R(0) : -ph.bottom_flux;
  }
}

// ------------------------------------------------------------------ gradient kernel

// Lifted gradients, then the one-sided normal viscous flux F_v . n_out on every face point,
// written for the neighbours: Tv[e][F][0..2] = tau n, Tv[e][F][3] = u.tau n - f.n.
// On a wall side (face-kernel mode) the energy entry holds instead the wall's conductive flux f.n
// with the top temperature imposed (used by k_face on the outer wall; Section 5).
// The values at the line's two end points of one component: lo = sum_s I[0][s] l[s], hi = sum_s I[N][s] l[s].
template <int N, class R>
__device__ __forceinline__ void line_ends(const R (&l)[N], const R (&w0)[N], const R (&wN)[N], R& lo, R& hi) {
  lo = R(0);
  hi = R(0);
#pragma unroll
  for (int s = 0; s < N; ++s) {
    lo += w0[s] * l[s];
    hi += wN[s] * l[s];
  }
}

// Component c's line of the gradient record (one 16-byte load for a xi line at N = 4 FP32).
template <int N, int D, class R>
__device__ __forceinline__ void load_grad_line(const R* sgc, int ln, R (&out)[N]) {
  if constexpr (D == 0 && N == 4 && sizeof(R) == 4 && kVecGradLoad) {
    const float4 v = *reinterpret_cast<const float4*>(sgc + line_sidx<N, 0, R>(ln, 0));
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) out[s] = sgc[line_sidx<N, D, R>(ln, s)];
  }
}

template <int N, bool PERT, class R, int EPB, int D, bool KR>
__device__ __forceinline__ void face_visc_dir(const KArgs<R>& A, const R* sm, int el, int ln, int e,
                                              const R (&s3f)[2][3]) {
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N2 = N * N, N3 = N * N * N;
  const R* sq = sm + L::oQ + el * L::SQ;
  const R* sbg = sm + L::oBG + el * L::SBG;
  const R* sgr0 = sm + L::oGR0 + el * L::SGR0;
  const R* sg = sm + L::oG + el * L::SG;
  const R* tI = sm + L::oTAB;
  if constexpr (face_ends<N>()) {
    // every line component is read once and reduced to its two end values at once
    R w0[N], wN[N];
#pragma unroll
    for (int s = 0; s < N; ++s) {
      w0[s] = tI[s];
      wN[s] = tI[N * N + s];
    }
    R qe[2][5], ge[2][kG], gre[2][3], r0e[2], E0e[2];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R l[N];
      load_line_lin<N, D>(sq + v * N3, ln, l);
      line_ends<N>(l, w0, wN, qe[0][v], qe[1][v]);
    }
#pragma unroll
    for (int c = 0; c < kG; ++c) {
      R l[N];
      load_grad_line<N, D>(sg + c * N3, ln, l);
      line_ends<N>(l, w0, wN, ge[0][c], ge[1][c]);
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      r0e[side] = R(0);
      E0e[side] = R(0);
#pragma unroll
      for (int n = 0; n < 3; ++n) gre[side][n] = R(0);
    }
    if (PERT) {
      R l[N];
      load_line_bg<N, D>(sbg, ln, l);
      line_ends<N>(l, w0, wN, r0e[0], r0e[1]);
      load_line_bg<N, D>(sbg + N3, ln, l);
      line_ends<N>(l, w0, wN, E0e[0], E0e[1]);
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        load_line_bg<N, D>(sgr0 + n * N3, ln, l);
        line_ends<N>(l, w0, wN, gre[0][n], gre[1][n]);
      }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {  // unrolled: the end values are picked by constant index
      const int f = side ? N : 0;
      const int kind = kFaceKernel ? __ldg(A.m.nbr + e * 6 + 2 * D + side) : 0;
      R qf[5], gf[kG], gr0f[3];
#pragma unroll
      for (int v = 0; v < 5; ++v) qf[v] = side ? qe[1][v] : qe[0][v];
#pragma unroll
      for (int c = 0; c < kG; ++c) gf[c] = side ? ge[1][c] : ge[0][c];
#pragma unroll
      for (int n = 0; n < 3; ++n) gr0f[n] = side ? gre[1][n] : gre[0][n];
      const R rho0f = side ? r0e[1] : r0e[0];
      const R E0f = side ? E0e[1] : E0e[0];
      R s3[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) s3[n] = side ? s3f[1][n] : s3f[0][n];
      const R sgn = side ? R(1) : R(-1);
      const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
      const R im = qdiv(sgn, mag);
      const R nh[3] = {im * s3[0], im * s3[1], im * s3[2]};
      const Pt<R> st = point_state<PERT>(qf, rho0f, E0f, A.ph);
      const R krf = kr_at<N, D, KR>(A, e, ln, f);
      R Fv[5];
      flux_visc<PERT>(st, gf, gr0f, rho0f, A.ph.gm1 * E0f, nh, A.ph, krf, Fv);
      if (kFaceKernel && kind < 0) Fv[4] = wall_conduction(gf, nh, krf, A.ph);
      R* o = A.Tv_out + ((size_t)e * 6 + 2 * D + side) * 4 * N2;
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v * N2 + ln] = Fv[1 + v];
    }
  } else {
    R qv[5][N], gv[kG][N], r0[N], E0l[N], g0[3][N];
#pragma unroll
    for (int v = 0; v < 5; ++v) load_line_lin<N, D>(sq + v * N3, ln, qv[v]);
    load_grad_lines<N, D>(sg, ln, gv);
    if (PERT) {
      load_line_bg<N, D>(sbg, ln, r0);
      load_line_bg<N, D>(sbg + N3, ln, E0l);
#pragma unroll
      for (int n = 0; n < 3; ++n) load_line_bg<N, D>(sgr0 + n * N3, ln, g0[n]);
    }
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const int f = side ? N : 0;
      const int kind = kFaceKernel ? __ldg(A.m.nbr + e * 6 + 2 * D + side) : 0;
      R w[N];
#pragma unroll
      for (int s = 0; s < N; ++s) w[s] = tI[f * N + s];
      R qf[5], gf[kG], gr0f[3] = {R(0), R(0), R(0)};
      R rho0f = R(0), E0f = R(0);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qf[v] = R(0);
#pragma unroll
        for (int s = 0; s < N; ++s) qf[v] += w[s] * qv[v][s];
      }
#pragma unroll
      for (int c = 0; c < kG; ++c) {
        gf[c] = R(0);
#pragma unroll
        for (int s = 0; s < N; ++s) gf[c] += w[s] * gv[c][s];
      }
      if (PERT) {
#pragma unroll
        for (int s = 0; s < N; ++s) {
          rho0f += w[s] * r0[s];
          E0f += w[s] * E0l[s];
#pragma unroll
          for (int n = 0; n < 3; ++n) gr0f[n] += w[s] * g0[n][s];
        }
      }
      R s3[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) s3[n] = side ? s3f[1][n] : s3f[0][n];
      const R sgn = side ? R(1) : R(-1);
      const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
      const R im = qdiv(sgn, mag);
      const R nh[3] = {im * s3[0], im * s3[1], im * s3[2]};
      const Pt<R> st = point_state<PERT>(qf, rho0f, E0f, A.ph);
      const R krf = kr_at<N, D, KR>(A, e, ln, f);
      R Fv[5];
      flux_visc<PERT>(st, gf, gr0f, rho0f, A.ph.gm1 * E0f, nh, A.ph, krf, Fv);
      if (kFaceKernel && kind < 0) Fv[4] = wall_conduction(gf, nh, krf, A.ph);
      R* o = A.Tv_out + ((size_t)e * 6 + 2 * D + side) * 4 * N2;
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v * N2 + ln] = Fv[1 + v];
    }
  }
}

// Lifting of tile `tile` (elements tile * EPB ...; threads beyond EPB * N^2 idle but take part in the
// barriers).  bar: the CTA's staging barrier (initialised), pbar: the parity of its next phase.
template <int N, bool PERT, class R, int EPB, bool KR>
__device__ __forceinline__ void grad_tile(const KArgs<R>& A, int64_t tile, uint64_t* bar, uint32_t& pbar) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int e0 = (int)(tile * EPB);
  const int ne = min(EPB, A.m.E - e0);
  const int e = e0 + el;
  const bool active = el < ne;
  fill_tables<N, R>(A.ops, sm + Layout<N, PERT, R, EPB>::oTAB);
  __syncthreads();
  LiftPre<N, R> pre;
  // the six (neighbour, face code) pairs of each element, for the later directions' prefetches
  __shared__ int snb[kGradNbShared ? EPB : 1][12];
  if (!stage_elements<N, PERT, R, EPB, false>(A, sm, bar, pbar, e0, ne, [&] {
        if (active) lift_prefetch<N, PERT, R, kLiftFused ? lift_dir_at<N, R>(0) : 0>(A, e, ln, pre);
        if (kGradNbShared && active && ln < 6) {
          snb[el][2 * ln] = __ldg(A.m.nbr + e * 6 + ln);
          snb[el][2 * ln + 1] = __ldg(A.m.code + e * 6 + ln);
        }
      }))
    return;
  lift_all<N, PERT, R, EPB>(A, sm, el, ln, e, active, pre, kGradNbShared ? snb[kGradNbShared ? el : 0] : nullptr);
  // face metrics of the viscous-flux pass, loaded before the record stores
  R s3f[3][2][3];
  if (active && A.Tv_out != nullptr) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int n = 0; n < 3; ++n)
          s3f[d][side][n] = __ldg(A.m.Sf + ((size_t)e * 3 + d) * 3 * (N + 1) * N2 + (n * (N + 1) + side * N) * N2 + ln);
  }
  // the gradient record out: one bulk store per element (issued by thread 0, overlapping the viscous
  // face pass, which only reads shared memory), else a strided copy
  using L = Layout<N, PERT, R, EPB>;
  constexpr int N3 = N * N * N;
  constexpr uint32_t kGBytes = kG * N3 * sizeof(R);
  const bool g_bulk = grad_bulk_store<N>() && A.G_out != nullptr && kGBytes % 16 == 0 && (L::SG * sizeof(R)) % 16 == 0 &&
                      ((uintptr_t)A.G_out & 15u) == 0;
  if (g_bulk) {
    if (threadIdx.x == 0) {
      for (int j = 0; j < ne; ++j) bulk_s2g(A.G_out + (size_t)(e0 + j) * kG * N3, sm + L::oG + j * L::SG, kGBytes);
      bulk_commit();
    }
  } else if (A.G_out != nullptr) {
    for (int i = threadIdx.x; i < ne * kG * N3; i += blockDim.x)
      A.G_out[(size_t)e0 * kG * N3 + i] = sm[L::oG + (i / (kG * N3)) * L::SG + i % (kG * N3)];
  }
  if (active && A.Tv_out != nullptr) {
    face_visc_dir<N, PERT, R, EPB, 0, KR>(A, sm, el, ln, e, s3f[0]);
    face_visc_dir<N, PERT, R, EPB, 1, KR>(A, sm, el, ln, e, s3f[1]);
    face_visc_dir<N, PERT, R, EPB, 2, KR>(A, sm, el, ln, e, s3f[2]);
  }
  if (g_bulk && threadIdx.x == 0) bulk_wait_read();  // the CTA's shared memory must outlive the reads
}

// FP32: 16 resident warps per SM at N = 3, 4 (register cap 128), as grad_min_blocks gives
template <int N, bool PERT, class R, int EPB, bool KR>
__global__ void __launch_bounds__(EPB * N * N, sizeof(R) == 4 ? grad_min_blocks<N, EPB>() : 1) k_grad(const KArgs<R> A) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);  // ordered by the tile's first barrier
  uint32_t ph = 0;
  grad_tile<N, PERT, R, EPB, KR>(A, blockIdx.x, &bar, ph);
}

// ------------------------------------------------------------------ flux sweep, one direction

// Transformed fluxes at the N+1 flux points of the thread's D-line (Eq. 12), common fluxes at
// the two ends (Rusanov + averaged viscous; walls per Section 5), derivative back to the solution
// points (Eq. 18), accumulated into the divergence array.
template <int N, bool PERT, class R, int EPB, int D, bool KR, bool X>
__device__ __forceinline__ void flux_dir(const KArgs<R>& A, R* sm, int el, int ln, int e, const FluxPre<R, X>& pre,
                                         const int* snb, const R* sS) {
  using L = Layout<N, PERT, R, EPB, true>;
  constexpr bool SMM = L::SM;  // metrics of this direction staged in shared memory at sS
  constexpr int N2 = N * N, N3 = N * N * N;
  const R* sq = sm + L::oQ + el * L::SQ;
  const R* sbg = sm + L::oBG + el * L::SBG;
  const R* sgr0 = sm + L::oGR0 + el * L::SGR0;
  const R* sg = sm + L::oG + el * L::SG;
  R* sdiv = sm + L::oDIV + el * L::SDIV;
  const PhysArg<R>& ph = A.ph;

  // line data in registers (FP32); the FP64 form re-reads the gradients from shared memory per
  // flux point to stay within the register file
  constexpr bool kRegGrad = sizeof(R) == 4 && reg_grad_lines<N>();
  R qv[5][N], gv[kRegGrad ? kG : 1][N];
#pragma unroll
  for (int v = 0; v < 5; ++v) load_line_lin<N, D>(sq + v * N3, ln, qv[v]);
  if constexpr (kRegGrad) {
    load_grad_lines<N, D>(sg, ln, gv);
  }
  // the background line is read from shared memory per flux point (register budget)
  const R* Sl = A.m.Sf + ((size_t)e * 3 + D) * 3 * (N + 1) * N2;

  R acc[5][N];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int i = 0; i < N; ++i) acc[v][i] = R(0);
  const R* tI = sm + L::oTAB;
  const R* tD = sm + L::oTAB + (N + 1) * N;

  // one rolled loop over the flux points keeps a single copy of the flux code per direction
  // Flux points in the order 1, ..., N, 0, so that the neighbour data (prefetched) are first needed
  // after the interior points; S^D at the next flux point is loaded one iteration ahead.
  constexpr bool EF = end_first<N, D>();
  constexpr int AH = SMM ? 0 : s3_ahead<N>();
  R s3n[3];
  if constexpr (!SMM) {
#pragma unroll
    for (int n = 0; n < 3; ++n) s3n[n] = pre.s3[n];
  }
  R s3nn[AH == 2 ? 3 : 1];
  if constexpr (AH == 2) {
#pragma unroll
    for (int n = 0; n < 3; ++n) s3nn[n] = pre.s3b[n];
  }
  NbFace<R> nbn;  // mode 2: the next end point's neighbour data
  nbn.kind = -1;
  // face-kernel mode: the end points' common fluxes F~ are read (both issued now), and the loop visits
  // the interior flux points 1..N-1 only
  constexpr bool FK = kFaceKernel;
  R Fc0[FK ? 5 : 1], FcN[FK ? 5 : 1];
  if constexpr (FK) {
    const R* c0 = A.Fc + ((size_t)e * 6 + 2 * D) * 5 * N2 + ln;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Fc0[v] = __ldg(c0 + v * N2);
      FcN[v] = __ldg(c0 + (5 + v) * N2);
    }
  }
#pragma unroll 1
  for (int it = 0; it < (FK ? N - 1 : N + 1); ++it) {
    const int f = flux_order<N, EF>(it);
    R s3[3];
    if constexpr (SMM) {
#pragma unroll
      for (int n = 0; n < 3; ++n) s3[n] = sS[(n * L::SFP + f - L::SF0) * N2 + ln];
    } else {
#pragma unroll
      for (int n = 0; n < 3; ++n) s3[n] = s3n[n];
    }
    if constexpr (SMM) {
    } else if constexpr (AH == 2) {
#pragma unroll
      for (int n = 0; n < 3; ++n) s3n[n] = s3nn[n];
      if (it + 2 <= N) {
        const int fnn = flux_order<N, EF>(it + 2);
#pragma unroll
        for (int n = 0; n < 3; ++n) s3nn[n] = __ldg(Sl + (n * (N + 1) + fnn) * N2 + ln);
      }
    } else if (it < N) {
      const int fn = flux_order<N, EF>(it + 1);
#pragma unroll
      for (int n = 0; n < 3; ++n) s3n[n] = __ldg(Sl + (n * (N + 1) + fn) * N2 + ln);
    }
    NbFace<R> nbc;  // mode 2: this end point's neighbour data
    if (!FK && flux_nb_mode<N>() == 2) {
      nbc = nbn;
      if (it == N - 2 || it == N - 1) nbn = load_nb_at<N, PERT, true>(A, pre.nbi[it == N - 2 ? 1 : 0]);
    }
    R w[N];
#pragma unroll
    for (int s = 0; s < N; ++s) w[s] = tI[f * N + s];
    FluxPointData<N, PERT, R> P;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R t = R(0);
#pragma unroll
      for (int s = 0; s < N; ++s) t += w[s] * qv[v][s];
      P.q[v] = t;
    }
#pragma unroll
    for (int c = 0; c < kG; ++c) {
      R t = R(0);
#pragma unroll
      for (int s = 0; s < N; ++s) {
        if constexpr (kRegGrad) t += w[s] * gv[c][s];
        else t += w[s] * sg[c * N3 + line_sidx<N, D, R>(ln, s)];
      }
      P.g[c] = t;
    }
    P.r0 = R(0);
    P.E0 = R(0);
#pragma unroll
    for (int n = 0; n < 3; ++n) P.gr0[n] = R(0);
    if (PERT) {
#pragma unroll
      for (int s = 0; s < N; ++s) {
        const int pt = line_bg<N, D, R>(ln, s);
        if constexpr (L::bgShared) {
          P.r0 += w[s] * sbg[pt];
          P.E0 += w[s] * sbg[N3 + pt];
#pragma unroll
          for (int n = 0; n < 3; ++n) P.gr0[n] += w[s] * sgr0[n * N3 + pt];
        } else {
          const float* bge = A.bg.bg + (size_t)e * 2 * N3;
          const float* gre = A.bg.grho0 + (size_t)e * 3 * N3;
          P.r0 += w[s] * (R)__ldg(bge + pt);
          P.E0 += w[s] * (R)__ldg(bge + N3 + pt);
#pragma unroll
          for (int n = 0; n < 3; ++n) P.gr0[n] += w[s] * (R)__ldg(gre + n * N3 + pt);
        }
      }
    }
    const Pt<R> st = point_state<PERT>(P.q, P.r0, P.E0, ph);
    const R p0f = ph.gm1 * P.E0;
    const R krf = kr_at<N, D, KR>(A, e, ln, f);
    R Ft[5];
    if (FK || (f > 0 && f < N)) {
      R Fi[5], Fv[5];
      flux_inv(P.q, st, s3, Fi);
      flux_visc<PERT>(st, P.g, P.gr0, P.r0, p0f, s3, ph, krf, Fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) Ft[v] = Fi[v] - Fv[v];
    } else {
      const int side = (f == N);
      NbFace<R> nb;
      if constexpr (EF) {
        nb = pre.nb[side];
      } else if constexpr (flux_nb_mode<N>() == 0) {
        nb = load_nb<N, PERT, true>(A, e, 2 * D + side, ln);
      } else if constexpr (flux_nb_mode<N>() == 1) {
        nb = load_nb_at<N, PERT, true>(A, pre.nbi[side]);
      } else if constexpr (flux_nb_mode<N>() == 2) {
        nb = nbc;
      } else {
        const int F = 2 * D + side, k = snb[2 * F], c = snb[2 * F + 1];
        NbIdx x;
        x.bf = k >= 0 ? k * 6 + (c >> 3) : k;
        x.tp = k >= 0 ? map_face_pt<N>(ln, c & 7) : 0;
        nb = load_nb_at<N, PERT, true>(A, x);
      }
      const R sgn = side ? R(1) : R(-1);
      const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
      const R im = qdiv(sgn, mag);
    const R nh[3] = {im * s3[0], im * s3[1], im * s3[2]};
      R Fh[5];
      if (nb.kind >= 0) {
        const Pt<R> sR = point_state<PERT>(nb.q, nb.r0, nb.E0, ph);
        rusanov<PERT>(P.q, st, P.r0, P.E0, nb.q, sR, nb.r0, nb.E0, nh, ph, Fh);
        R Fv[5];
        flux_visc<PERT>(st, P.g, P.gr0, P.r0, p0f, nh, ph, krf, Fv);
#pragma unroll
        for (int v = 1; v < 5; ++v)  // the neighbour stored F_v . n_out(neighbour) = -F_v . n
          Fh[v] -= R(0.5) * (Fv[v] - nb.tv[v - 1]);
      } else {
        wall_flux<PERT>(st, P.g, nh, nb.kind, krf, ph, Fh);  // walls (Section 5)
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) Ft[v] = sgn * mag * Fh[v];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const R dc = tD[i * (N + 1) + f];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v][i] += dc * Ft[v];
    }
  }
  if constexpr (FK) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const R d0 = tD[i * (N + 1)], dN = tD[i * (N + 1) + N];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v][i] += d0 * Fc0[v] + dN * FcN[v];
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int si = line_sidx<N, D, R>(ln, i);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (D == 0) sdiv[v * N3 + si] = acc[v][i];
      else sdiv[v * N3 + si] += acc[v][i];
    }
  }
}

// ------------------------------------------------------------------ residual kernel

// Residual (and RK stage) of tile `tile` (elements tile * EPB ...; threads beyond EPB * N^2 idle but
// take part in the barriers).  bar: the staging barrier, barS: the two staged-metric barriers (used
// when L::SM; all initialised), pbar / pbarS: the parities of their next phases.
template <int N, bool PERT, class R, int EPB, int MODE, bool KR>
__device__ __forceinline__ void resid_tile(const KArgs<R>& A, int64_t tile, uint64_t* bar, uint64_t* barS,
                                           uint32_t& pbar, uint32_t& pbarS) {
  using L = Layout<N, PERT, R, EPB, true>;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const int el = threadIdx.x / N2, ln = threadIdx.x % N2;
  const int e0 = (int)(tile * EPB);
  const int ne = min(EPB, A.m.E - e0);
  const int e = e0 + el;
  const bool active = el < ne;
  fill_tables<N, R>(A.ops, sm + L::oTAB);
  __syncthreads();
  // direction d's metric blocks of the CTA's elements into buffer `buf` (thread 0), on barrier b
  auto stage_dir = [&](int d, int buf, uint64_t* b) {
    if constexpr (L::SM) {
      if (threadIdx.x == 0) {
        fence_async_smem();  // the buffer's previous contents were read by the generic proxy
        mbar_expect_tx(b, ne * L::SSF * sizeof(R));
        for (int j = 0; j < ne; ++j)
          stage_metric_block<N, R, L>(A.m.Sf, e0 + j, d, sm + (buf ? L::oSF1 : L::oSF0) + j * L::SSF, b);
      }
    }
  };
  const R* sS0 = sm + L::oSF0 + el * L::SSF;
  const R* sS1 = sm + L::oSF1 + el * L::SSF;
  bool failed = false;
  FluxPre<R, !stage_metrics<N, R>() && ((N == 4 && kEndFirstD0) || s3_ahead<N>() == 2)> fp;
  __shared__ int snb[flux_nb_mode<N>() == 3 ? EPB : 1][12];  // (neighbour, face code) of the 6 faces
  if (!stage_elements<N, PERT, R, EPB, true>(A, sm, bar, pbar, e0, ne, [&] {
        if (active) flux_prefetch<N, PERT, R, 0>(A, e, ln, fp);
        if (!kFaceKernel && flux_nb_mode<N>() == 3 && active && ln < 6) {
          snb[el][2 * ln] = __ldg(A.m.nbr + e * 6 + ln);
          snb[el][2 * ln + 1] = __ldg(A.m.code + e * 6 + ln);
        }
      }))
    return;
  const uint32_t polls = wait_polls(A.err);
  const int* snb_el = snb[flux_nb_mode<N>() == 3 ? el : 0];
  stage_dir(1, 1, &barS[0]);
  if (active) {
    flux_dir<N, PERT, R, EPB, 0, KR>(A, sm, el, ln, e, fp, snb_el, sS0);
    flux_prefetch<N, PERT, R, 1>(A, e, ln, fp);
  }
  __syncthreads();
  stage_dir(2, 0, &barS[1]);
  if constexpr (L::SM) failed |= !mbar_wait(&barS[0], pbarS, A.err, polls);
  if (active) {
    flux_dir<N, PERT, R, EPB, 1, KR>(A, sm, el, ln, e, fp, snb_el, sS1);
    flux_prefetch<N, PERT, R, 2>(A, e, ln, fp);
  }
  __syncthreads();
  if constexpr (L::SM) {
    failed |= !mbar_wait(&barS[1], pbarS, A.err, polls);
    pbarS ^= 1u;  // both staged-metric barriers completed a phase
  }
  if (active) flux_dir<N, PERT, R, EPB, 2, KR>(A, sm, el, ln, e, fp, snb_el, sS0);

  // Global inputs of the epilogue, all issued before its first store.  The epilogue works point by
  // point, so thread ln takes the points ln + N^2 i (i < N): 16 consecutive threads read 64
  // consecutive bytes of each array.
  R xg[3][N], ijg[N], r0g[5][N], ung[5][N];
  if (active) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pt = ln + N2 * i;
#pragma unroll
      for (int n = 0; n < 3; ++n) xg[n][i] = __ldg(A.m.x + ((size_t)e * 3 + n) * N3 + pt);
      ijg[i] = __ldg(A.m.invJ + (size_t)e * N3 + pt);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const size_t oi = ((size_t)e * 5 + v) * N3 + pt;
        r0g[v][i] = (PERT && A.bg.R0) ? (R)__ldg(A.bg.R0 + oi) : R(0);
        // a stage whose combination has no u^n term (a = 0) does not read it
        ung[v][i] = (MODE == kModeRK && A.a != R(0)) ? A.un[oi] : R(0);
      }
    }
  }
  // a staged-metric wait that gave up (flag set, copies drained): no thread stores anything
  if (__syncthreads_or(failed)) return;

  // residual dQ/dt = -div/|J| - M (Eqs. 4, 11), sources of Eqs. 2-3, and the RK combination
  R* sq = sm + L::oQ + el * L::SQ;
  const R* sdiv = sm + L::oDIV + el * L::SDIV;
  const PhysArg<R>& ph = A.ph;
  if (active) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pt = ln + N2 * i;
      const int si = sidx<N, R>(ln % N, ln / N, i);
      R q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = sq[v * N3 + pt];
      const R x0 = xg[0][i], x1 = xg[1][i], x2 = xg[2][i];
      const R r2 = x0 * x0 + x1 * x1 + x2 * x2;
      const R gr = qdiv(ph.GM, r2 * sqrt(r2));  // g = gr * x points outward (the source uses -rho g_vec)
      const R g3[3] = {gr * x0, gr * x1, gr * x2};
      R M[5];
      M[0] = R(0);
      M[1] = q[0] * g3[0] - ph.twoOmega * q[2];
      M[2] = q[0] * g3[1] + ph.twoOmega * q[1];
      M[3] = q[0] * g3[2];
      M[4] = q[1] * g3[0] + q[2] * g3[1] + q[3] * g3[2];
      const R ij = ijg[i];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        R Rv = -sdiv[v * N3 + si] * ij - M[v];
        if (PERT) Rv += r0g[v][i];
        const size_t oi = ((size_t)e * 5 + v) * N3 + pt;
        if (A.radd) Rv += __ldg(A.radd + oi);
        if (MODE == kModeResidual) {
          A.out[oi] = Rv;
        } else {
          const R dR = A.dt * Rv;
          if (A.out2) A.out2[oi] = A.a2 * A.un2[oi] + A.b2 * q[v] + A.c2 * dR;
          const R nv = A.a * ung[v][i] + A.b * q[v] + A.c * dR;
          A.out[oi] = nv;
          sq[v * N3 + pt] = nv;
        }
      }
    }
  }
  if (MODE == kModeRK) {
    __syncthreads();
    if (active && A.T_out) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          R lo = R(0), hi = R(0);
#pragma unroll
          for (int s = 0; s < N; ++s) {
            const int pt = d == 0 ? line_pt<N, 0>(ln, s) : (d == 1 ? line_pt<N, 1>(ln, s) : line_pt<N, 2>(ln, s));
            const R val = sq[v * N3 + pt];
            lo += A.ops.I[0][s] * val;
            hi += A.ops.I[N][s] * val;
          }
          A.T_out[((size_t)e * 6 + 2 * d) * 5 * N2 + v * N2 + ln] = lo;
          A.T_out[((size_t)e * 6 + 2 * d + 1) * 5 * N2 + v * N2 + ln] = hi;
        }
    }
  }
}

// FP32: 12 resident warps per SM at N = 3, 4 (register cap ~168 per thread), as resid_min_blocks gives
template <int N, bool PERT, class R, int EPB, int MODE, bool KR>
__global__ void __launch_bounds__(EPB * N * N, sizeof(R) == 4 ? resid_min_blocks<N, EPB>() : 1) k_resid(const KArgs<R> A) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(8) uint64_t barS[2];  // staged metrics of directions 1 and 2
  if (threadIdx.x == 0) {  // ordered by the tile's first barrier
    mbar_init(&bar);
    if constexpr (Layout<N, PERT, R, EPB, true>::SM) {
      mbar_init(&barS[0]);
      mbar_init(&barS[1]);
    }
  }
  uint32_t ph = 0, phS = 0;
  resid_tile<N, PERT, R, EPB, MODE, KR>(A, blockIdx.x, &bar, barS, ph, phS);
}

// ------------------------------------------------------------------ face kernel

// Common flux of every interior face point, once per face (Section 3: Rusanov inviscid flux with the
// wave speed of both sides, average of the two one-sided normal viscous fluxes from the lifting
// kernel).  One thread per (face, point) of the face list (element, local face) of owner sides; the
// owner's metric gives the unit normal n and |S|.  Writes F~ = sigma |S| F_n at the owner's point and
// -sigma' |S| F_n at the neighbour's matching point (its outward normal is -n), so the two sides'
// fluxes are exactly opposite.
//
// Wall faces follow the interior ones in the list (entries nf..nf+nw-1): their common flux (Section 5)
// is formed from the element's own trace and the lifting kernel's wall data (the viscous traction
// tau n and the conductive flux with the top temperature imposed).
// One thread's face point g (of (nf + nw) * N^2).
template <int N, bool PERT, class R>
__device__ __forceinline__ void face_point(const KArgs<R>& A, const int2* __restrict__ faces, int nf, int nw, int64_t g) {
  constexpr int N2 = N * N;
  if (g < 0 || g >= (int64_t)(nf + nw) * N2) return;
  const int t = (int)(g % N2);
  const int2 fc = faces[g / N2];
  const int e = fc.x, F = fc.y, D = F >> 1, side = F & 1;
  const int k = __ldg(A.m.nbr + e * 6 + F), code = __ldg(A.m.code + e * 6 + F);
  if (k < 0) {  // wall
    const size_t o = (size_t)e * 6 + F;
    R q[5], tv[4];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = __ldg(A.T + (o * 5 + v) * N2 + t);
#pragma unroll
    for (int v = 0; v < 4; ++v) tv[v] = __ldg(A.Tv + (o * 4 + v) * N2 + t);
    R r0 = R(0), E0 = R(0);
    if (PERT) {
      r0 = (R)__ldg(A.bg.bgT + (o * 2) * N2 + t);
      E0 = (R)__ldg(A.bg.bgT + (o * 2 + 1) * N2 + t);
    }
    const R* Sl = A.m.Sf + ((size_t)e * 3 + D) * 3 * (N + 1) * N2;
    R s3[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) s3[n] = __ldg(Sl + (n * (N + 1) + (side ? N : 0)) * N2 + t);
    const R sgn = side ? R(1) : R(-1);
    const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
    const R im = qdiv(sgn, mag);
    const R nh[3] = {im * s3[0], im * s3[1], im * s3[2]};
    const Pt<R> st = point_state<PERT>(q, r0, E0, A.ph);
    // exact inviscid flux (0, p n, 0) minus the normal viscous traction; energy: f.n
    const R trac = tv[0] * nh[0] + tv[1] * nh[1] + tv[2] * nh[2];
    R Fh[5];
    Fh[0] = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) Fh[1 + a] = (st.p - trac) * nh[a];
    Fh[4] = k == -2 ? tv[3] : (PERT ? R(0) : -A.ph.bottom_flux);
#pragma unroll
    for (int v = 0; v < 5; ++v) A.Fc_out[(o * 5 + v) * N2 + t] = sgn * mag * Fh[v];
    return;
  }
  const int Fn = code >> 3, tp = map_face_pt<N>(t, code & 7);
  const size_t oL = (size_t)e * 6 + F, oR = (size_t)k * 6 + Fn;
  R qL[5], qR[5], tvL[4], tvR[4];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = __ldg(A.T + (oL * 5 + v) * N2 + t);
    qR[v] = __ldg(A.T + (oR * 5 + v) * N2 + tp);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    tvL[v] = __ldg(A.Tv + (oL * 4 + v) * N2 + t);
    tvR[v] = __ldg(A.Tv + (oR * 4 + v) * N2 + tp);
  }
  R r0L = R(0), E0L = R(0), r0R = R(0), E0R = R(0);
  if (PERT) {
    r0L = (R)__ldg(A.bg.bgT + (oL * 2) * N2 + t);
    E0L = (R)__ldg(A.bg.bgT + (oL * 2 + 1) * N2 + t);
    r0R = (R)__ldg(A.bg.bgT + (oR * 2) * N2 + tp);
    E0R = (R)__ldg(A.bg.bgT + (oR * 2 + 1) * N2 + tp);
  }
  const R* Sl = A.m.Sf + ((size_t)e * 3 + D) * 3 * (N + 1) * N2;
  R s3[3];
#pragma unroll
  for (int n = 0; n < 3; ++n) s3[n] = __ldg(Sl + (n * (N + 1) + (side ? N : 0)) * N2 + t);
  const R sgn = side ? R(1) : R(-1);
  const R mag = sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
  const R im = qdiv(sgn, mag);
  const R nh[3] = {im * s3[0], im * s3[1], im * s3[2]};
  const Pt<R> sL = point_state<PERT>(qL, r0L, E0L, A.ph);
  const Pt<R> sR = point_state<PERT>(qR, r0R, E0R, A.ph);
  R Fh[5];
  rusanov<PERT>(qL, sL, r0L, E0L, qR, sR, r0R, E0R, nh, A.ph, Fh);
#pragma unroll
  for (int v = 1; v < 5; ++v) Fh[v] -= R(0.5) * (tvL[v - 1] - tvR[v - 1]);  // tvR = F_v,R . (-n)
  const R sR_ = (Fn & 1) ? R(1) : R(-1);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    A.Fc_out[(oL * 5 + v) * N2 + t] = sgn * mag * Fh[v];
    A.Fc_out[(oR * 5 + v) * N2 + tp] = -sR_ * mag * Fh[v];
  }
}

template <int N, bool PERT, class R>
__global__ void __launch_bounds__(64) k_face(const KArgs<R> A, const int2* __restrict__ faces, int nf, int nw) {
  face_point<N, PERT, R>(A, faces, nf, nw, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
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
  static cudaError_t face(const KArgs<R>& A, const int2* faces, int nf, int nw, cudaStream_t st) {
    if (!kFaceKernel || nf + nw == 0) return cudaSuccess;
    if (A.Fc_out == nullptr || A.T == nullptr || A.Tv == nullptr) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)(nf + nw) * N * N;
    // 64-thread CTAs (p = 3: 1 % faster than 128, 2.5 % faster than 256)
    k_face<N, PERT, R><<<(unsigned)((n + 63) / 64), 64, 0, st>>>(A, faces, nf, nw);
    return cudaGetLastError();
  }
  static cudaError_t grad(const KArgs<R>& A, cudaStream_t st) {
    if (A.m.E == 0) return cudaSuccess;
    const size_t sm = (size_t)L::total_grad * sizeof(R);
    // the radiative-diffusivity profile is a compile-time option of the FP32 kernels (FP64 checks it
    // at run time)
    if constexpr (sizeof(R) == 8) {
      return grad_kr<true>(A, st, sm);
    } else {
      return A.m.kr != nullptr ? grad_kr<true>(A, st, sm) : grad_kr<false>(A, st, sm);
    }
  }
  template <bool KR>
  static cudaError_t grad_kr(const KArgs<R>& A, cudaStream_t st, size_t sm) {
    cudaError_t e = cudaFuncSetAttribute(k_grad<N, PERT, R, EPB, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_grad<N, PERT, R, EPB, KR><<<blocks(A.m.E), threads, sm, st>>>(A);
    return cudaGetLastError();
  }
  template <int MODE>
  static cudaError_t resid(const KArgs<R>& A, cudaStream_t st) {
    if (A.m.E == 0) return cudaSuccess;
    if (A.G_in == nullptr) return cudaErrorInvalidValue;  // the residual kernel reads the gradient record
    if (kFaceKernel && A.Fc == nullptr) return cudaErrorInvalidValue;  // and the common face fluxes
    const size_t sm = (size_t)Layout<N, PERT, R, EPB, true>::total_resid * sizeof(R);
    if constexpr (sizeof(R) == 8) {
      return resid_kr<MODE, true>(A, st, sm);
    } else {
      return A.m.kr != nullptr ? resid_kr<MODE, true>(A, st, sm) : resid_kr<MODE, false>(A, st, sm);
    }
  }
  template <int MODE, bool KR>
  static cudaError_t resid_kr(const KArgs<R>& A, cudaStream_t st, size_t sm) {
    cudaError_t e =
        cudaFuncSetAttribute(k_resid<N, PERT, R, EPB, MODE, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_resid<N, PERT, R, EPB, MODE, KR><<<blocks(A.m.E), threads, sm, st>>>(A);
    return cudaGetLastError();
  }
};

}  // namespace chorus
