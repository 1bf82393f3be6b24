// Persistent batch stage: one cooperative launch runs an RK stage of every order group of a batch
// (up to four union meshes, p = 2..5).  Its CTAs pull (order, tile) work items of each phase from a
// counter (the orders' tiles in one list, the most expensive order first) and run the same tile
// functions as the per-order kernels, specialised per order by template dispatch; between the phases
// (traces, lifting, face fluxes, residual) they meet at a grid barrier whose spin is bounded: a
// barrier that runs out of polls sets the error flag (CHORUS_ETIMEOUT) and the CTA stops, so that
// every other CTA's next barrier runs out too and the launch ends.  Nothing traps.
#include <cuda_runtime.h>

#include <algorithm>

#include "mesh_state.h"
#include "sd_kernels.cuh"

namespace chorus {
namespace {

constexpr int kPThreads = 128;     // threads per CTA, every order and phase
constexpr int kPMinBlocks = 3;     // resident CTAs per SM asked of the compiler (register cap 170)
// elements per CTA of order slot s = p - 2 in both element phases: the CTA stays within 128 threads
template <int S>
__host__ __device__ constexpr int p_epb() { return S == 0 ? 14 : S == 1 ? 8 : S == 2 ? 5 : 3; }

struct PersistArgs {
  KArgs<float> grad[4], face[4], resid[4];  // slot p - 2; an absent order has no work items
  const int2* faces[4];
  int nf[4], nw[4];
  int64_t items[4][4];  // [phase: traces, lifting, faces, residual][slot]
  int trace;            // 1: the stage starts with the traces of its input state
  unsigned* sync;       // [0] grid-barrier arrivals, [1 + phase] work counter (zero at launch)
  unsigned* err;        // the error flags (bit 0: a bounded wait gave up) and, in err[1], the wait limit
};
static_assert(sizeof(PersistArgs) <= 32000, "kernel parameters above the 32 KB limit");

// Bounded grid barrier: all CTAs of the launch arrive (the k-th barrier waits for k x gridDim.x
// arrivals).  The writes before it, generic and bulk, are visible to every CTA after it, for generic
// loads and bulk copies alike.  Returns false (flag set) when the polls run out.
__device__ bool grid_sync(unsigned* count, unsigned target, unsigned* err, uint32_t polls) {
  __shared__ int ok_s;
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    int ok = 0;
    for (uint32_t i = 0; i < polls; ++i) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) {
        ok = 1;
        break;
      }
      __nanosleep(i < 64 ? 32 : 256);
    }
    if (!ok) atomicOr(err, 1u);
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The work items of order slot S (N = S + 3 solution points per direction), one function per phase
// kept out of line: inlined into one kernel body, the 16 (phase, order) tile functions spill 3.3 KB a
// thread; out of line, 0-0.5 KB each.
template <int S>
__device__ __noinline__ void trace_item(const PersistArgs& P, int64_t t) {
  const KArgs<float>& A = P.grad[S];
  trace_tile<S + 3, float, p_epb<S>()>(A.m, A.ops, A.q, const_cast<float*>(A.T), t);
}
template <int S>
__device__ __noinline__ void grad_item(const PersistArgs& P, int64_t t, uint64_t* bar, uint32_t& pbar) {
  grad_tile<S + 3, true, float, p_epb<S>(), false>(P.grad[S], t, bar, pbar);
}
template <int S>
__device__ __noinline__ void face_item(const PersistArgs& P, int64_t t) {
  face_point<S + 3, true, float>(P.face[S], P.faces[S], P.nf[S], P.nw[S], t * kPThreads + threadIdx.x);
}
template <int S>
__device__ __noinline__ void resid_item(const PersistArgs& P, int64_t t, uint64_t* bar, uint64_t* barS, uint32_t& pbar,
                                        uint32_t& pbarS) {
  resid_tile<S + 3, true, float, p_epb<S>(), kModeRK, false>(P.resid[S], t, bar, barS, pbar, pbarS);
}
template <int S>
__device__ __forceinline__ void run_item(const PersistArgs& P, int phase, int64_t t, uint64_t* bar, uint64_t* barS,
                                         uint32_t& pbar, uint32_t& pbarS) {
  if (phase == 0) trace_item<S>(P, t);
  else if (phase == 1) grad_item<S>(P, t, bar, pbar);
  else if (phase == 2) face_item<S>(P, t);
  else resid_item<S>(P, t, bar, barS, pbar, pbarS);
}

__global__ void __launch_bounds__(kPThreads, kPMinBlocks) k_batch_stage(const __grid_constant__ PersistArgs P) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(8) uint64_t barS[2];
  __shared__ int64_t s_item;
  __shared__ int s_stop;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    mbar_init(&barS[0]);
    mbar_init(&barS[1]);
    s_stop = 0;
  }
  __syncthreads();
  uint32_t pbar = 0, pbarS = 0;
  unsigned barriers = 0;
  const uint32_t polls = wait_polls(P.err);  // the grid barriers' limit: the staging waits' own
  for (int phase = P.trace ? 0 : 1; phase < 4; ++phase) {
    const int64_t total = P.items[phase][0] + P.items[phase][1] + P.items[phase][2] + P.items[phase][3];
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(P.sync + 1 + phase, 1u);
      __syncthreads();
      const int64_t it = s_item;
      const int stop = s_stop;
      __syncthreads();  // every thread has read s_item before thread 0 takes the next one
      if (it >= total || stop) break;
      int slot = 3;  // the list holds p = 5's items first, then p = 4, 3, 2
      int64_t t = it;
      while (slot > 0 && t >= P.items[phase][slot]) {
        t -= P.items[phase][slot];
        --slot;
      }
      if (slot == 3) run_item<3>(P, phase, t, &bar, barS, pbar, pbarS);
      else if (slot == 2) run_item<2>(P, phase, t, &bar, barS, pbar, pbarS);
      else if (slot == 1) run_item<1>(P, phase, t, &bar, barS, pbar, pbarS);
      else run_item<0>(P, phase, t, &bar, barS, pbar, pbarS);
      __syncthreads();  // the tile's shared memory is free for the next one
      if (threadIdx.x == 0 && (*(volatile unsigned*)P.err & 1u)) s_stop = 1;  // a bounded wait gave up
    }
    if (phase == 1 && threadIdx.x == 0) bulk_wait_all();  // the gradient records are written out
    if (phase < 3 && !grid_sync(P.sync, ++barriers * gridDim.x, P.err, polls)) return;
  }
}

}  // namespace

namespace {

template <int S>
constexpr size_t slot_smem() {
  constexpr int N = S + 3, EPB = p_epb<S>();
  return std::max((size_t)Layout<N, true, float, EPB>::total_grad,
                  (size_t)Layout<N, true, float, EPB, true>::total_resid) * sizeof(float);
}
constexpr size_t kPSmem = std::max(std::max(slot_smem<0>(), slot_smem<1>()), std::max(slot_smem<2>(), slot_smem<3>()));

template <int S>
int64_t tiles_of(int64_t E) {
  return (E + p_epb<S>() - 1) / p_epb<S>();
}
int64_t tiles_of_slot(int s, int64_t E) {
  return s == 0 ? tiles_of<0>(E) : s == 1 ? tiles_of<1>(E) : s == 2 ? tiles_of<2>(E) : tiles_of<3>(E);
}

}  // namespace

int persist_grid() {
  static int grid = -1;
  if (grid >= 0) return grid;
  int dev = 0, sms = 0, coop = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaFuncSetAttribute(k_batch_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_stage, kPThreads, kPSmem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    grid = 0;
    return grid;
  }
  grid = nb * sms;
  return grid;
}

chorus_status persist_rk3_step(StagePtrs* const groups[4], double dt, unsigned* sync, cudaStream_t st) {
  const int grid = persist_grid();
  if (grid <= 0) return CHORUS_EUNSUPPORTED;
  if (!sync) return CHORUS_EINVAL;
  unsigned* err = nullptr;
  for (int s = 0; s < 4; ++s) {
    if (!groups[s]) continue;
    if (groups[s]->m.kr != nullptr) return CHORUS_EUNSUPPORTED;  // built for a constant kappa_r
    if (!err) err = groups[s]->err;
  }
  if (!err) return CHORUS_EINVAL;
  const std::vector<Stage>& stg = stages_of(0);
  for (int k = 0; k < (int)stg.size(); ++k) {
    const Stage& sg = stg[k];
    PersistArgs P{};
    for (int s = 0; s < 4; ++s) {
      if (!groups[s]) continue;
      const StagePtrs& G = *groups[s];
      const int N = s + 3;
      float* Tc = (k % 2 == 0) ? G.Ta : G.Tb;  // the traces of the stage's input state
      float* Tn = (k % 2 == 0) ? G.Tb : G.Ta;
      KArgs<float>& a = P.grad[s];
      a.m = G.m; a.ops = G.ops; a.ph = G.ph; a.bg = G.bg; a.q = G.buf[sg.src]; a.T = Tc; a.Tv_out = G.Tv;
      a.G_out = G.G; a.Fc_out = G.Fc; a.err = err;
      KArgs<float>& f = P.face[s];
      f.m = G.m; f.ph = G.ph; f.bg = G.bg; f.T = Tc; f.Tv = G.Tv; f.Fc_out = G.Fc; f.err = err;
      KArgs<float>& r = P.resid[s];
      r.m = G.m; r.ops = G.ops; r.ph = G.ph; r.bg = G.bg; r.q = G.buf[sg.src]; r.T = Tc; r.Tv = G.Tv;
      r.out = G.buf[sg.dst]; r.T_out = Tn; r.G_in = G.G; r.Fc = G.Fc;
      r.un = G.buf[sg.un]; r.a = (float)sg.a; r.b = (float)sg.b; r.c = (float)sg.c; r.dt = (float)dt; r.err = err;
      P.faces[s] = G.faces;
      P.nf[s] = G.nf;
      P.nw[s] = G.nw;
      const int64_t tiles = tiles_of_slot(s, G.m.E);
      P.items[0][s] = k == 0 ? tiles : 0;
      P.items[1][s] = tiles;
      P.items[2][s] = ((int64_t)(G.nf + G.nw) * N * N + kPThreads - 1) / kPThreads;
      P.items[3][s] = tiles;
    }
    P.trace = k == 0;
    P.sync = sync;
    P.err = err;
    if (cudaMemsetAsync(sync, 0, 5 * sizeof(unsigned), st) != cudaSuccess) return CHORUS_ECUDA;
    void* args[] = {&P};
    if (cudaLaunchCooperativeKernel((const void*)k_batch_stage, dim3(grid), dim3(kPThreads), args, kPSmem, st) !=
        cudaSuccess) {
      cudaGetLastError();
      return CHORUS_ECUDA;
    }
  }
  return CHORUS_OK;
}

}  // namespace chorus
