// Tensor-core forward pass of the closure network (135 -> 128 -> 128 -> 135, SiLU) for element
// states and plain sample rows, on the fifth-generation tensor cores: tcgen05.mma kind::f16 with
// BF16 operands in shared memory and FP32 accumulators in tensor memory (TMEM).
//
// Numerics: each layer's input is rounded to BF16 (round to nearest even) before its product with
// the BF16 weights; products are exact and accumulate in FP32; bias, SiLU and the output scale are
// applied in FP32 to the accumulator.  Element inputs are scaled by the reciprocal of the input
// scale (FP32; FP64 where the background is subtracted first).
//
// Work decomposition: persistent CTAs of 128 threads; a tile is 128 samples (the MMA M).  The three
// weight matrices are copied once per CTA into shared memory in the MMA operand layout; per tile
// the inputs are converted into the A operand, and the three products run back to back, each
// followed by an epilogue in which warp w reads TMEM lanes 32w..32w+31 (its tile rows).
//
// Operand layout (K-major, no swizzle): 8 x 8 BF16 core matrices of 128 contiguous bytes (8 rows of
// 16 bytes); the core matrix of row group g and K chunk c of an R x K operand starts at byte
// (g * K/8 + c) * 128, so the descriptors use a leading (K) byte offset of 128 and a stride (row
// group) byte offset of K/8 * 128.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "closure.h"

namespace chorus {
namespace {

constexpr int TM = 128;   // samples per tile (MMA M)
constexpr int NI = ClosureLayout::NI, NH = ClosureLayout::NH, NO = ClosureLayout::NO;
constexpr int KA = 144;   // 135 inputs padded to a multiple of 16 (the MMA K step)
constexpr int NOP = 144;  // 135 outputs padded to a multiple of 16 (MMA N)
constexpr int kTmemCols = 256;

// shared-memory plan (bytes); every operand block starts on a 1024-byte boundary
constexpr int oW1 = 0;                       // [NH][KA]
constexpr int oW2 = oW1 + NH * KA * 2;       // [NH][NH]
constexpr int oW3 = oW2 + NH * NH * 2;       // [NOP][NH]
constexpr int oA = oW3 + NOP * NH * 2;       // [TM][KA]   layer-1 input
constexpr int oH = oA + TM * KA * 2;         // [TM][NH]   layer-2 / layer-3 input
constexpr int oEnd = oH + TM * NH * 2;
constexpr int kOutStride = NO;               // FP32 output staging rows (overlays A and H); odd stride
static_assert(TM * kOutStride * 4 <= oEnd - oA, "output staging must fit in the A and H blocks");
static_assert(oW2 % 1024 == 0 && oW3 % 1024 == 0 && oA % 1024 == 0 && oH % 1024 == 0, "operand alignment");
constexpr size_t kSmemBytes = (size_t)oEnd + 1024;  // + alignment slack

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element index (BF16 units) of (row, k) in an R x K operand block
__device__ __forceinline__ int opnd(int row, int k, int K) {
  return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start address, leading byte offset 128 (next core matrix along
// K), stride byte offset K/8*128 (next 8-row group), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, int K) {
  const uint64_t sbo = (uint64_t)(K / 8) * 128;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both K-major, N, M = 128
__host__ __device__ constexpr uint32_t idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded poll of the given phase parity: at most 2^24 polls (about a second with the back-off).
__device__ __forceinline__ bool poll_phase(uint64_t* bar, uint32_t parity) {
  const uint32_t a = saddr(bar);
  for (uint32_t it = 0; it < (1u << 24); ++it) {
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

// Bounded wait for the given phase parity; false (and *err set) if the limit ran out, after one more
// bounded wait for the operation still in flight (the caller then frees its TMEM and returns).
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, unsigned* err) {
  if (poll_phase(bar, parity)) return true;
  if (err) atomicOr(err, 2u);
  poll_phase(bar, parity);
  return false;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

struct Rec {
  const __nv_bfloat16* W[3];
  const float* b[3];
  const float* in_scale;
  const float* out_scale;
};

__device__ __forceinline__ Rec rec_of(const void* w) {
  const unsigned char* p = (const unsigned char*)w;
  Rec r;
  r.W[0] = (const __nv_bfloat16*)(p + ClosureLayout::oW1);
  r.W[1] = (const __nv_bfloat16*)(p + ClosureLayout::oW2);
  r.W[2] = (const __nv_bfloat16*)(p + ClosureLayout::oW3);
  r.b[0] = (const float*)(p + ClosureLayout::ob1);
  r.b[1] = (const float*)(p + ClosureLayout::ob2);
  r.b[2] = (const float*)(p + ClosureLayout::ob3);
  r.in_scale = (const float*)(p + ClosureLayout::oin);
  r.out_scale = (const float*)(p + ClosureLayout::oout);
  return r;
}

// copy a row-major [n_out][n_in] BF16 matrix into the operand block [n_pad][k_pad], zero-padded
__device__ void stage_weights(const __nv_bfloat16* W, int n_out, int n_in, int n_pad, int k_pad, __nv_bfloat16* dst) {
  for (int i = threadIdx.x; i < n_pad * k_pad; i += blockDim.x) {
    const int n = i / k_pad, k = i % k_pad;
    dst[opnd(n, k, k_pad)] = (n < n_out && k < n_in) ? W[n * n_in + k] : __float2bfloat16_rn(0.0f);
  }
}

// Epilogue of a hidden layer: z = acc + b, h = SiLU(z), written as BF16 into the H operand block.
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, int col0, const float* bias, __nv_bfloat16* H) {
  const int w = threadIdx.x >> 5, row = threadIdx.x;
  const uint32_t lane = (uint32_t)(32 * w) << 16;
#pragma unroll 1
  for (int c = 0; c < NH; c += 16) {
    float v[16];
    tmem_ld16(tmem + lane + (uint32_t)(col0 + c), v);
    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(silu(v[i] + __ldg(bias + c + i)));
    // two 16-byte core-matrix rows (columns c..c+7 and c+8..c+15)
    *reinterpret_cast<uint4*>(H + opnd(row, c, NH)) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(H + opnd(row, c + 8, NH)) = *reinterpret_cast<const uint4*>(h + 8);
  }
}

// Forward pass over rows [0, n).
// Source: ELEM = true reads element states Q[e][135] (q' = Q - Q0 when Q0 != nullptr) and divides by
// in_scale per variable; false reads sample rows X[r][135] as they are.  Output: ELEM = true writes
// or adds out_scale * y into R[e][135]; false stores y into Y[r][135].
template <bool ELEM, class R>
__global__ void __launch_bounds__(128, 1)
    k_mlp_tc(const void* weights, const R* __restrict__ Q, const double* __restrict__ Q0, R* __restrict__ out,
             int64_t n, int accumulate, unsigned* err) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __nv_bfloat16* sW1 = (__nv_bfloat16*)(sm + oW1);
  __nv_bfloat16* sW2 = (__nv_bfloat16*)(sm + oW2);
  __nv_bfloat16* sW3 = (__nv_bfloat16*)(sm + oW3);
  __nv_bfloat16* sA = (__nv_bfloat16*)(sm + oA);
  __nv_bfloat16* sH = (__nv_bfloat16*)(sm + oH);
  float* sOut = (float*)(sm + oA);
  const Rec w = rec_of(weights);
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_holder)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  stage_weights(w.W[0], NH, NI, NH, KA, sW1);
  stage_weights(w.W[1], NH, NH, NH, NH, sW2);
  stage_weights(w.W[2], NO, NH, NOP, NH, sW3);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_holder;
  const uint32_t dA = tmem, dB = tmem + 128;  // accumulator columns: layers 1 and 3 in [0, 144), layer 2 in [128, 256)
  uint32_t phase = 0;
  const int64_t n_tiles = (n + TM - 1) / TM;
  float inv_in[5];
  double inv_in64[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    inv_in64[v] = 1.0 / (double)__ldg(w.in_scale + v);
    inv_in[v] = (float)inv_in64[v];
  }

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t r0 = t * TM;
    const int rows = (int)((n - r0) < TM ? (n - r0) : TM);
    // ---- layer-1 input, one 8-column chunk per thread step: 8 consecutive inputs of a row (coalesced
    // across the warp), scaled, rounded to BF16, stored as one 16-byte row of a core matrix
#pragma unroll 6
    for (int i = threadIdx.x; i < TM * (KA / 8); i += blockDim.x) {  // 18 steps: six chunks' loads in flight
      const int r = i / (KA / 8), c = i % (KA / 8);
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = 8 * c + u;
        float x = 0.0f;
        if (r < rows && k < NI) {
          const int64_t gi = (r0 + r) * NI + k;
          if (ELEM) {
            if (Q0) x = (float)(((double)Q[gi] - Q0[gi]) * inv_in64[k / 27]);  // the difference needs FP64
            else x = (float)Q[gi] * inv_in[k / 27];
          } else {
            x = (float)Q[gi];
          }
        }
        v[u] = __float2bfloat16_rn(x);
      }
      *reinterpret_cast<uint4*>(sA + opnd(r, 8 * c, KA)) = *reinterpret_cast<const uint4*>(v);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    // ---- three products, each followed by its epilogue
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      if (threadIdx.x == 0) {
        fence_after();
        const uint32_t a_base = saddr(layer == 0 ? sA : sH);
        const uint32_t b_base = saddr(layer == 0 ? sW1 : (layer == 1 ? sW2 : sW3));
        const int K = layer == 0 ? KA : NH;
        const int N = layer == 2 ? NOP : NH;
        const uint32_t d = layer == 1 ? dB : dA;
        for (int kk = 0; kk < K / 16; ++kk)  // K step 16: two core matrices of 128 bytes
          mma(d, sdesc(a_base + kk * 256, K), sdesc(b_base + kk * 256, K), idesc(N), kk > 0);
        mma_commit(&bar);
      }
      __syncwarp();
      if (!wait_phase(&bar, phase, err)) abort_flag = 1;
      phase ^= 1u;
      __syncthreads();
      if (abort_flag) break;
      fence_after();
      if (layer < 2) {
        hidden_epilogue(layer == 1 ? dB : dA, 0, w.b[layer], sH);
        fence_async_smem();
        fence_before();
        __syncthreads();
      } else {
        // output layer: y = acc + b3 (columns 0..134), staged as FP32 rows for coalesced stores
        const int row = threadIdx.x;
        const uint32_t lane = (uint32_t)(32 * warp) << 16;
#pragma unroll 1
        for (int c = 0; c < NOP; c += 16) {
          float v[16];
          tmem_ld16(dA + lane + (uint32_t)c, v);
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c + i < NO) sOut[row * kOutStride + c + i] = v[i] + __ldg(w.b[2] + c + i);
        }
        fence_before();
        __syncthreads();
        for (int i = threadIdx.x; i < rows * NO; i += blockDim.x) {
          const int r = i / NO, k = i % NO;
          const float y = sOut[r * kOutStride + k];
          R* o = out + (r0 + r) * NO + k;
          if (ELEM) {
            const R c = (R)(y * __ldg(w.out_scale + k / 27));
            *o = accumulate ? *o + c : c;
          } else {
            *o = (R)y;
          }
        }
        __syncthreads();  // the staging rows overlay the next tile's A block
      }
    }
    if (abort_flag) break;
  }
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

template <bool ELEM, class R>
cudaError_t launch_tc(const void* weights, const R* Q, const double* Q0, R* out, int64_t n, int accumulate,
                      unsigned* err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<ELEM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + TM - 1) / TM;
  const unsigned grid = (unsigned)(tiles < sm_count() ? tiles : sm_count());
  k_mlp_tc<ELEM, R><<<grid, 128, kSmemBytes, st>>>(weights, Q, Q0, out, n, accumulate, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_elements_tc(int prec, const void* weights, const void* Q, const double* Q0, void* out, int64_t E,
                            int accumulate, unsigned* err, cudaStream_t st) {
  if (prec == 0)
    return launch_tc<true, double>(weights, (const double*)Q, Q0, (double*)out, E, accumulate, err, st);
  return launch_tc<true, float>(weights, (const float*)Q, nullptr, (float*)out, E, accumulate, err, st);
}

cudaError_t mlp_forward_tc(const void* weights, const float* X, float* Y, int64_t n, unsigned* err, cudaStream_t st) {
  return launch_tc<false, float>(weights, X, nullptr, Y, n, 0, err, st);
}

}  // namespace chorus
