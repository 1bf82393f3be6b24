// Learned subgrid closure: record layout and entry points shared by closure.cu and the C ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <vector>

namespace chorus {

// Closure record (device, caller-owned): BF16 weights W1 [128][135], W2 [128][128], W3 [135][128],
// FP32 biases b1 [128], b2 [128], b3 [135], FP32 input scales [5] and output scales [5].
// The master parameter vector of training (FP32) lists W1, W2, W3, b1, b2, b3 in that order.
struct ClosureLayout {
  static constexpr int NI = 135, NH = 128, NO = 135;
  static constexpr size_t oW1 = 0;
  static constexpr size_t oW2 = oW1 + 2 * NH * NI;
  static constexpr size_t oW3 = oW2 + 2 * NH * NH;
  static constexpr size_t ob1 = oW3 + 2 * NO * NH;
  static constexpr size_t ob2 = ob1 + 4 * NH;
  static constexpr size_t ob3 = ob2 + 4 * NH;
  static constexpr size_t oin = ob3 + 4 * NO;
  static constexpr size_t oout = oin + 4 * 5;
  static constexpr size_t total_bytes = (oout + 4 * 5 + 15) / 16 * 16;
  static constexpr int mW1 = 0, mW2 = mW1 + NH * NI, mW3 = mW2 + NH * NH, mb1 = mW3 + NO * NH;
  static constexpr int mb2 = mb1 + NH, mb3 = mb2 + NH, n_params = mb3 + NO;
};

__host__ __device__ inline float closure_load_param(const void* w, int i) {
  const unsigned char* p = (const unsigned char*)w;
  using L = ClosureLayout;
  if (i < L::mb1) return __bfloat162float(((const __nv_bfloat16*)(p + L::oW1))[i]);  // W1, W2, W3 contiguous
  return ((const float*)(p + L::ob1))[i - L::mb1];                                  // b1, b2, b3 contiguous
}

__device__ inline void closure_store_param(void* w, int i, float v) {
  unsigned char* p = (unsigned char*)w;
  using L = ClosureLayout;
  if (i < L::mb1)
    ((__nv_bfloat16*)(p + L::oW1))[i] = __float2bfloat16_rn(v);
  else
    ((float*)(p + L::ob1))[i - L::mb1] = v;
}

size_t closure_record_bytes();
std::vector<double> projection_matrix(int Nf, int Nc);
std::vector<unsigned char> init_record(uint64_t seed, const float* in_scale, const float* out_scale);

cudaError_t launch_project(int64_t E, int Nf, int Nc, int prec, const void* Qf, void* Qc, const double* add_f,
                           const double* sub_c, int nvar, cudaStream_t st);
cudaError_t mlp_forward(const void* weights, const float* X, float* Y, int64_t n, cudaStream_t st);
// tensor-core forward (closure_tc.cu): BF16 layer inputs, FP32 accumulation; err (device) receives
// bit 2 if a bounded wait ran out (may be null)
cudaError_t mlp_elements_tc(int prec, const void* weights, const void* Q, const double* Q0, void* out, int64_t E,
                            int accumulate, unsigned* err, cudaStream_t st);
cudaError_t mlp_forward_tc(const void* weights, const float* X, float* Y, int64_t n, unsigned* err, cudaStream_t st);
cudaError_t mlp_backward(const void* weights, const float* X, const float* T, int64_t n, int64_t row0, int64_t rows,
                         float* grad, double* loss, cudaStream_t st);
cudaError_t make_pairs(int prec, const void* weights, const void* Qc, const double* Q0, const void* PRf,
                       const void* Rc, float* X, float* Y, int64_t E, cudaStream_t st);
cudaError_t adam(float* master, float* m1, float* m2, const float* grad, void* weights, float lr, float b1, float b2,
                 float eps, int64_t t, cudaStream_t st);
cudaError_t load_master(const void* weights, float* master, cudaStream_t st);

}  // namespace chorus
