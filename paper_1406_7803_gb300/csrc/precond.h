// precond.h -- launch wrappers of the learned preconditioner (precond.cu).
#pragma once

#include "kernels.h"

namespace fde {

constexpr int kPrecondWidth = 64;
constexpr int kPrecondParams = kPrecondWidth * 3 + kPrecondWidth + 2 * (kPrecondWidth * kPrecondWidth + kPrecondWidth) +
                               kPrecondWidth + 1;

// W[j][g] = K(y) exp(MLP(f)) R[j][g] for nb rows (in place allowed); wb: bf16 weights.
template <typename T>
void launch_precond_apply(const cplx<T>* R, int ldr, const T* kin, const double* tband, const double* sumsq, int nb,
                          int K, const void* wb, cplx<T>* W, int ldw, cudaStream_t st);

// Inference on the tensor cores (default) or on the CUDA cores; status bits of the
// tensor-core inference (read and cleared, synchronising); its mbarrier poll limit.
void set_precond_tensor_cores(bool on);
bool precond_tensor_cores();
unsigned precond_tc_take_status(cudaStream_t st);
bool set_precond_tc_spin(long long polls);

// Loss sum_j min_a |a m R_j - D_j|^2 / |D_j|^2 (a complex) and its gradient over nb x K pairs;
// part: precond_grad_blocks(nb, K) x (kPrecondParams + 1) floats; awork:
// precond_alpha_work(nb) doubles; wtmp: nb x K complex (the tensor-core path's m R with the
// master weights); out[kPrecondParams + 1] (gradient, then the loss) is overwritten.  Runs on
// the tensor cores when precond_tensor_cores(), else on the CUDA cores.
int precond_grad_blocks(int nb, int K);
size_t precond_alpha_work(int nb);
template <typename T>
void launch_precond_grad(const cplx<T>* R, const cplx<T>* D, int nb, int K, const T* kin, const double* tband,
                         const double* sumsq, const double* dnorm2, const float* wf, float* part, double* awork,
                         cplx<T>* wtmp, double* out, cudaStream_t st);

void launch_precond_adam(float* wf, void* wb, const double* grad, float* m1, float* m2, float lr, int step,
                         cudaStream_t st);
void launch_precond_to_bf16(const float* wf, void* wb, float* rounded, cudaStream_t st);

}  // namespace fde
