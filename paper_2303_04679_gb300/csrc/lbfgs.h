// Launchers of the limited-memory BFGS vector kernels (lbfgs.cu).
#pragma once
#include <cuda_runtime.h>

namespace modil {

// out = (mul ? *mul : 1) * (x . y); part: lb_dot_partials() doubles of scratch.
template <class T>
cudaError_t lb_dot(const T* x, const T* y, long long n, double* part, const double* mul, double* out,
                   cudaStream_t s);
// y += sign * (*a - (b ? *b : 0)) * x.
template <class T>
cudaError_t lb_axpy(T* y, const T* x, const double* a, const double* b, double sign, long long n,
                    cudaStream_t s);
// r = (*num / *den) * q.
template <class T>
cudaError_t lb_scale(T* r, const T* q, const double* num, const double* den, long long n, cudaStream_t s);
// z = x + a * y.
template <class T>
cudaError_t lb_axpby(T* z, const T* x, const T* y, double a, long long n, cudaStream_t s);
// z = x - y.
template <class T>
cudaError_t lb_sub(T* z, const T* x, const T* y, long long n, cudaStream_t s);
// z = a * x
template <class T>
cudaError_t lb_mul(T* z, const T* x, double a, long long n, cudaStream_t s);
int lb_dot_partials();
// out[d] = va[d] . vb[d] for d < ndots (device pointer arrays); part:
// lb_mdot_partials(ndots) doubles of scratch.
template <class T>
cudaError_t lb_mdot(const T* const* va, const T* const* vb, int ndots, long long n, double* part, double* out,
                    cudaStream_t s);
int lb_mdot_partials(int ndots);
// r = c0 g + sum_k coef[k] v[k] (device pointer and coefficient arrays).
template <class T>
cudaError_t lb_combine(T* r, const T* g, double c0, const T* const* v, const double* coef, int nv, long long n,
                       cudaStream_t s);

}  // namespace modil
