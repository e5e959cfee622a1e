// Vector kernels of the limited-memory BFGS optimiser over a problem's level
// arena (all fields and levels of one instance back to back): dot products
// reduced in FP64 in a fixed order (deterministic), and the axpy forms of the
// two-loop recursion whose coefficients stay on the device (no host round
// trip inside the recursion).
#include "lbfgs.h"
#include "modil_dev.cuh"

namespace modil {

constexpr int kDotBlocks = 2 * 152, kDotNT = 256;

// Per-block FP64 partial sums of x . y (grid-stride, fixed order).
template <class T>
__global__ void __launch_bounds__(kDotNT) k_dot(const T* __restrict__ x, const T* __restrict__ y,
                                                long long n, double* __restrict__ part) {
  __shared__ double ws[kDotNT / 32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)kDotNT + threadIdx.x; i < n; i += (long long)gridDim.x * kDotNT)
    s = fma((double)x[i], (double)y[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kDotNT / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

// out = (mul ? *mul : 1) * sum of the partials (one warp, fixed order).
__global__ void k_dot_final(const double* __restrict__ part, int nb, const double* mul, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += part[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = mul ? *mul * s : s;
}

// y += sign * (a - (b ? b : 0)) * x, coefficients read on the device.
template <class T>
__global__ void k_axpy_dev(T* __restrict__ y, const T* __restrict__ x, const double* a, const double* b,
                           double sign, long long n) {
  const double c = sign * (*a - (b ? *b : 0.0));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)fma(c, (double)x[i], (double)y[i]);
}

// r = (num / den) * q.
template <class T>
__global__ void k_scale_dev(T* __restrict__ r, const T* __restrict__ q, const double* num, const double* den,
                            long long n) {
  const double c = *num / *den;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = (T)(c * (double)q[i]);
}

// z = x + a * y (host coefficient).
template <class T>
__global__ void k_axpby(T* __restrict__ z, const T* __restrict__ x, const T* __restrict__ y, double a,
                        long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = (T)fma(a, (double)y[i], (double)x[i]);
}

// z = a * x (host coefficient).
template <class T>
__global__ void k_mul(T* __restrict__ z, const T* __restrict__ x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = (T)(a * (double)x[i]);
}

// z = x - y.
template <class T>
__global__ void k_sub(T* __restrict__ z, const T* __restrict__ x, const T* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = x[i] - y[i];
}

// Many dot products in one launch: block (c, d) sums chunk c of dot d (the
// chunks split n evenly, each summed in a fixed order); k_mdot_final adds a
// dot's chunks in order.  The vector pointers are device arrays.
constexpr int kMdotChunks = 64, kMdotNT = 256;

template <class T>
__global__ void __launch_bounds__(kMdotNT) k_mdot(const T* const* __restrict__ va, const T* const* __restrict__ vb,
                                                  long long n, double* __restrict__ part) {
  __shared__ double ws[kMdotNT / 32];
  const int d = blockIdx.y;
  const T* __restrict__ x = va[d];
  const T* __restrict__ y = vb[d];
  const long long len = (n + kMdotChunks - 1) / kMdotChunks;
  const long long i0 = blockIdx.x * len, i1 = min(n, i0 + len);
  double s = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kMdotNT) s = fma((double)x[i], (double)y[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kMdotNT / 32; ++w) t += ws[w];
    part[(long long)d * kMdotChunks + blockIdx.x] = t;
  }
}

__global__ void k_mdot_final(const double* __restrict__ part, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < kMdotChunks; i += 32) s += part[(long long)blockIdx.x * kMdotChunks + i];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// r = c0 g + sum_i coef[i] v_i (the compact form's H g): each element reads
// the nv vectors in a fixed order.
template <class T>
__global__ void k_combine(T* __restrict__ r, const T* __restrict__ g, double c0, const T* const* __restrict__ v,
                          const double* __restrict__ coef, int nv, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double a = c0 * (double)g[i];
    for (int k = 0; k < nv; ++k) a = fma(coef[k], (double)v[k][i], a);
    r[i] = (T)a;
  }
}

static dim3 vec_grid(long long n) {
  const long long b = (n + 255) / 256;
  return dim3((unsigned)(b < 4 * 152 ? (b > 0 ? b : 1) : 4 * 152));
}

template <class T>
cudaError_t lb_dot(const T* x, const T* y, long long n, double* part, const double* mul, double* out,
                   cudaStream_t s) {
  k_dot<T><<<kDotBlocks, kDotNT, 0, s>>>(x, y, n, part);
  k_dot_final<<<1, 32, 0, s>>>(part, kDotBlocks, mul, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_axpy(T* y, const T* x, const double* a, const double* b, double sign, long long n,
                    cudaStream_t s) {
  k_axpy_dev<T><<<vec_grid(n), 256, 0, s>>>(y, x, a, b, sign, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_scale(T* r, const T* q, const double* num, const double* den, long long n, cudaStream_t s) {
  k_scale_dev<T><<<vec_grid(n), 256, 0, s>>>(r, q, num, den, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_axpby(T* z, const T* x, const T* y, double a, long long n, cudaStream_t s) {
  k_axpby<T><<<vec_grid(n), 256, 0, s>>>(z, x, y, a, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_mul(T* z, const T* x, double a, long long n, cudaStream_t s) {
  k_mul<T><<<vec_grid(n), 256, 0, s>>>(z, x, a, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_sub(T* z, const T* x, const T* y, long long n, cudaStream_t s) {
  k_sub<T><<<vec_grid(n), 256, 0, s>>>(z, x, y, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_mdot(const T* const* va, const T* const* vb, int ndots, long long n, double* part, double* out,
                    cudaStream_t s) {
  if (ndots <= 0) return cudaSuccess;
  k_mdot<T><<<dim3(kMdotChunks, ndots), kMdotNT, 0, s>>>(va, vb, n, part);
  k_mdot_final<<<ndots, 32, 0, s>>>(part, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t lb_combine(T* r, const T* g, double c0, const T* const* v, const double* coef, int nv, long long n,
                       cudaStream_t s) {
  k_combine<T><<<vec_grid(n), 256, 0, s>>>(r, g, c0, v, coef, nv, n);
  return cudaGetLastError();
}

int lb_dot_partials() { return kDotBlocks; }
int lb_mdot_partials(int ndots) { return ndots * kMdotChunks; }

#define MODIL_LB_INST(T)                                                                              \
  template cudaError_t lb_dot<T>(const T*, const T*, long long, double*, const double*, double*,     \
                                 cudaStream_t);                                                        \
  template cudaError_t lb_axpy<T>(T*, const T*, const double*, const double*, double, long long,     \
                                  cudaStream_t);                                                       \
  template cudaError_t lb_scale<T>(T*, const T*, const double*, const double*, long long, cudaStream_t); \
  template cudaError_t lb_axpby<T>(T*, const T*, const T*, double, long long, cudaStream_t);         \
  template cudaError_t lb_mul<T>(T*, const T*, double, long long, cudaStream_t);                    \
  template cudaError_t lb_mdot<T>(const T* const*, const T* const*, int, long long, double*, double*,  \
                                  cudaStream_t);                                                       \
  template cudaError_t lb_combine<T>(T*, const T*, double, const T* const*, const double*, int, long long, \
                                     cudaStream_t);                                                    \
  template cudaError_t lb_sub<T>(T*, const T*, const T*, long long, cudaStream_t);
MODIL_LB_INST(float)
MODIL_LB_INST(double)

}  // namespace modil
