// PDE-independent kernels: the transposed prolongation chain with the fused
// Adam update of each coarse level, and the per-instance finalisation.
//
// Restriction.  The reverse of Horner's scheme gives dL/du_{i+1} = T_i^T
// dL/du_i (paper Section 2.2: the decomposition is linear, so its adjoint is
// the chain of transposed interpolation matrices).  Each thread gathers one
// coarse cell from at most 6 x 6 fine values of the level below (the column of
// the tensor-product interpolation matrix), then, in step mode, updates that
// level's parameter with Adam and stores the level gradient for the next
// restriction.
#include "modil_dev.cuh"
#include "launch.h"

namespace modil {

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_level(Arena<T> A, int l, int mode) {
  __shared__ DevInst D;
  const int gt = blockIdx.x;
  const int ii = A.tile_inst[l][gt];
  block_copy(&D, A.inst + ii);
  __syncthreads();
  const InstState st = A.st[ii];
  const int cur = (int)(st.t & 1);
  const AdamCoef ac = adam_coef(D, st);
  const int nz = D.n[l][0], ny = D.n[l][1], nx = D.n[l][2];
  const int fz = D.n[l - 1][0], fy = D.n[l - 1][1], fx = D.n[l - 1][2];
  const int local = gt - D.tile_base[l];
  const int tpz = D.nt[l][1] * D.nt[l][2];
  const int tz = local / tpz;
  const int rem = local - tz * tpz;
  const int ty = rem / D.nt[l][2], tx = rem - ty * D.nt[l][2];
  const bool store_g = (mode != MODE_STEP) || (l < D.nlev - 1);
  // Tiles are kLevTY x kLevTX in (y, x) and one plane deep in z.
  for (int idx = threadIdx.x; idx < kLevTY * kLevTX; idx += MODIL_NT) {
    const int oy = idx / kLevTX, ox = idx - oy * kLevTX;
    const int z = tz, y = ty * kLevTY + oy, x = tx * kLevTX + ox;
    if (z >= nz || y >= ny || x >= nx) continue;
    int iz[6], iy[6], ix[6];
    T wz[6], wy[6], wx[6];
    int cz = 1;
    if (D.ndim == 3) cz = restrict_taps<T>(z, nz, iz, wz);
    else { iz[0] = 0; wz[0] = T(1); }
    const int cy = restrict_taps<T>(y, ny, iy, wy);
    const int cx = restrict_taps<T>(x, nx, ix, wx);
    const long long e = ((long long)z * ny + y) * nx + x;
    for (int f = 0; f < D.nfield; ++f) {
      const T* __restrict__ gf = A.g + D.off[f][l - 1];
      T acc = T(0);
      for (int a = 0; a < cz; ++a) {
        T accy = T(0);
        for (int b = 0; b < cy; ++b) {
          const T* row = gf + ((long long)iz[a] * fy + iy[b]) * fx;
          T accx = T(0);
          for (int c = 0; c < cx; ++c) accx += wx[c] * row[ix[c]];
          accy += wy[b] * accx;
        }
        acc += wz[a] * accy;
      }
      const long long o = D.off[f][l] + e;
      if (store_g) A.g[o] = acc;
      if (mode == MODE_STEP) {
        T p = A.p[cur][o];
        T m = A.m[o];
        double v = A.v[o];
        adam_update(p, m, v, acc, ac);
        A.p[cur ^ 1][o] = p;
        A.m[o] = m;
        A.v[o] = v;
      }
    }
  }
  (void)fz;
}

// One block per instance: fixed-order FP64 sums of the per-tile partials,
// the regulariser, the loss terms, the conductivity-node gradient, Adam on
// the nodes and the step counter.
template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_finalize(Arena<T> A, int mode) {
  __shared__ DevInst D;
  __shared__ double sums[2 + MODIL_MAXK];
  const int ii = blockIdx.x;
  block_copy(&D, A.inst + ii);
  __syncthreads();
  const int nt0 = D.nt[0][0] * D.nt[0][1] * D.nt[0][2];
  const long long base = D.tile_base[0];
  const int nterm = (mode == MODE_LOSS) ? 2 : 2 + D.nk;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < nterm; j += MODIL_NT / 32) {
    double s = 0.0;
    for (int t = lane; t < nt0; t += 32) s += A.part[(base + t) * A.npart + j];
    s = warp_sum(s);
    if (lane == 0) sums[j] = s;
  }
  __syncthreads();
  InstState& st = A.st[ii];
  // regulariser w_reg * sum (q_{j+1} - 2 q_j + q_{j-1})^2 and its gradient
  const int nk = D.nk;
  if (threadIdx.x == 0) {
    double reg = 0.0;
    for (int j = 1; j + 1 < nk; ++j) {
      const double d2 = (double)A.kq[D.k_off + j + 1] - 2.0 * (double)A.kq[D.k_off + j] +
                        (double)A.kq[D.k_off + j - 1];
      reg += d2 * d2;
    }
    reg *= D.w_reg;
    const double res = D.w_res_dV * sums[0];
    const double dat = D.w_data_n * sums[1];
    const double tot = res + dat + reg;
    st.terms[0] = tot;
    st.terms[1] = res;
    st.terms[2] = dat;
    st.terms[3] = reg;
    if (!isfinite(tot)) st.nonfinite = 1;
  }
  if (mode != MODE_LOSS) {
    const AdamCoef ac = adam_coef(D, st);
    for (int j = threadIdx.x; j < nk; j += MODIL_NT) {
      double g = sums[2 + j];
      // d/dq_j of w_reg * sum_i d2_i^2, d2_i = q_{i+1} - 2 q_i + q_{i-1}
      auto q = [&](int i) { return (double)A.kq[D.k_off + i]; };
      for (int i = j - 1; i <= j + 1; ++i) {
        if (i < 1 || i + 1 >= nk) continue;
        const double d2 = q(i + 1) - 2.0 * q(i) + q(i - 1);
        const double c = (i == j) ? -2.0 : 1.0;
        g += D.w_reg * 2.0 * d2 * c;
      }
      A.kg[D.k_off + j] = (T)g;
      sums[2 + j] = g;
    }
    __syncthreads();
    if (mode == MODE_STEP) {
      for (int j = threadIdx.x; j < nk; j += MODIL_NT) {
        T p = A.kq[D.k_off + j];
        T m = A.km[D.k_off + j];
        double v = A.kv[D.k_off + j];
        adam_update(p, m, v, (T)sums[2 + j], ac);
        A.kq[D.k_off + j] = p;
        A.km[D.k_off + j] = m;
        A.kv[D.k_off + j] = v;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        st.t += 1;
        st.b1t *= D.b1;
        st.b2t *= D.b2;
      }
    }
  }
}

template <class T>
__global__ void k_reset(Arena<T> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.n_inst) {
    InstState s;
    s.t = 0;
    s.b1t = 1.0;
    s.b2t = 1.0;
    for (int j = 0; j < 4; ++j) s.terms[j] = 0.0;
    s.nonfinite = 0;
    s.pad = 0;
    A.st[i] = s;
  }
}

template <class T>
cudaError_t launch_level(const Arena<T>& A, int level, int mode, cudaStream_t s) {
  if (A.ntiles[level] == 0) return cudaSuccess;
  k_level<T><<<A.ntiles[level], MODIL_NT, 0, s>>>(A, level, mode);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_finalize(const Arena<T>& A, int mode, cudaStream_t s) {
  k_finalize<T><<<A.n_inst, MODIL_NT, 0, s>>>(A, mode);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_reset(const Arena<T>& A, cudaStream_t s) {
  k_reset<T><<<(A.n_inst + 255) / 256, 256, 0, s>>>(A);
  return cudaGetLastError();
}

template cudaError_t launch_level<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_level<double>(const Arena<double>&, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const Arena<float>&, int, cudaStream_t);
template cudaError_t launch_finalize<double>(const Arena<double>&, int, cudaStream_t);
template cudaError_t launch_reset<float>(const Arena<float>&, cudaStream_t);
template cudaError_t launch_reset<double>(const Arena<double>&, cudaStream_t);

}  // namespace modil
