// The Poisson family of Section 3.1 in d = 1, 2, 3 with the node-based
// (finite differences at N + 1 nodes per axis) or the cell-based (finite
// volumes at N cell centres per axis) layout, on [0,1]^d.  Grids are small
// (the paper uses N = 32), so each step of the method is its own kernel with
// one thread per cell or node; every sum has a fixed order.
//   k_gcompose  w_l = u_l + T w_{l+1} for one level l (coarse to fine; l = 0
//               writes the composed field), T the tensor product of the 1-D
//               node or cell interpolation (Section 2.2);
//   k_gresid    per fine cell/node: its residual and loss terms, and dL/du in
//               gather form -- the residual of the cell itself and of its
//               2d neighbours, each times its coefficient of u here -- plus
//               the data term, then Adam on level 0;
//   k_grestrict dL/du_l = T^T dL/du_{l-1} (transposed taps gathered per
//               coarse cell), then Adam on level l;
//   k_gfinal    the instance's loss terms from the per-block partial sums
//               (fixed order) and the step counter.
// Residuals (the paper's Section 3.1 discretisations):
//   cell: sum_a (u_{+a} - 2u + u_{-a}) / h_a^2 - f in every cell, the zero
//         wall value imposed by quadratic extrapolation through the wall and
//         the two nearest centres (ghost = -2 u_0 + u_1 / 3);
//   node: the same difference at interior nodes; the Dirichlet value is
//         imposed directly on the boundary nodes (the stencil reads 0 there),
//         whose unknowns then do not enter the residual part of the loss.
#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

// Interpolation taps of fine index i from a level of nc cells (node layout:
// nc + 1 nodes; fine node 2j copies coarse node j, fine node 2j+1 takes the
// mean of j and j+1).
template <class T>
__device__ __forceinline__ void taps1(int i, int nc, bool node, int& j0, int& j1, T& w0, T& w1) {
  if (node) {
    j0 = i >> 1;
    if (i & 1) { j1 = j0 + 1; w0 = T(0.5); w1 = T(0.5); }
    else { j1 = j0; w0 = T(1); w1 = T(0); }
    return;
  }
  prolong_taps<T>(i, nc, j0, j1, w0, w1);
}

// Transposed taps: the fine indices (and weights) whose interpolation reads
// coarse index j; nf fine entries per axis.  Returns the count (<= 6).
template <class T>
__device__ __forceinline__ int rtaps1(int j, int nc, bool node, int* idx, T* w) {
  if (node) {
    int c = 0;
    idx[c] = 2 * j; w[c] = T(1); ++c;
    if (j >= 1) { idx[c] = 2 * j - 1; w[c] = T(0.5); ++c; }
    if (j < nc) { idx[c] = 2 * j + 1; w[c] = T(0.5); ++c; }
    return c;
  }
  return restrict_taps<T>(j, nc, idx, w);
}

__device__ __forceinline__ void unflat(long long c, const int* n, int* q) {
  q[2] = (int)(c % n[2]);
  const long long r = c / n[2];
  q[1] = (int)(r % n[1]);
  q[0] = (int)(r / n[1]);
}

// Cells per axis of level l (node layout: the array has one more entry).
__device__ __forceinline__ int cells_of(const DevInst& D, int l, int a, bool node) {
  return node ? D.n[l][a] - 1 : D.n[l][a];
}

template <class T>
__global__ void __launch_bounds__(kGridNT) k_gcompose(const __grid_constant__ Arena<T> A, int l, int cur) {
  const int b = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.cblk_inst[l][b];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  const bool node = D.layout != 0;
  const int* n = D.n[l];
  const int* nc = D.n[l + 1];
  const long long cell = (long long)A.cblk_first[l][b] + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (cell >= (long long)n[0] * n[1] * n[2]) return;
  const T* __restrict__ P = A.p[cur];
  if (l + 1 >= D.nlev) {  // a single level: the composed field is level 0
    A.ufine[D.fine_off[0] + cell] = P[D.off[0][0] + cell];
    return;
  }
  int q[3];
  unflat(cell, n, q);
  const T* __restrict__ Wc = (l + 1 == D.nlev - 1) ? P + D.off[0][l + 1] : A.wl + D.off[0][l + 1];
  int j[3][2];
  T w[3][2];
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 1 && nc[a] == 1) {  // an unused leading axis
      j[a][0] = j[a][1] = 0; w[a][0] = T(1); w[a][1] = T(0);
    } else {
      taps1<T>(q[a], cells_of(D, l + 1, a, node), node, j[a][0], j[a][1], w[a][0], w[a][1]);
    }
  }
  T acc = T(0);
  for (int s = 0; s < 2; ++s) {
    T hy = T(0);
    for (int t = 0; t < 2; ++t) {
      const T* row = Wc + ((long long)j[0][s] * nc[1] + j[1][t]) * nc[2];
      hy += w[1][t] * (w[2][0] * row[j[2][0]] + w[2][1] * row[j[2][1]]);
    }
    acc += w[0][s] * hy;
  }
  const T v = P[D.off[0][l] + cell] + acc;
  if (l == 0) A.ufine[D.fine_off[0] + cell] = v;
  else A.wl[D.off[0][l] + cell] = v;
}

// Residual at q of the composed field U (n entries per axis), and the
// coefficient of U at c in it; real axes are those with more than one entry.
template <class T>
struct GridRes {
  const T* U;
  const int* n;
  bool node;
  T ih2[3];
  int real[3];
  __device__ T raw(int z, int y, int x) const { return U[((long long)z * n[1] + y) * n[2] + x]; }
  __device__ bool boundary(int z, int y, int x) const {
    const int c[3] = {z, y, x};
    for (int a = 0; a < 3; ++a)
      if (real[a] && (c[a] == 0 || c[a] == n[a] - 1)) return true;
    return false;
  }
  // the stencil's value: the node layout's boundary nodes hold the Dirichlet value 0
  __device__ T at(int z, int y, int x) const { return (node && boundary(z, y, x)) ? T(0) : raw(z, y, x); }
  // residual at q (which has one); f_q the right-hand side
  __device__ T res(const int* q, T f) const {
    T r = -f;
    const T uq = at(q[0], q[1], q[2]);
    for (int a = 0; a < 3; ++a) {
      if (!real[a]) continue;
      int lo[3] = {q[0], q[1], q[2]}, hi[3] = {q[0], q[1], q[2]};
      --lo[a];
      ++hi[a];
      T ul, uh;
      if (node) {
        ul = at(lo[0], lo[1], lo[2]);
        uh = at(hi[0], hi[1], hi[2]);
      } else {
        const bool hl = q[a] > 0, hh = q[a] < n[a] - 1;
        // a wall's ghost: quadratic extrapolation through the zero wall value
        // and the two nearest centres (each axis has >= 2 cells)
        int in1[3] = {q[0], q[1], q[2]};
        in1[a] += hl ? -1 : 1;
        int in2[3] = {q[0], q[1], q[2]};
        in2[a] += hh ? 1 : -1;
        const T u1 = at(in1[0], in1[1], in1[2]), u2 = at(in2[0], in2[1], in2[2]);
        ul = hl ? u1 : T(-2) * uq + u2 / T(3);
        uh = hh ? u2 : T(-2) * uq + u1 / T(3);
      }
      r += (uh - T(2) * uq + ul) * ih2[a];
    }
    return r;
  }
  // d r_q / d U_c for c = q + s e_a (s = +-1), or c = q (a < 0)
  __device__ T coef(const int* q, int a, int s) const {
    if (node) {
      if (a < 0) {
        T d = T(0);
        for (int b = 0; b < 3; ++b) if (real[b]) d += T(-2) * ih2[b];
        return d;
      }
      return ih2[a];
    }
    if (a < 0) {
      T d = T(0);
      for (int b = 0; b < 3; ++b) {
        if (!real[b]) continue;
        d += (T(-2) - (q[b] > 0 ? T(0) : T(2)) - (q[b] < n[b] - 1 ? T(0) : T(2))) * ih2[b];
      }
      return d;
    }
    // the neighbour q + s e_a, plus a third of it through q's ghost on the
    // other side when that side is a wall
    const bool wall_opposite = (s > 0) ? (q[a] == 0) : (q[a] == n[a] - 1);
    return (T(1) + (wall_opposite ? T(1) / T(3) : T(0))) * ih2[a];
  }
  __device__ bool has_res(const int* q) const {
    if (!node) return true;
    for (int a = 0; a < 3; ++a)
      if (real[a] && (q[a] == 0 || q[a] == n[a] - 1)) return false;
    return true;
  }
};

template <class T>
__global__ void __launch_bounds__(kGridNT) k_gresid(const __grid_constant__ Arena<T> A, int mode, int cur) {
  __shared__ double red[2][kGridNT / 32];
  const int gt = blockIdx.x, tid = threadIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  const bool node = D.layout != 0;
  const int* n = D.n[0];
  const long long ncell = (long long)n[0] * n[1] * n[2];
  const long long cell = (long long)(gt - D.tile_base[0]) * kGridNT + tid;
  const bool mine = cell < ncell;
  pdl_wait();
  pdl_trigger();
  GridRes<T> R;
  R.U = A.ufine + D.fine_off[0];
  R.n = n;
  R.node = node;
  for (int a = 0; a < 3; ++a) {
    R.real[a] = n[a] > 1;
    R.ih2[a] = T(1) / ((T)D.h[a] * (T)D.h[a]);
  }
  const T* F = A.aux + D.aux_off;  // right-hand side per fine cell/node
  const T lam_scale = T(2) * (T)D.w_res_dV;
  double rr = 0.0, dd = 0.0;
  T g = T(0);
  int q[3] = {0, 0, 0};
  if (mine) unflat(cell, n, q);
  // a boundary node is fixed: no residual term reads its unknown
  if (mine && !(node && R.boundary(q[0], q[1], q[2]))) {
    if (R.has_res(q)) {
      const T r = R.res(q, F[cell]);
      rr += (double)r * (double)r;
      g += lam_scale * r * R.coef(q, -1, 0);
    }
    // the neighbours' residuals that read this cell
    for (int a = 0; a < 3; ++a) {
      if (!R.real[a]) continue;
      for (int s = -1; s <= 1; s += 2) {
        int nb[3] = {q[0], q[1], q[2]};
        nb[a] += s;
        if (nb[a] < 0 || nb[a] >= n[a] || !R.has_res(nb)) continue;
        const long long cn = ((long long)nb[0] * n[1] + nb[1]) * n[2] + nb[2];
        const T r = R.res(nb, F[cn]);
        g += lam_scale * r * R.coef(nb, a, -s);
      }
    }
  }
  // data term: runs of this tile (unique cells)
  const T wd2 = T(2) * (T)D.w_data_n;
  for (int i = A.run_ptr[gt]; i < A.run_ptr[gt + 1]; ++i) {
    if (A.run_cell[i] != cell || !mine) continue;
    const T u = R.raw(q[0], q[1], q[2]);
    T sd = T(0), sq = T(0);
    for (int e = A.run_beg[i]; e < A.run_beg[i + 1]; ++e) {
      const T d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    dd += (double)sq;
    g += wd2 * sd;
  }
  // fixed-order block sums
  rr = warp_sum(rr);
  dd = warp_sum(dd);
  if ((tid & 31) == 0) { red[0][tid >> 5] = rr; red[1][tid >> 5] = dd; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kGridNT / 32; ++k) { a += red[0][k]; b += red[1][k]; }
    A.part[(long long)gt * A.npart + 0] = a;
    A.part[(long long)gt * A.npart + 1] = b;
  }
  if (mode == MODE_LOSS || !mine) return;
  g *= (T)A.gscale;
  const long long o = D.off[0][0] + cell;
  A.g[o] = g;
  if (mode == MODE_STEP) {
    const AdamCoef ac = adam_coef(D, A.st[ii]);
    T p = A.p[cur][o], m = A.m[o];
    double v = A.v[o];
    adam_update(p, m, v, g, ac);
    A.p[cur ^ 1][o] = p;
    A.m[o] = m;
    A.v[o] = v;
  }
}

template <class T>
__global__ void __launch_bounds__(kGridNT) k_grestrict(const __grid_constant__ Arena<T> A, int l, int mode, int cur) {
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[l][gt];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  const bool node = D.layout != 0;
  const int* n = D.n[l];
  const int* nf = D.n[l - 1];
  const long long cell = (long long)(gt - D.tile_base[l]) * kGridNT + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (cell >= (long long)n[0] * n[1] * n[2]) return;
  int q[3];
  unflat(cell, n, q);
  int idx[3][6], cnt[3];
  T w[3][6];
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 1 && nf[a] == 1) {
      cnt[a] = 1; idx[a][0] = 0; w[a][0] = T(1);
    } else {
      cnt[a] = rtaps1<T>(q[a], cells_of(D, l, a, node), node, idx[a], w[a]);
    }
  }
  const T* Gf = A.g + D.off[0][l - 1];
  T g = T(0);
  for (int i = 0; i < cnt[0]; ++i) {
    T hy = T(0);
    for (int j = 0; j < cnt[1]; ++j) {
      const T* row = Gf + ((long long)idx[0][i] * nf[1] + idx[1][j]) * nf[2];
      T hx = T(0);
      for (int k = 0; k < cnt[2]; ++k) hx += w[2][k] * row[idx[2][k]];
      hy += w[1][j] * hx;
    }
    g += w[0][i] * hy;
  }
  const long long o = D.off[0][l] + cell;
  if (mode != MODE_STEP || l < D.nlev - 1) A.g[o] = g;
  if (mode == MODE_STEP) {
    const AdamCoef ac = adam_coef(D, A.st[ii]);
    T p = A.p[cur][o], m = A.m[o];
    double v = A.v[o];
    adam_update(p, m, v, g, ac);
    A.p[cur ^ 1][o] = p;
    A.m[o] = m;
    A.v[o] = v;
  }
}

// One block per instance: loss terms from the tiles' partial sums (each
// thread a fixed stride of tiles, then a fixed-order block sum), the
// non-finite latch and, in step mode, the step counter.
template <class T>
__global__ void __launch_bounds__(kGridNT) k_gfinal(const __grid_constant__ Arena<T> A, int mode) {
  __shared__ double red[2][kGridNT / 32];
  const int ii = blockIdx.x, tid = threadIdx.x;
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  pdl_wait();
  pdl_trigger();
  const double* part = A.part + (long long)D.tile_base[0] * A.npart;
  double a = 0.0, b = 0.0;
  for (int t = tid; t < D.ntile0; t += kGridNT) {
    a += part[(long long)t * A.npart + 0];
    b += part[(long long)t * A.npart + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((tid & 31) == 0) { red[0][tid >> 5] = a; red[1][tid >> 5] = b; }
  __syncthreads();
  if (tid == 0) {
    double ra = 0.0, rb = 0.0;
    for (int k = 0; k < kGridNT / 32; ++k) { ra += red[0][k]; rb += red[1][k]; }
    InstState& S = A.st[ii];
    const double res = D.w_res_dV * ra, dat = D.w_data_n * rb, tot = res + dat;
    S.terms[0] = tot;
    S.terms[1] = res;
    S.terms[2] = dat;
    S.terms[3] = 0.0;
    if (!isfinite(tot)) S.nonfinite |= kStatusNonfinite;
    if (mode == MODE_STEP) advance_step(S, D.b1, D.b2);
  }
}

// ---------------------------------------------------------------------------
static cudaLaunchConfig_t grid_cfg(dim3 grid, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kGridNT);
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <class T>
cudaError_t launch_gcompose(const Arena<T>& A, int level, int cur, cudaStream_t s) {
  if (A.ncblk[level] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = grid_cfg(dim3(A.ncblk[level]), s, at);
  return cudaLaunchKernelEx(&cfg, k_gcompose<T>, A, level, cur);
}
template <class T>
cudaError_t launch_gresid(const Arena<T>& A, int mode, int cur, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = grid_cfg(dim3(A.ntiles[0]), s, at);
  return cudaLaunchKernelEx(&cfg, k_gresid<T>, A, mode, cur);
}
template <class T>
cudaError_t launch_grestrict(const Arena<T>& A, int level, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[level] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = grid_cfg(dim3(A.ntiles[level]), s, at);
  return cudaLaunchKernelEx(&cfg, k_grestrict<T>, A, level, mode, cur);
}
template <class T>
cudaError_t launch_gfinal(const Arena<T>& A, int mode, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = grid_cfg(dim3(A.n_inst), s, at);
  return cudaLaunchKernelEx(&cfg, k_gfinal<T>, A, mode);
}

template cudaError_t launch_gcompose<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_gcompose<double>(const Arena<double>&, int, int, cudaStream_t);
template cudaError_t launch_gresid<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_gresid<double>(const Arena<double>&, int, int, cudaStream_t);
template cudaError_t launch_grestrict<float>(const Arena<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_grestrict<double>(const Arena<double>&, int, int, int, cudaStream_t);
template cudaError_t launch_gfinal<float>(const Arena<float>&, int, cudaStream_t);
template cudaError_t launch_gfinal<double>(const Arena<double>&, int, cudaStream_t);

}  // namespace modil
