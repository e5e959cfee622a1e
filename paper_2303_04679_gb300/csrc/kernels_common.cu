// PDE-independent kernels: the transposed prolongation chain with the fused
// Adam update of each coarse level, and the per-instance tail that closes a
// pass (loss terms, conductivity-node gradient and Adam, the smallest levels,
// the step counter).
//
// Restriction.  The reverse of Horner's scheme gives dL/du_{i+1} = T_i^T
// dL/du_i (paper Section 2.2: the decomposition is linear, so its adjoint is
// the chain of transposed interpolation matrices).  Column X of the 1-D cell
// interpolation matrix is nonzero only on fine cells 2X-2 .. 2X+3, so the
// transposed operator is a 6-tap window with weights that depend only on X
// and the level size; the tensor product is applied separably (rows, then
// columns) from a copy of the finer level staged in shared memory.
//
// k_level handles one level over all instances that still have a level
// larger than the tail threshold; k_tail runs the remaining small levels of
// one instance in shared memory, spread over a few blocks that each update a
// slice of the cells.
#include <cooperative_groups.h>

#include "launch.h"
#include "modil_dev.cuh"

namespace cg = cooperative_groups;

namespace modil {

// Weights of coarse cell X (level of nc cells) on fine cells 2X-2 .. 2X+3:
// 1/4, 3/4, 3/4, 1/4 in the interior; the extrapolated end rows of the
// interpolation matrix give 5/4 and -1/4 near the ends; one coarse cell
// copies into both fine cells.
template <class T>
__device__ __forceinline__ void rwin(int X, int nc, T* w) {
  if (nc == 1) {
    w[0] = T(0); w[1] = T(0); w[2] = T(1); w[3] = T(1); w[4] = T(0); w[5] = T(0);
    return;
  }
  w[0] = (X == 1) ? T(-0.25) : T(0);
  w[1] = (X >= 1) ? T(0.25) : T(0);
  w[2] = (X == 0) ? T(1.25) : T(0.75);
  w[3] = (X == nc - 1) ? T(1.25) : T(0.75);
  w[4] = (X <= nc - 2) ? T(0.25) : T(0);
  w[5] = (X == nc - 2) ? T(-0.25) : T(0);
}

// Separable restriction of a staged 2-D region of the finer level.
//   S: fine values, rows fy0 .. fy0+fh-1, cols fx0 .. fx0+fw-1, row stride ss
//   H: scratch, fh rows x cw cols (row stride cw)
//   output coarse rows Y0 .. Y0+ch-1, cols X0 .. X0+cw-1 of a level ny x nx
//   (finer level nfy x nfx) to out(k, value) for k = (Y-Y0)*cw + (X-X0).
// Fine indices outside the level only meet zero weights; they are clamped
// to stay inside the staged region.
template <class T, int NT, class Out>
__device__ __forceinline__ void restrict_sep(const T* S, int ss, int fy0, int fh, int fx0, int fw,
                                             T* H, int Y0, int ch, int X0, int cw, int ny, int nx,
                                             Out out) {
  const int tid = threadIdx.x;
  for (int i = tid; i < fh * cw; i += NT) {
    const int r = i / cw, X = X0 + (i - (i / cw) * cw);
    T w[6];
    rwin<T>(X, nx, w);
    const T* row = S + r * ss;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int f = min(max(2 * X - 2 + k - fx0, 0), fw - 1);
      acc += w[k] * row[f];
    }
    H[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < ch * cw; i += NT) {
    const int Yr = i / cw, c = i - (i / cw) * cw;
    const int Y = Y0 + Yr;
    T w[6];
    rwin<T>(Y, ny, w);
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int f = min(max(2 * Y - 2 + k - fy0, 0), fh - 1);
      acc += w[k] * H[f * cw + c];
    }
    out(i, acc);
  }
}

constexpr int kLevFY = 2 * kLevTY + 4, kLevFX = 2 * kLevTX + 4;  // staged fine region

// restrict_sep for the fixed tile of k_level: the loops run over the
// constant-size boxes (divisions by constants) with bounds checks.
template <class T, int NT, class Out>
__device__ __forceinline__ void restrict_box(const T* S, int fy0, int fh, int fx0, int fw, T* H, int Y0, int ch,
                                             int X0, int cw, int ny, int nx, Out out) {
  const int tid = threadIdx.x;
  for (int i = tid; i < kLevFY * kLevTX; i += NT) {
    const int r = i / kLevTX, c = i % kLevTX;
    if (r >= fh || c >= cw) continue;
    const int X = X0 + c;
    T w[6];
    rwin<T>(X, nx, w);
    const T* row = S + r * kLevFX;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int f = min(max(2 * X - 2 + k - fx0, 0), fw - 1);
      acc += w[k] * row[f];
    }
    H[r * kLevTX + c] = acc;
  }
  __syncthreads();
  // cells packed as k = Yr * cw + c, so that k == threadIdx.x: each thread
  // finishes the cell whose Adam state it holds
  for (int i = tid; i < ch * cw; i += NT) {
    const int Yr = i / cw, c = i - (i / cw) * cw;
    const int Y = Y0 + Yr;
    T w[6];
    rwin<T>(Y, ny, w);
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int f = min(max(2 * Y - 2 + k - fy0, 0), fh - 1);
      acc += w[k] * H[f * kLevTX + c];
    }
    out(Yr * cw + c, acc);
  }
}

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_level(const __grid_constant__ Arena<T> A, int l, int mode, int cur) {
  static_assert(kLevTY * kLevTX == MODIL_NT, "one coarse cell per thread");
  __shared__ DevInst D;
  __shared__ __align__(16) T fineS[kLevFY * kLevFX];
  __shared__ __align__(16) T H[kLevFY * kLevTX];
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[l][gt];
  load_inst(&D, A, ii);
  __syncthreads();
  const int nf = D.nfield;
  const int ny = D.n[l][1], nx = D.n[l][2];
  const int fy = D.n[l - 1][1], fx = D.n[l - 1][2];
  const int local = gt - D.tile_base[l];
  const int ty = local / D.nt[l][2], tx = local - ty * D.nt[l][2];
  const int y0 = ty * kLevTY, x0 = tx * kLevTX;
  const int ch = min(kLevTY, ny - y0), cw = min(kLevTX, nx - x0);
  const bool store_g = (mode != MODE_STEP) || (l < D.nlev - 1);
  // Prologue: this level's parameters and moments were last written by the
  // same kernel one step earlier, two or more launches back.
  const int oy = threadIdx.x / cw, ox = threadIdx.x - (threadIdx.x / cw) * cw;
  const bool mine = threadIdx.x < ch * cw;
  const long long e = (long long)(y0 + oy) * nx + (x0 + ox);
  T pv[MODIL_MAXF], mv[MODIL_MAXF];
  double vv[MODIL_MAXF];
#pragma unroll
  for (int f = 0; f < MODIL_MAXF; ++f) {
    pv[f] = T(0); mv[f] = T(0); vv[f] = 0.0;
    if (f < nf && mode == MODE_STEP && mine) {
      const long long o = D.off[f][l] + e;
      pv[f] = A.p[cur][o];
      mv[f] = A.m[o];
      vv[f] = A.v[o];
    }
  }
  __shared__ AdamCoef acS;
  if (threadIdx.x == 0) acS = adam_coef(D, A.st[ii]);  // once per block: no per-thread FP64
  pdl_wait();
  pdl_trigger();
  const int fy0 = max(0, 2 * y0 - 2), fy1 = min(fy, 2 * (y0 + ch) + 2);
  const int fx0 = max(0, 2 * x0 - 2), fx1 = min(fx, 2 * (x0 + cw) + 2);
  const int fw = fx1 - fx0, fh = fy1 - fy0;
#pragma unroll
  for (int f = 0; f < MODIL_MAXF; ++f) {
    if (f >= nf) break;
    // stage field f of the finer level's gradient over the tile's footprint
    const T* __restrict__ gf = A.g + D.off[f][l - 1];
    for (int i = threadIdx.x; i < kLevFY * kLevFX; i += MODIL_NT) {
      const int r = i / kLevFX, c = i % kLevFX;
      if (r < fh && c < fw) cp_async(fineS + i, gf + (long long)(fy0 + r) * fx + (fx0 + c));
    }
    cp_async_wait_all();
    __syncthreads();
    const AdamCoef ac = acS;
    const long long o = D.off[f][l] + e;
    restrict_box<T, MODIL_NT>(fineS, fy0, fh, fx0, fw, H, y0, ch, x0, cw, ny, nx,
                              [&](int k, T g) {
                                // k == threadIdx.x: each thread finishes its own cell
                                if (store_g) A.g[o] = g;
                                if (mode == MODE_STEP) {
                                  adam_update(pv[f], mv[f], vv[f], g, ac);
                                  A.p[cur ^ 1][o] = pv[f];
                                  A.m[o] = mv[f];
                                  A.v[o] = vv[f];
                                }
                              });
    __syncthreads();  // fineS and H are reused by the next field
  }
}

// ---------------------------------------------------------------------------
// Tail: one thread-block cluster of kTailC blocks per instance.  The tail
// levels are split by rows over the blocks of the cluster; each level is
// restricted from the rows of the level above, read from global memory (first
// tail level) or from the owning blocks' shared memory over the cluster's
// distributed shared memory, with a cluster barrier between levels.  The
// per-tile partials are summed in slices by every block and combined in
// block order by block 0, which also steps the conductivity nodes and, at the
// very end, the step counter.
// ---------------------------------------------------------------------------
constexpr int kTailNT = 256;

// Shared-memory layout of one tail block (identical on host and device).
struct TailLayout {
  int rp[MODIL_MAXL];       // rows per block of each tail level
  int own_off[MODIL_MAXL];  // offset of the block's own rows of each level (one field)
  int own_cells;            // cells of one field owned by one block (upper bound)
  int nf;                   // fields
  int st_elems, h_elems;    // staging of the level above, separable scratch
  size_t bytes(int esz) const {
    const size_t oc = (size_t)own_cells * nf;
    return 8 * oc + (size_t)esz * (3 * oc + st_elems + h_elems) + 64;
  }
};

__host__ __device__ inline void tail_layout(int L, int ts, const int (*n)[3], int nf, TailLayout& t) {
  int acc = 0, st = 0, h = 0;
  for (int l = 0; l < MODIL_MAXL; ++l) { t.rp[l] = 0; t.own_off[l] = 0; }
  for (int l = ts; l < L; ++l) {
    const int ny = n[l][1], nx = n[l][2];
    const int rp = (ny + kTailC - 1) / kTailC;
    t.rp[l] = rp;
    t.own_off[l] = acc;
    acc += rp * nx;
    const int rows = 2 * rp + 4;
    st = max(st, rows * n[l - 1][2]);
    h = max(h, rows * nx);
  }
  t.own_cells = acc;
  t.nf = nf;
  t.st_elems = st;
  t.h_elems = h;
}

template <class T>
__global__ void __cluster_dims__(kTailC, 1, 1) __launch_bounds__(kTailNT)
k_tail(const __grid_constant__ Arena<T> A, int mode, int cur) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevInst D;
  __shared__ TailLayout TL;
  __shared__ double psum[2 + MODIL_MAXK];
  __shared__ double qs[MODIL_MAXK];
  __shared__ double chunk[kTailNT];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int ii = blockIdx.x / kTailC;
  const int tid = threadIdx.x;
  load_inst(&D, A, ii);
  __syncthreads();
  if (tid == 0) tail_layout(D.nlev, D.tail, D.n, D.nfield, TL);
  __syncthreads();
  const int L = D.nlev, ts = D.tail;
  const bool levels = (mode == MODE_GRAD || mode == MODE_STEP) && ts < L;
  const int nf = D.nfield;
  const int oc = TL.own_cells;  // per field; field f of the own arrays starts at f * oc
  double* vS = reinterpret_cast<double*>(smem);
  T* gO = reinterpret_cast<T*>(smem + 8 * (size_t)oc * nf);
  T* pS = gO + oc * nf;
  T* mS = pS + oc * nf;
  T* Pst = mS + oc * nf;
  T* H = Pst + TL.st_elems;

  // Prologue: the tail levels' parameters and moments and the bias-correction
  // powers were last written by this kernel one step earlier.
  if (mode == MODE_STEP && levels) {
    for (int f = 0; f < nf; ++f)
      for (int l = ts; l < L; ++l) {
        const int ny = D.n[l][1], nx = D.n[l][2];
        const int a = r * TL.rp[l], b = min(ny, a + TL.rp[l]);
        for (int i = tid; i < (b > a ? (b - a) * nx : 0); i += kTailNT) {
          const long long o = D.off[f][l] + (long long)a * nx + i;
          const int k = f * oc + TL.own_off[l] + i;
          cp_async(pS + k, A.p[cur] + o);
          cp_async(mS + k, A.m + o);
          cp_async(vS + k, A.v + o);
        }
      }
  }
  InstState& S = A.st[ii];
  __shared__ AdamCoef acS;
  if (tid == 0) acS = adam_coef(D, S);  // once per block: no per-thread FP64
  pdl_wait();
  pdl_trigger();

  // ---- partial sums: block r adds tiles [r*nt0/C, (r+1)*nt0/C) -------------
  const int nk = D.nk;
  const int nterm = (mode == MODE_LOSS) ? 2 : 2 + nk;
  {
    const int nt0 = D.ntile0, np = A.npart;
    const int t0 = (int)((long long)r * nt0 / kTailC), t1 = (int)((long long)(r + 1) * nt0 / kTailC);
    const double* part = A.part + (long long)D.tile_base[0] * np;
    const int sub = kTailNT / nterm;  // sub-chunks per term
    double s = 0.0;
    const int j = tid % nterm, c = tid / nterm;
    if (c < sub)
      for (int tb = t0 + c; tb < t1; tb += 8 * sub) {
        double v[8];  // loads first, then the adds in order
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = tb + u * sub;
          v[u] = (t < t1) ? __ldcg(part + (long long)t * np + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
      }
    chunk[tid] = s;
    __syncthreads();
    if (tid < nterm) {
      double a = 0.0;
      for (int cc = 0; cc < sub; ++cc) a += chunk[cc * nterm + tid];
      psum[tid] = a;
    }
  }

  // ---- the small levels, distributed by rows over the cluster ---------------
  for (int l = ts; l < (levels ? L : ts); ++l) {
    const int ny = D.n[l][1], nx = D.n[l][2];
    const int fy = D.n[l - 1][1], fx = D.n[l - 1][2];
    const int a = r * TL.rp[l], b = min(ny, a + TL.rp[l]);
    if (b > a) {
      const int pa = max(0, 2 * a - 2), pb = min(fy, 2 * b + 2);
      const int prow = pb - pa;
      for (int f = 0; f < nf; ++f) {
        if (l == ts) {
          const T* src = A.g + D.off[f][l - 1] + (long long)pa * fx;
          for (int i = tid; i < prow * fx; i += kTailNT) cp_async(Pst + i, src + i);
          cp_async_wait_all();
        } else {
          const int rpp = TL.rp[l - 1];
          for (int i = tid; i < prow * fx; i += kTailNT) {
            const int y = pa + i / fx, x = i - (i / fx) * fx;
            const int owner = y / rpp;
            const T* rem = cluster.map_shared_rank(gO, owner);
            Pst[i] = rem[f * oc + TL.own_off[l - 1] + (y - owner * rpp) * fx + x];
          }
        }
        __syncthreads();
        T* dst = gO + f * oc + TL.own_off[l];
        restrict_sep<T, kTailNT>(Pst, fx, pa, prow, 0, fx, H, a, b - a, 0, nx, ny, nx,
                                 [&](int k, T g) { dst[k] = g; });
        __syncthreads();  // Pst and H are reused by the next field
      }
    }
    cluster.sync();
    // every block has read the bias-correction powers: advance them now (off the
    // critical path of the remaining levels)
    if (l == ts && mode == MODE_STEP && r == 0 && tid == 0) advance_step(S, D.b1, D.b2);
  }
  if (!levels) {
    cluster.sync();  // partial sums visible cluster-wide; powers read by all blocks
    if (mode == MODE_STEP && r == 0 && tid == 0) advance_step(S, D.b1, D.b2);
  }

  // ---- block 0: loss terms, dL/dq, Adam on the nodes -------------------------
  if (r == 0) {
    __shared__ double d2s[MODIL_MAXK];
    for (int j = tid; j < nk; j += kTailNT) qs[j] = (double)A.kq[D.k_off + j];
    if (tid < nterm) {
      double v[kTailC];
#pragma unroll
      for (int rr = 0; rr < kTailC; ++rr) v[rr] = *cluster.map_shared_rank(psum + tid, rr);
      double a = 0.0;
#pragma unroll
      for (int rr = 0; rr < kTailC; ++rr) a += v[rr];
      chunk[tid] = a;
    }
    __syncthreads();
    // second differences d2_j = q_{j+1} - 2 q_j + q_{j-1}, j = 1 .. nk-2, in parallel
    double dd = 0.0;
    if (tid < MODIL_MAXK) {
      d2s[tid] = 0.0;
      if (tid >= 1 && tid + 1 < nk) {
        dd = qs[tid + 1] - 2.0 * qs[tid] + qs[tid - 1];
        d2s[tid] = dd;
      }
    }
    double reg = 0.0;
    if (tid < 64) {
      reg = warp_sum(dd * dd);
      if ((tid & 31) == 0) chunk[nterm + (tid >> 5)] = reg;
    }
    __syncthreads();
    if (tid == 0) {
      const double rg = D.w_reg * (chunk[nterm] + chunk[nterm + 1]);
      const double res = D.w_res_dV * chunk[0];
      const double dat = D.w_data_n * chunk[1];
      const double tot = res + dat + rg;
      S.terms[0] = tot;
      S.terms[1] = res;
      S.terms[2] = dat;
      S.terms[3] = rg;
      if (!isfinite(tot)) S.nonfinite = 1;
    }
    if (mode != MODE_LOSS)
      for (int j = tid; j < nk; j += kTailNT) {
        const AdamCoef ac = acS;
        // d/dq_j of w_reg * sum_i d2_i^2 = 2 w_reg (d2_{j-1} - 2 d2_j + d2_{j+1})
        const double dm = (j >= 1) ? d2s[j - 1] : 0.0;
        const double dp = (j + 1 < MODIL_MAXK) ? d2s[j + 1] : 0.0;
        const double g = chunk[2 + j] + 2.0 * D.w_reg * (dm - 2.0 * d2s[j] + dp);
        A.kg[D.k_off + j] = (T)g;
        if (mode == MODE_STEP) {
          T p = (T)qs[j];
          T m = A.km[D.k_off + j];
          double v = A.kv[D.k_off + j];
          adam_update(p, m, v, (T)g, ac);
          A.kq[D.k_off + j] = p;
          A.km[D.k_off + j] = m;
          A.kv[D.k_off + j] = v;
        }
      }
  }

  // ---- Adam on the block's own rows of every tail level ---------------------
  if (levels) {
    cp_async_wait_all();
    __syncthreads();
    for (int f = 0; f < nf; ++f)
    for (int l = ts; l < L; ++l) {
      const int ny = D.n[l][1], nx = D.n[l][2];
      const int a = r * TL.rp[l], b = min(ny, a + TL.rp[l]);
      for (int i = tid; i < (b > a ? (b - a) * nx : 0); i += kTailNT) {
        const int k = f * oc + TL.own_off[l] + i;
        const long long o = D.off[f][l] + (long long)a * nx + i;
        const T g = gO[k];
        if (mode != MODE_STEP || l < L - 1) A.g[o] = g;
        if (mode == MODE_STEP) {
          const AdamCoef ac = acS;
          T p = pS[k], m = mS[k];
          double v = vS[k];
          adam_update(p, m, v, g, ac);
          A.p[cur ^ 1][o] = p;
          A.m[o] = m;
          A.v[o] = v;
        }
      }
    }
  }
  // no block may exit while another still reads its shared memory
  cluster.sync();
}

template <class T>
__global__ void k_reset(const __grid_constant__ Arena<T> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.n_inst) {
    InstState s;
    const DevInst& D = A.inst[i];
    s.t = 0;
    s.b1t = 1.0;
    s.b2t = 1.0;
    s.c1 = 1.0 / (1.0 - D.b1);
    s.c2 = 1.0 / (1.0 - D.b2);
    for (int j = 0; j < 4; ++j) s.terms[j] = 0.0;
    s.nonfinite = 0;
    s.pad = 0;
    A.st[i] = s;
  }
}

// Holds the stream for about ns nanoseconds (bounded loop) so that launches
// queued behind it run back to back when they are timed one by one.
__global__ void k_delay(long long ns) {
  if (threadIdx.x != 0) return;
  const long long t0 = clock64();
  const long long cycles = ns * 2;  // at most ~2 cycles per ns at the top clock
  for (int i = 0; i < (1 << 20); ++i) {
    if (clock64() - t0 >= cycles) break;
    __nanosleep(1000);
  }
}

static cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <class T>
cudaError_t launch_level(const Arena<T>& A, int level, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[level] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = pdl_config(dim3(A.ntiles[level]), dim3(MODIL_NT), 0, s, at);
  return cudaLaunchKernelEx(&cfg, k_level<T>, A, level, mode, cur);
}

size_t tail_smem_bytes(const TailPlan& tp, int elem) { return tp.smem_bytes; }

// Shared-memory bytes the tail blocks of one instance need.
size_t tail_instance_bytes(int L, int ts, const int (*n)[3], int nf, int elem) {
  TailLayout t;
  tail_layout(L, ts, n, nf, t);
  return t.bytes(elem);
}

template <class T>
cudaError_t prepare_tail(const TailPlan& tp) {
  return raise_smem_limit(k_tail<T>, tp.smem_bytes);
}

template <class T>
cudaError_t launch_tail(const Arena<T>& A, int mode, int cur, const TailPlan& tp, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = pdl_config(dim3(A.n_inst * kTailC), dim3(kTailNT), tp.smem_bytes, s, at);
  return cudaLaunchKernelEx(&cfg, k_tail<T>, A, mode, cur);
}

template <class T>
cudaError_t launch_reset(const Arena<T>& A, cudaStream_t s) {
  k_reset<T><<<(A.n_inst + 255) / 256, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_delay(long long ns, cudaStream_t s) {
  k_delay<<<1, 32, 0, s>>>(ns);
  return cudaGetLastError();
}

template cudaError_t launch_level<float>(const Arena<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_level<double>(const Arena<double>&, int, int, int, cudaStream_t);
template cudaError_t prepare_tail<float>(const TailPlan&);
template cudaError_t prepare_tail<double>(const TailPlan&);
template cudaError_t launch_tail<float>(const Arena<float>&, int, int, const TailPlan&, cudaStream_t);
template cudaError_t launch_tail<double>(const Arena<double>&, int, int, const TailPlan&, cudaStream_t);
template cudaError_t launch_reset<float>(const Arena<float>&, cudaStream_t);
template cudaError_t launch_reset<double>(const Arena<double>&, cudaStream_t);

}  // namespace modil
