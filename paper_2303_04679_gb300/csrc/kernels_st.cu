// Fused fine-tile kernel of the space-time PDE family (viscous Burgers,
// heat conduction with unknown conductivity).  One block owns a TY x TX tile
// of the fine grid (axes t, x) and in one pass:
//   0. issues every global load it needs at once (cp.async into shared
//      memory; 16-byte copies where rows are 4-element aligned): the tile's
//      region of every level (tile plus a halo of 2 fine cells, and at each
//      coarser level half that plus one cell), the level-1 Adam moments of
//      the tile, its measurement runs, the conductivity nodes;
//   1. composes the field on the tile by Horner's scheme on that pyramid
//      (w_L = u_L, w_i = u_i + T_i w_{i+1}; paper Section 2.2), the fine
//      level streamed down columns;
//   2. evaluates every residual that touches the tile (tile plus 1 cell) and
//      its local Jacobian, dr/du at the 4 stencil points, streamed down
//      columns, and keeps lambda * dr/du (lambda = 2 w dV r);
//   3. adds the data term of the measurements inside the tile to the cell's
//      own term, and that of the off-grid points whose corner cells the tile
//      owns (d-linear samples of the composed field; per owned corner cell a
//      fixed-order sum over the points reaching it);
//   4. reduces r^2 and the data misfit over what it owns (FP64 partials per
//      tile);
//   5. forms dL/du in gather form (each cell sums lambda * dr/du over the
//      residuals that read it), writes it and applies Adam to level 1 (step
//      mode), 2 or 4 cells of a row per thread;
//   6. for the heat problem reduces dL/dq of the conductivity nodes into a
//      per-tile partial (deterministic warp-range binning).
// The per-tile partials are summed by the per-instance tail kernel.
// The stencils are the discretisations of the paper's Sections 3.2 and 3.4:
//   Burgers, rows n >= 1:
//     r = (u^n_i - u^{n-1}_i)/dt + (F_{i+1/2} - F_{i-1/2})/dx
//         - nu (u^n_{i+1} - 2u^n_i + u^n_{i-1})/dx^2,
//     F = Engquist-Osher upwind flux of u^2/2, through a wall the same flux
//     against the zero wall value, odd ghosts for the viscous term;
//   heat, rows n >= 1 (row 0: (u^0_i - u_init_i)/dt):
//     r = (u^n_i - u^{n-1}_i)/dt
//         - [k_{i+1/2}(u^n_{i+1}-u^n_i) - k_{i-1/2}(u^n_i-u^n_{i-1})]/dx^2,
//     k_{i+1/2} = k((u^n_i + u^n_{i+1})/2), k piecewise linear in the nodes q;
//   Poisson (Section 3.1, cell layout on [0,1]^2, axes (y, x)), every cell:
//     r = (u_E - 2u + u_W)/dx^2 + (u_N - 2u + u_S)/dy^2 - f, a wall's ghost
//     -2 u_0 + u_1/3 (quadratic extrapolation through the zero wall value).
#include <algorithm>

#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

template <int TY, int TX>
struct StGeom {
  static constexpr int HU = 2;                    // halo of the composed field
  static constexpr int UH = TY + 2 * HU;          // rows of the staged / composed region
  static constexpr int SX = 4;                    // region column of x0 (staging from x0 - 4)
  static constexpr int SW = TX + 2 * SX;          // row stride of the staged / composed region
  static constexpr int UW = TX + 2 * HU;          // composed columns x0 - 2 .. x0 + TX + 1
  static constexpr int RH = TY + 2, RW = TX + 2;  // residual region: tile plus 1
  static constexpr int NA = RH * RW;
  // residuals streamed down columns: one task = one column x a chunk of
  // rows, at most one task per thread
  static constexpr int NC1 = (MODIL_NT / RW) > 0 ? MODIL_NT / RW : 1;
  static constexpr int RC1 = (RH + NC1 - 1) / NC1;
  static constexpr int NRUN = MODIL_NT;           // measurement runs staged per tile
  // cells of a row per Adam task: 4 when that still gives every thread a task
  static constexpr int VW = (TY * TX >= 4 * MODIL_NT) ? 4 : 2;
  static constexpr int NFACE = (TX + 1) * TY;      // heat: faces of the owned rows
  static constexpr int FPT = (NFACE + MODIL_NT - 1) / MODIL_NT;
  static_assert(TX % 4 == 0, "tile width: whole 4-element vectors");
};

// Shared-memory layout in bytes (the pyramid of coarse levels goes last).
template <class T, int PDE, int TY, int TX>
struct StSmem {
  using G = StGeom<TY, TX>;
  static constexpr bool HEAT = (PDE == PDE_HEAT);
  static constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_inst = 0;
  static constexpr size_t o_reg = a16(o_inst + sizeof(DevInst));        // 5 x MAXL ints + misc
  static constexpr size_t o_red = a16(o_reg + 4 * (6 * MODIL_MAXL + 4));
  static constexpr size_t o_p0 = a16(o_red + 8 * 16);                   // staged level 0
  static constexpr size_t o_u = a16(o_p0 + sizeof(T) * G::UH * G::SW);  // composed field
  static constexpr size_t o_a = a16(o_u + sizeof(T) * G::UH * G::SW);   // lambda * dr/du
  // lambda * dr/du per stencil neighbour: W, centre, E, S (and N for Poisson)
  static constexpr int NJ = (PDE == PDE_POISSON) ? 5 : 4;
  static constexpr size_t o_m = a16(o_a + sizeof(T) * NJ * G::NA);
  static constexpr size_t o_v = a16(o_m + sizeof(T) * TY * TX);
  static constexpr size_t o_rc = a16(o_v + sizeof(double) * TY * TX);  // runs: cell
  static constexpr size_t o_rb = a16(o_rc + 4 * G::NRUN);              // runs: first value index
  static constexpr size_t o_rv = a16(o_rb + 4 * (G::NRUN + 1));        // runs: first value
  static constexpr size_t o_mu = a16(o_rv + sizeof(T) * G::NRUN);      // heat: lambda * dr/dk
  static constexpr size_t o_q = a16(o_mu + (HEAT ? sizeof(T) * 2 * TY * TX : 0));
  static constexpr size_t o_ic = a16(o_q + (HEAT ? sizeof(T) * MODIL_MAXK : 0));
  static constexpr size_t o_pyr = a16(o_ic + (HEAT ? sizeof(T) * G::SW : 0));
  static size_t bytes(size_t pyr_elems) { return o_pyr + sizeof(T) * pyr_elems; }
  // heat: the dL/dq bins reuse the lambda * dr/du arrays once the gather is done
  static_assert(!HEAT || sizeof(T) * 4 * G::NA >= 8 * (MODIL_NT / 32) * MODIL_MAXK, "bins");
};

// Coefficients of a tile in the working precision, converted once per block.
template <class T>
struct StCoef {
  T idt, idx1, idx2, idy2, nu, lam_scale, wd2, gscale;
};

// 16-byte asynchronous copies (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
template <class T>
__device__ __forceinline__ void cp_async_x4(T* dst, const T* src) {
  cp_async16(dst, src);
  if (sizeof(T) == 8) cp_async16(dst + 2, src + 2);
}
// VW (2 or 4) consecutive elements: asynchronous copy, load, store
template <int VW, class T>
__device__ __forceinline__ void cp_async_v(T* dst, const T* src) {
  if constexpr (VW * sizeof(T) == 8)
    cp_async(reinterpret_cast<double*>(dst), reinterpret_cast<const double*>(src));
  else if constexpr (VW * sizeof(T) == 16)
    cp_async16(dst, src);
  else
    cp_async_x4(dst, src);
}
template <int VW, class T>
__device__ __forceinline__ void ldv(const T* s, T* v) {
  if constexpr (VW == 4 && sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(s);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (VW == 2 && sizeof(T) == 4) {
    const float2 a = *reinterpret_cast<const float2*>(s);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int k = 0; k < VW; k += 2) {
      const double2 a = *reinterpret_cast<const double2*>(s + k);
      v[k] = a.x; v[k + 1] = a.y;
    }
  }
}
template <int VW, class T>
__device__ __forceinline__ void stv(T* d, const T* v) {
  if constexpr (VW == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (VW == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(d) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int k = 0; k < VW; k += 2) *reinterpret_cast<double2*>(d + k) = make_double2(v[k], v[k + 1]);
  }
}

// Block sums of two per-thread values (compensated FP32 or FP64), fixed
// order, two barriers; every thread gets both results.  scratch: 128 bytes.
template <int NT>
__device__ __forceinline__ void block_sum2(float a, float b, void* scratch, double& sa, double& sb) {
  float ah = a, al = 0.f, bh = b, bl = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float x0 = __shfl_xor_sync(0xffffffffu, ah, o), x1 = __shfl_xor_sync(0xffffffffu, al, o);
    const float y0 = __shfl_xor_sync(0xffffffffu, bh, o), y1 = __shfl_xor_sync(0xffffffffu, bl, o);
    ff_add(ah, al, x0, x1);
    ff_add(bh, bl, y0, y1);
  }
  float* sc = reinterpret_cast<float*>(scratch);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sc[4 * w] = ah; sc[4 * w + 1] = al; sc[4 * w + 2] = bh; sc[4 * w + 3] = bl; }
  __syncthreads();
  float h0 = sc[0], l0 = sc[1], h1 = sc[2], l1 = sc[3];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) {
    ff_add(h0, l0, sc[4 * i], sc[4 * i + 1]);
    ff_add(h1, l1, sc[4 * i + 2], sc[4 * i + 3]);
  }
  sa = (double)h0 + (double)l0;
  sb = (double)h1 + (double)l1;
}
template <int NT>
__device__ __forceinline__ void block_sum2(double a, double b, void* scratch, double& sa, double& sb) {
  a = warp_sum(a);
  b = warp_sum(b);
  double* sc = reinterpret_cast<double*>(scratch);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sc[2 * w] = a; sc[2 * w + 1] = b; }
  __syncthreads();
  sa = 0.0;
  sb = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) { sa += sc[2 * i]; sb += sc[2 * i + 1]; }
}

// Conductivity k(u), piecewise linear in nodes q_0..q_K at u_j = j/K, constant
// outside [0, 1].  Returns k; s, th are the segment and local coordinate.
template <class T>
__device__ __forceinline__ T kcond(T u, const T* q, int K, int& s, T& th, T& dk) {
  const T ub = tmin(tmax(u, T(0)), T(1));
  const T x = ub * T(K);
  int si = (int)tfloor(x);
  si = si > K - 1 ? K - 1 : si;
  s = si;
  th = x - T(si);
  const T d = q[si + 1] - q[si];
  dk = (u >= T(0) && u <= T(1)) ? T(K) * d : T(0);
  return q[si] + th * d;
}

template <class T>
__device__ __forceinline__ T eo_flux(T a, T b, T& da, T& db) {
  const T ap = tmax(a, T(0));
  const T bm = tmin(b, T(0));
  da = ap;
  db = bm;
  return T(0.5) * ap * ap + T(0.5) * bm * bm;
}

// FP32: four blocks per SM (64 registers a thread), so that a 512 x 512 grid
// in 16 x 32 tiles runs in one wave on 152 SMs.
template <class T, int PDE, int TY, int TX>
__global__ void __launch_bounds__(MODIL_NT, sizeof(T) == 4 ? 4 : 2)
k_fine_st(const __grid_constant__ Arena<T> A, int mode, int cur) {
  using G = StGeom<TY, TX>;
  using S = StSmem<T, PDE, TY, TX>;
  extern __shared__ __align__(16) unsigned char smem[];
  DevInst& D = *reinterpret_cast<DevInst*>(smem + S::o_inst);
  int* reg = reinterpret_cast<int*>(smem + S::o_reg);
  int* loy = reg;
  int* lox = reg + MODIL_MAXL;
  int* hgt = reg + 2 * MODIL_MAXL;
  int* wid = reg + 3 * MODIL_MAXL;
  int* poff = reg + 4 * MODIL_MAXL;
  // 1 / (region width) per level: row = floor((idx + 1/2) / width) in FP32 is
  // exact for these region sizes (quotients below a few hundred)
  float* winv = reinterpret_cast<float*>(reg + 5 * MODIL_MAXL + 1);
  void* red = smem + S::o_red;
  T* P0 = reinterpret_cast<T*>(smem + S::o_p0);
  T* uR = reinterpret_cast<T*>(smem + S::o_u);
  T* aJ = reinterpret_cast<T*>(smem + S::o_a);
  T* mS = reinterpret_cast<T*>(smem + S::o_m);
  double* vS = reinterpret_cast<double*>(smem + S::o_v);
  int* rcS = reinterpret_cast<int*>(smem + S::o_rc);
  int* rbS = reinterpret_cast<int*>(smem + S::o_rb);
  T* rvS = reinterpret_cast<T*>(smem + S::o_rv);
  T* muE = reinterpret_cast<T*>(smem + S::o_mu);
  T* muW = muE + TY * TX;
  T* qS = reinterpret_cast<T*>(smem + S::o_q);
  T* icS = reinterpret_cast<T*>(smem + S::o_ic);
  T* pyr = reinterpret_cast<T*>(smem + S::o_pyr);
  double* bins = reinterpret_cast<double*>(aJ);  // heat, after the gather
  __shared__ AdamCoef acS[1];
  __shared__ StCoef<T> cS[1];

  const int tid = threadIdx.x;
  // One tile; `first` is the block's first tile (the only one that waits on
  // the previous launch).  A persistent launch calls it for every tile it
  // takes from the queue, an ordinary launch once for tile blockIdx.x.
  auto tile = [&](const int gt, const bool first) {
  // ---- prologue: data no kernel of a step writes -----------------------------
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  const int nrun = re - rb;              // runs hold distinct cells of the tile
  const int nst = min(nrun, G::NRUN);    // runs staged in shared memory
  // Pyramid regions, computed by warp 0.  Level 0 covers the tile plus the
  // halo; level l+1 covers what interpolating level l needs,
  // [lo/2 - 1, hi/2 + 1], clipped to the level.  Unrolled, level l starts at
  // (lo0 - 2^(l+1) + 2) >> l and ends at (hi0 + 2^(l+1) - 2) >> l, so lane l
  // computes level l directly.
  auto regions = [&]() {
    const int L = D.nlev;
    const int ny = D.n[0][1], nx = D.n[0][2];
    const int local = gt - D.tile_base[0];
    const int ty = local / D.nt[0][2], tx = local - ty * D.nt[0][2];
    const int y0 = ty * TY, x0 = tx * TX;
    const int a0 = max(0, y0 - G::HU), b0 = min(ny - 1, y0 + TY - 1 + G::HU);
    const int c0 = max(0, x0 - G::HU), d0 = min(nx - 1, x0 + TX - 1 + G::HU);
    int ly = 0, lx = 0, h = 0, w = 1;
    if (tid < L) {
      const int k = (1 << (tid + 1)) - 2;
      ly = max(0, (a0 - k) >> tid);
      lx = max(0, (c0 - k) >> tid);
      h = min(D.n[tid][1] - 1, (b0 + k) >> tid) - ly + 1;
      w = min(D.n[tid][2] - 1, (d0 + k) >> tid) - lx + 1;
    }
    // the pyramid holds levels 1 .. L-1 back to back: exclusive prefix sum
    const int sz = (tid >= 1 && tid < L) ? h * w : 0;
    int inc = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (tid >= o) inc += v;
    }
    if (tid < L) {
      loy[tid] = ly; lox[tid] = lx; hgt[tid] = h; wid[tid] = w;
      winv[tid] = 1.0f / (float)w;
      poff[tid] = inc - sz;
    }
  };
  load_inst(&D, A, ii);
  __syncthreads();
  if (tid < 32) regions();
  __syncthreads();

  const int L = D.nlev;
  const int ny = D.n[0][1], nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int ty = local / D.nt[0][2], tx = local - ty * D.nt[0][2];
  const int y0 = ty * TY, x0 = tx * TX;
  const int hy = min(TY, ny - y0), hx = min(TX, nx - x0);  // owned extent (ragged edge)
  const int K = D.nk - 1;
  // once per block (read after the staging barrier): no per-thread
  // conversions of FP64 coefficients
  if (tid == 32) {
    StCoef<T> c;
    const T dt = (T)D.h[1], dx = (T)D.h[2];
    c.idt = T(1) / dt;
    c.idx1 = T(1) / dx;
    c.idx2 = T(1) / (dx * dx);
    c.idy2 = T(1) / (dt * dt);
    c.nu = (T)D.coef[0];
    c.lam_scale = T(2) * (T)D.w_res_dV;
    c.wd2 = T(2) * (T)D.w_data_n;
    c.gscale = (T)A.gscale;
    *cS = c;
  }

  const T* __restrict__ P = A.p[cur];
  const long long o0 = D.off[0][0];
  // 16-byte vectors need rows and the level start on 4-element boundaries
  // (the tile origin x0 is a multiple of TX, so of 4; so is the owned width)
  const bool vec = ((nx & 3) == 0) && ((o0 & 3) == 0);
  auto stage_level = [&](int l) {
    const T* src = P + D.off[0][l];
    if (l == 0) {  // rows y0-2 .. y0+TY+1, columns x0-4 .. x0+TX+3, 4 elements per copy
      constexpr int CW = G::SW / 4;
      for (int k = tid; k < G::UH * CW; k += MODIL_NT) {
        const int ry = k / CW, cx = k - ry * CW;
        const int y = y0 - G::HU + ry, x = x0 - G::SX + 4 * cx;
        if (y < 0 || y >= ny) continue;
        T* dst = P0 + ry * G::SW + 4 * cx;
        const T* s0 = src + (long long)y * nx + x;
        if (vec) {
          if (x >= 0 && x < nx) cp_async_x4(dst, s0);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (x + j >= 0 && x + j < nx) cp_async(dst + j, s0 + j);
        }
      }
      return;
    }
    const int nxl = D.n[l][2];
    for (int idx = tid; idx < hgt[l] * wid[l]; idx += MODIL_NT) {
      const int ry = (int)(((float)idx + 0.5f) * winv[l]), rx = idx - ry * wid[l];
      const int y = loy[l] + ry, x = lox[l] + rx;
      cp_async(pyr + poff[l] + idx, src + (long long)y * nxl + x);
    }
  };
  // Levels below the tail and the level-1 Adam state were last written two
  // or more launches ago; the tail levels are written by the previous launch.
  const int pre = min(L, D.tail);
  for (int l = 0; l < pre; ++l) stage_level(l);
  constexpr int VW = G::VW, QW = TX / VW;
  if (mode == MODE_STEP) {
    for (int k = tid; k < TY * QW; k += MODIL_NT) {
      const int oy = k / QW, ox = VW * (k - oy * QW);
      if (oy >= hy || ox >= hx) continue;
      const long long e = o0 + (long long)(y0 + oy) * nx + (x0 + ox);
      const int s = oy * TX + ox;
      if (vec) {
        cp_async_v<VW>(mS + s, A.m + e);
        cp_async_v<VW>(vS + s, A.v + e);
      } else {
#pragma unroll
        for (int j = 0; j < VW; ++j)
          if (ox + j < hx) {
            cp_async(mS + s + j, A.m + e + j);
            cp_async(vS + s + j, A.v + e + j);
          }
      }
    }
  }
  // the tile's measurement runs (static)
  for (int i = tid; i < nst; i += MODIL_NT) {
    cp_async(reinterpret_cast<float*>(rcS + i), reinterpret_cast<const float*>(A.run_cell + rb + i));
    cp_async(reinterpret_cast<float*>(rbS + i), reinterpret_cast<const float*>(A.run_beg + rb + i));
    cp_async(rvS + i, A.run_v0 + rb + i);
  }
  if (tid == 0 && nst > 0)
    cp_async(reinterpret_cast<float*>(rbS + nst), reinterpret_cast<const float*>(A.run_beg + rb + nst));
  if (PDE == PDE_HEAT) {
    if (y0 == 0)
      for (int x = lox[0] + tid; x < lox[0] + wid[0]; x += MODIL_NT)
        cp_async(icS + (x - x0 + G::SX), A.aux + D.aux_off + x);
  }

  if (first) {
    pdl_wait();
    pdl_trigger();
  }
  if (tid == 0) *acS = adam_coef(D, A.st[ii]);  // once per block: no per-thread FP64
  for (int l = pre; l < L; ++l) stage_level(l);
  // the nodes are stepped by the tail kernel, the previous launch
  if (PDE == PDE_HEAT)
    for (int j = tid; j < D.nk; j += MODIL_NT) cp_async(qS + j, A.kq + D.k_off + j);
  cp_async_wait_all();
  __syncthreads();

  // ---- 1. Horner on the pyramid: w_l = u_l + T w_{l+1}, coarse to fine -------
  auto horner_level = [&](int l, int first, int stride) {  // l >= 1, in place
    const int nyc = D.n[l + 1][1], nxc = D.n[l + 1][2];
    const T* wc = pyr + poff[l + 1];
    const int cw = wid[l + 1], cly = loy[l + 1], clx = lox[l + 1];
    const int nreg = hgt[l] * wid[l];
    for (int idx = first; idx < nreg; idx += stride) {
      const int ry = (int)(((float)idx + 0.5f) * winv[l]), rx = idx - ry * wid[l];
      const int y = loy[l] + ry, x = lox[l] + rx;
      int jy0, jy1, jx0, jx1;
      T wy0, wy1, wx0, wx1;
      prolong_taps<T>(y, nyc, jy0, jy1, wy0, wy1);
      prolong_taps<T>(x, nxc, jx0, jx1, wx0, wx1);
      const T* r0 = wc + (jy0 - cly) * cw - clx;
      const T* r1 = wc + (jy1 - cly) * cw - clx;
      pyr[poff[l] + idx] += wy0 * (wx0 * r0[jx0] + wx1 * r0[jx1]) + wy1 * (wx0 * r1[jx0] + wx1 * r1[jx1]);
    }
  };
  // the small coarse regions (levels >= 2) by one warp, warp-synchronously
  if (tid < 32) {
    for (int l = L - 2; l >= 2; --l) {
      horner_level(l, tid, 32);
      __syncwarp();
    }
  }
  __syncthreads();
  if (L >= 3) {
    horner_level(1, tid, MODIL_NT);
    __syncthreads();
  }
  // Level 0 streamed down columns of the region: a task is a column and a
  // chunk of rows; the column's taps into level 1 are fixed, the row taps have
  // the closed form below, and each row of level 1 is interpolated in x once
  // per task.
  if (L >= 2) {
    constexpr int NC0 = (MODIL_NT / G::UW) > 0 ? MODIL_NT / G::UW : 1;
    constexpr int RC0 = (G::UH + NC0 - 1) / NC0;
    const int nyc = D.n[1][1], nxc = D.n[1][2];
    const int cw = wid[1];
    const T* wb = pyr + poff[1] - loy[1] * cw - lox[1];  // wb[Y * cw + X] = w_1(Y, X)
    for (int t = tid; t < G::UW * NC0; t += MODIL_NT) {
      const int ch = t / G::UW, col = t - ch * G::UW;
      const int x = x0 - G::HU + col;
      if (x < 0 || x >= nx) continue;
      int jx0, jx1;
      T wx0, wx1;
      prolong_taps<T>(x, nxc, jx0, jx1, wx0, wx1);
      const int r0 = max(ch * RC0, G::HU - y0);
      const int r1 = min(min((ch + 1) * RC0, G::UH), ny - y0 + G::HU);
      int ja = -2;
      T va = T(0), vb = T(0);
      for (int ry = r0; ry < r1; ++ry) {
        const int y = y0 - G::HU + ry;
        // fine row y between coarse rows lo and lo + 1: weights 5/4 - t/2 and
        // t/2 - 1/4 with t = y - 2 lo in {0, 1, 2, 3} (3/4 and 1/4 inside,
        // the extrapolated 5/4 and -1/4 at the ends); one coarse row: a copy
        int lo = 0, hi = 0;
        T wl = T(1), wh = T(0);
        if (nyc > 1) {
          lo = min(max((y - 1) >> 1, 0), nyc - 2);
          hi = lo + 1;
          wl = T(1.25) - T(0.5) * (T)(y - 2 * lo);
          wh = T(1) - wl;
        }
        if (lo != ja) {
          va = (lo == ja + 1) ? vb : wx0 * wb[lo * cw + jx0] + wx1 * wb[lo * cw + jx1];
          vb = wx0 * wb[hi * cw + jx0] + wx1 * wb[hi * cw + jx1];
          ja = lo;
        }
        const int o = ry * G::SW + col + (G::SX - G::HU);
        uR[o] = P0[o] + (wl * va + wh * vb);
      }
    }
  }
  __syncthreads();
  const T* Ub = (L >= 2) ? uR : P0;  // composed field, region layout
  auto U = [&](int y, int x) -> T { return Ub[(y - y0 + G::HU) * G::SW + (x - x0 + G::SX)]; };

  if (mode == MODE_COMPOSE) {
    T* out = A.ufine + D.fine_off[0];
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      if (oy < hy && ox < hx) out[(long long)(y0 + oy) * nx + (x0 + ox)] = U(y0 + oy, x0 + ox);
    }
    return;
  }

  // ---- 2./3. residuals, local Jacobians, owned r^2 (streamed down columns) --
  const StCoef<T> cf = *cS;
  const bool adj = (mode != MODE_LOSS);
  float racc_f = 0.f;
  double racc_d = 0.0;  // FP64 problems
  for (int t = tid; t < G::RW * G::NC1; t += MODIL_NT) {
    const int ch = t / G::RW, rx = t - ch * G::RW;
    const int x = x0 - 1 + rx;
    const bool xin = (x >= 0 && x < nx);
    const bool hw = (x > 0), he = (x < nx - 1);
    const bool ocol = (rx >= 1 && rx <= hx);
    const T* up = Ub + G::SW + (rx - 1 + G::SX);  // row ry of the residual region: up[ry * SW]
    const int r0 = ch * G::RC1, r1 = min(r0 + G::RC1, G::RH);
    T uprev = up[(r0 - 1) * G::SW];
    for (int ry = r0; ry < r1; ++ry) {
      const int y = y0 - 1 + ry;
      const T* uq = up + ry * G::SW;
      const T uc = uq[0], uo = uprev;
      uprev = uc;
      T r = T(0), J0 = T(0), J1 = T(0), J2 = T(0), J3 = T(0), J4 = T(0), dE = T(0), dW = T(0);
      bool valid = xin && (y >= 0 && y < ny);
      if (PDE == PDE_BURGERS && y == 0) valid = false;
      if (valid && PDE == PDE_POISSON) {
        // 5-point Laplacian minus f; a wall's ghost value is the quadratic
        // extrapolation -2 u_0 + u_1 / 3 through the zero wall value (both
        // axes have >= 2 cells, so the inner neighbour exists)
        const bool hs = (y > 0), hn = (y < ny - 1);
        const T third = T(1) / T(3);
        const T uw = uq[-1], ue = uq[1], un = uq[G::SW];
        const T gw = hw ? uw : T(-2) * uc + ue * third;
        const T ge = he ? ue : T(-2) * uc + uw * third;
        const T gs = hs ? uo : T(-2) * uc + un * third;
        const T gn = hn ? un : T(-2) * uc + uo * third;
        const T f = A.aux[D.aux_off + (long long)y * nx + x];
        r = (ge - T(2) * uc + gw) * cf.idx2 + (gn - T(2) * uc + gs) * cf.idy2 - f;
        J1 = (T(-2) - (hw ? T(0) : T(2)) - (he ? T(0) : T(2))) * cf.idx2 +
             (T(-2) - (hs ? T(0) : T(2)) - (hn ? T(0) : T(2))) * cf.idy2;
        J0 = hw ? (T(1) + (he ? T(0) : third)) * cf.idx2 : T(0);  // dr/du at x - 1
        J2 = he ? (T(1) + (hw ? T(0) : third)) * cf.idx2 : T(0);  // x + 1
        J3 = hs ? (T(1) + (hn ? T(0) : third)) * cf.idy2 : T(0);  // y - 1
        J4 = hn ? (T(1) + (hs ? T(0) : third)) * cf.idy2 : T(0);  // y + 1
      } else if (valid) {
        if (PDE == PDE_HEAT && y == 0) {
          r = (uc - icS[x - x0 + G::SX]) * cf.idt;
          J1 = cf.idt;
        } else {
          const T uw = hw ? uq[-1] : -uc;
          const T ue = he ? uq[1] : -uc;
          if (PDE == PDE_BURGERS) {
            // the flux through a wall is the upwind flux against the zero wall value
            T dFEc, dFEe, dFWw, dFWc;
            const T FE = eo_flux(uc, he ? ue : T(0), dFEc, dFEe);
            const T FW = eo_flux(hw ? uw : T(0), uc, dFWw, dFWc);
            const T lap = (ue - T(2) * uc + uw) * cf.idx2;
            r = (uc - uo) * cf.idt + (FE - FW) * cf.idx1 - cf.nu * lap;
            const T cdiag = T(-2) - (hw ? T(0) : T(1)) - (he ? T(0) : T(1));
            J1 = cf.idt + (dFEc - dFWc) * cf.idx1 - cf.nu * cdiag * cf.idx2;
            J0 = hw ? (-dFWw * cf.idx1 - cf.nu * cf.idx2) : T(0);
            J2 = he ? (dFEe * cf.idx1 - cf.nu * cf.idx2) : T(0);
            J3 = -cf.idt;
          } else {
            int s;
            T th, dk;
            T kE, kW, dEc, dEe, dWc, dWw;
            const T duE = ue - uc, duW = uc - uw;
            if (he) {
              kE = kcond(T(0.5) * (uc + ue), qS, K, s, th, dk);
              dEc = -kE + T(0.5) * dk * duE;
              dEe = kE + T(0.5) * dk * duE;
            } else {
              kE = qS[0];
              dEc = T(-2) * kE;
              dEe = T(0);
            }
            if (hw) {
              kW = kcond(T(0.5) * (uw + uc), qS, K, s, th, dk);
              dWc = kW + T(0.5) * dk * duW;
              dWw = -kW + T(0.5) * dk * duW;
            } else {
              kW = qS[0];
              dWc = T(2) * kW;
              dWw = T(0);
            }
            r = (uc - uo) * cf.idt - (kE * duE - kW * duW) * cf.idx2;
            J1 = cf.idt - (dEc - dWc) * cf.idx2;
            J2 = -dEe * cf.idx2;
            J0 = dWw * cf.idx2;
            J3 = -cf.idt;
            dE = -duE * cf.idx2;  // dr/dk_E
            dW = duW * cf.idx2;   // dr/dk_W
          }
        }
      }
      const bool owned = valid && ry >= 1 && ry <= hy && ocol;
      if (owned) {
        if (sizeof(T) == 4) racc_f += (float)(r * r);
        else racc_d += (double)(r * r);
      }
      if (adj) {
        const T lam = cf.lam_scale * r;
        const int c = ry * G::RW + rx;
        aJ[0 * G::NA + c] = lam * J0;
        aJ[1 * G::NA + c] = lam * J1;
        aJ[2 * G::NA + c] = lam * J2;
        aJ[3 * G::NA + c] = lam * J3;
        if (PDE == PDE_POISSON) aJ[4 * G::NA + c] = lam * J4;
        if (PDE == PDE_HEAT && ry >= 1 && ry <= TY && rx >= 1 && rx <= TX) {
          const int o = (ry - 1) * TX + (rx - 1);
          muE[o] = owned ? lam * dE : T(0);
          muW[o] = owned ? lam * dW : T(0);
        }
      }
    }
  }
  // ---- 3b. off-grid points whose corner cells the tile owns: the sampled
  // value minus the measurement per record (the tile of a point's lower
  // corner counts its misfit) --------------------------------------------------
  float dacc_f = 0.f;
  double dacc_d = 0.0;
  if (A.pt_ptr) {
    const int p1 = A.pt_ptr[gt + 1];
    for (int j = A.pt_ptr[gt] + tid; j < p1; j += MODIL_NT) {
      T smp = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int cell = A.pt_cell[4 * (long long)j + k];
        const int yy = cell / nx, xx = cell - (cell / nx) * nx;
        smp += A.pt_w[4 * (long long)j + k] * U(yy, xx);
      }
      const T dd = smp - A.pt_val[j];
      A.pt_diff[j] = dd;
      if (A.pt_own[j]) {
        if (sizeof(T) == 4) dacc_f += (float)(dd * dd);
        else dacc_d += (double)(dd * dd);
      }
    }
  }
  __syncthreads();  // aJ / muE complete; point misfits written

  // ---- 4. data term: runs of equal cells inside the tile; its gradient joins
  // the cell's own residual term ----------------------------------------------
  for (int i = tid; i < nrun; i += MODIL_NT) {
    int cell, e0, e1;
    T v0;
    if (i < nst) {
      cell = rcS[i]; e0 = rbS[i]; e1 = rbS[i + 1]; v0 = rvS[i];
    } else {  // more runs than staged (dense measurements)
      cell = A.run_cell[rb + i]; e0 = A.run_beg[rb + i]; e1 = A.run_beg[rb + i + 1]; v0 = A.run_v0[rb + i];
    }
    const int y = cell / nx, x = cell - (cell / nx) * nx;
    const T u = U(y, x);
    T d = u - v0;
    T sd = d, sq = d * d;
    for (int e = e0 + 1; e < e1; ++e) {  // repeated measurements of a cell
      d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    if (sizeof(T) == 4) dacc_f += (float)sq;
    else dacc_d += (double)sq;
    if (adj) aJ[1 * G::NA + (y - y0 + 1) * G::RW + (x - x0 + 1)] += cf.wd2 * sd;
  }

  double rsum, dsum;  // the barriers inside also publish the data gradient
  if (sizeof(T) == 4) block_sum2<MODIL_NT>(racc_f, dacc_f, red, rsum, dsum);
  else block_sum2<MODIL_NT>(racc_d, dacc_d, red, rsum, dsum);
  if (tid == 0) {
    A.part[(long long)gt * A.npart + 0] = rsum;
    A.part[(long long)gt * A.npart + 1] = dsum;
  }

  // the points' gradient: each owned corner cell sums weight * misfit over
  // the records that reach it (fixed order)
  if (adj && A.pc_ptr && A.pc_ptr[gt + 1] > A.pc_ptr[gt]) {
    const int c1 = A.pc_ptr[gt + 1];
    for (int rr = A.pc_ptr[gt] + tid; rr < c1; rr += MODIL_NT) {
      const int cell = A.pc_cell[rr];
      const int yy = cell / nx, xx = cell - (cell / nx) * nx;
      T acc = T(0);
      for (int e = A.pc_beg[rr]; e < A.pc_beg[rr + 1]; ++e) acc += A.pe_w[e] * A.pt_diff[A.pe_rec[e]];
      aJ[1 * G::NA + (yy - y0 + 1) * G::RW + (xx - x0 + 1)] += cf.wd2 * acc;
    }
    __syncthreads();
  }

  if (adj) {
    // ---- 5. gather dL/du (each cell sums lambda * dr/du over the residuals
    // that read it), write it, Adam on level 1; VW cells of a row per task ---
    const AdamCoef ac = *acS;
    T* __restrict__ Gp = A.g + o0;
    for (int q = tid; q < TY * QW; q += MODIL_NT) {
      const int oy = q / QW, ox = VW * (q - oy * QW);
      if (oy >= hy || ox >= hx) continue;
      const int c = (oy + 1) * G::RW + (ox + 1);
      T g[VW];
#pragma unroll
      for (int k = 0; k < VW; ++k)
        g[k] = (aJ[1 * G::NA + c + k] + aJ[0 * G::NA + c + k + 1] + aJ[2 * G::NA + c + k - 1] +
                aJ[3 * G::NA + c + k + G::RW] + (PDE == PDE_POISSON ? aJ[4 * G::NA + c + k - G::RW] : T(0))) *
               cf.gscale;
      const long long e = (long long)(y0 + oy) * nx + (x0 + ox);
      const int sp = (oy + G::HU) * G::SW + ox + G::SX, sm = oy * TX + ox;
      if (vec) {  // VW owned cells, aligned
        stv<VW>(Gp + e, g);
        if (mode == MODE_STEP) {
          T p[VW], m[VW];
          double v[VW];
          ldv<VW>(P0 + sp, p);
          ldv<VW>(mS + sm, m);
          ldv<VW>(vS + sm, v);
#pragma unroll
          for (int k = 0; k < VW; ++k) adam_update(p[k], m[k], v[k], g[k], ac);
          stv<VW>(A.p[cur ^ 1] + o0 + e, p);
          stv<VW>(A.m + o0 + e, m);
          stv<VW>(A.v + o0 + e, v);
        }
      } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          if (ox + k >= hx) break;
          Gp[e + k] = g[k];
          if (mode == MODE_STEP) {
            T p = P0[sp + k], m = mS[sm + k];
            double v = vS[sm + k];
            adam_update(p, m, v, g[k], ac);
            A.p[cur ^ 1][o0 + e + k] = p;
            A.m[o0 + e + k] = m;
            A.v[o0 + e + k] = v;
          }
        }
      }
    }

    // ---- 6. heat: dL/dq partial by deterministic warp-range binning -------
    if (PDE == PDE_HEAT) {
      __syncthreads();  // the bins reuse the gathered arrays
      for (int i = tid; i < (MODIL_NT / 32) * MODIL_MAXK; i += MODIL_NT) bins[i] = 0.0;
      int fs[G::FPT];
      T fa0[G::FPT], fa1[G::FPT];
      int smin = 1 << 30, smax = -1;
#pragma unroll
      for (int k = 0; k < G::FPT; ++k) {
        const int f = tid + k * MODIL_NT;
        fs[k] = -1;
        fa0[k] = T(0);
        fa1[k] = T(0);
        if (f < G::NFACE) {
          const int fy = f / (TX + 1), fx = f - fy * (TX + 1);
          const int y = y0 + fy;
          const int xl = x0 + fx - 1, xr = x0 + fx;
          if (fy < hy && fx <= hx && y >= 1) {
            T mu = T(0);
            if (fx >= 1) mu += muE[fy * TX + fx - 1];
            if (fx < hx) mu += muW[fy * TX + fx];
            int s = 0;
            T th = T(0), dk;
            if (xl >= 0 && xr < nx) kcond(T(0.5) * (U(y, xl) + U(y, xr)), qS, K, s, th, dk);
            fs[k] = s;
            fa0[k] = mu * (T(1) - th);
            fa1[k] = mu * th;
            smin = min(smin, s);
            smax = max(smax, s + 1);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
        smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      }
      __syncthreads();  // bins zeroed
      const int w = tid >> 5, lane = tid & 31;
      for (int j = smin; j <= smax; ++j) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < G::FPT; ++k) {
          if (fs[k] == j) acc += fa0[k];
          if (fs[k] >= 0 && fs[k] + 1 == j) acc += fa1[k];
        }
        const double s = (sizeof(T) == 4) ? warp_sum_ff((float)acc) : warp_sum((double)acc);
        if (lane == 0) bins[w * MODIL_MAXK + j] = s;
      }
      __syncthreads();
      for (int j = tid; j < D.nk; j += MODIL_NT) {
        double s = 0.0;
#pragma unroll
        for (int ww = 0; ww < MODIL_NT / 32; ++ww) s += bins[ww * MODIL_MAXK + j];
        A.part[(long long)gt * A.npart + 2 + j] = s;
      }
    }
  }
  };  // tile

  if (!A.persistent) {
    tile(blockIdx.x, true);
    return;
  }
  // persistent launch: take tiles from the queue until it is empty
  __shared__ int s_tile;
  if (tid == 0) s_tile = atomicAdd(A.queue, 1);
  __syncthreads();
  bool first = true;
  for (;;) {
    const int gt = s_tile;
    if (gt >= A.ntiles[0]) break;
    int nxt = 0;
    if (tid == 0) nxt = atomicAdd(A.queue, 1);  // the next tile, taken while this one runs
    tile(gt, first);
    first = false;
    // every thread read s_tile before the tile's first barrier
    if (tid == 0) s_tile = nxt;
    __syncthreads();  // shared memory is reused by the next tile; s_tile published
  }
  if (first) {  // no tile: still complete the dependency protocol
    pdl_wait();
    pdl_trigger();
  }
  // the last block out rewinds the queue for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(A.queue + 1, 1) == (int)gridDim.x - 1) {
      A.queue[0] = 0;
      A.queue[1] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <class T, int PDE, int TY, int TX>
static cudaError_t launch_one(const Arena<T>& A, int mode, int cur, size_t pyr, cudaStream_t s) {
  const size_t smem = StSmem<T, PDE, TY, TX>::bytes(pyr);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(A.persistent ? std::min(A.ntiles[0], A.persistent) : A.ntiles[0]);
  cfg.blockDim = dim3(MODIL_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fine_st<T, PDE, TY, TX>, A, mode, cur);
}

template <class T, int TY, int TX>
static cudaError_t launch_cfg(const Arena<T>& A, int pde, int mode, int cur, size_t pyr,
                              cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  if (pde == PDE_BURGERS) return launch_one<T, PDE_BURGERS, TY, TX>(A, mode, cur, pyr, s);
  if (pde == PDE_HEAT) return launch_one<T, PDE_HEAT, TY, TX>(A, mode, cur, pyr, s);
  if (pde == PDE_POISSON) return launch_one<T, PDE_POISSON, TY, TX>(A, mode, cur, pyr, s);
  return cudaErrorInvalidValue;
}

template <class T, int TY, int TX>
static cudaError_t prepare_cfg(int pde, size_t pyr) {
  if (pde == PDE_BURGERS)
    return raise_smem_limit(k_fine_st<T, PDE_BURGERS, TY, TX>, StSmem<T, PDE_BURGERS, TY, TX>::bytes(pyr));
  if (pde == PDE_HEAT)
    return raise_smem_limit(k_fine_st<T, PDE_HEAT, TY, TX>, StSmem<T, PDE_HEAT, TY, TX>::bytes(pyr));
  if (pde == PDE_POISSON)
    return raise_smem_limit(k_fine_st<T, PDE_POISSON, TY, TX>, StSmem<T, PDE_POISSON, TY, TX>::bytes(pyr));
  return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of the kernel a problem will use
// (called once at creation, outside any stream capture).
template <class T>
cudaError_t prepare_fine_st(int pde, int cfg, size_t pyr) {
  switch (cfg) {
    case 0: return prepare_cfg<T, 16, 32>(pde, pyr);
    case 1: return prepare_cfg<T, 16, 64>(pde, pyr);
    case 2: return prepare_cfg<T, 8, 64>(pde, pyr);
    case 3: return prepare_cfg<T, 32, 32>(pde, pyr);
    case 4: return prepare_cfg<T, 8, 128>(pde, pyr);
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t launch_fine_st(const Arena<T>& A, int pde, int cfg, int mode, int cur, size_t pyr,
                           cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_cfg<T, 16, 32>(A, pde, mode, cur, pyr, s);
    case 1: return launch_cfg<T, 16, 64>(A, pde, mode, cur, pyr, s);
    case 2: return launch_cfg<T, 8, 64>(A, pde, mode, cur, pyr, s);
    case 3: return launch_cfg<T, 32, 32>(A, pde, mode, cur, pyr, s);
    case 4: return launch_cfg<T, 8, 128>(A, pde, mode, cur, pyr, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, int PDE, int TY, int TX>
static cudaError_t occ(size_t pyr, int* n) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_fine_st<T, PDE, TY, TX>, MODIL_NT,
                                                       StSmem<T, PDE, TY, TX>::bytes(pyr));
}

template <class T, int TY, int TX>
static cudaError_t occ_pde(int pde, size_t pyr, int* n) {
  if (pde == PDE_POISSON) return occ<T, PDE_POISSON, TY, TX>(pyr, n);
  return pde == PDE_HEAT ? occ<T, PDE_HEAT, TY, TX>(pyr, n) : occ<T, PDE_BURGERS, TY, TX>(pyr, n);
}

// Resident fine-kernel blocks per SM (sizes the persistent launch).
cudaError_t fine_st_blocks_per_sm(int pde, int cfg, size_t pyr, int elem, int* n) {
  const bool d = (elem == 8);
  switch (cfg) {
    case 0: return d ? occ_pde<double, 16, 32>(pde, pyr, n) : occ_pde<float, 16, 32>(pde, pyr, n);
    case 1: return d ? occ_pde<double, 16, 64>(pde, pyr, n) : occ_pde<float, 16, 64>(pde, pyr, n);
    case 2: return d ? occ_pde<double, 8, 64>(pde, pyr, n) : occ_pde<float, 8, 64>(pde, pyr, n);
    case 3: return d ? occ_pde<double, 32, 32>(pde, pyr, n) : occ_pde<float, 32, 32>(pde, pyr, n);
    case 4: return d ? occ_pde<double, 8, 128>(pde, pyr, n) : occ_pde<float, 8, 128>(pde, pyr, n);
    default: return cudaErrorInvalidValue;
  }
}

template <int PDE>
static size_t smem_pde(int cfg, size_t pyr, bool d) {
  switch (cfg) {
    case 0: return d ? StSmem<double, PDE, 16, 32>::bytes(pyr) : StSmem<float, PDE, 16, 32>::bytes(pyr);
    case 1: return d ? StSmem<double, PDE, 16, 64>::bytes(pyr) : StSmem<float, PDE, 16, 64>::bytes(pyr);
    case 2: return d ? StSmem<double, PDE, 8, 64>::bytes(pyr) : StSmem<float, PDE, 8, 64>::bytes(pyr);
    case 3: return d ? StSmem<double, PDE, 32, 32>::bytes(pyr) : StSmem<float, PDE, 32, 32>::bytes(pyr);
    case 4: return d ? StSmem<double, PDE, 8, 128>::bytes(pyr) : StSmem<float, PDE, 8, 128>::bytes(pyr);
    default: return 0;
  }
}

size_t fine_st_smem_bytes(int pde, int cfg, size_t pyr, int elem) {
  const bool d = (elem == 8);
  if (pde == PDE_POISSON) return smem_pde<PDE_POISSON>(cfg, pyr, d);
  return pde == PDE_HEAT ? smem_pde<PDE_HEAT>(cfg, pyr, d) : smem_pde<PDE_BURGERS>(cfg, pyr, d);
}

template cudaError_t prepare_fine_st<float>(int, int, size_t);
template cudaError_t prepare_fine_st<double>(int, int, size_t);
template cudaError_t launch_fine_st<float>(const Arena<float>&, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_fine_st<double>(const Arena<double>&, int, int, int, int, size_t, cudaStream_t);

}  // namespace modil
