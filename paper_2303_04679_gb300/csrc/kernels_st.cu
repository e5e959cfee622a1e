// Fused fine-tile kernel of the space-time PDE family (viscous Burgers,
// heat conduction with unknown conductivity).  One block owns a TY x TX tile
// of the fine grid (axes t, x) and in one pass:
//   0. issues every global load it needs at once (cp.async into shared
//      memory): the tile's region of every level (tile plus a halo of 2 fine
//      cells, and at each coarser level half that plus one cell), the level-1
//      parameters and Adam moments of the tile, the conductivity nodes;
//   1. composes the field on the tile by Horner's scheme on that pyramid
//      (w_L = u_L, w_i = u_i + T_i w_{i+1}; paper Section 2.2);
//   2. evaluates every residual that touches the tile (tile plus 1 cell) and
//      its local Jacobian, dr/du at the 4 stencil points;
//   3. reduces r^2 over the residuals it owns (FP64 partial per tile);
//   4. forms dL/du on the tile in gather form: each cell sums
//      lambda * dr/du over the residuals that read it (lambda = 2 w dV r);
//   5. adds the data term of the measurements inside the tile;
//   6. writes the fine gradient, applies Adam to level 1 (step mode), and for
//      the heat problem reduces dL/dq of the conductivity nodes into a
//      per-tile partial (deterministic warp-range binning).
// The per-tile partials are summed by the per-instance tail kernel.
// The stencils are the discretisations of the paper's Sections 3.2 and 3.4:
//   Burgers, rows n >= 1:
//     r = (u^n_i - u^{n-1}_i)/dt + (F_{i+1/2} - F_{i-1/2})/dx
//         - nu (u^n_{i+1} - 2u^n_i + u^n_{i-1})/dx^2,
//     F = Engquist-Osher upwind flux of u^2/2, zero convective flux through
//     the walls, odd ghosts for the viscous term;
//   heat, rows n >= 1 (row 0: (u^0_i - u_init_i)/dt):
//     r = (u^n_i - u^{n-1}_i)/dt
//         - [k_{i+1/2}(u^n_{i+1}-u^n_i) - k_{i-1/2}(u^n_i-u^n_{i-1})]/dx^2,
//     k_{i+1/2} = k((u^n_i + u^n_{i+1})/2), k piecewise linear in the nodes q.
#include <algorithm>

#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

template <int TY, int TX>
struct StGeom {
  static constexpr int HU = 2;                    // halo of the composed field
  static constexpr int UH = TY + 2 * HU, UW = TX + 2 * HU;
  static constexpr int RH = TY + 2, RW = TX + 2;  // residual region: tile plus 1
  static constexpr int NFACE = (TX + 1) * TY;      // heat: faces of the owned rows
  static constexpr int FPT = (NFACE + MODIL_NT - 1) / MODIL_NT;
};

// Shared-memory layout in bytes (the pyramid of coarse levels goes last).
template <class T, int TY, int TX>
struct StSmem {
  using G = StGeom<TY, TX>;
  static constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_inst = 0;
  static constexpr size_t o_reg = a16(o_inst + sizeof(DevInst));        // 5 x MAXL ints + misc
  static constexpr size_t o_red = a16(o_reg + 4 * (6 * MODIL_MAXL + 4));
  static constexpr size_t o_sums = a16(o_red + 8 * 16);                 // 2 + MAXK doubles
  static constexpr size_t o_bins = a16(o_sums + 8 * (2 + MODIL_MAXK));  // 8 warps x MAXK
  static constexpr size_t o_u = a16(o_bins + 8 * 8 * MODIL_MAXK);
  static constexpr size_t o_a = a16(o_u + sizeof(T) * G::UH * G::UW);
  static constexpr size_t o_g = a16(o_a + sizeof(T) * 4 * G::RH * G::RW);
  static constexpr size_t o_mu = a16(o_g + sizeof(T) * TY * TX);
  static constexpr size_t o_p = a16(o_mu + sizeof(T) * 2 * TY * TX);
  static constexpr size_t o_m = a16(o_p + sizeof(T) * TY * TX);
  static constexpr size_t o_v = a16(o_m + sizeof(T) * TY * TX);
  static constexpr size_t o_q = a16(o_v + sizeof(double) * TY * TX);
  static constexpr size_t o_ic = a16(o_q + sizeof(T) * MODIL_MAXK);
  static constexpr size_t o_rc = a16(o_ic + sizeof(T) * G::UW);    // runs: cell
  static constexpr size_t o_rb = a16(o_rc + 4 * TY * TX);            // runs: first value index
  static constexpr size_t o_rv = a16(o_rb + 4 * (TY * TX + 1));      // runs: first value
  static constexpr size_t o_pyr = a16(o_rv + sizeof(T) * TY * TX);
  static size_t bytes(size_t pyr_elems) { return o_pyr + sizeof(T) * pyr_elems; }
};

// Conductivity k(u), piecewise linear in nodes q_0..q_K at u_j = j/K, constant
// outside [0, 1].  Returns k; s, th are the segment and local coordinate.
template <class T>
__device__ __forceinline__ T kcond(T u, const T* q, int K, int& s, T& th, T& dk) {
  const T ub = fmin(fmax(u, T(0)), T(1));
  const T x = ub * T(K);
  int si = (int)floor(x);
  si = si > K - 1 ? K - 1 : si;
  s = si;
  th = x - T(si);
  const T d = q[si + 1] - q[si];
  dk = (u >= T(0) && u <= T(1)) ? T(K) * d : T(0);
  return q[si] + th * d;
}

template <class T>
__device__ __forceinline__ T eo_flux(T a, T b, T& da, T& db) {
  const T ap = fmax(a, T(0));
  const T bm = fmin(b, T(0));
  da = ap;
  db = bm;
  return T(0.5) * ap * ap + T(0.5) * bm * bm;
}

template <class T, int PDE, int TY, int TX>
__global__ void __launch_bounds__(MODIL_NT)
k_fine_st(const __grid_constant__ Arena<T> A, int mode, int cur) {
  using G = StGeom<TY, TX>;
  using S = StSmem<T, TY, TX>;
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
  double* red = reinterpret_cast<double*>(smem + S::o_red);
  double* bins = reinterpret_cast<double*>(smem + S::o_bins);
  T* uR = reinterpret_cast<T*>(smem + S::o_u);
  T* aJ = reinterpret_cast<T*>(smem + S::o_a);
  T* gS = reinterpret_cast<T*>(smem + S::o_g);
  T* muE = reinterpret_cast<T*>(smem + S::o_mu);
  T* muW = muE + TY * TX;
  T* pS = reinterpret_cast<T*>(smem + S::o_p);
  T* mS = reinterpret_cast<T*>(smem + S::o_m);
  double* vS = reinterpret_cast<double*>(smem + S::o_v);
  T* qS = reinterpret_cast<T*>(smem + S::o_q);
  T* icS = reinterpret_cast<T*>(smem + S::o_ic);
  T* pyr = reinterpret_cast<T*>(smem + S::o_pyr);
  int* rcS = reinterpret_cast<int*>(smem + S::o_rc);
  int* rbS = reinterpret_cast<int*>(smem + S::o_rb);
  T* rvS = reinterpret_cast<T*>(smem + S::o_rv);
  float* redf = reinterpret_cast<float*>(red);
  __shared__ AdamCoef acS[1];

  const int tid = threadIdx.x;
  // One tile; `first` is the block's first tile (the only one that waits on
  // the previous launch).  A persistent launch calls it for every tile it
  // takes from the queue, an ordinary launch once for tile blockIdx.x.
  auto tile = [&](const int gt, const bool first) {
  // ---- prologue: data no kernel of a step writes -----------------------------
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  const int nrun = min(re - rb, TY * TX);  // runs hold distinct cells of the tile
  __syncthreads();

  const int L = D.nlev;
  const int ny = D.n[0][1], nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int ty = local / D.nt[0][2], tx = local - ty * D.nt[0][2];
  const int y0 = ty * TY, x0 = tx * TX;
  const int hy = min(TY, ny - y0), hx = min(TX, nx - x0);  // owned extent (ragged edge)
  const int K = D.nk - 1;
  // Pyramid regions.  Level 0 covers the tile plus the halo; level l+1 covers
  // what interpolating level l needs, [lo/2 - 1, hi/2 + 1], clipped to the
  // level.  Unrolled, level l starts at (lo0 - 2^(l+1) + 2) >> l and ends at
  // (hi0 + 2^(l+1) - 2) >> l, so thread l computes level l directly.
  if (tid < L) {
    const int a0 = max(0, y0 - G::HU), b0 = min(ny - 1, y0 + TY - 1 + G::HU);
    const int c0 = max(0, x0 - G::HU), d0 = min(nx - 1, x0 + TX - 1 + G::HU);
    auto region = [&](int l, int& ly, int& lx, int& h, int& w) {
      const int k = (1 << (l + 1)) - 2;
      ly = max(0, (a0 - k) >> l);
      lx = max(0, (c0 - k) >> l);
      h = min(D.n[l][1] - 1, (b0 + k) >> l) - ly + 1;
      w = min(D.n[l][2] - 1, (d0 + k) >> l) - lx + 1;
    };
    int ly, lx, h, w, tot = 0;
    for (int k = 1; k < tid; ++k) {
      region(k, ly, lx, h, w);
      tot += h * w;
    }
    region(tid, ly, lx, h, w);
    loy[tid] = ly; lox[tid] = lx; hgt[tid] = h; wid[tid] = w;
    winv[tid] = 1.0f / (float)w;
    poff[tid] = tot;
  }
  __syncthreads();

  const T* __restrict__ P = A.p[cur];
  auto stage_level = [&](int l) {
    const T* src = P + D.off[0][l];
    if (l == 0) {  // the fixed window of the fine level (compile-time extents)
      for (int idx = tid; idx < G::UH * G::UW; idx += MODIL_NT) {
        const int ry = idx / G::UW, rx = idx - ry * G::UW;
        const int y = y0 - G::HU + ry, x = x0 - G::HU + rx;
        if (y >= 0 && y < ny && x >= 0 && x < nx) cp_async(uR + idx, src + (long long)y * nx + x);
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
  const long long o0 = D.off[0][0];
  if (mode == MODE_STEP) {
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      if (oy >= hy || ox >= hx) continue;
      const long long e = o0 + (long long)(y0 + oy) * nx + (x0 + ox);
      cp_async(pS + idx, P + e);
      cp_async(mS + idx, A.m + e);
      cp_async(vS + idx, A.v + e);
    }
  }
  // the tile's measurement runs (static)
  for (int i = tid; i < nrun; i += MODIL_NT) {
    cp_async(reinterpret_cast<float*>(rcS + i), reinterpret_cast<const float*>(A.run_cell + rb + i));
    cp_async(reinterpret_cast<float*>(rbS + i), reinterpret_cast<const float*>(A.run_beg + rb + i));
    cp_async(rvS + i, A.run_v0 + rb + i);
  }
  if (tid == 0 && nrun > 0)
    cp_async(reinterpret_cast<float*>(rbS + nrun), reinterpret_cast<const float*>(A.run_beg + rb + nrun));
  if (PDE == PDE_HEAT) {
    if (y0 == 0)
      for (int x = lox[0] + tid; x < lox[0] + wid[0]; x += MODIL_NT)
        cp_async(icS + (x - (x0 - G::HU)), A.aux + D.aux_off + x);
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

  // ---- 1. Horner on the pyramid: w_l += T w_{l+1}, coarse to fine ----------
  auto horner_level = [&](int l, int first, int stride) {
    const int nyc = D.n[l + 1][1], nxc = D.n[l + 1][2];
    const T* wc = pyr + poff[l + 1];
    const int cw = wid[l + 1], cly = loy[l + 1], clx = lox[l + 1];
    const int nreg = (l == 0) ? G::UH * G::UW : hgt[l] * wid[l];
    for (int idx = first; idx < nreg; idx += stride) {
      int y, x;
      if (l == 0) {
        const int ry = idx / G::UW, rx = idx - ry * G::UW;
        y = y0 - G::HU + ry;
        x = x0 - G::HU + rx;
        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
      } else {
        const int ry = (int)(((float)idx + 0.5f) * winv[l]), rx = idx - ry * wid[l];
        y = loy[l] + ry;
        x = lox[l] + rx;
      }
      int jy0, jy1, jx0, jx1;
      T wy0, wy1, wx0, wx1;
      prolong_taps<T>(y, nyc, jy0, jy1, wy0, wy1);
      prolong_taps<T>(x, nxc, jx0, jx1, wx0, wx1);
      const T* r0 = wc + (jy0 - cly) * cw - clx;
      const T* r1 = wc + (jy1 - cly) * cw - clx;
      const T add = wy0 * (wx0 * r0[jx0] + wx1 * r0[jx1]) + wy1 * (wx0 * r1[jx0] + wx1 * r1[jx1]);
      T* dst = (l == 0) ? uR + idx : pyr + poff[l] + idx;
      *dst += add;
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
  for (int l = min(1, L - 2); l >= 0; --l) {
    horner_level(l, tid, MODIL_NT);
    __syncthreads();
  }

  auto U = [&](int y, int x) -> T { return uR[(y - y0 + G::HU) * G::UW + (x - x0 + G::HU)]; };

  if (mode == MODE_COMPOSE) {
    T* out = A.ufine + D.fine_off[0];
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      if (oy < hy && ox < hx) out[(long long)(y0 + oy) * nx + (x0 + ox)] = U(y0 + oy, x0 + ox);
    }
    return;
  }

  // ---- 2./3. residuals, local Jacobians, owned r^2 -------------------------
  const T dt = (T)D.h[1], dx = (T)D.h[2];
  const T idt = T(1) / dt, idx1 = T(1) / dx, idx2 = T(1) / (dx * dx);
  const T nu = (T)D.coef[0];
  const T lam_scale = T(2) * (T)D.w_res_dV;
  const bool adj = (mode != MODE_LOSS);
  float racc_f = 0.f;
  double racc_d = 0.0;  // FP64 problems
  for (int idx = tid; idx < G::RH * G::RW; idx += MODIL_NT) {
    const int ry = idx / G::RW, rx = idx - ry * G::RW;
    const int y = y0 - 1 + ry, x = x0 - 1 + rx;
    T r = T(0), J0 = T(0), J1 = T(0), J2 = T(0), J3 = T(0), dE = T(0), dW = T(0);
    bool valid = (y >= 0 && y < ny && x >= 0 && x < nx);
    if (PDE == PDE_BURGERS && y == 0) valid = false;
    if (valid) {
      const T uc = U(y, x);
      if (PDE == PDE_HEAT && y == 0) {
        r = (uc - icS[x - (x0 - G::HU)]) * idt;
        J1 = idt;
      } else {
        const T uo = U(y - 1, x);
        const bool hw = (x > 0), he = (x < nx - 1);
        const T uw = hw ? U(y, x - 1) : -uc;
        const T ue = he ? U(y, x + 1) : -uc;
        if (PDE == PDE_BURGERS) {
          T dFEc = T(0), dFEe = T(0), dFWw = T(0), dFWc = T(0), FE = T(0), FW = T(0);
          if (he) FE = eo_flux(uc, ue, dFEc, dFEe);
          if (hw) FW = eo_flux(uw, uc, dFWw, dFWc);
          const T lap = (ue - T(2) * uc + uw) * idx2;
          r = (uc - uo) * idt + (FE - FW) * idx1 - nu * lap;
          const T cdiag = T(-2) - (hw ? T(0) : T(1)) - (he ? T(0) : T(1));
          J1 = idt + (dFEc - dFWc) * idx1 - nu * cdiag * idx2;
          J0 = hw ? (-dFWw * idx1 - nu * idx2) : T(0);
          J2 = he ? (dFEe * idx1 - nu * idx2) : T(0);
          J3 = -idt;
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
          r = (uc - uo) * idt - (kE * duE - kW * duW) * idx2;
          J1 = idt - (dEc - dWc) * idx2;
          J2 = -dEe * idx2;
          J0 = dWw * idx2;
          J3 = -idt;
          dE = -duE * idx2;  // dr/dk_E
          dW = duW * idx2;   // dr/dk_W
        }
      }
    }
    const bool owned = valid && ry >= 1 && ry <= hy && rx >= 1 && rx <= hx;
    if (owned) {
      if (sizeof(T) == 4) racc_f += (float)(r * r);
      else racc_d += (double)(r * r);
    }
    if (adj) {
      const T lam = lam_scale * r;
      aJ[0 * G::RH * G::RW + idx] = lam * J0;
      aJ[1 * G::RH * G::RW + idx] = lam * J1;
      aJ[2 * G::RH * G::RW + idx] = lam * J2;
      aJ[3 * G::RH * G::RW + idx] = lam * J3;
      if (PDE == PDE_HEAT && ry >= 1 && ry <= TY && rx >= 1 && rx <= TX) {
        const int o = (ry - 1) * TX + (rx - 1);
        muE[o] = owned ? lam * dE : T(0);
        muW[o] = owned ? lam * dW : T(0);
      }
    }
  }

  const T wd2 = T(2) * (T)D.w_data_n;
  __syncthreads();  // aJ / muE complete

  // ---- 4. gather dL/du on the tile ------------------------------------------
  if (adj) {
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      const int c = (oy + 1) * G::RW + (ox + 1);
      gS[idx] = aJ[1 * G::RH * G::RW + c] + aJ[0 * G::RH * G::RW + c + 1] +
                aJ[2 * G::RH * G::RW + c - 1] + aJ[3 * G::RH * G::RW + c + G::RW];
    }
    __syncthreads();
  }

  // ---- 5. data term: runs of equal cells inside the tile ---------------------
  float dacc_f = 0.f;
  double dacc_d = 0.0;
  for (int i = tid; i < nrun; i += MODIL_NT) {
    const int cell = rcS[i];
    const int y = cell / nx, x = cell - (cell / nx) * nx;
    const T u = U(y, x);
    T d = u - rvS[i];
    T sd = d, sq = d * d;
    for (int e = rbS[i] + 1; e < rbS[i + 1]; ++e) {  // repeated measurements of a cell
      d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    if (sizeof(T) == 4) dacc_f += (float)sq;
    else dacc_d += (double)sq;
    if (adj) gS[(y - y0) * TX + (x - x0)] += wd2 * sd;
  }

  double rsum, dsum;
  if (sizeof(T) == 4) {
    rsum = block_sum_ff<MODIL_NT>(racc_f, redf);
    dsum = block_sum_ff<MODIL_NT>(dacc_f, redf + 16);
  } else {
    rsum = block_sum<MODIL_NT>(racc_d, red);
    dsum = block_sum<MODIL_NT>(dacc_d, red + 8);
  }
  if (tid == 0) {
    A.part[(long long)gt * A.npart + 0] = rsum;
    A.part[(long long)gt * A.npart + 1] = dsum;
  }

  if (adj) {
    __syncthreads();  // gS complete (data added)
    // ---- 6. write dL/du, Adam on level 1 ------------------------------------
    const AdamCoef ac = *acS;
    T* __restrict__ Gp = A.g + o0;
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      if (oy >= hy || ox >= hx) continue;
      const long long e = (long long)(y0 + oy) * nx + (x0 + ox);
      const T g = gS[idx] * (T)A.gscale;
      Gp[e] = g;
      if (mode == MODE_STEP) {
        T p = pS[idx];
        T m = mS[idx];
        double v = vS[idx];
        adam_update(p, m, v, g, ac);
        A.p[cur ^ 1][o0 + e] = p;
        A.m[o0 + e] = m;
        A.v[o0 + e] = v;
      }
    }

    // ---- 6b. heat: dL/dq partial by deterministic warp-range binning -------
    if (PDE == PDE_HEAT) {
      for (int i = tid; i < 8 * MODIL_MAXK; i += MODIL_NT) bins[i] = 0.0;
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
  bool first = true;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(A.queue, 1);
    __syncthreads();
    const int gt = s_tile;
    __syncthreads();
    if (gt >= A.ntiles[0]) break;
    tile(gt, first);
    first = false;
    __syncthreads();  // shared memory is reused by the next tile
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
  const size_t smem = StSmem<T, TY, TX>::bytes(pyr);
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
  return cudaErrorInvalidValue;
}

template <class T, int TY, int TX>
static cudaError_t prepare_cfg(int pde, size_t pyr) {
  const int smem = (int)StSmem<T, TY, TX>::bytes(pyr);
  if (pde == PDE_BURGERS)
    return raise_smem_limit(k_fine_st<T, PDE_BURGERS, TY, TX>, (size_t)smem);
  if (pde == PDE_HEAT)
    return raise_smem_limit(k_fine_st<T, PDE_HEAT, TY, TX>, (size_t)smem);
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
                                                       StSmem<T, TY, TX>::bytes(pyr));
}

template <class T, int TY, int TX>
static cudaError_t occ_pde(int pde, size_t pyr, int* n) {
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

size_t fine_st_smem_bytes(int cfg, size_t pyr, int elem) {
  const bool d = (elem == 8);
  switch (cfg) {
    case 0: return d ? StSmem<double, 16, 32>::bytes(pyr) : StSmem<float, 16, 32>::bytes(pyr);
    case 1: return d ? StSmem<double, 16, 64>::bytes(pyr) : StSmem<float, 16, 64>::bytes(pyr);
    case 2: return d ? StSmem<double, 8, 64>::bytes(pyr) : StSmem<float, 8, 64>::bytes(pyr);
    case 3: return d ? StSmem<double, 32, 32>::bytes(pyr) : StSmem<float, 32, 32>::bytes(pyr);
    case 4: return d ? StSmem<double, 8, 128>::bytes(pyr) : StSmem<float, 8, 128>::bytes(pyr);
    default: return 0;
  }
}

template cudaError_t prepare_fine_st<float>(int, int, size_t);
template cudaError_t prepare_fine_st<double>(int, int, size_t);
template cudaError_t launch_fine_st<float>(const Arena<float>&, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_fine_st<double>(const Arena<double>&, int, int, int, int, size_t, cudaStream_t);

}  // namespace modil
