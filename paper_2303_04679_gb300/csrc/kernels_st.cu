// Fused fine-tile kernel of the space-time PDE family (viscous Burgers,
// heat conduction with unknown conductivity).  One block owns a TY x TX tile
// of the fine grid (axes t, x) and in one pass:
//   1. composes the field on the tile plus a halo of 2 cells by Horner's
//      scheme, rebuilding the coarse-level pyramid of just this tile in shared
//      memory (w_L = u_L, w_i = u_i + T_i w_{i+1}; paper Section 2.2);
//   2. evaluates every residual that touches the tile (tile plus 1 cell) and
//      its local Jacobian, dr/du at the 4 stencil points;
//   3. reduces r^2 over the residuals it owns (FP64 partial per tile);
//   4. forms dL/du on the tile in gather form: each cell sums
//      lambda * dr/du over the residuals that read it (lambda = 2 w dV r);
//   5. adds the data term of the measurements inside the tile;
//   6. writes the fine gradient, applies Adam to level 1 (step mode), and for
//      the heat problem reduces dL/dq of the 32 conductivity nodes into a
//      per-tile partial (deterministic warp-range binning).
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
#include "modil_dev.cuh"
#include "launch.h"

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
  static constexpr size_t a8(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_inst = 0;
  static constexpr size_t o_red = a8(o_inst + sizeof(DevInst));
  static constexpr size_t o_bins = a8(o_red + 8 * 40);  // 8 warps x MODIL_MAXK bins
  static constexpr size_t o_u = a8(o_bins + 8 * 8 * MODIL_MAXK);
  static constexpr size_t o_a = a8(o_u + sizeof(T) * G::UH * G::UW);
  static constexpr size_t o_g = a8(o_a + sizeof(T) * 4 * G::RH * G::RW);
  static constexpr size_t o_mu = a8(o_g + sizeof(T) * TY * TX);
  static constexpr size_t o_q = a8(o_mu + sizeof(T) * 2 * TY * TX);
  static constexpr size_t o_pyr = a8(o_q + sizeof(T) * MODIL_MAXK);
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
k_fine_st(Arena<T> A, int mode) {
  using G = StGeom<TY, TX>;
  using S = StSmem<T, TY, TX>;
  extern __shared__ __align__(16) unsigned char smem[];
  DevInst& D = *reinterpret_cast<DevInst*>(smem + S::o_inst);
  double* red = reinterpret_cast<double*>(smem + S::o_red);
  double* bins = reinterpret_cast<double*>(smem + S::o_bins);
  T* uR = reinterpret_cast<T*>(smem + S::o_u);
  T* aJ = reinterpret_cast<T*>(smem + S::o_a);
  T* gS = reinterpret_cast<T*>(smem + S::o_g);
  T* muE = reinterpret_cast<T*>(smem + S::o_mu);
  T* muW = muE + TY * TX;
  T* qS = reinterpret_cast<T*>(smem + S::o_q);
  T* pyr = reinterpret_cast<T*>(smem + S::o_pyr);

  const int tid = threadIdx.x;
  const int gt = blockIdx.x;
  const int ii = A.tile_inst[0][gt];
  block_copy(&D, A.inst + ii);
  __syncthreads();

  const InstState st = A.st[ii];
  const int cur = (int)(st.t & 1);
  const int L = D.nlev;
  const int ny = D.n[0][1], nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int ty = local / D.nt[0][2], tx = local - ty * D.nt[0][2];
  const int y0 = ty * TY, x0 = tx * TX;
  const int hy = min(TY, ny - y0), hx = min(TX, nx - x0);  // owned extent (ragged edge)
  const T* __restrict__ P = A.p[cur];
  const int K = D.nk - 1;

  if (PDE == PDE_HEAT) {
    for (int j = tid; j < D.nk; j += MODIL_NT) qS[j] = A.kq[D.k_off + j];
  }

  // ---- 1. compose by Horner's scheme on the tile's pyramid ----------------
  int loy[MODIL_MAXL], lox[MODIL_MAXL], wid[MODIL_MAXL], hgt[MODIL_MAXL], poff[MODIL_MAXL];
  loy[0] = max(0, y0 - G::HU);
  lox[0] = max(0, x0 - G::HU);
  int hiy = min(ny - 1, y0 + TY - 1 + G::HU), hix = min(nx - 1, x0 + TX - 1 + G::HU);
  hgt[0] = hiy - loy[0] + 1;
  wid[0] = hix - lox[0] + 1;
  poff[0] = 0;
  int tot = 0;
  for (int l = 1; l < L; ++l) {
    const int nyl = D.n[l][1], nxl = D.n[l][2];
    const int ly = max(0, (loy[l - 1] >> 1) - 1), lx = max(0, (lox[l - 1] >> 1) - 1);
    const int uy = min(nyl - 1, ((loy[l - 1] + hgt[l - 1] - 1) >> 1) + 1);
    const int ux = min(nxl - 1, ((lox[l - 1] + wid[l - 1] - 1) >> 1) + 1);
    loy[l] = ly; lox[l] = lx; hgt[l] = uy - ly + 1; wid[l] = ux - lx + 1;
    poff[l] = tot;
    tot += hgt[l] * wid[l];
  }
  for (int l = L - 1; l >= 0; --l) {
    const T* __restrict__ Pl = P + D.off[0][l];
    const int nxl = D.n[l][2];
    const bool top = (l == L - 1);
    const int nyc = top ? 1 : D.n[l + 1][1], nxc = top ? 1 : D.n[l + 1][2];
    const T* wc = top ? nullptr : pyr + poff[l + 1];
    const int cw = top ? 0 : wid[l + 1];
    const int cly = top ? 0 : loy[l + 1], clx = top ? 0 : lox[l + 1];
    for (int idx = tid; idx < hgt[l] * wid[l]; idx += MODIL_NT) {
      const int ry = idx / wid[l], rx = idx - ry * wid[l];
      const int y = loy[l] + ry, x = lox[l] + rx;
      T val = Pl[(long long)y * nxl + x];
      if (!top) {
        int jy0, jy1, jx0, jx1;
        T wy0, wy1, wx0, wx1;
        prolong_taps<T>(y, nyc, jy0, jy1, wy0, wy1);
        prolong_taps<T>(x, nxc, jx0, jx1, wx0, wx1);
        const T* r0 = wc + (jy0 - cly) * cw - clx;
        const T* r1 = wc + (jy1 - cly) * cw - clx;
        val += wy0 * (wx0 * r0[jx0] + wx1 * r0[jx1]) + wy1 * (wx0 * r1[jx0] + wx1 * r1[jx1]);
      }
      if (l == 0) uR[(y - (y0 - G::HU)) * G::UW + (x - (x0 - G::HU))] = val;
      else pyr[poff[l] + idx] = val;
    }
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
  double racc_d = 0.0;
  for (int idx = tid; idx < G::RH * G::RW; idx += MODIL_NT) {
    const int ry = idx / G::RW, rx = idx - ry * G::RW;
    const int y = y0 - 1 + ry, x = x0 - 1 + rx;
    T r = T(0), J0 = T(0), J1 = T(0), J2 = T(0), J3 = T(0), dE = T(0), dW = T(0);
    bool valid = (y >= 0 && y < ny && x >= 0 && x < nx);
    if (PDE == PDE_BURGERS && y == 0) valid = false;
    if (valid) {
      const T uc = U(y, x);
      if (PDE == PDE_HEAT && y == 0) {
        r = (uc - A.aux[D.aux_off + x]) * idt;
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
  double racc = racc_d + (double)racc_f;

  // ---- 5. data term (its loss is needed in every mode) ---------------------
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  const T wd2 = T(2) * (T)D.w_data_n;
  double dacc = 0.0;
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
  for (int r = rb + tid; r < re; r += MODIL_NT) {
    const int cell = A.run_cell[r];
    const int y = cell / nx, x = cell - (cell / nx) * nx;
    const T u = U(y, x);
    T sd = T(0);
    double sq = 0.0;
    for (int e = A.run_beg[r]; e < A.run_beg[r + 1]; ++e) {
      const T d = u - A.meas_val[e];
      sd += d;
      sq += (double)d * (double)d;
    }
    dacc += sq;
    if (adj) gS[(y - y0) * TX + (x - x0)] += wd2 * sd;
  }

  const double rsum = block_sum<MODIL_NT>(racc, red);
  const double dsum = block_sum<MODIL_NT>(dacc, red + 8);
  if (tid == 0) {
    A.part[(long long)gt * A.npart + 0] = rsum;
    A.part[(long long)gt * A.npart + 1] = dsum;
  }
  if (!adj) return;
  __syncthreads();  // gS complete (data added)

  // ---- 6. write dL/du, Adam on level 1 --------------------------------------
  {
    const long long o = D.off[0][0];
    const AdamCoef ac = adam_coef(D, st);
    T* __restrict__ Gp = A.g + o;
    for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
      const int oy = idx / TX, ox = idx - oy * TX;
      if (oy >= hy || ox >= hx) continue;
      const long long e = (long long)(y0 + oy) * nx + (x0 + ox);
      const T g = gS[idx];
      Gp[e] = g;
      if (mode == MODE_STEP) {
        T p = P[o + e];
        T m = A.m[o + e];
        double v = A.v[o + e];
        adam_update(p, m, v, g, ac);
        A.p[cur ^ 1][o + e] = p;
        A.m[o + e] = m;
        A.v[o + e] = v;
      }
    }
  }

  // ---- 6b. heat: dL/dq partial by deterministic warp-range binning ---------
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
      const double s = warp_sum((double)acc);
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

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <class T, int TY, int TX>
static cudaError_t launch_cfg(const Arena<T>& A, int pde, int mode, size_t pyr, cudaStream_t s) {
  const size_t smem = StSmem<T, TY, TX>::bytes(pyr);
  const int grid = A.ntiles[0];
  if (grid == 0) return cudaSuccess;
  if (pde == PDE_BURGERS) {
    k_fine_st<T, PDE_BURGERS, TY, TX><<<grid, MODIL_NT, smem, s>>>(A, mode);
  } else if (pde == PDE_HEAT) {
    k_fine_st<T, PDE_HEAT, TY, TX><<<grid, MODIL_NT, smem, s>>>(A, mode);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class T, int TY, int TX>
static cudaError_t prepare_cfg(int pde, size_t pyr) {
  const int smem = (int)StSmem<T, TY, TX>::bytes(pyr);
  if (pde == PDE_BURGERS)
    return cudaFuncSetAttribute(k_fine_st<T, PDE_BURGERS, TY, TX>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (pde == PDE_HEAT)
    return cudaFuncSetAttribute(k_fine_st<T, PDE_HEAT, TY, TX>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
cudaError_t launch_fine_st(const Arena<T>& A, int pde, int cfg, int mode, size_t pyr,
                           cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_cfg<T, 16, 32>(A, pde, mode, pyr, s);
    case 1: return launch_cfg<T, 16, 64>(A, pde, mode, pyr, s);
    case 2: return launch_cfg<T, 8, 64>(A, pde, mode, pyr, s);
    case 3: return launch_cfg<T, 32, 32>(A, pde, mode, pyr, s);
    case 4: return launch_cfg<T, 8, 128>(A, pde, mode, pyr, s);
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
template cudaError_t launch_fine_st<float>(const Arena<float>&, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_fine_st<double>(const Arena<double>&, int, int, int, size_t, cudaStream_t);

}  // namespace modil
