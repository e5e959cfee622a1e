// Fused fine-tile kernel of the steady incompressible Navier-Stokes cavity
// (paper Section 3.3): three fields u, v, p on a cell-centred grid, axes
// (y, x), unit square, no-slip walls with a moving lid u = 1 at y = 1.
//
// Discretisation (collocated finite volumes), residuals at cell P:
//   r_u = (F_e - F_w + G_n - G_s)/h + (p_E - p_W)/(2h) - nu lap(u),
//         F_e = ((u_P+u_E)/2)^2, G_n = ((v_P+v_N)/2)((u_P+u_N)/2), ...
//   r_v = the same for v with F_e = ((u_P+u_E)/2)((v_P+v_E)/2), G_n = ((v_P+v_N)/2)^2
//   r_c = (U_e - U_w + V_n - V_s)/h with Rhie-Chow face velocities
//         U_e = (u_P+u_E)/2 - tau [ (p_E-p_P)/h - (g_P+g_E)/2 ],  g = (p_E-p_W)/(2h)
// Convective and mass fluxes through walls are zero; the viscous term and
// the pressure gradient use ghost cells (wall velocity = mean of ghost and
// cell, ghost p = cell p).  The pressure level is fixed by the residual
// p(0,0).  nu = 1/Re, tau = tau_factor * h.
//
// One block owns a TY x TX tile: stages the pyramid of all three fields,
// composes them (Horner), forms every residual within 2 cells of the tile
// with its local Jacobian (37 entries: 11 + 11 for the momentum equations,
// written out by the product rule; 15 for the linear continuity equation,
// obtained by evaluating it on unit vectors), gathers dL/du, dL/dv, dL/dp on
// the tile, adds the velocity measurements, applies Adam to level 1 and
// writes per-tile FP64 partials.
#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

namespace ns2d {
constexpr int F = 3;
constexpr int NK = 37;
// stencil entries: field, dy, dx (equation by range: [0,11) x-momentum,
// [11,22) y-momentum, [22,37) continuity)
__constant__ int kField[NK] = {0, 0, 0, 0, 0, 1, 1, 1, 2, 2, 2,
                               1, 1, 1, 1, 1, 0, 0, 0, 2, 2, 2,
                               0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2};
__constant__ int kDy[NK] = {0, 0, 0, 1, -1, 0, 1, -1, 0, 0, 0,
                            0, 0, 0, 1, -1, 0, 0, 0, 1, -1, 0,
                            0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 1, -1, 2, -2};
__constant__ int kDx[NK] = {0, 1, -1, 0, 0, 0, 0, 0, 1, -1, 0,
                            0, 1, -1, 0, 0, 0, 1, -1, 0, 0, 0,
                            0, 1, -1, 0, 0, 0, 0, 1, -1, 2, -2, 0, 0, 0, 0};
}  // namespace ns2d

template <int TY, int TX>
struct NsGeom {
  static constexpr int HU = 4;                    // composed-field halo
  static constexpr int UH = TY + 2 * HU, UW = TX + 2 * HU;
  static constexpr int HR = 2;                    // residual halo
  static constexpr int RH = TY + 2 * HR, RW = TX + 2 * HR;
};

template <class T, int TY, int TX>
struct NsSmem {
  using G = NsGeom<TY, TX>;
  static constexpr int F = ns2d::F;
  static constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_inst = 0;
  static constexpr size_t o_reg = a16(o_inst + sizeof(DevInst));
  static constexpr size_t o_red = a16(o_reg + 4 * (6 * MODIL_MAXL + 4));
  static constexpr size_t o_u = a16(o_red + 8 * 16);
  static constexpr size_t o_a = a16(o_u + sizeof(T) * F * G::UH * G::UW);
  static constexpr size_t o_g = a16(o_a + sizeof(T) * ns2d::NK * G::RH * G::RW);
  static constexpr size_t o_p = a16(o_g + sizeof(T) * F * TY * TX);
  static constexpr size_t o_m = a16(o_p + sizeof(T) * F * TY * TX);
  static constexpr size_t o_v = a16(o_m + sizeof(T) * F * TY * TX);
  static constexpr size_t o_rc = a16(o_v + sizeof(double) * F * TY * TX);
  static constexpr size_t o_rf = a16(o_rc + 4 * F * TY * TX);
  static constexpr size_t o_rb = a16(o_rf + 4 * F * TY * TX);
  static constexpr size_t o_rv = a16(o_rb + 4 * (F * TY * TX + 1));
  static constexpr size_t o_pyr = a16(o_rv + sizeof(T) * F * TY * TX);
  static size_t bytes(size_t pyr_elems) { return o_pyr + sizeof(T) * F * pyr_elems; }
};

// Continuity residual times h from the 15 stencil values (linear in them).
// s: u_P u_E u_W v_P v_N v_S p_P p_E p_W p_EE p_WW p_N p_S p_NN p_SS.
template <class T>
__device__ __forceinline__ T cont_h(const T* s, bool iE, bool iW, bool iN, bool iS, bool iEE,
                                    bool iWW, bool iNN, bool iSS, T tf) {
  const T q = T(0.25) * tf;
  const T pP = s[6];
  const T pE = iE ? s[7] : pP, pW = iW ? s[8] : pP;
  const T pEE = iEE ? s[9] : pE, pWW = iWW ? s[10] : pW;
  const T pN = iN ? s[11] : pP, pS = iS ? s[12] : pP;
  const T pNN = iNN ? s[13] : pN, pSS = iSS ? s[14] : pS;
  T r = T(0);
  if (iE) r += T(0.5) * (s[0] + s[1]) - tf * (pE - pP) + q * (pE - pW + pEE - pP);
  if (iW) r -= T(0.5) * (s[2] + s[0]) - tf * (pP - pW) + q * (pP - pWW + pE - pW);
  if (iN) r += T(0.5) * (s[3] + s[4]) - tf * (pN - pP) + q * (pN - pS + pNN - pP);
  if (iS) r -= T(0.5) * (s[5] + s[3]) - tf * (pP - pS) + q * (pP - pSS + pN - pS);
  return r;
}

template <class T, int TY, int TX>
__global__ void __launch_bounds__(MODIL_NT)
k_fine_ns2d(const __grid_constant__ Arena<T> A, int mode, int cur) {
  using G = NsGeom<TY, TX>;
  using S = NsSmem<T, TY, TX>;
  constexpr int F = ns2d::F;
  constexpr int NR = G::RH * G::RW;
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
  float* redf = reinterpret_cast<float*>(red);
  T* uR = reinterpret_cast<T*>(smem + S::o_u);
  T* aJ = reinterpret_cast<T*>(smem + S::o_a);
  T* gS = reinterpret_cast<T*>(smem + S::o_g);
  T* pS = reinterpret_cast<T*>(smem + S::o_p);
  T* mS = reinterpret_cast<T*>(smem + S::o_m);
  double* vS = reinterpret_cast<double*>(smem + S::o_v);
  int* rcS = reinterpret_cast<int*>(smem + S::o_rc);
  int* rfS = reinterpret_cast<int*>(smem + S::o_rf);
  int* rbS = reinterpret_cast<int*>(smem + S::o_rb);
  T* rvS = reinterpret_cast<T*>(smem + S::o_rv);
  T* pyr = reinterpret_cast<T*>(smem + S::o_pyr);
  __shared__ AdamCoef acS[1];
  __shared__ int pyr_stride[1];

  const int tid = threadIdx.x;
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  const int nrun = min(re - rb, F * TY * TX);
  __syncthreads();

  const int L = D.nlev;
  const int ny = D.n[0][1], nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int ty = local / D.nt[0][2], tx = local - ty * D.nt[0][2];
  const int y0 = ty * TY, x0 = tx * TX;
  const int hy = min(TY, ny - y0), hx = min(TX, nx - x0);
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
    if (tid == L - 1) *pyr_stride = tot + ((L > 1) ? h * w : 0);
  }
  __syncthreads();
  const int PS = *pyr_stride;  // pyramid elements per field

  const T* __restrict__ P = A.p[cur];
  auto stage_level = [&](int f, int l) {
    const T* src = P + D.off[f][l];
    if (l == 0) {
      T* dst = uR + f * G::UH * G::UW;
      for (int idx = tid; idx < G::UH * G::UW; idx += MODIL_NT) {
        const int ry = idx / G::UW, rx = idx - ry * G::UW;
        const int y = y0 - G::HU + ry, x = x0 - G::HU + rx;
        if (y >= 0 && y < ny && x >= 0 && x < nx) cp_async(dst + idx, src + (long long)y * nx + x);
      }
      return;
    }
    const int nxl = D.n[l][2];
    for (int idx = tid; idx < hgt[l] * wid[l]; idx += MODIL_NT) {
      const int ry = (int)(((float)idx + 0.5f) * winv[l]), rx = idx - ry * wid[l];
      const int y = loy[l] + ry, x = lox[l] + rx;
      cp_async(pyr + f * PS + poff[l] + idx, src + (long long)y * nxl + x);
    }
  };
  const int pre = min(L, D.tail);
  for (int f = 0; f < F; ++f)
    for (int l = 0; l < pre; ++l) stage_level(f, l);
  if (mode == MODE_STEP) {
    for (int idx = tid; idx < F * TY * TX; idx += MODIL_NT) {
      const int f = idx / (TY * TX), c = idx - f * (TY * TX);
      const int oy = c / TX, ox = c - oy * TX;
      if (oy >= hy || ox >= hx) continue;
      const long long e = D.off[f][0] + (long long)(y0 + oy) * nx + (x0 + ox);
      cp_async(pS + idx, P + e);
      cp_async(mS + idx, A.m + e);
      cp_async(vS + idx, A.v + e);
    }
  }
  for (int i = tid; i < nrun; i += MODIL_NT) {
    cp_async(reinterpret_cast<float*>(rcS + i), reinterpret_cast<const float*>(A.run_cell + rb + i));
    cp_async(reinterpret_cast<float*>(rfS + i), reinterpret_cast<const float*>(A.run_field + rb + i));
    cp_async(reinterpret_cast<float*>(rbS + i), reinterpret_cast<const float*>(A.run_beg + rb + i));
    cp_async(rvS + i, A.run_v0 + rb + i);
  }
  if (tid == 0 && nrun > 0)
    cp_async(reinterpret_cast<float*>(rbS + nrun), reinterpret_cast<const float*>(A.run_beg + rb + nrun));

  pdl_wait();
  pdl_trigger();
  if (tid == 0) *acS = adam_coef(D, A.st[ii]);
  for (int f = 0; f < F; ++f)
    for (int l = pre; l < L; ++l) stage_level(f, l);
  cp_async_wait_all();
  __syncthreads();

  // ---- Horner, all three fields ------------------------------------------------
  auto horner_level = [&](int f, int l, int first, int stride) {
    const int nyc = D.n[l + 1][1], nxc = D.n[l + 1][2];
    const T* wc = pyr + f * PS + poff[l + 1];
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
      T* dst = (l == 0) ? uR + f * G::UH * G::UW + idx : pyr + f * PS + poff[l] + idx;
      *dst += add;
    }
  };
  if (tid < 32 * F) {  // small levels: one warp per field
    const int f = tid >> 5;
    for (int l = L - 2; l >= 2; --l) {
      horner_level(f, l, tid & 31, 32);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int l = min(1, L - 2); l >= 0; --l) {
    for (int f = 0; f < F; ++f) horner_level(f, l, tid, MODIL_NT);
    __syncthreads();
  }

  auto V = [&](int f, int y, int x) -> T {
    return uR[f * G::UH * G::UW + (y - y0 + G::HU) * G::UW + (x - x0 + G::HU)];
  };

  if (mode == MODE_COMPOSE) {
    for (int f = 0; f < F; ++f) {
      T* out = A.ufine + D.fine_off[f];
      for (int idx = tid; idx < TY * TX; idx += MODIL_NT) {
        const int oy = idx / TX, ox = idx - oy * TX;
        if (oy < hy && ox < hx) out[(long long)(y0 + oy) * nx + (x0 + ox)] = V(f, y0 + oy, x0 + ox);
      }
    }
    return;
  }

  // ---- residuals and local Jacobians -------------------------------------------
  const T h = (T)D.h[2];
  const T ih = T(1) / h, i2h = T(0.5) / h, nuh2 = (T(1) / (T)D.coef[0]) / (h * h);
  const T tf = (T)D.coef[1];
  const T lam_scale = T(2) * (T)D.w_res_dV;
  const bool adj = (mode != MODE_LOSS);
  float racc_f = 0.f;
  double racc_d = 0.0;
  for (int idx = tid; idx < NR; idx += MODIL_NT) {
    const int ry = idx / G::RW, rx = idx - ry * G::RW;
    const int y = y0 - G::HR + ry, x = x0 - G::HR + rx;
    T J[ns2d::NK];
#pragma unroll
    for (int k = 0; k < ns2d::NK; ++k) J[k] = T(0);
    T ru = T(0), rv = T(0), rc = T(0);
    const bool valid = (y >= 0 && y < ny && x >= 0 && x < nx);
    if (valid) {
      const bool iE = x < nx - 1, iW = x > 0, iN = y < ny - 1, iS = y > 0;
      const T uP = V(0, y, x), vP = V(1, y, x), pP = V(2, y, x);
      const T uE = iE ? V(0, y, x + 1) : -uP, uW = iW ? V(0, y, x - 1) : -uP;
      const T uN = iN ? V(0, y + 1, x) : T(2) - uP, uS = iS ? V(0, y - 1, x) : -uP;
      const T vE = iE ? V(1, y, x + 1) : -vP, vW = iW ? V(1, y, x - 1) : -vP;
      const T vN = iN ? V(1, y + 1, x) : -vP, vS = iS ? V(1, y - 1, x) : -vP;
      const T pE = iE ? V(2, y, x + 1) : pP, pW = iW ? V(2, y, x - 1) : pP;
      const T pN = iN ? V(2, y + 1, x) : pP, pS = iS ? V(2, y - 1, x) : pP;
      const T fE = iE ? T(1) : T(0), fW = iW ? T(1) : T(0), fN = iN ? T(1) : T(0), fS = iS ? T(1) : T(0);
      const T nwall = T(4) - fE - fW - fN - fS;
      // x-momentum
      const T ae = T(0.5) * (uP + uE), aw = T(0.5) * (uW + uP);
      const T bn = T(0.5) * (vP + vN), cn = T(0.5) * (uP + uN);
      const T bs = T(0.5) * (vS + vP), cs = T(0.5) * (uS + uP);
      ru = (fE * ae * ae - fW * aw * aw + fN * bn * cn - fS * bs * cs) * ih + (pE - pW) * i2h -
           nuh2 * (uE + uW + uN + uS - T(4) * uP);
      J[0] = (fE * ae - fW * aw + T(0.5) * (fN * bn - fS * bs)) * ih + nuh2 * (T(4) + nwall);
      J[1] = fE * (ae * ih - nuh2);
      J[2] = fW * (-aw * ih - nuh2);
      J[3] = fN * (T(0.5) * bn * ih - nuh2);
      J[4] = fS * (-T(0.5) * bs * ih - nuh2);
      J[5] = T(0.5) * (fN * cn - fS * cs) * ih;
      J[6] = fN * T(0.5) * cn * ih;
      J[7] = -fS * T(0.5) * cs * ih;
      J[8] = fE * i2h;
      J[9] = -fW * i2h;
      J[10] = (fW - fE) * i2h;  // ghost pressures copy p_P
      // y-momentum
      const T Ae = T(0.5) * (uP + uE), Be = T(0.5) * (vP + vE);
      const T Aw = T(0.5) * (uW + uP), Bw = T(0.5) * (vW + vP);
      const T dn = T(0.5) * (vP + vN), ds = T(0.5) * (vS + vP);
      rv = (fE * Ae * Be - fW * Aw * Bw + fN * dn * dn - fS * ds * ds) * ih + (pN - pS) * i2h -
           nuh2 * (vE + vW + vN + vS - T(4) * vP);
      J[11] = (T(0.5) * (fE * Ae - fW * Aw) + fN * dn - fS * ds) * ih + nuh2 * (T(4) + nwall);
      J[12] = fE * (T(0.5) * Ae * ih - nuh2);
      J[13] = fW * (-T(0.5) * Aw * ih - nuh2);
      J[14] = fN * (dn * ih - nuh2);
      J[15] = fS * (-ds * ih - nuh2);
      J[16] = T(0.5) * (fE * Be - fW * Bw) * ih;
      J[17] = fE * T(0.5) * Be * ih;
      J[18] = -fW * T(0.5) * Bw * ih;
      J[19] = fN * i2h;
      J[20] = -fS * i2h;
      J[21] = (fS - fN) * i2h;
      // continuity (linear): value, and the Jacobian from unit vectors
      const bool iEE = x < nx - 2, iWW = x > 1, iNN = y < ny - 2, iSS = y > 1;
      T s[15];
      s[0] = uP; s[1] = iE ? uE : T(0); s[2] = iW ? uW : T(0);
      s[3] = vP; s[4] = iN ? vN : T(0); s[5] = iS ? vS : T(0);
      s[6] = pP; s[7] = iE ? pE : T(0); s[8] = iW ? pW : T(0);
      s[9] = iEE ? V(2, y, x + 2) : T(0); s[10] = iWW ? V(2, y, x - 2) : T(0);
      s[11] = iN ? pN : T(0); s[12] = iS ? pS : T(0);
      s[13] = iNN ? V(2, y + 2, x) : T(0); s[14] = iSS ? V(2, y - 2, x) : T(0);
      rc = cont_h(s, iE, iW, iN, iS, iEE, iWW, iNN, iSS, tf) * ih;
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        T e[15];
#pragma unroll
        for (int j = 0; j < 15; ++j) e[j] = (j == k) ? T(1) : T(0);
        J[22 + k] = cont_h(e, iE, iW, iN, iS, iEE, iWW, iNN, iSS, tf) * ih;
      }
    }
    const bool owned = valid && ry >= G::HR && ry < G::HR + hy && rx >= G::HR && rx < G::HR + hx;
    if (owned) {
      if (sizeof(T) == 4) racc_f += (float)(ru * ru + rv * rv + rc * rc);
      else racc_d += (double)(ru * ru + rv * rv + rc * rc);
    }
    if (adj) {
      const T lu = lam_scale * ru, lv = lam_scale * rv, lc = lam_scale * rc;
#pragma unroll
      for (int k = 0; k < ns2d::NK; ++k) {
        const T lam = (k < 11) ? lu : (k < 22) ? lv : lc;
        aJ[k * NR + idx] = lam * J[k];
      }
    }
  }
  // pressure gauge: residual p(0,0) on the tile that owns the corner
  const bool corner = (y0 == 0 && x0 == 0);
  if (corner && tid == 0) {
    const T p00 = V(2, 0, 0);
    if (sizeof(T) == 4) racc_f += (float)(p00 * p00);
    else racc_d += (double)(p00 * p00);
  }
  const T wd2 = T(2) * (T)D.w_data_n;
  __syncthreads();

  if (adj) {
    for (int idx = tid; idx < F * TY * TX; idx += MODIL_NT) {
      const int f = idx / (TY * TX), c = idx - f * (TY * TX);
      const int oy = c / TX, ox = c - oy * TX;
      T g = T(0);
#pragma unroll
      for (int k = 0; k < ns2d::NK; ++k) {
        if (ns2d::kField[k] != f) continue;
        const int rr = (oy + G::HR - ns2d::kDy[k]) * G::RW + (ox + G::HR - ns2d::kDx[k]);
        g += aJ[k * NR + rr];
      }
      if (corner && f == 2 && c == 0) g += lam_scale * V(2, 0, 0);
      gS[idx] = g;
    }
    __syncthreads();
  }

  // ---- velocity measurements -------------------------------------------------
  float dacc_f = 0.f;
  double dacc_d = 0.0;
  for (int i = tid; i < nrun; i += MODIL_NT) {
    const int cell = rcS[i], f = rfS[i];
    const int y = cell / nx, x = cell - (cell / nx) * nx;
    const T u = V(f, y, x);
    T d = u - rvS[i];
    T sd = d, sq = d * d;
    for (int e = rbS[i] + 1; e < rbS[i + 1]; ++e) {
      d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    if (sizeof(T) == 4) dacc_f += (float)sq;
    else dacc_d += (double)sq;
    if (adj) gS[f * TY * TX + (y - y0) * TX + (x - x0)] += wd2 * sd;
  }
  // off-grid points whose corner cells the tile owns: the sampled value of
  // the record's field (its four corners lie in the composed region) minus
  // the measurement; the tile of a point's lower corner counts its misfit
  if (A.pt_ptr) {
    const int p1 = A.pt_ptr[gt + 1];
    for (int j = A.pt_ptr[gt] + tid; j < p1; j += MODIL_NT) {
      const int f = A.pt_field[j];
      T smp = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int cell = A.pt_cell[4 * (long long)j + k];
        const int yy = cell / nx, xx = cell - yy * nx;
        smp += A.pt_w[4 * (long long)j + k] * V(f, yy, xx);
      }
      const T dd = smp - A.pt_val[j];
      A.pt_diff[j] = dd;
      if (A.pt_own[j]) {
        if (sizeof(T) == 4) dacc_f += (float)(dd * dd);
        else dacc_d += (double)(dd * dd);
      }
    }
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
  if (!adj) return;
  // the points' gradient: each owned (field, corner cell) sums weight x
  // misfit over the records reaching it, in a fixed order (the block sums'
  // barriers above published the misfits)
  if (A.pc_ptr) {
    const int c1 = A.pc_ptr[gt + 1];
    for (int rr = A.pc_ptr[gt] + tid; rr < c1; rr += MODIL_NT) {
      const int cell = A.pc_cell[rr], f = A.pc_field[rr];
      const int yy = cell / nx, xx = cell - yy * nx;
      T acc = T(0);
      for (int e = A.pc_beg[rr]; e < A.pc_beg[rr + 1]; ++e) acc += A.pe_w[e] * A.pt_diff[A.pe_rec[e]];
      gS[f * TY * TX + (yy - y0) * TX + (xx - x0)] += wd2 * acc;
    }
  }
  __syncthreads();
  const AdamCoef ac = *acS;
  for (int idx = tid; idx < F * TY * TX; idx += MODIL_NT) {
    const int f = idx / (TY * TX), c = idx - f * (TY * TX);
    const int oy = c / TX, ox = c - oy * TX;
    if (oy >= hy || ox >= hx) continue;
    const long long o = D.off[f][0] + (long long)(y0 + oy) * nx + (x0 + ox);
    const T g = gS[idx] * (T)A.gscale;
    A.g[o] = g;
    if (mode == MODE_STEP) {
      T p = pS[idx], m = mS[idx];
      double v = vS[idx];
      adam_update(p, m, v, g, ac);
      A.p[cur ^ 1][o] = p;
      A.m[o] = m;
      A.v[o] = v;
    }
  }
}

template <class T, int TY, int TX>
static cudaError_t ns_launch(const Arena<T>& A, int mode, int cur, size_t pyr, cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(A.ntiles[0]);
  cfg.blockDim = dim3(MODIL_NT);
  cfg.dynamicSmemBytes = NsSmem<T, TY, TX>::bytes(pyr);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fine_ns2d<T, TY, TX>, A, mode, cur);
}

// NS2D uses the (8, 32) and (16, 32) tile shapes (configs 5 and 0).
template <class T>
cudaError_t launch_fine_ns2d(const Arena<T>& A, int cfg, int mode, int cur, size_t pyr,
                             cudaStream_t s) {
  if (cfg == 0) return ns_launch<T, 16, 32>(A, mode, cur, pyr, s);
  return ns_launch<T, 8, 32>(A, mode, cur, pyr, s);
}

template <class T>
cudaError_t prepare_fine_ns2d(int cfg, size_t pyr) {
  if (cfg == 0)
    return raise_smem_limit(k_fine_ns2d<T, 16, 32>, NsSmem<T, 16, 32>::bytes(pyr));
  return raise_smem_limit(k_fine_ns2d<T, 8, 32>, NsSmem<T, 8, 32>::bytes(pyr));
}

size_t fine_ns2d_smem_bytes(int cfg, size_t pyr, int elem) {
  if (cfg == 0) return elem == 8 ? NsSmem<double, 16, 32>::bytes(pyr) : NsSmem<float, 16, 32>::bytes(pyr);
  return elem == 8 ? NsSmem<double, 8, 32>::bytes(pyr) : NsSmem<float, 8, 32>::bytes(pyr);
}

template cudaError_t launch_fine_ns2d<float>(const Arena<float>&, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_fine_ns2d<double>(const Arena<double>&, int, int, int, size_t, cudaStream_t);
template cudaError_t prepare_fine_ns2d<float>(int, size_t);
template cudaError_t prepare_fine_ns2d<double>(int, size_t);

}  // namespace modil
