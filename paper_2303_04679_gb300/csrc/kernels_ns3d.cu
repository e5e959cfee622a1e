// Penalised steady Navier-Stokes in 3-D (body shape, paper Section 3.5,
// equation eq_nschi3): fields u, v, w, p, chihat on (z, y, x) cells of
// [0,1] x [0,1] x [0,2], chi = 1/(1 + exp(-(chihat + 5))).
//
//   momentum   r = (1 - chi)(conv + grad p - (D/Re) lap) + lambda chi u_c
//   continuity r = sum over axes of Rhie-Chow face fluxes (tau = tau_factor h)
//
// with the cavity's finite-volume discretisation in 3-D: face-averaged mass
// fluxes and face values, central pressure gradient, 7-point viscous term.
// Boundaries by ghost cells: inlet x = 0, u = (1, 0, 0), zero normal pressure
// gradient; outlet x = 2, p = 0, zero-gradient velocity; free-slip walls in
// y and z.  Mass fluxes through the x ends carry the boundary values (1 at
// the inlet, the cell's u at the outlet); walls carry none.
//
// Kernels of one pass:
//   k_compose3  per 3-D tile: stage the tile's pyramid of every level and
//               field, compose by Horner's scheme (Section 2.2), write the
//               composed fields (recomputed every pass, no per-level storage);
//   k_resid3    per 3-D tile: stage the composed fields with a halo of 4,
//               evaluate the momentum residuals on the tile plus 1 cell and
//               the continuity residuals on the tile plus 2 cells, each with
//               its local Jacobian, scatter lambda * dr/du into the tile's
//               gradient (shared-memory atomics: a stored 3-D Jacobian does
//               not fit), add the measurements, write dL/du and apply Adam to
//               level 1;
// then k_level3 restricts and steps each coarser level.
#include <algorithm>

#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

constexpr int C3Z = k3TZ, C3Y = k3TY, C3X = k3TX;  // fine tile (owned cells)
constexpr int NC3 = C3Z * C3Y * C3X;
constexpr int H3 = 4;                       // staged halo of the composed fields
constexpr int S3Z = C3Z + 2 * H3, S3Y = C3Y + 2 * H3, S3X = C3X + 2 * H3;
constexpr int NS3 = S3Z * S3Y * S3X;
constexpr int F3 = 5;

// Region of a level needed to interpolate a fine box [a0, b0] (one axis):
// unrolled, level l covers [(a0 - k) >> l, (b0 + k) >> l] with k = 2^(l+1) - 2.
__device__ __forceinline__ void lev_range(int a0, int b0, int l, int n, int& lo, int& cnt) {
  const int k = (1 << (l + 1)) - 2;
  lo = max(0, (a0 - k) >> l);
  cnt = min(n - 1, (b0 + k) >> l) - lo + 1;
}

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_compose3(const __grid_constant__ Arena<T> A, int cur) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevInst D;
  __shared__ int lo[MODIL_MAXL][3], cnt[MODIL_MAXL][3], poff[MODIL_MAXL + 1];
  T* pyr = reinterpret_cast<T*>(smem);
  const int tid = threadIdx.x;
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  __syncthreads();
  const int L = D.nlev;
  const int local = gt - D.tile_base[0];
  const int per_z = D.nt[0][1] * D.nt[0][2];
  const int tz = local / per_z, tr = local - tz * per_z;
  const int ty = tr / D.nt[0][2], tx = tr - ty * D.nt[0][2];
  const int z0 = tz * C3Z, y0 = ty * C3Y, x0 = tx * C3X;
  if (tid == 0) {
    int tot = 0;
    for (int l = 0; l < L; ++l) {
      lev_range(z0, min(D.n[0][0], z0 + C3Z) - 1, l, D.n[l][0], lo[l][0], cnt[l][0]);
      lev_range(y0, min(D.n[0][1], y0 + C3Y) - 1, l, D.n[l][1], lo[l][1], cnt[l][1]);
      lev_range(x0, min(D.n[0][2], x0 + C3X) - 1, l, D.n[l][2], lo[l][2], cnt[l][2]);
      poff[l] = tot;
      tot += cnt[l][0] * cnt[l][1] * cnt[l][2];
    }
    poff[L] = tot;
  }
  __syncthreads();
  const int PS = poff[L];
  pdl_wait();
  pdl_trigger();
  const T* __restrict__ P = A.p[cur];
  for (int f = 0; f < D.nfield; ++f)
    for (int l = 0; l < L; ++l) {
      const int cz = cnt[l][0], cy = cnt[l][1], cx = cnt[l][2];
      const T* src = P + D.off[f][l];
      for (int i = tid; i < cz * cy * cx; i += MODIL_NT) {
        const int a = i / (cy * cx), r = i - a * (cy * cx), b = r / cx, c = r - b * cx;
        const long long g = ((long long)(lo[l][0] + a) * D.n[l][1] + (lo[l][1] + b)) * D.n[l][2] + (lo[l][2] + c);
        cp_async(pyr + f * PS + poff[l] + i, src + g);
      }
    }
  cp_async_wait_all();
  __syncthreads();
  for (int l = L - 2; l >= 0; --l) {
    for (int f = 0; f < D.nfield; ++f) {
      const int cz = cnt[l][0], cy = cnt[l][1], cx = cnt[l][2];
      const int qy = cnt[l + 1][1], qx = cnt[l + 1][2];
      const T* wc = pyr + f * PS + poff[l + 1];
      for (int i = tid; i < cz * cy * cx; i += MODIL_NT) {
        const int a = i / (cy * cx), r = i - a * (cy * cx), b = r / cx, c = r - b * cx;
        const int z = lo[l][0] + a, y = lo[l][1] + b, x = lo[l][2] + c;
        int jz0, jz1, jy0, jy1, jx0, jx1;
        T wz0, wz1, wy0, wy1, wx0, wx1;
        prolong_taps<T>(z, D.n[l + 1][0], jz0, jz1, wz0, wz1);
        prolong_taps<T>(y, D.n[l + 1][1], jy0, jy1, wy0, wy1);
        prolong_taps<T>(x, D.n[l + 1][2], jx0, jx1, wx0, wx1);
        jz0 -= lo[l + 1][0]; jz1 -= lo[l + 1][0];
        jy0 -= lo[l + 1][1]; jy1 -= lo[l + 1][1];
        jx0 -= lo[l + 1][2]; jx1 -= lo[l + 1][2];
        auto at = [&](int zz, int yy, int xx) { return wc[(zz * qy + yy) * qx + xx]; };
        const T add =
            wz0 * (wy0 * (wx0 * at(jz0, jy0, jx0) + wx1 * at(jz0, jy0, jx1)) +
                   wy1 * (wx0 * at(jz0, jy1, jx0) + wx1 * at(jz0, jy1, jx1))) +
            wz1 * (wy0 * (wx0 * at(jz1, jy0, jx0) + wx1 * at(jz1, jy0, jx1)) +
                   wy1 * (wx0 * at(jz1, jy1, jx0) + wx1 * at(jz1, jy1, jx1)));
        pyr[f * PS + poff[l] + i] += add;
      }
    }
    __syncthreads();
  }
  for (int f = 0; f < D.nfield; ++f) {
    const int cz = cnt[0][0], cy = cnt[0][1], cx = cnt[0][2];
    T* out = A.ufine + D.fine_off[f];
    for (int i = tid; i < cz * cy * cx; i += MODIL_NT) {
      const int a = i / (cy * cx), r = i - a * (cy * cx), b = r / cx, c = r - b * cx;
      const long long g = ((long long)(lo[0][0] + a) * D.n[0][1] + (lo[0][1] + b)) * D.n[0][2] + (lo[0][2] + c);
      out[g] = pyr[f * PS + i];
    }
  }
}

// Ghost coefficient alpha and offset beta of field f beyond face (axis, side)
// of the domain: ghost = alpha * (value of the adjacent cell) + beta.
template <class T>
__device__ __forceinline__ void ghost3(int f, int axis, int side, T& alpha, T& beta) {
  beta = T(0);
  if (axis == 2) {           // x
    if (side == 0) {         // inlet
      alpha = (f == 3) ? T(1) : T(-1);
      beta = (f == 0) ? T(2) : T(0);
    } else {                 // outlet
      alpha = (f == 3) ? T(-1) : T(1);
    }
  } else if (axis == 1) {    // y walls, v normal
    alpha = (f == 1) ? T(-1) : T(1);
  } else {                   // z walls, w normal
    alpha = (f == 2) ? T(-1) : T(1);
  }
}

template <class T>
struct Ns3Coef {
  T ih[3], ih2[3], i2h[3];  // per axis (z, y, x): 1/h, 1/h^2, 1/(2h)
  T nu, lam, tf;
};

// Continuity residual from its 22 stencil values (affine in them).
// s: u P E W | v P N S | w P T B | p P E W EE WW N S NN SS T B TT BB
template <class T>
__device__ __forceinline__ T cont3(const T* s, const bool* in, const Ns3Coef<T>& c) {
  // in: E W EE WW N S NN SS T B TT BB (neighbour inside the domain)
  const T q = T(0.25) * c.tf, tf = c.tf;
  const T pP = s[9];
  const T pE = in[0] ? s[10] : -pP, pW = in[1] ? s[11] : pP;      // outlet odd, inlet even
  const T pEE = in[2] ? s[12] : -pE, pWW = in[3] ? s[13] : pW;
  const T pN = in[4] ? s[14] : pP, pS = in[5] ? s[15] : pP;        // walls even
  const T pNN = in[6] ? s[16] : pN, pSS = in[7] ? s[17] : pS;
  const T pT = in[8] ? s[18] : pP, pB = in[9] ? s[19] : pP;
  const T pTT = in[10] ? s[20] : pT, pBB = in[11] ? s[21] : pB;
  T fe, fw, fn, fs, ft, fb;
  fe = in[0] ? T(0.5) * (s[0] + s[1]) - tf * (pE - pP) + q * ((pE - pW) + (pEE - pP)) : s[0];
  fw = in[1] ? T(0.5) * (s[2] + s[0]) - tf * (pP - pW) + q * ((pP - pWW) + (pE - pW)) : T(1);
  fn = in[4] ? T(0.5) * (s[3] + s[4]) - tf * (pN - pP) + q * ((pN - pS) + (pNN - pP)) : T(0);
  fs = in[5] ? T(0.5) * (s[5] + s[3]) - tf * (pP - pS) + q * ((pP - pSS) + (pN - pS)) : T(0);
  ft = in[8] ? T(0.5) * (s[6] + s[7]) - tf * (pT - pP) + q * ((pT - pB) + (pTT - pP)) : T(0);
  fb = in[9] ? T(0.5) * (s[8] + s[6]) - tf * (pP - pB) + q * ((pP - pBB) + (pT - pB)) : T(0);
  return (fe - fw) * c.ih[2] + (fn - fs) * c.ih[1] + (ft - fb) * c.ih[0];
}

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_resid3(const __grid_constant__ Arena<T> A, int mode, int cur) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevInst D;
  __shared__ double red[16];
  __shared__ AdamCoef acS;
  T* uS = reinterpret_cast<T*>(smem);              // F3 x NS3, staged composed fields
  T* gS = uS + F3 * NS3;                           // F3 x NC3, tile gradient
  float* redf = reinterpret_cast<float*>(red);
  const int tid = threadIdx.x;
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  __syncthreads();
  const int nz = D.n[0][0], ny = D.n[0][1], nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int per_z = D.nt[0][1] * D.nt[0][2];
  const int tz = local / per_z, tr = local - tz * per_z;
  const int ty = tr / D.nt[0][2], tx = tr - ty * D.nt[0][2];
  const int z0 = tz * C3Z, y0 = ty * C3Y, x0 = tx * C3X;
  const int hz = min(C3Z, nz - z0), hy = min(C3Y, ny - y0), hx = min(C3X, nx - x0);
  if (tid == 0) acS = adam_coef(D, A.st[ii]);
  for (int i = tid; i < F3 * NC3; i += MODIL_NT) gS[i] = T(0);
  pdl_wait();
  pdl_trigger();
  // stage the composed fields (written by the previous launch) with a halo of 4
  for (int f = 0; f < F3; ++f) {
    const T* src = A.ufine + D.fine_off[f];
    for (int i = tid; i < NS3; i += MODIL_NT) {
      const int a = i / (S3Y * S3X), r = i - a * (S3Y * S3X), b = r / S3X, c = r - b * S3X;
      const int z = z0 - H3 + a, y = y0 - H3 + b, x = x0 - H3 + c;
      if (z >= 0 && z < nz && y >= 0 && y < ny && x >= 0 && x < nx)
        cp_async(uS + f * NS3 + i, src + ((long long)z * ny + y) * nx + x);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  Ns3Coef<T> cf;
  const double hh[3] = {D.h[0], D.h[1], D.h[2]};
  for (int a = 0; a < 3; ++a) {
    cf.ih[a] = (T)(1.0 / hh[a]);
    cf.ih2[a] = (T)(1.0 / (hh[a] * hh[a]));
    cf.i2h[a] = (T)(0.5 / hh[a]);
  }
  cf.nu = (T)(D.coef[1] / D.coef[0]);  // D / Re
  cf.lam = (T)D.coef[2];
  cf.tf = (T)D.coef[3];
  const int dims[3] = {nz, ny, nx};
  auto Vs = [&](int f, int z, int y, int x) -> T {
    return uS[f * NS3 + ((z - z0 + H3) * S3Y + (y - y0 + H3)) * S3X + (x - x0 + H3)];
  };
  auto owned = [&](int z, int y, int x) {
    return z >= z0 && z < z0 + hz && y >= y0 && y < y0 + hy && x >= x0 && x < x0 + hx;
  };
  auto scatter = [&](int f, int z, int y, int x, T val) {
    if (owned(z, y, x)) atomicAdd(gS + f * NC3 + ((z - z0) * C3Y + (y - y0)) * C3X + (x - x0), val);
  };
  const T lam_scale = T(2) * (T)D.w_res_dV;
  const bool adj = (mode != MODE_LOSS);
  float racc = 0.f;
  double raccd = 0.0;

  // ---- momentum on the tile plus one cell ------------------------------------
  constexpr int MZ = C3Z + 2, MY = C3Y + 2, MX = C3X + 2;
  for (int i = tid; i < MZ * MY * MX; i += MODIL_NT) {
    const int a = i / (MY * MX), rr = i - a * (MY * MX), b = rr / MX, c = rr - b * MX;
    const int z = z0 - 1 + a, y = y0 - 1 + b, x = x0 - 1 + c;
    if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) continue;
    const int P[3] = {z, y, x};
    // neighbour values along each axis with ghost substitution
    T nv[F3][3][2], al[F3][3][2];
    bool gh[3][2];
    T cen[F3];
#pragma unroll
    for (int f = 0; f < 4; ++f) cen[f] = Vs(f, z, y, x);
    cen[4] = Vs(4, z, y, x);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        int q[3] = {P[0], P[1], P[2]};
        q[ax] += sd ? 1 : -1;
        const bool inside = q[ax] >= 0 && q[ax] < dims[ax];
        gh[ax][sd] = !inside;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (inside) {
            nv[f][ax][sd] = Vs(f, q[0], q[1], q[2]);
            al[f][ax][sd] = T(0);
          } else {
            T alpha, beta;
            ghost3<T>(f, ax, sd, alpha, beta);
            nv[f][ax][sd] = alpha * cen[f] + beta;
            al[f][ax][sd] = alpha;
          }
        }
      }
    // chi and 1 - chi each from its own logistic: 1 - chi is never formed by
    // subtraction, which loses all digits in FP32 where chi is near 1
    const T chi = T(1) / (T(1) + exp(-(cen[4] + T(5))));
    const T om = T(1) / (T(1) + exp(cen[4] + T(5)));
    const bool own = owned(z, y, x);
    // mass-flux masks: x faces always carry flux, y and z walls none
    T mk[3][2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) mk[ax][sd] = (ax == 2 || !gh[ax][sd]) ? T(1) : T(0);
    // face-normal velocities (axis ax carried by component 2 - ax: z<-w, y<-v, x<-u)
    T Vf[3][2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int cmp = 2 - ax;
      Vf[ax][1] = mk[ax][1] * T(0.5) * (cen[cmp] + nv[cmp][ax][1]);
      Vf[ax][0] = mk[ax][0] * T(0.5) * (nv[cmp][ax][0] + cen[cmp]);
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {   // u (x), v (y), w (z)
      const int cax = 2 - comp;               // axis of this component
      const T phi = cen[comp];
      T conv = T(0), lap = T(0);
      // raw partials: own field at P and the 6 neighbours, face velocities
      T Jphi[3][2], JphiP = T(0), Jvel[3][2], JvelP[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const T fp = T(0.5) * (phi + nv[comp][ax][1]), fm = T(0.5) * (nv[comp][ax][0] + phi);
        conv += (Vf[ax][1] * fp - Vf[ax][0] * fm) * cf.ih[ax];
        lap += (nv[comp][ax][1] - T(2) * phi + nv[comp][ax][0]) * cf.ih2[ax];
        // d(conv)/d phi
        JphiP += T(0.5) * (Vf[ax][1] - Vf[ax][0]) * cf.ih[ax];
        Jphi[ax][1] = T(0.5) * Vf[ax][1] * cf.ih[ax];
        Jphi[ax][0] = -T(0.5) * Vf[ax][0] * cf.ih[ax];
        // d(conv)/d face velocity component (component 2 - ax)
        JvelP[ax] = T(0.5) * (mk[ax][1] * fp - mk[ax][0] * fm) * cf.ih[ax];
        Jvel[ax][1] = T(0.5) * mk[ax][1] * fp * cf.ih[ax];
        Jvel[ax][0] = -T(0.5) * mk[ax][0] * fm * cf.ih[ax];
        // viscous
        JphiP += T(2) * cf.nu * cf.ih2[ax];
        Jphi[ax][1] -= cf.nu * cf.ih2[ax];
        Jphi[ax][0] -= cf.nu * cf.ih2[ax];
      }
      const T gp = (nv[3][cax][1] - nv[3][cax][0]) * cf.i2h[cax];
      const T M = conv + gp - cf.nu * lap;
      const T r = om * M + cf.lam * chi * phi;
      if (own) {
        if (sizeof(T) == 4) racc += (float)(r * r);
        else raccd += (double)(r * r);
      }
      if (!adj) continue;
      const T lamr = lam_scale * r;
      // combine partials per field and slot (the face velocity of axis ax is
      // component 2 - ax; when it is this component the slots coincide)
      T jP[4] = {T(0), T(0), T(0), T(0)};
      T jn[4][3][2];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) { jn[f][ax][0] = T(0); jn[f][ax][1] = T(0); }
      jP[comp] += JphiP;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        jn[comp][ax][0] += Jphi[ax][0];
        jn[comp][ax][1] += Jphi[ax][1];
        const int vc = 2 - ax;
        jP[vc] += JvelP[ax];
        jn[vc][ax][0] += Jvel[ax][0];
        jn[vc][ax][1] += Jvel[ax][1];
      }
      jn[3][cax][1] += cf.i2h[cax];
      jn[3][cax][0] -= cf.i2h[cax];
      // fold ghost neighbours into the centre cell
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
          for (int sd = 0; sd < 2; ++sd)
            if (gh[ax][sd]) {
              jP[f] += al[f][ax][sd] * jn[f][ax][sd];
              jn[f][ax][sd] = T(0);
            }
      // penalisation
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T extra = (f == comp) ? cf.lam * chi : T(0);
        scatter(f, z, y, x, lamr * (om * jP[f] + extra));
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            if (gh[ax][sd] || jn[f][ax][sd] == T(0)) continue;
            int q[3] = {z, y, x};
            q[ax] += sd ? 1 : -1;
            scatter(f, q[0], q[1], q[2], lamr * om * jn[f][ax][sd]);
          }
      }
      scatter(4, z, y, x, lamr * chi * om * (cf.lam * phi - M));
    }
  }

  // ---- continuity on the tile plus two cells ---------------------------------
  constexpr int QZ = C3Z + 4, QY = C3Y + 4, QX = C3X + 4;
  // slot -> (field, dz, dy, dx)
  const int sf[22] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3};
  const int sz[22] = {0, 0, 0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2};
  const int sy[22] = {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2, 0, 0, 0, 0};
  const int sx[22] = {0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = tid; i < QZ * QY * QX; i += MODIL_NT) {
    const int a = i / (QY * QX), rr = i - a * (QY * QX), b = rr / QX, c = rr - b * QX;
    const int z = z0 - 2 + a, y = y0 - 2 + b, x = x0 - 2 + c;
    if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) continue;
    bool in[12];
    in[0] = x < nx - 1; in[1] = x > 0; in[2] = x < nx - 2; in[3] = x > 1;
    in[4] = y < ny - 1; in[5] = y > 0; in[6] = y < ny - 2; in[7] = y > 1;
    in[8] = z < nz - 1; in[9] = z > 0; in[10] = z < nz - 2; in[11] = z > 1;
    T s[22];
#pragma unroll
    for (int k = 0; k < 22; ++k) {
      const int zz = z + sz[k], yy = y + sy[k], xx = x + sx[k];
      const bool ok = zz >= 0 && zz < nz && yy >= 0 && yy < ny && xx >= 0 && xx < nx;
      s[k] = ok ? Vs(sf[k], zz, yy, xx) : T(0);
    }
    const T r = cont3(s, in, cf);
    if (owned(z, y, x)) {
      if (sizeof(T) == 4) racc += (float)(r * r);
      else raccd += (double)(r * r);
    }
    if (!adj) continue;
    const T lamr = lam_scale * r;
    T e[22];
#pragma unroll
    for (int k = 0; k < 22; ++k) e[k] = T(0);
    const T r0 = cont3(e, in, cf);  // constant part (inlet flux)
#pragma unroll
    for (int k = 0; k < 22; ++k) {
      e[k] = T(1);
      const T jk = cont3(e, in, cf) - r0;
      e[k] = T(0);
      if (jk != T(0)) scatter(sf[k], z + sz[k], y + sy[k], x + sx[k], lamr * jk);
    }
  }

  // ---- measurements --------------------------------------------------------------
  float dacc = 0.f;
  double daccd = 0.0;
  const T wd2 = T(2) * (T)D.w_data_n;
  __syncthreads();
  for (int i = rb + tid; i < re; i += MODIL_NT) {
    const int cell = A.run_cell[i], f = A.run_field[i];
    const int z = cell / (ny * nx), rem = cell - z * (ny * nx), y = rem / nx, x = rem - y * nx;
    const T u = Vs(f, z, y, x);
    T sd = T(0), sq = T(0);
    for (int e = A.run_beg[i]; e < A.run_beg[i + 1]; ++e) {
      const T d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    if (sizeof(T) == 4) dacc += (float)sq;
    else daccd += (double)sq;
    if (adj) gS[f * NC3 + ((z - z0) * C3Y + (y - y0)) * C3X + (x - x0)] += wd2 * sd;
  }
  double rsum, dsum;
  if (sizeof(T) == 4) {
    rsum = block_sum_ff<MODIL_NT>(racc, redf);
    dsum = block_sum_ff<MODIL_NT>(dacc, redf + 16);
  } else {
    rsum = block_sum<MODIL_NT>(raccd, red);
    dsum = block_sum<MODIL_NT>(daccd, red + 8);
  }
  if (tid == 0) {
    A.part[(long long)gt * A.npart + 0] = rsum;
    A.part[(long long)gt * A.npart + 1] = dsum;
  }
  if (!adj) return;
  __syncthreads();
  const AdamCoef ac = acS;
  for (int i = tid; i < F3 * NC3; i += MODIL_NT) {
    const int f = i / NC3, cidx = i - f * NC3;
    const int a = cidx / (C3Y * C3X), rr = cidx - a * (C3Y * C3X), b = rr / C3X, c = rr - b * C3X;
    if (a >= hz || b >= hy || c >= hx) continue;
    const long long o = D.off[f][0] + ((long long)(z0 + a) * ny + (y0 + b)) * nx + (x0 + c);
    const T g = gS[i] * (T)A.gscale;
    A.g[o] = g;
    if (mode == MODE_STEP) {
      T p = A.p[cur][o], m = A.m[o];
      double v = A.v[o];
      adam_update(p, m, v, g, ac);
      A.p[cur ^ 1][o] = p;
      A.m[o] = m;
      A.v[o] = v;
    }
  }
}

// 3-D restriction with Adam for one level: coarse tile 2 x 8 x 16, staged
// fine region, separable x, y, z passes of the transposed interpolation.
constexpr int L3Z = k3LZ, L3Y = k3LY, L3X = k3LX;
constexpr int L3FZ = 2 * L3Z + 4, L3FY = 2 * L3Y + 4, L3FX = 2 * L3X + 4;

template <class T>
__device__ __forceinline__ void rwin3(int X, int nc, T* w) {
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

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_level3(const __grid_constant__ Arena<T> A, int l, int mode, int cur) {
  static_assert(L3Z * L3Y * L3X == MODIL_NT, "one coarse cell per thread");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevInst D;
  __shared__ AdamCoef acS;
  T* S = reinterpret_cast<T*>(smem);   // staged fine region
  T* Hx = S + L3FZ * L3FY * L3FX;      // after the x pass
  T* Hy = Hx + L3FZ * L3FY * L3X;      // after the y pass
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[l][gt];
  load_inst(&D, A, ii);
  __syncthreads();
  const int nz = D.n[l][0], ny = D.n[l][1], nx = D.n[l][2];
  const int fz = D.n[l - 1][0], fy = D.n[l - 1][1], fx = D.n[l - 1][2];
  const int local = gt - D.tile_base[l];
  const int per_z = D.nt[l][1] * D.nt[l][2];
  const int tz = local / per_z, tr = local - tz * per_z;
  const int ty = tr / D.nt[l][2], tx = tr - ty * D.nt[l][2];
  const int Z0 = tz * L3Z, Y0 = ty * L3Y, X0 = tx * L3X;
  const int cz = min(L3Z, nz - Z0), cy = min(L3Y, ny - Y0), cx = min(L3X, nx - X0);
  const int t = threadIdx.x;
  const int oz = t / (L3Y * L3X), orr = t - oz * (L3Y * L3X), oy = orr / L3X, ox = orr - oy * L3X;
  const bool mine = oz < cz && oy < cy && ox < cx;
  const long long e = ((long long)(Z0 + oz) * ny + (Y0 + oy)) * nx + (X0 + ox);
  const bool store_g = (mode != MODE_STEP) || (l < D.nlev - 1);
  if (t == 0) acS = adam_coef(D, A.st[ii]);
  pdl_wait();
  pdl_trigger();
  const int fz0 = max(0, 2 * Z0 - 2), fz1 = min(fz, 2 * (Z0 + cz) + 2);
  const int fy0 = max(0, 2 * Y0 - 2), fy1 = min(fy, 2 * (Y0 + cy) + 2);
  const int fx0 = max(0, 2 * X0 - 2), fx1 = min(fx, 2 * (X0 + cx) + 2);
  const int dz = fz1 - fz0, dy = fy1 - fy0, dx = fx1 - fx0;
  for (int f = 0; f < D.nfield; ++f) {
    const T* __restrict__ gf = A.g + D.off[f][l - 1];
    for (int i = t; i < dz * dy * dx; i += MODIL_NT) {
      const int a = i / (dy * dx), r = i - a * (dy * dx), b = r / dx, c = r - b * dx;
      cp_async(S + (a * L3FY + b) * L3FX + c, gf + ((long long)(fz0 + a) * fy + (fy0 + b)) * fx + (fx0 + c));
    }
    // this thread's parameter and moments (plain loads overlap the copies)
    T pv = T(0), mv = T(0);
    double vv = 0.0;
    const long long o = D.off[f][l] + e;
    if (mode == MODE_STEP && mine) {
      pv = A.p[cur][o];
      mv = A.m[o];
      vv = A.v[o];
    }
    cp_async_wait_all();
    __syncthreads();
    // x pass: (dz, dy, cx)
    for (int i = t; i < dz * dy * cx; i += MODIL_NT) {
      const int a = i / (dy * cx), r = i - a * (dy * cx), b = r / cx, c = r - b * cx;
      const int X = X0 + c;
      T w[6];
      rwin3<T>(X, nx, w);
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int q = min(max(2 * X - 2 + k - fx0, 0), dx - 1);
        acc += w[k] * S[(a * L3FY + b) * L3FX + q];
      }
      Hx[(a * L3FY + b) * L3X + c] = acc;
    }
    __syncthreads();
    // y pass: (dz, cy, cx)
    for (int i = t; i < dz * cy * cx; i += MODIL_NT) {
      const int a = i / (cy * cx), r = i - a * (cy * cx), b = r / cx, c = r - b * cx;
      const int Y = Y0 + b;
      T w[6];
      rwin3<T>(Y, ny, w);
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int q = min(max(2 * Y - 2 + k - fy0, 0), dy - 1);
        acc += w[k] * Hx[(a * L3FY + q) * L3X + c];
      }
      Hy[(a * L3Y + b) * L3X + c] = acc;
    }
    __syncthreads();
    // z pass and the update of this thread's cell
    if (mine) {
      const int Z = Z0 + oz;
      T w[6];
      rwin3<T>(Z, nz, w);
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int q = min(max(2 * Z - 2 + k - fz0, 0), dz - 1);
        acc += w[k] * Hy[(q * L3Y + oy) * L3X + ox];
      }
      if (store_g) A.g[o] = acc;
      if (mode == MODE_STEP) {
        const AdamCoef ac = acS;
        adam_update(pv, mv, vv, acc, ac);
        A.p[cur ^ 1][o] = pv;
        A.m[o] = mv;
        A.v[o] = vv;
      }
    }
    __syncthreads();  // S, Hx and Hy are reused by the next field
  }
}

static cudaLaunchConfig_t cfg3(dim3 grid, size_t smem, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t c = {};
  c.gridDim = grid;
  c.blockDim = dim3(MODIL_NT);
  c.dynamicSmemBytes = smem;
  c.stream = s;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = at;
  c.numAttrs = 1;
  return c;
}

size_t compose3_smem_bytes(size_t pyr_elems, int elem) { return (size_t)elem * F3 * pyr_elems + 64; }
size_t resid3_smem_bytes(int elem) { return (size_t)elem * (F3 * NS3 + F3 * NC3) + 64; }
size_t level3_smem_bytes(int elem) {
  return (size_t)elem * (L3FZ * L3FY * L3FX + L3FZ * L3FY * L3X + L3FZ * L3Y * L3X) + 64;
}

template <class T>
cudaError_t prepare_ns3d(size_t pyr_elems) {
  cudaError_t e = raise_smem_limit(k_compose3<T>, compose3_smem_bytes(pyr_elems, sizeof(T)));
  if (e == cudaSuccess) e = raise_smem_limit(k_resid3<T>, resid3_smem_bytes(sizeof(T)));
  if (e == cudaSuccess) e = raise_smem_limit(k_level3<T>, level3_smem_bytes(sizeof(T)));
  return e;
}

template <class T>
cudaError_t launch_compose3(const Arena<T>& A, int cur, size_t pyr, cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[0]), compose3_smem_bytes(pyr, sizeof(T)), s, at);
  return cudaLaunchKernelEx(&c, k_compose3<T>, A, cur);
}

template <class T>
cudaError_t launch_resid3(const Arena<T>& A, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[0]), resid3_smem_bytes(sizeof(T)), s, at);
  return cudaLaunchKernelEx(&c, k_resid3<T>, A, mode, cur);
}

template <class T>
cudaError_t launch_level3(const Arena<T>& A, int level, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[level] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[level]), level3_smem_bytes(sizeof(T)), s, at);
  return cudaLaunchKernelEx(&c, k_level3<T>, A, level, mode, cur);
}

template cudaError_t prepare_ns3d<float>(size_t);
template cudaError_t prepare_ns3d<double>(size_t);
template cudaError_t launch_compose3<float>(const Arena<float>&, int, size_t, cudaStream_t);
template cudaError_t launch_compose3<double>(const Arena<double>&, int, size_t, cudaStream_t);
template cudaError_t launch_resid3<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_resid3<double>(const Arena<double>&, int, int, cudaStream_t);
template cudaError_t launch_level3<float>(const Arena<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_level3<double>(const Arena<double>&, int, int, int, cudaStream_t);

}  // namespace modil
