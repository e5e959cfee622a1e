// Penalised steady Navier-Stokes in 3-D (body shape, paper Section 3.5,
// equation eq_nschi3): fields u, v, w, p, chihat on (z, y, x) cells of
// [0,1] x [0,1] x [0,2], chi = 1/(1 + exp(-(chihat - 5))) (the initial guess
// chihat = 0 is chi = 1/(1 + e^5), almost no body, as Section 3.5 states).
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
//   k_prolong3  one launch per level, coarse to fine: the composed level
//               w_l = u_l + T w_{l+1} (Horner's scheme, Section 2.2), the finest
//               into the composed-field buffer;
//   k_resid3    per 3-D tile: stage the composed fields with a halo of 4,
//               residuals and their adjoint in gather form (each cell collects
//               the adjoint of the fluxes through its six faces and of the
//               neighbouring pressure-gradient and continuity terms; no
//               atomics), the measurements, dL/du and Adam on level 1;
//   k_level3    one block per (coarse tile, field): restriction of the level
//               above (transposed interpolation) and Adam.
#include <cuda.h>

#include <algorithm>

#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

// Polls of one bounded mbarrier wait before the block gives up; a test can
// lower it (set_spin_limit) to make a wait run out on purpose.
constexpr long long kSpinPolls = 1LL << 24;
__device__ long long g_spin_limit = kSpinPolls;

cudaError_t set_spin_limit(long long polls) {
  if (polls < 0) polls = kSpinPolls;
  return cudaMemcpyToSymbol(g_spin_limit, &polls, sizeof(polls));
}

constexpr int C3Z = k3TZ, C3Y = k3TY, C3X = k3TX;  // fine tile (owned cells)
constexpr int NC3 = C3Z * C3Y * C3X;
constexpr int H3 = 4;                       // staged halo of the composed fields
constexpr int S3Z = C3Z + 2 * H3, S3Y = C3Y + 2 * H3, S3X = C3X + 2 * H3;
constexpr int NS3 = S3Z * S3Y * S3X;
constexpr int F3 = 5;

// ---------------------------------------------------------------------------
// Composition, one level per launch (Horner's scheme, Section 2.2):
// w_l = u_l + T w_{l+1}; the coarsest composed level is u_{L-1} itself (read
// from the parameters), w_0 goes to the composed-field buffer, the others to
// the per-level scratch.  One block per (coarse tile of level l+1, field): the
// coarse tile and a halo of one cell are staged in shared memory, and each
// thread writes the 8 fine children of its coarse cell (separable weights: per
// axis the even child takes 1/4, 3/4 of cells j-1, j and the odd child 3/4,
// 1/4 of cells j, j+1; past the first or last coarse centre the line through
// the two outermost centres is extended, 5/4 and -1/4; a single coarse cell
// is copied).
// ---------------------------------------------------------------------------
constexpr int PZ = k3LZ + 2, PY = k3LY + 2, PX = k3LX + 2;  // staged coarse region

template <class T>
__device__ __forceinline__ void child_weights(int j, int nc, T* we, T* wo) {
  // coefficients of (c[j-1], c[j], c[j+1]) for the even and the odd child of j
  if (nc == 1) {
    we[0] = T(0); we[1] = T(1); we[2] = T(0);
    wo[0] = T(0); wo[1] = T(1); wo[2] = T(0);
    return;
  }
  if (j == 0) { we[0] = T(0); we[1] = T(1.25); we[2] = T(-0.25); }
  else { we[0] = T(0.25); we[1] = T(0.75); we[2] = T(0); }
  if (j == nc - 1) { wo[0] = T(-0.25); wo[1] = T(1.25); wo[2] = T(0); }
  else { wo[0] = T(0); wo[1] = T(0.75); wo[2] = T(0.25); }
}

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_prolong3(const __grid_constant__ Arena<T> A, int l, int cur) {
  static_assert(k3LZ * k3LY * k3LX == MODIL_NT, "one coarse cell per thread");
  __shared__ DevInst D;
  __shared__ T cS[PZ * PY * PX];
  const int gt = blockIdx.x, f = blockIdx.y;
  const int lc = l + 1;  // the coarse level
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[lc][gt];
  load_inst(&D, A, ii);
  __syncthreads();
  const bool blk = f < D.nfield && lc <= D.nlev - 1;
  const int local = gt - D.tile_base[lc];
  const int per_z = D.nt[lc][1] * D.nt[lc][2];
  const int bz = local / per_z, br = local - bz * per_z;
  const int by = br / D.nt[lc][2], bx = br - by * D.nt[lc][2];
  const int cz = D.n[lc][0], cy = D.n[lc][1], cx = D.n[lc][2];
  const int Z0 = bz * k3LZ, Y0 = by * k3LY, X0 = bx * k3LX;
  const int t = threadIdx.x;
  const int oz = t / (k3LY * k3LX), oy = (t / k3LX) % k3LY, ox = t % k3LX;
  const int Z = Z0 + oz, Y = Y0 + oy, Xc = X0 + ox;
  const bool mine = blk && Z < cz && Y < cy && Xc < cx;
  const int nyf = 2 * cy, nxf = 2 * cx;
  // this level's own values (the 8 children of the thread's coarse cell) were
  // last written one step earlier: read them before the dependency wait
  T uo[2][2][2];
  {
    const T* __restrict__ u = A.p[cur] + D.off[blk ? f : 0][l];
#pragma unroll
    for (int cz2 = 0; cz2 < 2; ++cz2)
#pragma unroll
      for (int cy2 = 0; cy2 < 2; ++cy2) {
        const long long rowo = ((long long)(2 * Z + cz2) * nyf + (2 * Y + cy2)) * nxf + 2 * Xc;
#pragma unroll
        for (int cx2 = 0; cx2 < 2; ++cx2) uo[cz2][cy2][cx2] = mine ? u[rowo + cx2] : T(0);
      }
  }
  pdl_wait();
  pdl_trigger();
  if (!blk) return;
  const T* __restrict__ w = (lc == D.nlev - 1 ? A.p[cur] : A.wl) + D.off[f][lc];
  // stage the coarse tile with a halo of one cell (clamped at the grid edge;
  // clamped copies only meet zero weights)
  for (int i = threadIdx.x; i < PZ * PY * PX; i += MODIL_NT) {
    const int a = i / (PY * PX), r = i - a * (PY * PX), b = r / PX, c = r - b * PX;
    const int z = min(max(Z0 - 1 + a, 0), cz - 1), y = min(max(Y0 - 1 + b, 0), cy - 1),
              x = min(max(X0 - 1 + c, 0), cx - 1);
    cS[i] = w[((long long)z * cy + y) * cx + x];
  }
  __syncthreads();
  if (!mine) return;
  T ez[3], odz[3], ey[3], ody[3], ex[3], odx[3];
  child_weights<T>(Z, cz, ez, odz);
  child_weights<T>(Y, cy, ey, ody);
  child_weights<T>(Xc, cx, ex, odx);
  // along x: for the 3 x 3 (z, y) rows around the cell, the even and odd x children
  T hx[2][3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T* row = cS + ((oz + a) * PY + (oy + b)) * PX + ox;
      hx[0][a][b] = ex[0] * row[0] + ex[1] * row[1] + ex[2] * row[2];
      hx[1][a][b] = odx[0] * row[0] + odx[1] * row[1] + odx[2] * row[2];
    }
  T* __restrict__ out = l == 0 ? A.ufine + D.fine_off[f] : A.wl + D.off[f][l];
#pragma unroll
  for (int cz2 = 0; cz2 < 2; ++cz2) {
    const T* wz = cz2 ? odz : ez;
#pragma unroll
    for (int cy2 = 0; cy2 < 2; ++cy2) {
      const T* wy = cy2 ? ody : ey;
      const long long rowo = ((long long)(2 * Z + cz2) * nyf + (2 * Y + cy2)) * nxf + 2 * Xc;
#pragma unroll
      for (int cx2 = 0; cx2 < 2; ++cx2) {
        T v = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          v += wz[a] * (wy[0] * hx[cx2][a][0] + wy[1] * hx[cx2][a][1] + wy[2] * hx[cx2][a][2]);
        out[rowo + cx2] = uo[cz2][cy2][cx2] + v;
      }
    }
  }
}

// Single-level instances: the composed field is level 0 itself.
template <class T>
__global__ void k_copy3(const __grid_constant__ Arena<T> A, int cur) {
  __shared__ DevInst D;
  const int gt = blockIdx.x, f = blockIdx.y;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  if (f >= D.nfield || D.nlev != 1) return;
  const int local = gt - D.tile_base[0];
  const int per_z = D.nt[0][1] * D.nt[0][2];
  const int bz = local / per_z, br = local - bz * per_z;
  const int by = br / D.nt[0][2], bx = br - by * D.nt[0][2];
  const int nz = D.n[0][0], ny = D.n[0][1], nx = D.n[0][2];
  for (int t = threadIdx.x; t < C3Z * C3Y * C3X; t += blockDim.x) {
    const int z = bz * C3Z + t / (C3Y * C3X), y = by * C3Y + (t / C3X) % C3Y, x = bx * C3X + t % C3X;
    if (z >= nz || y >= ny || x >= nx) continue;
    const long long o = ((long long)z * ny + y) * nx + x;
    A.ufine[D.fine_off[f] + o] = A.p[cur][D.off[f][0] + o];
  }
}

// Ghost coefficient alpha and offset beta of field f (0..3) beyond face
// (axis, side) of the domain: ghost = alpha * (value of the adjacent cell) + beta.
template <class T>
__device__ __forceinline__ void ghost3(int f, int axis, int side, T& alpha, T& beta) {
  beta = T(0);
  if (axis == 2) {           // x
    if (side == 0) {         // inlet: u = 2 - u_P (face value 1), v, w odd, p even
      alpha = (f == 3) ? T(1) : T(-1);
      beta = (f == 0) ? T(2) : T(0);
    } else {                 // outlet: p odd (p = 0 on the face), velocity even
      alpha = (f == 3) ? T(-1) : T(1);
    }
  } else if (axis == 1) {    // y walls: v odd, the rest even
    alpha = (f == 1) ? T(-1) : T(1);
  } else {                   // z walls: w odd, the rest even
    alpha = (f == 2) ? T(-1) : T(1);
  }
}

template <class T>
struct Ns3Coef {
  T ih[3], ih2[3], i2h[3];  // per axis (z, y, x): 1/h, 1/h^2, 1/(2h)
  T nu, lam, tf;
};

// Continuity residual from its 22 stencil values.
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

// d(axis part of the continuity residual of cell P)/d(value at P + o e_axis)
// for the normal velocity (vel = true, |o| <= 1) or the pressure (|o| <= 2).
// P's position along the axis: i in [0, n); x axis: inflow face at i = 0
// (flux 1), outflow at n - 1 (flux u_P, odd pressure ghost); y, z: walls
// (no flux, even pressure ghosts).
template <class T, bool INTR>
__device__ __forceinline__ T cont_coef(bool xaxis, int i, int n, int o, bool vel, T tf, T ih) {
  const bool in0 = INTR || i < n - 1, in1 = INTR || i > 0, in2 = INTR || i < n - 2, in3 = INTR || i > 1;
  const T q = T(0.25) * tf, h = T(0.5);
  T ce = T(0), cw = T(0);  // partials of the + face flux and of the - face flux
  if (vel) {
    if (in0) { if (o == 0 || o == 1) ce = h; }
    else if (xaxis && o == 0) ce = T(1);   // outflow flux u_P
    if (in1) { if (o == 0 || o == -1) cw = h; }
  } else {
    const T godd = xaxis ? T(-1) : T(1);   // sign of the + end's pressure ghost
    if (in0) {
      if (o == 0) ce = tf - q + (in1 ? T(0) : -q);
      else if (o == 1) ce = -tf + q + (in2 ? T(0) : godd * q);
      else if (o == -1) ce = in1 ? -q : T(0);
      else if (o == 2) ce = in2 ? q : T(0);
    }
    if (in1) {
      if (o == 0) cw = -tf + q + (in0 ? T(0) : godd * q);
      else if (o == -1) cw = tf - q + (in3 ? T(0) : -q);
      else if (o == -2) cw = in3 ? -q : T(0);
      else if (o == 1) cw = in0 ? q : T(0);
    }
  }
  return (ce - cw) * ih;
}

// ---------------------------------------------------------------------------
// Residuals, adjoint, data term and level-1 Adam for one fine tile.
//   phase 1  momentum residuals on the tile plus one cell: the adjoint weights
//            A_c = 2 w dV r_c (1 - chi) of the three components, and for owned
//            cells the terms of their own residual that do not pass through a
//            face (penalisation, body fraction); continuity residuals on the
//            tile plus two cells (weights B = 2 w dV r);
//   phase 2  each owned cell gathers, per face, the adjoint of the convective
//            and viscous fluxes through that face, the pressure-gradient terms
//            of its neighbours and the continuity terms of the cells within two
//            cells along each axis, adds the data term, writes dL/du and steps
//            level 1 with Adam.  No atomics: every cell is written by one thread.
// ---------------------------------------------------------------------------
constexpr int MZ = C3Z + 2, MY = C3Y + 2, MX = C3X + 2, NM = MZ * MY * MX;    // tile + 1
constexpr int QZ = C3Z + 4, QY = C3Y + 4, QX = C3X + 4, NQ = QZ * QY * QX;    // tile + 2

// chihat is staged on the tile plus one cell in z and y and plus four in x
// (a TMA box starts on a 16-byte boundary): [CZ3][CY3][CX3], x offset 4.
constexpr int CZ3 = C3Z + 2, CY3 = C3Y + 2, CX3 = C3X + 8, NC3S = CZ3 * CY3 * CX3;

template <class T>
struct R3 {  // per-tile context of the residual kernel
  T *uS, *cS, *aS, *bS, *gS;
  int z0, y0, x0, hz, hy, hx, nz, ny, nx;
  Ns3Coef<T> cf;
  T Rs;
  __device__ int sidx(int z, int y, int x) const {
    return ((z - z0 + H3) * S3Y + (y - y0 + H3)) * S3X + (x - x0 + H3);
  }
  __device__ int cidx(int z, int y, int x) const {
    return ((z - z0 + 1) * CY3 + (y - y0 + 1)) * CX3 + (x - x0 + 4);
  }
  __device__ int midx(int z, int y, int x) const {
    return ((z - z0 + 1) * MY + (y - y0 + 1)) * MX + (x - x0 + 1);
  }
  __device__ bool owned(int z, int y, int x) const {
    return z >= z0 && z < z0 + hz && y >= y0 && y < y0 + hy && x >= x0 && x < x0 + hx;
  }
};

// Phase 1: momentum weights on the tile plus one cell, own-residual terms of
// owned cells, continuity weights on the tile plus two cells.  INTR: the tile
// and four cells around it lie inside the grid (no ghost, wall or flag logic).
template <class T, bool INTR>
__device__ __forceinline__ void r3_phase1(const R3<T>& c, bool adj, float& racc, double& raccd) {
  const Ns3Coef<T>& cf = c.cf;
  const int dims[3] = {c.nz, c.ny, c.nx};
  auto addsq = [&](T r) {
    if (sizeof(T) == 4) racc += (float)(r * r);
    else raccd += (double)(r * r);
  };
  for (int i = threadIdx.x; i < NM; i += MODIL_NT) {
    const int a = i / (MY * MX), rr = i - a * (MY * MX), b = rr / MX, cc = rr - b * MX;
    const int z = c.z0 - 1 + a, y = c.y0 - 1 + b, x = c.x0 - 1 + cc;
    if (!INTR && (z < 0 || z >= c.nz || y < 0 || y >= c.ny || x < 0 || x >= c.nx)) continue;
    const int P[3] = {z, y, x};
    const int sp = c.sidx(z, y, x);
    T cen[4], nv[4][3][2];
    bool gh[3][2];
#pragma unroll
    for (int f = 0; f < 4; ++f) cen[f] = c.uS[f * NS3 + sp];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int q = P[ax] + (sd ? 1 : -1);
        const bool inside = INTR || (q >= 0 && q < dims[ax]);
        gh[ax][sd] = !inside;
        const int stride = ax == 0 ? S3Y * S3X : (ax == 1 ? S3X : 1);
        const int sq = sp + (sd ? stride : -stride);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (inside) {
            nv[f][ax][sd] = c.uS[f * NS3 + sq];
          } else {
            T alpha, beta;
            ghost3<T>(f, ax, sd, alpha, beta);
            nv[f][ax][sd] = alpha * cen[f] + beta;
          }
        }
      }
    const T chat = c.cS[c.cidx(z, y, x)];
    // chi and 1 - chi each from its own logistic: 1 - chi is never formed by
    // subtraction, which loses all digits in FP32 where chi is near 1
    const T chi = T(1) / (T(1) + texp(-(chat - T(5))));
    const T om = T(1) / (T(1) + texp(chat - T(5)));
    T Vf[3][2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int n = 2 - ax;  // velocity component normal to the faces of this axis
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const T mk = (ax == 2 || !gh[ax][sd]) ? T(1) : T(0);  // mass flux through walls is zero
        Vf[ax][sd] = mk * T(0.5) * (cen[n] + nv[n][ax][sd]);
      }
    }
    const bool own = c.owned(z, y, x);
    const int ot = ((z - c.z0) * C3Y + (y - c.y0)) * C3X + (x - c.x0);
    T gch = T(0);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const int cax = 2 - comp;
      const T phi = cen[comp];
      T conv = T(0), lap = T(0);
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        conv += (Vf[ax][1] * T(0.5) * (phi + nv[comp][ax][1]) - Vf[ax][0] * T(0.5) * (nv[comp][ax][0] + phi)) *
                cf.ih[ax];
        lap += (nv[comp][ax][1] - T(2) * phi + nv[comp][ax][0]) * cf.ih2[ax];
      }
      const T M = conv + (nv[3][cax][1] - nv[3][cax][0]) * cf.i2h[cax] - cf.nu * lap;
      const T r = om * M + cf.lam * chi * phi;
      if (own) addsq(r);
      const T R = c.Rs * r;
      c.aS[comp * NM + i] = R * om;
      if (own && adj) {
        c.gS[comp * NC3 + ot] = R * cf.lam * chi;
        gch += R * chi * om * (cf.lam * phi - M);
      }
    }
    if (own && adj) c.gS[4 * NC3 + ot] = gch;
  }
  const int sf[22] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3};
  const int sz[22] = {0, 0, 0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2};
  const int sy[22] = {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2, 0, 0, 0, 0};
  const int sx[22] = {0, 1, -1, 0, 0, 0, 0, 0, 0, 0, 1, -1, 2, -2, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < NQ; i += MODIL_NT) {
    const int a = i / (QY * QX), rr = i - a * (QY * QX), b = rr / QX, cc = rr - b * QX;
    const int z = c.z0 - 2 + a, y = c.y0 - 2 + b, x = c.x0 - 2 + cc;
    if (!INTR && (z < 0 || z >= c.nz || y < 0 || y >= c.ny || x < 0 || x >= c.nx)) continue;
    bool in[12];
    in[0] = INTR || x < c.nx - 1; in[1] = INTR || x > 0; in[2] = INTR || x < c.nx - 2; in[3] = INTR || x > 1;
    in[4] = INTR || y < c.ny - 1; in[5] = INTR || y > 0; in[6] = INTR || y < c.ny - 2; in[7] = INTR || y > 1;
    in[8] = INTR || z < c.nz - 1; in[9] = INTR || z > 0; in[10] = INTR || z < c.nz - 2; in[11] = INTR || z > 1;
    T sv[22];
    const int sp = c.sidx(z, y, x);
    // every slot lies inside the staged box; slots outside the grid hold
    // unused values (cont3 takes the ghost instead, by the flags)
#pragma unroll
    for (int k = 0; k < 22; ++k) sv[k] = c.uS[sf[k] * NS3 + sp + (sz[k] * S3Y + sy[k]) * S3X + sx[k]];
    const T r = cont3(sv, in, cf);
    if (c.owned(z, y, x)) addsq(r);
    c.bS[i] = c.Rs * r;
  }
}

// Adam state of a thread's two owned cells, loaded at kernel start so that
// its DRAM latency overlaps the staging and phase 1.
template <class T>
struct AdamPre {
  T p[2][F3], m[2][F3];
  double v[2][F3];
};

// Phase 2: gather of the adjoint for every owned cell; dL/du and Adam.
template <class T, bool INTR>
__device__ __forceinline__ void r3_phase2(const R3<T>& c, const Arena<T>& A, const DevInst& D, int mode, int cur,
                                          const AdamCoef& ac, const AdamPre<T>& pre) {
  static_assert(NC3 == 2 * MODIL_NT, "two owned cells per thread");
  const Ns3Coef<T>& cf = c.cf;
  const int dims[3] = {c.nz, c.ny, c.nx};
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int t = threadIdx.x + kk * MODIL_NT;
    const int a = t / (C3Y * C3X), rr = t - a * (C3Y * C3X), b = rr / C3X, cc = rr - b * C3X;
    if (!INTR && (a >= c.hz || b >= c.hy || cc >= c.hx)) continue;
    const int z = c.z0 + a, y = c.y0 + b, x = c.x0 + cc;
    const int X[3] = {z, y, x};
    const int sp = c.sidx(z, y, x), mp = c.midx(z, y, x);
    const int qp = ((a + 2) * QY + (b + 2)) * QX + (cc + 2);
    T g[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) g[f] = c.gS[f * NC3 + t];
    T cen[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) cen[f] = c.uS[f * NS3 + sp];
    T AX[3];
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) AX[c3] = c.aS[c3 * NM + mp];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int n = 2 - ax;
      const int sstr = ax == 0 ? S3Y * S3X : (ax == 1 ? S3X : 1);
      const int mstr = ax == 0 ? MY * MX : (ax == 1 ? MX : 1);
      const int qstr = ax == 0 ? QY * QX : (ax == 1 ? QX : 1);
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int s = sd ? 1 : -1;
        const bool ghost = !INTR && ((X[ax] + s < 0) || (X[ax] + s >= dims[ax]));
        T nb[4], al[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (ghost) {
            T alpha, beta;
            ghost3<T>(f, ax, sd, alpha, beta);
            nb[f] = alpha * cen[f] + beta;
            al[f] = alpha;
          } else {
            nb[f] = c.uS[f * NS3 + sp + s * sstr];
            al[f] = T(0);
          }
        }
        const T mk = (ax == 2 || !ghost) ? T(1) : T(0);
        const T Vn = mk * T(0.5) * (cen[n] + nb[n]);
        T tn = T(0);
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
          const T AY = ghost ? T(0) : c.aS[c3 * NM + mp + s * mstr];
          const T Wc = T(s) * (AX[c3] - AY) * cf.ih[ax];
          tn += Wc * T(0.5) * (cen[c3] + nb[c3]);
          // convective flux through this face via the transported component
          g[c3] += T(0.5) * Vn * Wc * (ghost ? (T(1) + al[c3]) : T(1));
          // viscous flux through this face
          g[c3] += ghost ? -cf.nu * cf.ih2[ax] * AX[c3] * (al[c3] - T(1)) : cf.nu * cf.ih2[ax] * (AX[c3] - AY);
        }
        // convective flux through this face via the normal (transporting) velocity
        g[n] += T(0.5) * mk * tn * (ghost ? (T(1) + al[n]) : T(1));
        // pressure gradient of the component normal to this axis
        if (ghost) g[3] += T(s) * al[3] * AX[n] * cf.i2h[ax];
        else g[3] -= T(s) * c.aS[n * NM + mp + s * mstr] * cf.i2h[ax];
      }
      // continuity: cells P = X + d e_ax (|d| <= 2) that read X along this axis
      const bool xaxis = (ax == 2);
#pragma unroll
      for (int d = -2; d <= 2; ++d) {
        const int pi = X[ax] + d;
        if (!INTR && (pi < 0 || pi >= dims[ax])) continue;
        const T B = c.bS[qp + d * qstr];
        g[3] += B * cont_coef<T, INTR>(xaxis, pi, dims[ax], -d, false, cf.tf, cf.ih[ax]);
        if (d >= -1 && d <= 1) g[n] += B * cont_coef<T, INTR>(xaxis, pi, dims[ax], -d, true, cf.tf, cf.ih[ax]);
      }
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const long long o = D.off[f][0] + ((long long)z * c.ny + y) * c.nx + x;
      const T gg = g[f] * (T)A.gscale;
      A.g[o] = gg;
      if (mode == MODE_STEP) {
        T p = pre.p[kk][f], m = pre.m[kk][f];
        double v = pre.v[kk][f];
        adam_update(p, m, v, gg, ac);
        A.p[cur ^ 1][o] = p;
        A.m[o] = m;
        A.v[o] = v;
      }
    }
  }
}

__device__ __forceinline__ uint32_t smem_addr3(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <class T>
__global__ void __launch_bounds__(MODIL_NT)
k_resid3(const __grid_constant__ Arena<T> A, int mode, int cur, const __grid_constant__ CUtensorMap tm_u,
         const __grid_constant__ CUtensorMap tm_c, int use_tma) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ DevInst D;
  __shared__ double red[16];
  __shared__ AdamCoef acS;
  __shared__ Ns3Coef<T> cfS;
  __shared__ __align__(8) uint64_t bar;
  __shared__ int tma_ok;
  R3<T> c;
  c.uS = reinterpret_cast<T*>(smem);   // u, v, w, p with a halo of 4: 4 x NS3
  c.cS = c.uS + 4 * NS3;               // chihat: NC3S
  c.aS = c.cS + NC3S;                  // momentum adjoint weights: 3 x NM
  c.bS = c.aS + 3 * NM;                // continuity adjoint weights: NQ
  c.gS = c.bS + NQ;                    // own-residual and data terms: F3 x NC3
  float* redf = reinterpret_cast<float*>(red);
  const int tid = threadIdx.x;
  const int gt = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  load_inst(&D, A, ii);
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  __syncthreads();
  c.nz = D.n[0][0]; c.ny = D.n[0][1]; c.nx = D.n[0][2];
  const int local = gt - D.tile_base[0];
  const int per_z = D.nt[0][1] * D.nt[0][2];
  const int tz = local / per_z, tr = local - tz * per_z;
  const int ty = tr / D.nt[0][2], tx = tr - ty * D.nt[0][2];
  c.z0 = tz * C3Z; c.y0 = ty * C3Y; c.x0 = tx * C3X;
  c.hz = min(C3Z, c.nz - c.z0); c.hy = min(C3Y, c.ny - c.y0); c.hx = min(C3X, c.nx - c.x0);
  if (tid == 0) {
    acS = adam_coef(D, A.st[ii]);
    // stencil coefficients: FP64 divisions by one thread (GB300 runs FP64 at
    // 1/64 of the FP32 rate; per thread they would cost more than the stencils)
    for (int a = 0; a < 3; ++a) {
      const double hh = D.h[a];
      cfS.ih[a] = (T)(1.0 / hh);
      cfS.ih2[a] = (T)(1.0 / (hh * hh));
      cfS.i2h[a] = (T)(0.5 / hh);
    }
    cfS.nu = (T)(D.coef[1] / D.coef[0]);  // D / Re
    cfS.lam = (T)D.coef[2];
    cfS.tf = (T)D.coef[3];
    tma_ok = 1;
    if (use_tma) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr3(&bar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  for (int i = tid; i < F3 * NC3; i += MODIL_NT) c.gS[i] = T(0);
  // level-1 parameters and moments were last written one step earlier (many
  // launches back), so they may be read before the dependency wait
  AdamPre<T> pre;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int t = tid + kk * MODIL_NT;
    const int a = t / (C3Y * C3X), b = (t / C3X) % C3Y, cc = t % C3X;
    const bool ok = mode == MODE_STEP && a < c.hz && b < c.hy && cc < c.hx;
    const long long e = ((long long)(c.z0 + a) * c.ny + (c.y0 + b)) * c.nx + (c.x0 + cc);
#pragma unroll
    for (int f = 0; f < F3; ++f) {
      const long long o = D.off[f][0] + e;
      pre.p[kk][f] = ok ? A.p[cur][o] : T(0);
      pre.m[kk][f] = ok ? A.m[o] : T(0);
      pre.v[kk][f] = ok ? A.v[o] : 0.0;
    }
  }
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  if (use_tma) {
    // one 4-D box (x, y, z, field 0..3) and one chihat box; reads outside the
    // grid return zeros (never used: ghosts are formed from the cell values)
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(sizeof(T) * (4 * NS3 + NC3S));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr3(&bar)), "r"(bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr3(c.uS)),
          "l"(reinterpret_cast<uint64_t>(&tm_u)), "r"(smem_addr3(&bar)), "r"(c.x0 - H3), "r"(c.y0 - H3),
          "r"(c.z0 - H3), "r"(0)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr3(c.cS)),
          "l"(reinterpret_cast<uint64_t>(&tm_c)), "r"(smem_addr3(&bar)), "r"(c.x0 - 4), "r"(c.y0 - 1),
          "r"(c.z0 - 1), "r"(4)
          : "memory");
    }
    // bounded wait for the copies; on timeout the block flags it, then waits
    // (bounded again) for the copies still in flight into its shared memory
    // before it skips the tile and returns
    auto wait_copies = [&](long long polls) {
      bool done = false;
      for (long long it = 0; it < polls && !done; ++it) {
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(r)
            : "r"(smem_addr3(&bar))
            : "memory");
        done = r != 0;
      }
      return done;
    };
    if (!wait_copies(g_spin_limit)) {
      tma_ok = 0;
      wait_copies(kSpinPolls);
    }
  } else {
    for (int f = 0; f < 4; ++f) {
      const T* src = A.ufine + D.fine_off[f];
      for (int i = tid; i < NS3; i += MODIL_NT) {
        const int a = i / (S3Y * S3X), r = i - a * (S3Y * S3X), b = r / S3X, cc = r - b * S3X;
        const int z = c.z0 - H3 + a, y = c.y0 - H3 + b, x = c.x0 - H3 + cc;
        if (z >= 0 && z < c.nz && y >= 0 && y < c.ny && x >= 0 && x < c.nx)
          cp_async(c.uS + f * NS3 + i, src + ((long long)z * c.ny + y) * c.nx + x);
      }
    }
    const T* src = A.ufine + D.fine_off[4];
    for (int i = tid; i < NC3S; i += MODIL_NT) {
      const int a = i / (CY3 * CX3), r = i - a * (CY3 * CX3), b = r / CX3, cc = r - b * CX3;
      const int z = c.z0 - 1 + a, y = c.y0 - 1 + b, x = c.x0 - 4 + cc;
      if (z >= 0 && z < c.nz && y >= 0 && y < c.ny && x >= 0 && x < c.nx)
        cp_async(c.cS + i, src + ((long long)z * c.ny + y) * c.nx + x);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  if (!tma_ok) {  // the wait for a copy ran out: flag it, skip the tile
    if (tid == 0) atomicOr(&A.st[ii].nonfinite, kStatusTimeout);
    return;
  }
  c.cf = cfS;
  c.Rs = T(2) * (T)D.w_res_dV;
  const bool adj = (mode != MODE_LOSS);
  const bool interior = c.z0 >= 4 && c.z0 + C3Z + 4 <= c.nz && c.y0 >= 4 && c.y0 + C3Y + 4 <= c.ny &&
                        c.x0 >= 4 && c.x0 + C3X + 4 <= c.nx;
  float racc = 0.f;
  double raccd = 0.0;
  if (interior) r3_phase1<T, true>(c, adj, racc, raccd);
  else r3_phase1<T, false>(c, adj, racc, raccd);

  // ---- data term (unique (field, cell) per run) ------------------------------
  float dacc = 0.f;
  double daccd = 0.0;
  const T wd2 = T(2) * (T)D.w_data_n;
  __syncthreads();
  for (int i = rb + tid; i < re; i += MODIL_NT) {
    const int cell = A.run_cell[i], f = A.run_field[i];
    const int z = cell / (c.ny * c.nx), rem = cell - z * (c.ny * c.nx), y = rem / c.nx, x = rem - y * c.nx;
    const T u = (f < 4) ? c.uS[f * NS3 + c.sidx(z, y, x)] : c.cS[c.cidx(z, y, x)];
    T sd = T(0), sq = T(0);
    for (int e = A.run_beg[i]; e < A.run_beg[i + 1]; ++e) {
      const T d = u - A.meas_val[e];
      sd += d;
      sq += d * d;
    }
    if (sizeof(T) == 4) dacc += (float)sq;
    else daccd += (double)sq;
    if (adj) c.gS[f * NC3 + ((z - c.z0) * C3Y + (y - c.y0)) * C3X + (x - c.x0)] += wd2 * sd;
  }
  // off-grid points whose corner cells the tile owns: trilinear sample of the
  // record's field from the composed fields (eight corners) minus the
  // measurement; the tile of a point's lower corner counts its misfit
  if (A.pt_ptr) {
    const int p1 = A.pt_ptr[gt + 1];
    for (int j = A.pt_ptr[gt] + tid; j < p1; j += MODIL_NT) {
      const T* uf = A.ufine + D.fine_off[A.pt_field[j]];
      T smp = T(0);
#pragma unroll
      for (int k = 0; k < 8; ++k) smp += A.pt_w[8 * (long long)j + k] * uf[A.pt_cell[8 * (long long)j + k]];
      const T dd = smp - A.pt_val[j];
      A.pt_diff[j] = dd;
      if (A.pt_own[j]) {
        if (sizeof(T) == 4) dacc += (float)(dd * dd);
        else daccd += (double)(dd * dd);
      }
    }
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
  // the points' gradient: each owned (field, corner cell) sums weight x
  // misfit over the records reaching it, in a fixed order (the block sums'
  // barriers above published the misfits)
  if (A.pc_ptr) {
    const int c1 = A.pc_ptr[gt + 1];
    for (int rr = A.pc_ptr[gt] + tid; rr < c1; rr += MODIL_NT) {
      const int cell = A.pc_cell[rr], f = A.pc_field[rr];
      const int z = cell / (c.ny * c.nx), rem = cell - z * (c.ny * c.nx), y = rem / c.nx, x = rem - y * c.nx;
      T acc = T(0);
      for (int e = A.pc_beg[rr]; e < A.pc_beg[rr + 1]; ++e) acc += A.pe_w[e] * A.pt_diff[A.pe_rec[e]];
      c.gS[f * NC3 + ((z - c.z0) * C3Y + (y - c.y0)) * C3X + (x - c.x0)] += wd2 * acc;
    }
  }
  __syncthreads();
  const AdamCoef ac = acS;
  if (interior) r3_phase2<T, true>(c, A, D, mode, cur, ac, pre);
  else r3_phase2<T, false>(c, A, D, mode, cur, ac, pre);
}

// 3-D restriction with Adam for one level: coarse tile 2 x 8 x 16, staged
// fine region, separable x, y, z passes of the transposed interpolation.
constexpr int L3Z = k3LZ, L3Y = k3LY, L3X = k3LX;
// staged finer region: rows 2 Z0 - 2 .. and 2 Y0 - 2 .., columns 2 X0 - 4 ..
// (a 4-element boundary, so that rows copy in 16-byte chunks)
constexpr int L3FZ = 2 * L3Z + 4, L3FY = 2 * L3Y + 4, L3FX = 2 * L3X + 8;

// 16-byte asynchronous copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16_3(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}

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
  const int gt = blockIdx.x, f = blockIdx.y;
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
  // this thread's parameter and moments: written by this kernel one step
  // earlier (many launches back), so read before the dependency wait
  T pv = T(0), mv = T(0);
  double vv = 0.0;
  const long long o = D.off[min(f, D.nfield - 1)][l] + e;
  if (mode == MODE_STEP && mine && f < D.nfield) {
    pv = A.p[cur][o];
    mv = A.m[o];
    vv = A.v[o];
  }
  pdl_wait();
  pdl_trigger();
  const int fz0 = max(0, 2 * Z0 - 2), fz1 = min(fz, 2 * (Z0 + cz) + 2);
  const int fy0 = max(0, 2 * Y0 - 2), fy1 = min(fy, 2 * (Y0 + cy) + 2);
  const int fx0 = max(0, 2 * X0 - 2), fx1 = min(fx, 2 * (X0 + cx) + 2);
  const int dz = fz1 - fz0, dy = fy1 - fy0;
  if (f >= D.nfield) return;
  {
    const long long fo = D.off[f][l - 1];
    const T* __restrict__ gf = A.g + fo;
    const int oX = 2 * X0 - 4;  // x of the region's first column
    // loops run over the constant-size boxes (divisions by constants) with bounds
    // checks; 4-element chunks wholly inside the level where rows and the level
    // start are 16-byte aligned, single elements otherwise
    const bool vec = ((fx & 3) == 0) && ((fo & 3) == 0) && (sizeof(T) == 4);
    if (vec) {
      constexpr int CW = L3FX / 4;
      for (int i = t; i < L3FZ * L3FY * CW; i += MODIL_NT) {
        const int a = i / (L3FY * CW), b = (i / CW) % L3FY, c = 4 * (i % CW);
        const int xx = oX + c;
        if (a < dz && b < dy && xx >= 0 && xx + 3 < fx && xx + 3 >= fx0 && xx < fx1)
          cp_async16_3(S + (a * L3FY + b) * L3FX + c, gf + ((long long)(fz0 + a) * fy + (fy0 + b)) * fx + xx);
      }
    } else {
      for (int i = t; i < L3FZ * L3FY * L3FX; i += MODIL_NT) {
        const int a = i / (L3FY * L3FX), b = (i / L3FX) % L3FY, c = i % L3FX;
        const int xx = oX + c;
        if (a < dz && b < dy && xx >= fx0 && xx < fx1)
          cp_async(S + i, gf + ((long long)(fz0 + a) * fy + (fy0 + b)) * fx + xx);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // x pass: (dz, dy, cx)
    for (int i = t; i < L3FZ * L3FY * L3X; i += MODIL_NT) {
      const int a = i / (L3FY * L3X), b = (i / L3X) % L3FY, c = i % L3X;
      if (a >= dz || b >= dy || c >= cx) continue;
      const int X = X0 + c;
      T w[6];
      rwin3<T>(X, nx, w);
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {  // taps outside the level have zero weight: clamp them into it
        const int q = min(max(2 * X - 2 + k, fx0), fx1 - 1) - oX;
        acc += w[k] * S[(a * L3FY + b) * L3FX + q];
      }
      Hx[(a * L3FY + b) * L3X + c] = acc;
    }
    __syncthreads();
    // y pass: (dz, cy, cx)
    for (int i = t; i < L3FZ * L3Y * L3X; i += MODIL_NT) {
      const int a = i / (L3Y * L3X), b = (i / L3X) % L3Y, c = i % L3X;
      if (a >= dz || b >= cy || c >= cx) continue;
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

size_t resid3_smem_bytes(int elem) { return (size_t)elem * (4 * NS3 + NC3S + 3 * NM + NQ + F3 * NC3) + 128; }
size_t level3_smem_bytes(int elem) {
  return (size_t)elem * (L3FZ * L3FY * L3FX + L3FZ * L3FY * L3X + L3FZ * L3Y * L3X) + 64;
}

template <class T>
cudaError_t prepare_ns3d(size_t) {
  cudaError_t e = raise_smem_limit(k_resid3<T>, resid3_smem_bytes(sizeof(T)));
  if (e == cudaSuccess) e = raise_smem_limit(k_level3<T>, level3_smem_bytes(sizeof(T)));
  return e;
}

template <class T>
cudaError_t launch_prolong3(const Arena<T>& A, int level, int nfield, int cur, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  if (level < 0) {  // single-level instances: copy level 0
    if (A.ntiles[0] == 0) return cudaSuccess;
    cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[0], nfield), 0, s, at);
    return cudaLaunchKernelEx(&c, k_copy3<T>, A, cur);
  }
  if (A.ntiles[level + 1] == 0) return cudaSuccess;
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[level + 1], nfield), 0, s, at);
  return cudaLaunchKernelEx(&c, k_prolong3<T>, A, level, cur);
}

template <class T>
cudaError_t launch_resid3(const Arena<T>& A, int mode, int cur, const Ns3Maps* maps, cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[0]), resid3_smem_bytes(sizeof(T)), s, at);
  static const CUtensorMap zero{};
  const bool tma = maps && maps->ok;
  return cudaLaunchKernelEx(&c, k_resid3<T>, A, mode, cur, tma ? maps->u : zero, tma ? maps->c : zero,
                            tma ? 1 : 0);
}

// TMA maps of the composed fields of a single-instance 3-D problem: a 4-D view
// (x, y, z, field) of the buffer, boxes of 24 x 16 x 12 x 4 (u, v, w, p) and
// 24 x 10 x 6 x 1 (chihat).  ok = false where TMA cannot address the buffer
// (row pitch not a multiple of 16 bytes): the kernel then stages with cp.async.
typedef CUresult (*EncodeTiled3)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_ns3_maps(Ns3Maps* m, const void* ufine, int nz, int ny, int nx, int elem) {
  m->ok = false;
  if (((long long)nx * elem) % 16 || (reinterpret_cast<uintptr_t>(ufine) & 15)) return 0;
  static EncodeTiled3 enc = nullptr;
  if (!enc) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      return -1;
    enc = reinterpret_cast<EncodeTiled3>(p);
  }
  const CUtensorMapDataType dt = elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)F3};
  cuuint64_t strides[3] = {(cuuint64_t)nx * elem, (cuuint64_t)nx * ny * elem, (cuuint64_t)nx * ny * nz * elem};
  cuuint32_t es[4] = {1, 1, 1, 1};
  cuuint32_t bu[4] = {S3X, S3Y, S3Z, 4};
  cuuint32_t bc[4] = {CX3, CY3, CZ3, 1};
  void* base = const_cast<void*>(ufine);
  if (enc(&m->u, dt, 4, base, dims, strides, bu, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return -2;
  if (enc(&m->c, dt, 4, base, dims, strides, bc, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return -2;
  m->ok = true;
  return 0;
}

template <class T>
cudaError_t launch_level3(const Arena<T>& A, int level, int nfield, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[level] == 0) return cudaSuccess;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t c = cfg3(dim3(A.ntiles[level], nfield), level3_smem_bytes(sizeof(T)), s, at);
  return cudaLaunchKernelEx(&c, k_level3<T>, A, level, mode, cur);
}

template cudaError_t prepare_ns3d<float>(size_t);
template cudaError_t prepare_ns3d<double>(size_t);
template cudaError_t launch_prolong3<float>(const Arena<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_prolong3<double>(const Arena<double>&, int, int, int, cudaStream_t);
template cudaError_t launch_resid3<float>(const Arena<float>&, int, int, const Ns3Maps*, cudaStream_t);
template cudaError_t launch_resid3<double>(const Arena<double>&, int, int, const Ns3Maps*, cudaStream_t);
template cudaError_t launch_level3<float>(const Arena<float>&, int, int, int, int, cudaStream_t);
template cudaError_t launch_level3<double>(const Arena<double>&, int, int, int, int, cudaStream_t);

}  // namespace modil
