// Warp-streaming fine kernel of the viscous Burgers problem (paper Section
// 3.2; axes (t, x)) and the level-by-level composition pass it reads.
//
// Composition pass, coarse to fine: w_l = u_l + T_l w_{l+1}, w_{L-1} = u_{L-1}
// (Horner's scheme of Section 2.2, T the tensor product of the cell-based 1-D
// interpolation), stored in the scratch arrays wl at the offsets of the
// levels: levels L-2 .. 2 of each instance by one block (k_compose2_small),
// then level 1 of every instance in one grid (k_compose2).
//
// Fine kernel (k_fine_stream): one warp owns a strip of kSW = 60 columns and
// kSR = 32 rows of the fine grid.  Lane j holds the two columns
// a = x0 - 2 + 2j and b = a + 1, so the warp covers the owned columns plus two
// on each side: the composed field is needed two columns out, the residuals
// one column out.  Two columns per lane share the per-row work (copies,
// shuffles, addresses, bookkeeping) and move as one 8- or 16-byte access.
// The warp walks down the rows of its strip (from one row above it to one row
// below); per row it
//   1. composes u = u_0 + T w_1 (level 0 of the row, the two rows of w_1 it
//      interpolates between, interpolated in x once per row of w_1);
//   2. evaluates the residual of the row and lambda * dr/du at its four
//      stencil points (lambda = 2 w_res dV r), the neighbours u(a-1) and
//      u(b+1) taken from the adjacent lanes by shuffles;
//   3. adds the data term of the measured cells of the row;
//   4. finishes the previous row: dL/du(n-1, x) gathers lambda dr/du of the
//      residuals that read u(n-1, x) -- its own, those of x-1 and x+1 of row
//      n-1 (one of them in the adjacent lane) and that of (n, x) -- writes it
//      and applies Adam.
// Everything stays in registers: no shared-memory tiles and no block
// barriers.  Level 0's parameters and Adam moments stream through a per-warp
// ring of kRing rows in shared memory, copied asynchronously kRing - 1 rows
// ahead.  Rows go in pairs (2k+1, 2k+2), which interpolate between the same
// two rows k, k+1 of w_1 with the fixed weights (3/4, 1/4) and (1/4, 3/4);
// inside the strip a pair runs with every row condition known to hold (no
// bounds checks, no weight arithmetic), the pairs at the strip's edges and
// the level's ends take the general path.  The next row of w_1 is loaded one
// pair ahead.  The kernel is compiled per mode (loss, gradient, step,
// compose).  Each lane sums its r^2 (at most 64 cells) in FP32, the warp
// combines the lanes in compensated FP32, and each warp writes FP64 partial
// sums (r^2 and the data misfit) for the per-instance tail kernel.
// The stencil (rows n >= 1, the implicit step of the reading of Section 3.2):
//   r = (u^n_i - u^{n-1}_i)/dt + (F_{i+1/2} - F_{i-1/2})/dx
//       - nu (u^n_{i+1} - 2u^n_i + u^n_{i-1})/dx^2,
//   F = Engquist-Osher upwind flux of u^2/2; through a wall the same flux
//   against the zero wall value (Dirichlet data); odd ghosts (u_{-1} = -u_0)
//   for the viscous term.
#include "launch.h"
#include "modil_dev.cuh"

namespace modil {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRing = 4;  // rows of level 0 in flight per warp (a power of two)

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Asynchronous 4- or 8-byte copy to a shared-memory address.
__device__ __forceinline__ void cp_async_at(unsigned saddr, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_at(unsigned saddr, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(src) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <class T>
__device__ __forceinline__ T eo_flux_s(T a, T b, T& da, T& db) {
  const T ap = tmax(a, T(0));
  const T bm = tmin(b, T(0));
  da = ap;
  db = bm;
  return T(0.5) * ap * ap + T(0.5) * bm * bm;
}

// ---------------------------------------------------------------------------
// Composition: one cell of w_l = u_l + T w_{l+1}
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T compose_cell(const T* __restrict__ Pl, const T* __restrict__ Wc, int y, int x,
                                          int nx, int nyc, int nxc) {
  int jy0, jy1, jx0, jx1;
  T wy0, wy1, wx0, wx1;
  prolong_taps<T>(y, nyc, jy0, jy1, wy0, wy1);
  prolong_taps<T>(x, nxc, jx0, jx1, wx0, wx1);
  const T* r0 = Wc + (long long)jy0 * nxc;
  const T* r1 = Wc + (long long)jy1 * nxc;
  const T c = wy0 * (wx0 * r0[jx0] + wx1 * r0[jx1]) + wy1 * (wx0 * r1[jx0] + wx1 * r1[jx1]);
  return Pl[(long long)y * nx + x] + c;
}

// Level 1 of every instance with L >= 3: four consecutive cells of a row per
// thread (16-byte load and store where the row and the level start allow).
template <class T>
__global__ void __launch_bounds__(kComposeNT) k_compose2(const __grid_constant__ Arena<T> A, int l, int cur) {
  const int b = blockIdx.x;
  const int ii = (A.n_inst == 1) ? 0 : A.cblk_inst[l][b];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  const int ny = D.n[l][1], nx = D.n[l][2];
  const int nyc = D.n[l + 1][1], nxc = D.n[l + 1][2];
  const long long cell = (long long)A.cblk_first[l][b] + 4 * threadIdx.x;
  // the levels are written by the previous step's last kernels and, for
  // w_{l+1}, by the previous launch
  pdl_wait();
  pdl_trigger();
  const long long ncell = (long long)ny * nx;
  if (cell >= ncell) return;
  const T* __restrict__ P = A.p[cur];
  const T* __restrict__ Pl = P + D.off[0][l];
  const T* __restrict__ Wc = (l + 1 == D.nlev - 1) ? P + D.off[0][l + 1] : A.wl + D.off[0][l + 1];
  T* __restrict__ Wl = A.wl + D.off[0][l];
  const int y = (int)(cell / nx), x = (int)(cell - (long long)y * nx);
  if (sizeof(T) == 4 && (nx & 3) == 0 && ((D.off[0][l] + cell) & 3) == 0) {
    T v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = compose_cell<T>(Pl, Wc, y, x + k, nx, nyc, nxc);
    *reinterpret_cast<float4*>(Wl + cell) = make_float4(v[0], v[1], v[2], v[3]);
    return;
  }
  for (int k = 0; k < 4 && cell + k < ncell; ++k) {
    const int yy = (int)((cell + k) / nx), xx = (int)((cell + k) - (long long)yy * nx);
    Wl[cell + k] = compose_cell<T>(Pl, Wc, yy, xx, nx, nyc, nxc);
  }
}

// Levels L-2 .. 2 of one instance per block, coarse to fine, a barrier
// between levels (the block's own writes of w_{l+1} are then visible).
template <class T>
__global__ void __launch_bounds__(kComposeSmallNT) k_compose2_small(const __grid_constant__ Arena<T> A, int cur) {
  const int ii = (A.n_inst == 1) ? 0 : A.csmall_inst[blockIdx.x];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  pdl_wait();
  pdl_trigger();
  const T* __restrict__ P = A.p[cur];
  for (int l = D.nlev - 2; l >= 2; --l) {
    const int ny = D.n[l][1], nx = D.n[l][2];
    const int nyc = D.n[l + 1][1], nxc = D.n[l + 1][2];
    const T* __restrict__ Wc = (l + 1 == D.nlev - 1) ? P + D.off[0][l + 1] : A.wl + D.off[0][l + 1];
    const T* __restrict__ Pl = P + D.off[0][l];
    T* __restrict__ Wl = A.wl + D.off[0][l];
    for (int c = threadIdx.x; c < ny * nx; c += kComposeSmallNT) {
      const int y = c / nx, x = c - y * nx;
      Wl[c] = compose_cell<T>(Pl, Wc, y, x, nx, nyc, nxc);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The streaming fine kernel
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void acc_add(float& hi, float& lo, T x) {
  ff_add(hi, lo, (float)x, 0.f);
}

template <class T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// Asynchronous copy of two consecutive elements (8 bytes of FP32, 16 of FP64).
__device__ __forceinline__ void cp_async_pair(unsigned saddr, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_pair(unsigned saddr, const double* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(src) : "memory");
}

// Loop-invariant coefficients of a strip in the working precision, computed
// once per warp into shared memory: under register pressure the compiler
// reloads them from there instead of recomputing conversions and divisions.
template <class T>
struct StreamCoef {
  AdamCoef ac;
  T idt, idx1, idx2, nu, lam_scale, wd2, gscale;
};

// Residual of cell (n, x) and lambda dr/du (lambda = 2 w_res dV r) at its
// four stencil points: (n, x-1) -> lJ0, (n, x) -> lJ1, (n, x+1) -> lJ2,
// (n-1, x) -> lJ3.  uW, uE: the neighbours in the row (unused at a wall, where
// the odd ghost -u stands in for the viscous term and the flux through the
// wall is the upwind flux against the zero wall value).  ls = 2 w_res dV, or
// 0 for a column without a residual (every lambda dr/du then vanishes, so
// that both columns of a lane run the same instructions without branches).
template <class T>
__device__ __forceinline__ T burgers_cell(T u, T uo, T uW, T uE, bool hw, bool he, T cdiag, T ls,
                                          const StreamCoef<T>& cf, T& lJ0, T& lJ1, T& lJ2, T& lJ3) {
  const T uw = hw ? uW : -u;
  const T ue = he ? uE : -u;
  T dFEc, dFEe, dFWw, dFWc;
  const T FE = eo_flux_s(u, he ? ue : T(0), dFEc, dFEe);
  const T FW = eo_flux_s(hw ? uw : T(0), u, dFWw, dFWc);
  const T lap = (ue - T(2) * u + uw) * cf.idx2;
  const T r = (u - uo) * cf.idt + (FE - FW) * cf.idx1 - cf.nu * lap;
  const T lam = ls * r;
  lJ1 = lam * (cf.idt + (dFEc - dFWc) * cf.idx1 - cf.nu * cdiag * cf.idx2);
  lJ0 = hw ? lam * (-dFWw * cf.idx1 - cf.nu * cf.idx2) : T(0);
  lJ2 = he ? lam * (dFEe * cf.idx1 - cf.nu * cf.idx2) : T(0);
  lJ3 = lam * (-cf.idt);
  return r;
}

template <class T, int MODE>
__global__ void __launch_bounds__(kStreamNT, sizeof(T) == 4 ? kStreamBlocksF32 : kStreamBlocksF64)
k_fine_stream(const __grid_constant__ Arena<T> A, int cur) {
  constexpr bool step = (MODE == MODE_STEP), adj = (MODE != MODE_LOSS), comp_only = (MODE == MODE_COMPOSE);
  using T2 = typename Pair<T>::type;
  // per warp: a ring of kRing rows (64 columns) of level 0's parameters and
  // Adam moments, filled with asynchronous copies kRing - 1 rows ahead of use
  __shared__ __align__(16) T sP[kStreamNT / 32][kRing][64];
  __shared__ __align__(16) T sM[kStreamNT / 32][kRing][64];
  __shared__ __align__(16) double sV[kStreamNT / 32][kRing][64];
  __shared__ StreamCoef<T> sC[kStreamNT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gt = blockIdx.x * (kStreamNT / 32) + w;
  if (gt >= A.ntiles[0]) return;
  const int ii = (A.n_inst == 1) ? 0 : A.tile_inst[0][gt];
  const DevInst& D = (A.n_inst == 1) ? A.inst0 : A.inst[ii];
  const int ny = D.n[0][1], nx = D.n[0][2];
  const int L = D.nlev;
  const int local = gt - D.tile_base[0];
  const int sty = local / D.nt[0][2], stx = local - sty * D.nt[0][2];
  const int y0 = sty * kSR, x0 = stx * kSW;
  const int y1 = min(y0 + kSR, ny), xo1 = min(x0 + kSW, nx);  // owned rows [y0, y1), columns [x0, xo1)
  // the lane's two columns: a = x0 - 2 + 2 lane, b = a + 1
  const int xa = x0 - 2 + 2 * lane, xb = xa + 1;
  const bool ina = xa >= 0 && xa < nx, inb = xb >= 0 && xb < nx;
  const bool owna = xa >= x0 && xa < xo1, ownb = xb >= x0 && xb < xo1;
  // residual columns [x0 - 1, xo1]
  const bool resa = ina && xa >= x0 - 1 && xa <= xo1, resb = inb && xb >= x0 - 1 && xb <= xo1;
  const bool hwa = xa > 0, hea = xa < nx - 1, hwb = xb > 0, heb = xb < nx - 1;
  // per-instance bases; indices within an instance's level fit 32 bits
  const long long o0 = D.off[0][0];
  const T* __restrict__ P0 = A.p[cur] + o0;
  const T* __restrict__ M0 = A.m + o0;
  const double* __restrict__ V0 = A.v + o0;
  T* __restrict__ G0 = A.g + o0;               // level 0's gradient
  T* __restrict__ Pn = A.p[cur ^ 1] + o0;      // level 0 after the step
  // both columns of a lane move as one 8- or 16-byte access when every row
  // and array starts on a pair boundary (x0 and a are even); else element by
  // element
  const bool vec = (nx % 2 == 0) &&
                   ((reinterpret_cast<uintptr_t>(P0) | reinterpret_cast<uintptr_t>(Pn) |
                     reinterpret_cast<uintptr_t>(M0) | reinterpret_cast<uintptr_t>(G0)) % (2 * sizeof(T))) == 0 &&
                   reinterpret_cast<uintptr_t>(V0) % 16 == 0;
  const int nstart = max(y0 - 1, 0);
  const int rmax = min(y1, ny - 1);  // last row of level 0 the strip reads
  // level 0 of row r (and m, v of owned rows) -> ring slot r % kRing; one copy
  // group per row, committed even when empty.  chk = false: the caller knows
  // y0 <= r <= rmax.  Shared addresses of the lane's ring columns and global
  // pointers of its columns are formed once; a row adds offsets only.
  const unsigned sPa = (unsigned)__cvta_generic_to_shared(&sP[w][0][2 * lane]);
  const unsigned sMa = (unsigned)__cvta_generic_to_shared(&sM[w][0][2 * lane]);
  const unsigned sVa = (unsigned)__cvta_generic_to_shared(&sV[w][0][2 * lane]);
  const T* gP = P0 + xa;
  const T* gM = M0 + xa;
  const double* gV = V0 + xa;
  auto issue = [&](int r, bool chk) {
    if (!chk || r <= rmax) {
      const unsigned so = (unsigned)(r & (kRing - 1)) * 64u;  // slot offset in elements
      const int ro = r * nx;
      const bool mv = step && (!chk || r >= y0);
      if (vec) {  // ina == inb and owna == ownb
        if (ina) {
          cp_async_pair(sPa + so * (unsigned)sizeof(T), gP + ro);
          if (mv && owna) {
            cp_async_pair(sMa + so * (unsigned)sizeof(T), gM + ro);
            cp_async_pair(sVa + so * 8u, gV + ro);
          }
        }
      } else {
        if (ina) cp_async_at(sPa + so * (unsigned)sizeof(T), gP + ro);
        if (inb) cp_async_at(sPa + (so + 1u) * (unsigned)sizeof(T), gP + ro + 1);
        if (mv && owna) {
          cp_async_at(sMa + so * (unsigned)sizeof(T), gM + ro);
          cp_async_at(sVa + so * 8u, gV + ro);
        }
        if (mv && ownb) {
          cp_async_at(sMa + (so + 1u) * (unsigned)sizeof(T), gM + ro + 1);
          cp_async_at(sVa + (so + 1u) * 8u, gV + ro + 1);
        }
      }
    }
    cp_async_commit();
  };
  // level 0, m and v were last written by this kernel one step earlier
#pragma unroll
  for (int k = 0; k < kRing - 1; ++k) issue(nstart + k, true);
  const T cdga = T(-2) - (hwa ? T(0) : T(1)) - (hea ? T(0) : T(1));
  const T cdgb = T(-2) - (hwb ? T(0) : T(1)) - (heb ? T(0) : T(1));
  // level 1 composed (w_1; the coarsest level itself when L == 2) and the
  // column taps into it of the lane's two columns
  const int nyc = L >= 2 ? D.n[1][1] : 1, nxc = L >= 2 ? D.n[1][2] : 1;
  int ja0 = 0, ja1 = 0, jb0 = 0, jb1 = 0;
  T wa0 = T(0), wa1 = T(0), wb0 = T(0), wb1 = T(0);
  if (L >= 2) {
    if (ina) prolong_taps<T>(xa, nxc, ja0, ja1, wa0, wa1);
    if (inb) prolong_taps<T>(xb, nxc, jb0, jb1, wb0, wb1);
  }
  const T* __restrict__ W1 = (L >= 3) ? A.wl + D.off[0][1] : A.p[cur] + D.off[0][1];
  // fine row n lies between rows lo(n) and lo(n) + 1 of w_1
  auto lo_of = [&](int n) { return nyc > 1 ? min(max((n - 1) >> 1, 0), nyc - 2) : 0; };
  const int rb = A.run_ptr[gt], re = A.run_ptr[gt + 1];
  // the cell of the next measurement run (runs sorted by cell)
  auto run_cell = [&](int r) { return r < re ? A.run_cell[r] : 0x7fffffff; };

  pdl_wait();  // w_1 (previous launch) and the step state (previous step's tail)
  pdl_trigger();
  if (lane == 0) {
    StreamCoef<T> c;
    const T dt = (T)D.h[1], dx = (T)D.h[2];
    c.idt = T(1) / dt;
    c.idx1 = T(1) / dx;
    c.idx2 = T(1) / (dx * dx);
    c.nu = (T)D.coef[0];
    c.lam_scale = T(2) * (T)D.w_res_dV;
    c.wd2 = T(2) * (T)D.w_data_n;
    c.gscale = (T)A.gscale;
    c.ac = adam_coef(D, A.st[ii]);
    sC[w] = c;
  }
  __syncwarp();
  const StreamCoef<T>& cf = sC[w];
  const AdamCoef& ac = cf.ac;
  // per column: lambda scale (0 without a residual), 1 for an owned cell
  const T lsa = resa ? cf.lam_scale : T(0), lsb = resb ? cf.lam_scale : T(0);
  const T ooa = owna ? T(1) : T(0), oob = ownb ? T(1) : T(0);

  // per column (a, b): va, vb the rows clo and clo + 1 of w_1 interpolated in
  // x (zero when L == 1); ca, cb the raw taps of row clo + 2, loaded one shift
  // ahead
  int clo = lo_of(nstart);
  T vaa = T(0), vba = T(0), caa = T(0), cba = T(0);  // column a
  T vab = T(0), vbb = T(0), cab = T(0), cbb = T(0);  // column b
  if (L >= 2) {
    const int hi = nyc > 1 ? clo + 1 : 0;
    const T* r0 = W1 + clo * nxc;
    const T* r1 = W1 + hi * nxc;
    vaa = wa0 * r0[ja0] + wa1 * r0[ja1];
    vba = wa0 * r1[ja0] + wa1 * r1[ja1];
    vab = wb0 * r0[jb0] + wb1 * r0[jb1];
    vbb = wb0 * r1[jb0] + wb1 * r1[jb1];
    if (clo + 2 <= nyc - 1) {
      const T* r2 = W1 + (clo + 2) * nxc;
      caa = r2[ja0]; cba = r2[ja1];
      cab = r2[jb0]; cbb = r2[jb1];
    }
  }
  auto shift = [&]() {  // advance to rows clo + 1, clo + 2 of w_1
    vaa = vba;
    vab = vbb;
    vba = wa0 * caa + wa1 * cba;
    vbb = wb0 * cab + wb1 * cbb;
    ++clo;
    if (L >= 2 && clo + 2 <= nyc - 1) {
      const T* r2 = W1 + (clo + 2) * nxc;
      caa = r2[ja0]; cba = r2[ja1];
      cab = r2[jb0]; cbb = r2[jb1];
    }
  };
  // FP32 problems: r^2 per lane in plain FP32 (<= 64 terms), data misfit compensated
  float rh = 0.f, rl = 0.f, dh = 0.f, dl = 0.f;
  double rd = 0.0, dd = 0.0;                     // FP64 problems
  // row n - 1 (pending gradient) of columns a and b
  T lJ0pa = T(0), lJ1pa = T(0), lJ2pa = T(0), datpa = T(0), p0pa = T(0), mpa = T(0);
  T lJ0pb = T(0), lJ1pb = T(0), lJ2pb = T(0), datpb = T(0), p0pb = T(0), mpb = T(0);
  double vpa = 0.0, vpb = 0.0;
  int rr = rb, nc = run_cell(rb);
  T uoa = T(0), uob = T(0);  // u(n-1, a), u(n-1, b)

  // Row n: the field, the residual and the data term of row n; the gradient
  // and the Adam update of row n - 1.  Row y1 (< ny) supplies the residual
  // that reads the last owned row; the pass with n == ny only finishes rows.
  // gen = false: a row of the strip's interior (y0 < n, n + kRing - 1 <=
  // rmax), where every row condition holds and the copies need no check.
  auto row = [&](const int n, const T wlo, const T whi, const bool gen) {
    issue(n + kRing - 1, gen);
    cp_async_wait_group<kRing - 1>();  // this lane's copies of row n have landed
    const bool row_ok = !gen || n < ny;
    const bool own_row = !gen || (n >= y0 && n < y1);
    const bool res_row = !gen || (n >= 1 && n >= y0 && n < ny);
    const bool grad_row = !gen || (n - 1 >= y0 && n - 1 < y1);
    const int sl = n & (kRing - 1);
    // No branches on the lane's columns: slots of columns outside the level
    // (or of rows not copied) hold stale values, which are selected away
    // (level 0) or used only in results that are never stored (m, v).  A
    // column outside the level has u = 0 (its w_1 taps have weight 0).
    const T2 pp = *reinterpret_cast<const T2*>(&sP[w][sl][2 * lane]);
    const T p0a = (row_ok && ina) ? pp.x : T(0), p0b = (row_ok && inb) ? pp.y : T(0);
    const T ua = p0a + (wlo * vaa + whi * vba);
    const T ub = p0b + (wlo * vab + whi * vbb);
    T mna = T(0), mnb = T(0);
    double vna = 0.0, vnb = 0.0;
    if (step) {
      const T2 mm = *reinterpret_cast<const T2*>(&sM[w][sl][2 * lane]);
      const double2 vv = *reinterpret_cast<const double2*>(&sV[w][sl][2 * lane]);
      mna = mm.x; mnb = mm.y;
      vna = vv.x; vnb = vv.y;
    }
    if (comp_only) {
      if (row_ok && own_row) {
        T* uf = A.ufine + D.fine_off[0] + n * nx;
        if (owna) uf[xa] = ua;
        if (ownb) uf[xb] = ub;
      }
      return;
    }
    const T uWa = __shfl_up_sync(kFull, ub, 1);    // u(n, a - 1): column b of lane - 1
    const T uEb = __shfl_down_sync(kFull, ua, 1);  // u(n, b + 1): column a of lane + 1
    T lJ0a, lJ1a, lJ2a, lJ3a, lJ0b, lJ1b, lJ2b, lJ3b;
    {
      const T ra = burgers_cell<T>(ua, uoa, uWa, ub, hwa, hea, cdga, res_row ? lsa : T(0), cf,
                                   lJ0a, lJ1a, lJ2a, lJ3a);
      const T rb = burgers_cell<T>(ub, uob, ua, uEb, hwb, heb, cdgb, res_row ? lsb : T(0), cf,
                                   lJ0b, lJ1b, lJ2b, lJ3b);
      // r^2 of the owned cells of residual rows (x 1) and of the others (x 0)
      const bool rrow = own_row && res_row;
      const T oa = rrow ? ooa : T(0), ob = rrow ? oob : T(0);
      if (sizeof(T) == 4) {
        rh = fmaf((float)oa, (float)(ra * ra), rh);
        rh = fmaf((float)ob, (float)(rb * rb), rh);
      } else {
        rd = fma((double)oa, (double)(ra * ra), rd);
        rd = fma((double)ob, (double)(rb * rb), rd);
      }
    }
    // data term of the measured cells of row n (runs sorted by cell; every
    // run of this strip lies in its owned columns)
    T data = T(0), datb = T(0);
    const int rowbase = n * nx;
    if (nc < rowbase + nx && own_row) {
      for (; rr < re; ++rr) {
        const int off = A.run_cell[rr] - rowbase;
        if (off >= nx) break;
        const bool ha = xa == off;
        if (ha || xb == off) {
          const T u = ha ? ua : ub;
          const int e0 = A.run_beg[rr], e1 = A.run_beg[rr + 1];
          T d = u - A.run_v0[rr];
          T sd = d, sq = d * d;
          for (int k = e0 + 1; k < e1; ++k) {  // repeated measurements of a cell
            d = u - A.meas_val[k];
            sd += d;
            sq += d * d;
          }
          if (sizeof(T) == 4) acc_add(dh, dl, sq);
          else dd += (double)sq;
          if (ha) data = cf.wd2 * sd;
          else datb = cf.wd2 * sd;
        }
      }
      nc = run_cell(rr);
    }
    // gradient and Adam of row n - 1: dL/du(n-1, x) gathers lambda dr/du of
    // the residuals (n-1, x-1), (n-1, x), (n-1, x+1) and (n, x)
    const T fromWa = __shfl_up_sync(kFull, lJ2pb, 1);    // residual (n-1, a-1): lane - 1
    const T fromEb = __shfl_down_sync(kFull, lJ0pa, 1);  // residual (n-1, b+1): lane + 1
    if (adj && grad_row) {
      const T ga = ((lJ1pa + datpa) + lJ0pb + fromWa + lJ3a) * cf.gscale;
      const T gb = ((lJ1pb + datpb) + fromEb + lJ2pa + lJ3b) * cf.gscale;
      const int em = rowbase - nx + xa;
      T pa = p0pa, ma = mpa, pb = p0pb, mb = mpb;
      double va = vpa, vb = vpb;
      if (step) {
        adam_update(pa, ma, va, ga, ac);
        adam_update(pb, mb, vb, gb, ac);
      }
      if (vec) {
        if (owna) {  // == ownb
          *reinterpret_cast<T2*>(G0 + em) = T2{ga, gb};
          if (step) {
            *reinterpret_cast<T2*>(Pn + em) = T2{pa, pb};
            *reinterpret_cast<T2*>(const_cast<T*>(M0) + em) = T2{ma, mb};
            *reinterpret_cast<double2*>(const_cast<double*>(V0) + em) = double2{va, vb};
          }
        }
      } else {
        if (owna) {
          G0[em] = ga;
          if (step) {
            Pn[em] = pa;
            const_cast<T*>(M0)[em] = ma;
            const_cast<double*>(V0)[em] = va;
          }
        }
        if (ownb) {
          G0[em + 1] = gb;
          if (step) {
            Pn[em + 1] = pb;
            const_cast<T*>(M0)[em + 1] = mb;
            const_cast<double*>(V0)[em + 1] = vb;
          }
        }
      }
    }
    lJ0pa = lJ0a; lJ1pa = lJ1a; lJ2pa = lJ2a; datpa = data;
    lJ0pb = lJ0b; lJ1pb = lJ1b; lJ2pb = lJ2b; datpb = datb;
    p0pa = p0a; mpa = mna; vpa = vna;
    p0pb = p0b; mpb = mnb; vpb = vnb;
    uoa = ua; uob = ub;
  };
  // a row at the strip's edges: weights of w_1 rows clo, clo + 1 from its
  // position (3/4, 1/4 inside; 5/4, -1/4 at the level's ends; a copy when
  // w_1 has one row)
  auto edge_row = [&](const int n) {
    T wlo = T(1), whi = T(0);
    if (nyc > 1) {
      wlo = T(1.25) - T(0.5) * (T)(n - 2 * clo);
      whi = T(1) - wlo;
    }
    row(n, wlo, whi, true);
  };
  int n = nstart;
  if (n == 0) edge_row(n++);  // row 0 has no partner row -1
  // rows in pairs (2k + 1, 2k + 2), both between rows k and k + 1 of w_1
  for (; n <= y1; n += 2) {
    const int k = (n - 1) >> 1;
    if (k > clo && k <= nyc - 2) shift();
    const bool inner = n > y0 && n + kRing <= rmax && (L < 2 || k <= nyc - 2);
    if (inner) {
      row(n, T(0.75), T(0.25), false);
      row(n + 1, T(0.25), T(0.75), false);
    } else {
      edge_row(n);
      if (n + 1 <= y1) edge_row(n + 1);
    }
  }
  cp_async_wait_all();  // the ring's trailing (empty or unused) copies
  if (comp_only) return;
  double rs, ds;
  if (sizeof(T) == 4) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a0 = __shfl_xor_sync(kFull, rh, o), a1 = __shfl_xor_sync(kFull, rl, o);
      const float b0 = __shfl_xor_sync(kFull, dh, o), b1 = __shfl_xor_sync(kFull, dl, o);
      ff_add(rh, rl, a0, a1);
      ff_add(dh, dl, b0, b1);
    }
    rs = (double)rh + (double)rl;
    ds = (double)dh + (double)dl;
  } else {
    rs = warp_sum(rd);
    ds = warp_sum(dd);
  }
  if (lane == 0) {
    A.part[(long long)gt * A.npart + 0] = rs;
    A.part[(long long)gt * A.npart + 1] = ds;
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static cudaLaunchConfig_t pdl_cfg(dim3 grid, dim3 block, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <class T>
cudaError_t launch_compose2(const Arena<T>& A, int level, int cur, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  if (level >= 2) {  // every level from 2 up, one block per instance
    if (A.ncsmall == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = pdl_cfg(dim3(A.ncsmall), dim3(kComposeSmallNT), s, at);
    return cudaLaunchKernelEx(&cfg, k_compose2_small<T>, A, cur);
  }
  if (A.ncblk[level] == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = pdl_cfg(dim3(A.ncblk[level]), dim3(kComposeNT), s, at);
  return cudaLaunchKernelEx(&cfg, k_compose2<T>, A, level, cur);
}

template <class T>
cudaError_t launch_fine_stream(const Arena<T>& A, int mode, int cur, cudaStream_t s) {
  if (A.ntiles[0] == 0) return cudaSuccess;
  constexpr int wpb = kStreamNT / 32;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = pdl_cfg(dim3((A.ntiles[0] + wpb - 1) / wpb), dim3(kStreamNT), s, at);
  switch (mode) {
    case MODE_LOSS: return cudaLaunchKernelEx(&cfg, k_fine_stream<T, MODE_LOSS>, A, cur);
    case MODE_GRAD: return cudaLaunchKernelEx(&cfg, k_fine_stream<T, MODE_GRAD>, A, cur);
    case MODE_STEP: return cudaLaunchKernelEx(&cfg, k_fine_stream<T, MODE_STEP>, A, cur);
    default: return cudaLaunchKernelEx(&cfg, k_fine_stream<T, MODE_COMPOSE>, A, cur);
  }
}

template cudaError_t launch_compose2<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_compose2<double>(const Arena<double>&, int, int, cudaStream_t);
template cudaError_t launch_fine_stream<float>(const Arena<float>&, int, int, cudaStream_t);
template cudaError_t launch_fine_stream<double>(const Arena<double>&, int, int, cudaStream_t);

}  // namespace modil
