// C ABI of the mODIL library: problem planning, the device arena, uploads,
// the per-step launch sequence (optionally captured once in a CUDA graph and
// replayed) and read-back.  The declarations and their contracts are in
// include/modil.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "modil.h"
#include "launch.h"
#include "lbfgs.h"
#include "modil_dev.cuh"

using namespace modil;

namespace {

thread_local std::string g_err;

modil_status fail(modil_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

namespace modil {
// Shared with the other translation units of the library (learned warm start).
int set_last_error(int status, const std::string& msg) {
  g_err = msg;
  return status;
}
}  // namespace modil

namespace {

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(MODIL_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct InstPlan {
  int nlev = 1, nfield = 1, nk = 0;
  int n[MODIL_MAXL][3] = {};
  int nt[MODIL_MAXL][3] = {};
  long long lev_size[MODIL_MAXL] = {};
};

// Everything derived from the descriptors before any device memory exists.
struct Plan {
  int n_inst = 0, pde = 0, dtype = 0, ndim = 2, nfield = 1, cfg = 1, max_lev = 1, min_lev = MODIL_MAXL, nk = 0;
  int max_tail = 1;        // level kernels run for levels 1 .. max_tail-1
  TailPlan tail;
  int npart = 2;
  size_t esz = 4;
  std::vector<InstPlan> inst;
  std::vector<DevInst> dev;
  std::vector<int> tile_inst[MODIL_MAXL];
  long long n_param = 0;   // elements of one level arena (all instances, fields, levels)
  long long n_fine = 0;    // elements of the composed-field scratch
  long long n_k = 0;       // conductivity nodes over all instances
  long long n_aux = 0;
  // measurements, grouped into runs of equal (tile, cell)
  std::vector<int> run_ptr, run_cell, run_field, run_beg;
  std::vector<double> meas_val, run_v0;
  // off-grid points: records per tile and runs of corner contributions
  long long n_points = 0;
  std::vector<int> pt_ptr, pt_cell, pt_own, pt_field, pc_ptr, pc_cell, pc_field, pc_beg, pe_rec;
  int pt_nc = 4;           // corner cells per record (2^d)
  std::vector<double> pt_w, pt_val, pe_w;
  size_t pyr_elems = 0;
  bool stream = false;     // warp-streaming fine kernel and composition pass (Burgers)
  bool grid = false;       // Poisson in d = 1, 3 or the node layout: one kernel per step
  std::vector<int> cblk_inst[MODIL_MAXL], cblk_first[MODIL_MAXL], csmall_inst;
  size_t o_cbi[MODIL_MAXL], o_cbf[MODIL_MAXL], o_csm;
  // arena offsets (bytes)
  size_t o_p0, o_p1, o_m, o_v, o_g, o_uf, o_wl, o_kq, o_km, o_kv, o_kg, o_aux, o_part, o_rptr, o_rcell,
      o_rfield, o_rbeg, o_mval, o_rv0, o_inst, o_st, o_cnt, o_q, o_ti[MODIL_MAXL], total;
  size_t o_pptr, o_pcell, o_pw, o_pval, o_pown, o_pdiff, o_cptr, o_ccell, o_cbeg, o_erec, o_ew, o_pfield, o_cfield;
};

int find_cfg(int ty, int tx) {
  for (int c = 0; c < kNumTileCfg; ++c)
    if (kTileCfg[c][0] == ty && kTileCfg[c][1] == tx) return c;
  return -1;
}

modil_status make_plan(const modil_desc* d, int n, Plan& P, bool allow_stream = true) {
  if (!d || n < 1) return fail(MODIL_ERR_ARG, "descs is NULL or n < 1");
  P = Plan();
  P.n_inst = n;
  // Tail kernel: 8 blocks per instance while the batch's clusters fit in one
  // wave (152 SMs x 4 resident tail blocks), otherwise fewer (and the tail
  // takes correspondingly smaller levels, so that its blocks stay small)
  P.tail.cluster = kTailC;
  while (P.tail.cluster > 1 && (long long)n * P.tail.cluster > 152 * 4) P.tail.cluster /= 2;
  P.pde = d[0].pde;
  P.dtype = d[0].dtype;
  P.ndim = d[0].ndim;
  if (P.pde != MODIL_PDE_BURGERS && P.pde != MODIL_PDE_HEAT && P.pde != MODIL_PDE_NS2D &&
      P.pde != MODIL_PDE_NS3D && P.pde != MODIL_PDE_POISSON)
    return fail(MODIL_ERR_UNSUPPORTED, "unknown pde " + std::to_string(P.pde));
  if (P.dtype != MODIL_F32 && P.dtype != MODIL_F64) return fail(MODIL_ERR_ARG, "dtype");
  const bool three = P.pde == MODIL_PDE_NS3D;
  if (P.pde == MODIL_PDE_POISSON) {
    if (P.ndim < 1 || P.ndim > 3) return fail(MODIL_ERR_ARG, "Poisson: ndim 1, 2 or 3");
    if (d[0].layout != MODIL_CELL && d[0].layout != MODIL_NODE) return fail(MODIL_ERR_ARG, "layout");
    P.grid = P.ndim != 2 || d[0].layout == MODIL_NODE;
  } else if (P.ndim != (three ? 3 : 2)) {
    return fail(MODIL_ERR_ARG, three ? "NS3D needs ndim = 3" : "this PDE family is 2-D (ndim = 2)");
  } else if (d[0].layout != MODIL_CELL) {
    return fail(MODIL_ERR_ARG, "only the Poisson family has a node layout");
  }
  const bool grid = P.grid;
  P.esz = P.dtype == MODIL_F64 ? 8 : 4;
  P.nfield = (P.pde == MODIL_PDE_NS2D) ? 3 : (three ? 5 : 1);
  // tile configuration (same for the batch)
  int ty = d[0].tile[0], tx = d[0].tile[1];
  if (three && (ty != 0 || tx != 0)) return fail(MODIL_ERR_ARG, "NS3D takes the library tile (tile = 0)");
  bool any_points = false;
  for (int i = 0; i < n; ++i) any_points |= d[i].n_points > 0;
  if (ty == 0 && tx == 0) {
    ty = (P.pde == MODIL_PDE_NS2D) ? 8 : 16;
    tx = 32;
    // Burgers: the warp-streaming kernel (one warp per strip) when the batch
    // has enough strips to fill the GPU and no off-grid points need the tile
    // kernel; small grids keep the tile kernel's 256 threads per tile
    long long strips = 0;
    for (int i = 0; i < n; ++i) {
      const int sy = d[i].shape[0], sx = d[i].shape[1];
      strips += (long long)((sy + kSR - 1) / kSR) * ((sx + kSW - 1) / kSW);
    }
    if (P.pde == MODIL_PDE_BURGERS && !any_points && allow_stream && strips >= kStreamMinStrips) {
      ty = kSR;
      tx = kSW;
    }
  }
  P.cfg = find_cfg(ty, tx);
  if (P.cfg < 0) return fail(MODIL_ERR_ARG, "unsupported tile shape");
  if (P.cfg == kStreamCfg) {
    if (P.pde != MODIL_PDE_BURGERS) return fail(MODIL_ERR_ARG, "the 32 x 60 strip is the Burgers streaming kernel's");
    if (any_points) return fail(MODIL_ERR_UNSUPPORTED, "off-grid points need a tile kernel shape (not 32 x 60)");
    if (!allow_stream) P.cfg = 0;
  }
  P.stream = (P.cfg == kStreamCfg);
  if (P.pde == MODIL_PDE_NS2D && P.cfg != 0 && P.cfg != 5)
    return fail(MODIL_ERR_ARG, "NS2D tiles are 8x32 or 16x32");
  if (P.pde != MODIL_PDE_NS2D && P.cfg == 5)
    return fail(MODIL_ERR_ARG, "unsupported tile shape");
  const int TY = kTileCfg[P.cfg][0], TX = kTileCfg[P.cfg][1];

  P.inst.resize(n);
  P.dev.resize(n);
  long long off = 0, foff = 0, koff = 0, aoff = 0;
  for (int i = 0; i < n; ++i) {
    const modil_desc& q = d[i];
    if (q.pde != P.pde || q.dtype != P.dtype || q.ndim != P.ndim || q.layout != d[0].layout)
      return fail(MODIL_ERR_ARG, "a batch must share pde, dtype, ndim and layout");
    if (q.k_fixed && q.pde != MODIL_PDE_HEAT)
      return fail(MODIL_ERR_ARG, "k_fixed: only the heat family has conductivity nodes");
    if (!(q.k_scale >= 0.0 && q.k_scale < HUGE_VAL) || (q.k_scale != 0.0 && q.pde != MODIL_PDE_HEAT))
      return fail(MODIL_ERR_ARG, "k_scale: a finite value >= 0, for the heat family only");
    if (q.tile[0] != d[0].tile[0] || q.tile[1] != d[0].tile[1])
      return fail(MODIL_ERR_ARG, "a batch must share the tile shape");
    // 2-D problems: (1, ny, nx); 3-D: (nz, ny, nx); the grid path also 1-D
    // (1, 1, nx); cells per axis (the node layout stores one more per axis)
    const int nd = P.ndim;
    const int nz = (nd == 3) ? q.shape[0] : 1;
    const int ny = (nd == 3) ? q.shape[1] : (nd == 2 ? q.shape[0] : 1);
    const int nx = q.shape[nd - 1];
    const int ex = (grid && q.layout == MODIL_NODE) ? 1 : 0;  // extra entry per real axis
    if (nz < 1 || ny < 1 || nx < 1) return fail(MODIL_ERR_ARG, "shape must be positive");
    if (q.n_levels < 1 || q.n_levels > MODIL_MAXL) return fail(MODIL_ERR_ARG, "n_levels");
    const int L = q.n_levels;
    if ((nd == 3 && (nz % (1 << (L - 1)))) || (nd >= 2 && (ny % (1 << (L - 1)))) || (nx % (1 << (L - 1))))
      return fail(MODIL_ERR_ARG, "every axis must be divisible by 2^(n_levels-1)");
    if ((long long)nz * ny * nx > (1LL << 30)) return fail(MODIL_ERR_ARG, "grid too large");
    if (three) {
      if (!(q.coef[0] > 0)) return fail(MODIL_ERR_ARG, "NS3D needs coef[0] = Re > 0");
      if (!(q.coef[1] >= 0) || !(q.coef[2] >= 0) || !(q.coef[3] >= 0))
        return fail(MODIL_ERR_ARG, "NS3D needs D, lambda and the Rhie-Chow factor >= 0");
    }
    if (P.pde == MODIL_PDE_BURGERS && ny < 2) return fail(MODIL_ERR_ARG, "Burgers needs >= 2 rows");
    if (P.pde == MODIL_PDE_BURGERS && !(q.coef[0] >= 0)) return fail(MODIL_ERR_ARG, "Burgers needs coef[0] = nu >= 0");
    // physical domain: all zero = the family's own
    bool dom = false;
    for (int a = 0; a < 3; ++a) dom |= (q.domain_lo[a] != 0.0 || q.domain_hi[a] != 0.0);
    if (dom) {
      if (P.pde == MODIL_PDE_NS2D || three)
        return fail(MODIL_ERR_UNSUPPORTED, "the cavity and the body take only their own domain");
      if (!(q.domain_hi[0] > q.domain_lo[0]) || !(q.domain_hi[1] > q.domain_lo[1]) ||
          !std::isfinite(q.domain_lo[0]) || !std::isfinite(q.domain_hi[0]) ||
          !std::isfinite(q.domain_lo[1]) || !std::isfinite(q.domain_hi[1]))
        return fail(MODIL_ERR_ARG, "domain_hi must exceed domain_lo (finite) on both axes");
    }
    if (P.pde == MODIL_PDE_NS2D) {
      if (ny != nx) return fail(MODIL_ERR_ARG, "the cavity grid must be square");
      if (!(q.coef[0] > 0)) return fail(MODIL_ERR_ARG, "NS2D needs coef[0] = Re > 0");
      if (!(q.coef[1] >= 0)) return fail(MODIL_ERR_ARG, "NS2D needs coef[1] = tau factor >= 0");
    }
    if (P.stream) {  // composition pass: level 1 in blocks of 4 kComposeNT cells,
                     // levels 2 .. L-2 one block per instance
      if (L >= 3) {
        const long long cells = (long long)(ny >> 1) * (nx >> 1);
        for (long long c = 0; c < cells; c += 4 * kComposeNT) {
          P.cblk_inst[1].push_back(i);
          P.cblk_first[1].push_back((int)c);
        }
      }
      if (L >= 4) P.csmall_inst.push_back(i);
    }
    if (P.pde == MODIL_PDE_POISSON) {
      const long long ent = (long long)(nd == 3 ? nz + ex : 1) * (nd >= 2 ? ny + ex : 1) * (nx + ex);
      if (q.n_aux != ent || !q.aux)
        return fail(MODIL_ERR_ARG, "Poisson needs aux[] with one right-hand side value per fine cell or node");
      if (!ex && ((nd >= 2 && ny < 2) || nx < 2 || (nd == 3 && nz < 2)))
        return fail(MODIL_ERR_ARG, "Poisson (cell layout) needs >= 2 cells per axis");
      if (grid && q.n_points > 0)
        return fail(MODIL_ERR_UNSUPPORTED, "off-grid points: the 2-D cell layout of the Poisson family only");
    }
    if (P.pde == MODIL_PDE_HEAT) {
      if (q.n_aux != nx || !q.aux) return fail(MODIL_ERR_ARG, "heat needs aux[nx] (initial profile)");
      if (q.n_knodes < 2 || q.n_knodes > MODIL_MAXK || !q.knodes)
        return fail(MODIL_ERR_ARG, "heat needs 2..64 conductivity nodes");
    }
    if (q.n_meas < 0 || (q.n_meas > 0 && (!q.meas_cell || !q.meas_value)))
      return fail(MODIL_ERR_ARG, "measurement arrays");
    if (q.n_points < 0 || (q.n_points > 0 && (!q.point_coord || !q.point_value)))
      return fail(MODIL_ERR_ARG, "point arrays");

    if (!(q.adam_lr >= 0) || !(q.adam_beta1 >= 0 && q.adam_beta1 < 1) ||
        !(q.adam_beta2 >= 0 && q.adam_beta2 < 1) || !(q.adam_eps >= 0))
      return fail(MODIL_ERR_ARG, "Adam parameters");
    InstPlan& ip = P.inst[i];
    DevInst& D = P.dev[i];
    std::memset(&D, 0, sizeof(D));
    ip.nlev = L;
    ip.nfield = P.nfield;
    ip.nk = P.pde == MODIL_PDE_HEAT ? q.n_knodes : 0;
    P.nk = std::max(P.nk, ip.nk);
    P.max_lev = std::max(P.max_lev, L);
    P.min_lev = std::min(P.min_lev, L);
    D.nlev = L;
    D.nfield = P.nfield;
    D.nk = ip.nk;
    D.ndim = three ? 3 : 2;
    // first level small enough for the per-instance tail kernel (2-D only: the
    // 3-D levels are all restricted by the level kernel, the tail finalises)
    // (per field: the tail restricts the fields of a level one after another)
    const long long tcap =
        (P.dtype == MODIL_F64 ? kTailCellsF64 : kTailCellsF32) * P.tail.cluster / (kTailC * P.nfield);
    int tail = L;
    if (!three && !grid)
      for (int l = 1; l < L; ++l)
        if ((long long)(ny >> l) * (nx >> l) <= tcap) { tail = l; break; }
    D.tail = tail;
    P.max_tail = std::max(P.max_tail, tail);
    if (!grid) {
      size_t tc = 0;
      for (int l = tail; l < L; ++l) tc += (size_t)(ny >> l) * (nx >> l);
      P.tail.tail_cells = std::max(P.tail.tail_cells, tc);
      if (tail < L)
        P.tail.prev_cells = std::max(P.tail.prev_cells, (size_t)(ny >> (tail - 1)) * (nx >> (tail - 1)));
      int nn[MODIL_MAXL][3] = {};
      for (int l = 0; l < L; ++l) { nn[l][0] = nz >> l; nn[l][1] = ny >> l; nn[l][2] = nx >> l; }
      P.tail.smem_bytes = std::max(P.tail.smem_bytes, tail_instance_bytes(L, tail, nn, P.nfield, P.tail.cluster, (int)P.esz));
    }
    for (int l = 0; l < L; ++l) {
      ip.n[l][0] = three ? nz >> l : (nd == 3 ? (nz >> l) + ex : 1);
      ip.n[l][1] = (nd >= 2) ? (ny >> l) + ex : 1;
      ip.n[l][2] = (nx >> l) + ex;
      int tzl = 1, tyl, txl;
      if (grid) {
        // flat blocks of kGridNT cells of every level
        const long long sz = (long long)ip.n[l][0] * ip.n[l][1] * ip.n[l][2];
        ip.nt[l][0] = ip.nt[l][1] = 1;
        ip.nt[l][2] = (int)((sz + kGridNT - 1) / kGridNT);
        ip.lev_size[l] = sz;
        for (int a = 0; a < 3; ++a) { D.n[l][a] = ip.n[l][a]; D.nt[l][a] = ip.nt[l][a]; }
        D.tile_base[l] = (int)P.tile_inst[l].size();
        if (l == 0) D.ntile0 = ip.nt[l][2];
        for (int t = 0; t < ip.nt[l][2]; ++t) P.tile_inst[l].push_back(i);
        if (l == 0 || l + 1 < L)  // composition of this level (l = 0 writes the composed field)
          for (long long c = 0; c < sz; c += kGridNT) {
            P.cblk_inst[l].push_back(i);
            P.cblk_first[l].push_back((int)c);
          }
        continue;
      }
      if (three) {
        tzl = l == 0 ? k3TZ : k3LZ;
        tyl = l == 0 ? k3TY : k3LY;
        txl = l == 0 ? k3TX : k3LX;
      } else {
        tyl = l == 0 ? TY : kLevTY;
        txl = l == 0 ? TX : kLevTX;
      }
      ip.nt[l][0] = (ip.n[l][0] + tzl - 1) / tzl;
      ip.nt[l][1] = (ip.n[l][1] + tyl - 1) / tyl;
      ip.nt[l][2] = (ip.n[l][2] + txl - 1) / txl;
      ip.lev_size[l] = (long long)ip.n[l][0] * ip.n[l][1] * ip.n[l][2];
      for (int a = 0; a < 3; ++a) { D.n[l][a] = ip.n[l][a]; D.nt[l][a] = ip.nt[l][a]; }
      D.tile_base[l] = (int)P.tile_inst[l].size();
      const int ntl = ip.nt[l][0] * ip.nt[l][1] * ip.nt[l][2];
      if (l == 0) D.ntile0 = ntl;
      if (l == 0 || l < tail)
        for (int t = 0; t < ntl; ++t) P.tile_inst[l].push_back(i);
    }
    for (int f = 0; f < P.nfield; ++f) {
      for (int l = 0; l < L; ++l) {
        D.off[f][l] = off;
        off += ip.lev_size[l];
      }
      D.fine_off[f] = foff;
      foff += ip.lev_size[0];
    }
    D.k_off = koff;
    koff += ip.nk;
    D.aux_off = aoff;
    aoff += (P.pde == MODIL_PDE_HEAT) ? nx : (P.pde == MODIL_PDE_POISSON ? ip.lev_size[0] : 0);
    D.layout = q.layout;
    if (grid) {
      // [0,1]^d; unused leading axes keep spacing 1
      D.h[0] = (nd == 3) ? 1.0 / nz : 1.0;
      D.h[1] = (nd >= 2) ? 1.0 / ny : 1.0;
      D.h[2] = 1.0 / nx;
    } else if (dom) {
      D.h[0] = 1.0; D.h[1] = (q.domain_hi[0] - q.domain_lo[0]) / ny; D.h[2] = (q.domain_hi[1] - q.domain_lo[1]) / nx;
    } else if (P.pde == MODIL_PDE_BURGERS) {
      D.h[0] = 1.0; D.h[1] = 1.0 / ny; D.h[2] = 2.0 / nx;
    } else if (three) {
      D.h[0] = 1.0 / nz; D.h[1] = 1.0 / ny; D.h[2] = 2.0 / nx;
    } else {
      D.h[0] = 1.0; D.h[1] = 1.0 / ny; D.h[2] = 1.0 / nx;
    }
    const double dV = D.h[0] * D.h[1] * D.h[2];
    for (int c = 0; c < 4; ++c) D.coef[c] = q.coef[c];

    D.w_res_dV = q.w_res * dV;
    D.w_data_n = (q.n_meas + q.n_points) > 0 ? q.w_data / (q.n_meas + q.n_points) : 0.0;
    D.w_reg = q.w_reg;
    D.k_fixed = q.k_fixed != 0;
    D.k_scale = q.k_scale > 0.0 ? q.k_scale : 1.0;
    D.lr = q.adam_lr; D.b1 = q.adam_beta1; D.b2 = q.adam_beta2; D.eps = q.adam_eps;
    // pyramid bound of this instance (unclipped worst case, clipped by level size)
    if (three || grid) {
      // composition is level by level (no per-tile pyramid)
    } else {
      const int hu = (P.pde == MODIL_PDE_NS2D) ? 4 : 2;  // halo of the composed field
      long long hy = TY + 2 * hu, hx = TX + 2 * hu, tot = 0;
      for (int l = 1; l < L; ++l) {
        hy = std::min<long long>((hy + 7) / 2, ip.n[l][1]);
        hx = std::min<long long>((hx + 7) / 2, ip.n[l][2]);
        tot += hy * hx;
      }
      P.pyr_elems = std::max<size_t>(P.pyr_elems, (size_t)tot);
    }
  }
  P.n_param = off;
  P.n_fine = foff;
  P.n_k = koff;
  P.n_aux = aoff;
  P.npart = 2 + P.nk;
  P.tail.level_kernels = P.max_tail - 1;
  if (tail_smem_bytes(P.tail, (int)P.esz) > 200 * 1024)  // plus about 23 KB of static shared memory
    return fail(MODIL_ERR_UNSUPPORTED, "coarse levels too large for the tail kernel");

  // measurements -> runs sorted by (global fine tile, cell)
  const int nft = (int)P.tile_inst[0].size();
  struct M { int tile, cell, field; double val; };
  std::vector<M> all;
  for (int i = 0; i < n; ++i) {
    const modil_desc& q = d[i];
    const InstPlan& ip = P.inst[i];
    const int nz = ip.n[0][0], ny = ip.n[0][1], nx = ip.n[0][2];
    const int tz = three ? k3TZ : 1, ty3 = three ? k3TY : TY, tx3 = three ? k3TX : TX;
    for (int k = 0; k < q.n_meas; ++k) {
      const int c = q.meas_cell[k];
      const int f = q.meas_field ? q.meas_field[k] : 0;
      if (c < 0 || (long long)c >= (long long)nz * ny * nx)
        return fail(MODIL_ERR_ARG, "measurement cell out of range");
      if (f < 0 || f >= P.nfield) return fail(MODIL_ERR_ARG, "measurement field out of range");
      if (!std::isfinite(q.meas_value[k])) return fail(MODIL_ERR_ARG, "measurement value not finite");
      const int z = c / (ny * nx), y = (c / nx) % ny, x = c % nx;
      const int t = grid ? P.dev[i].tile_base[0] + c / kGridNT
                         : P.dev[i].tile_base[0] + ((z / tz) * ip.nt[0][1] + (y / ty3)) * ip.nt[0][2] + (x / tx3);
      all.push_back({t, c, f, q.meas_value[k]});
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const M& a, const M& b) {
    if (a.tile != b.tile) return a.tile < b.tile;
    if (a.field != b.field) return a.field < b.field;
    return a.cell < b.cell;
  });
  P.run_ptr.assign(nft + 1, 0);
  for (size_t k = 0; k < all.size(); ++k) {
    const bool start = k == 0 || all[k].tile != all[k - 1].tile || all[k].cell != all[k - 1].cell ||
                       all[k].field != all[k - 1].field;
    if (start) {
      P.run_cell.push_back(all[k].cell);
      P.run_field.push_back(all[k].field);
      P.run_beg.push_back((int)k);
      P.run_v0.push_back(all[k].val);
      P.run_ptr[all[k].tile + 1]++;
    }
    P.meas_val.push_back(all[k].val);
  }
  P.run_beg.push_back((int)all.size());
  for (int t = 0; t < nft; ++t) P.run_ptr[t + 1] += P.run_ptr[t];

  // off-grid points -> records of every tile owning one of a point's 2^d
  // corner cells (the tile of the lower corner counts the misfit), and per
  // tile runs of (record, weight) entries sorted by (field, target cell)
  {
    const int nd = three ? 3 : 2, nc = 1 << nd;
    P.pt_nc = nc;
    struct R { int tile, field; int cell[8]; double w[8]; double val; int own; };
    std::vector<R> recs;
    for (int i = 0; i < n; ++i) {
      const modil_desc& q = d[i];
      if (q.n_points <= 0) continue;
      const InstPlan& ip = P.inst[i];
      const int nn[3] = {ip.n[0][0], ip.n[0][1], ip.n[0][2]};  // (1, ny, nx) in 2-D
      bool dom = false;
      for (int a = 0; a < 3; ++a) dom |= (q.domain_lo[a] != 0.0 || q.domain_hi[a] != 0.0);
      // origin and length of the axes (z,) y, x
      double org[3] = {0.0, 0.0, 0.0}, len[3] = {1.0, 1.0, 1.0};
      if (three) {
        len[2] = 2.0;  // the body: [0,1] x [0,1] x [0,2]
      } else if (dom) {
        org[1] = q.domain_lo[0]; len[1] = q.domain_hi[0] - q.domain_lo[0];
        org[2] = q.domain_lo[1]; len[2] = q.domain_hi[1] - q.domain_lo[1];
      } else if (P.pde == MODIL_PDE_BURGERS) {
        org[2] = -1.0; len[2] = 2.0;
      }
      // position along one axis in units of cell centres, clamped to the
      // outermost centres; lower centre i0 and fraction t towards i0 + 1
      auto axis = [](double pos, double o, double l, int m, int& i0, double& t) {
        double sc = (pos - o) / (l / m) - 0.5;
        sc = std::min(std::max(sc, 0.0), (double)(m - 1));
        if (m == 1) { i0 = 0; t = 0.0; return; }
        i0 = std::min((int)std::floor(sc), m - 2);
        t = sc - i0;
      };
      const int tz = three ? k3TZ : 1, ty = three ? k3TY : TY, tx = three ? k3TX : TX;
      auto tile_of = [&](int z, int y, int x) {
        return P.dev[i].tile_base[0] + ((z / tz) * ip.nt[0][1] + (y / ty)) * ip.nt[0][2] + (x / tx);
      };
      for (int k = 0; k < q.n_points; ++k) {
        double pc[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < nd; ++a) pc[3 - nd + a] = q.point_coord[nd * k + a];
        const double v = q.point_value[k];
        const int f = q.point_field ? q.point_field[k] : 0;
        bool fin = std::isfinite(v);
        for (int a = 0; a < 3; ++a) fin = fin && std::isfinite(pc[a]);
        if (!fin) return fail(MODIL_ERR_ARG, "point coordinate or value not finite");
        if (f < 0 || f >= P.nfield) return fail(MODIL_ERR_ARG, "point field out of range");
        int i0[3];
        double t[3];
        for (int a = 0; a < 3; ++a) {
          if (a < 3 - nd) { i0[a] = 0; t[a] = 0.0; continue; }
          axis(pc[a], org[a], len[a], nn[a], i0[a], t[a]);
        }
        R r;
        r.val = v;
        r.field = f;
        int tiles[8];
        for (int c = 0; c < nc; ++c) {
          // corner c: bit 0 -> x, bit 1 -> y, bit 2 -> z (upper neighbour when set)
          int cc[3];
          double w = 1.0;
          for (int a = 0; a < 3; ++a) {
            const int bit = (a == 2) ? (c & 1) : (a == 1 ? (c >> 1) & 1 : (c >> 2) & 1);
            if (a < 3 - nd) { cc[a] = 0; continue; }
            cc[a] = bit ? std::min(i0[a] + 1, nn[a] - 1) : i0[a];
            w *= bit ? t[a] : 1.0 - t[a];
          }
          r.cell[c] = (cc[0] * nn[1] + cc[1]) * nn[2] + cc[2];
          r.w[c] = w;
          tiles[c] = tile_of(cc[0], cc[1], cc[2]);
        }
        for (int c = 0; c < nc; ++c) {
          bool seen = false;
          for (int e = 0; e < c; ++e) seen |= tiles[e] == tiles[c];
          if (seen) continue;
          r.tile = tiles[c];
          r.own = (tiles[c] == tiles[0]) ? 1 : 0;
          recs.push_back(r);
        }
        P.n_points++;
      }
    }
    if (!recs.empty()) {
      std::stable_sort(recs.begin(), recs.end(), [](const R& a, const R& b) { return a.tile < b.tile; });
      P.pt_ptr.assign(nft + 1, 0);
      struct E { int tile, field, cell, rec; double w; };
      std::vector<E> ents;
      for (size_t j = 0; j < recs.size(); ++j) {
        const R& r = recs[j];
        P.pt_ptr[r.tile + 1]++;
        for (int c = 0; c < nc; ++c) {
          P.pt_cell.push_back(r.cell[c]);
          P.pt_w.push_back(r.w[c]);
        }
        P.pt_val.push_back(r.val);
        P.pt_own.push_back(r.own);
        P.pt_field.push_back(r.field);
      }
      for (int t = 0; t < nft; ++t) P.pt_ptr[t + 1] += P.pt_ptr[t];
      // entries: the corners each record's tile owns
      for (size_t j = 0; j < recs.size(); ++j) {
        const R& r = recs[j];
        const int ii = P.tile_inst[0][r.tile];
        const InstPlan& ip = P.inst[ii];
        const int ny = ip.n[0][1], nx = ip.n[0][2];
        const int tz = three ? k3TZ : 1, ty = three ? k3TY : TY, tx = three ? k3TX : TX;
        for (int c = 0; c < nc; ++c) {
          const int z = r.cell[c] / (ny * nx), y = (r.cell[c] / nx) % ny, x = r.cell[c] % nx;
          const int t = P.dev[ii].tile_base[0] + ((z / tz) * ip.nt[0][1] + (y / ty)) * ip.nt[0][2] + (x / tx);
          if (t == r.tile) ents.push_back({t, r.field, r.cell[c], (int)j, r.w[c]});
        }
      }
      std::stable_sort(ents.begin(), ents.end(), [](const E& a, const E& b) {
        if (a.tile != b.tile) return a.tile < b.tile;
        if (a.field != b.field) return a.field < b.field;
        if (a.cell != b.cell) return a.cell < b.cell;
        return a.rec < b.rec;
      });
      P.pc_ptr.assign(nft + 1, 0);
      for (size_t k = 0; k < ents.size(); ++k) {
        if (k == 0 || ents[k].tile != ents[k - 1].tile || ents[k].cell != ents[k - 1].cell ||
            ents[k].field != ents[k - 1].field) {
          P.pc_cell.push_back(ents[k].cell);
          P.pc_field.push_back(ents[k].field);
          P.pc_beg.push_back((int)k);
          P.pc_ptr[ents[k].tile + 1]++;
        }
        P.pe_rec.push_back(ents[k].rec);
        P.pe_w.push_back(ents[k].w);
      }
      P.pc_beg.push_back((int)ents.size());
      for (int t = 0; t < nft; ++t) P.pc_ptr[t + 1] += P.pc_ptr[t];
    }
  }

  // arena layout
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t r = o; o = align256(o + std::max<size_t>(bytes, 1)); return r; };
  P.o_p0 = take(P.esz * P.n_param);
  P.o_p1 = take(P.esz * P.n_param);
  P.o_m = take(P.esz * P.n_param);
  P.o_v = take(8 * P.n_param);
  P.o_g = take(P.esz * P.n_param);
  P.o_uf = take(P.esz * P.n_fine);
  P.o_wl = take((P.pde == MODIL_PDE_NS3D || P.stream || P.grid) ? P.esz * P.n_param : 0);
  P.o_kq = take(P.esz * P.n_k);
  P.o_km = take(P.esz * P.n_k);
  P.o_kv = take(8 * P.n_k);
  P.o_kg = take(P.esz * P.n_k);
  P.o_aux = take(P.esz * P.n_aux);
  P.o_part = take(8 * (size_t)nft * P.npart);
  P.o_rptr = take(4 * P.run_ptr.size());
  P.o_rcell = take(4 * P.run_cell.size());
  P.o_rfield = take(4 * P.run_field.size());
  P.o_rbeg = take(4 * P.run_beg.size());
  P.o_mval = take(P.esz * P.meas_val.size());
  P.o_rv0 = take(P.esz * P.run_v0.size());
  P.o_pptr = take(4 * P.pt_ptr.size());
  P.o_pcell = take(4 * P.pt_cell.size());
  P.o_pw = take(P.esz * P.pt_w.size());
  P.o_pval = take(P.esz * P.pt_val.size());
  P.o_pown = take(4 * P.pt_own.size());
  P.o_pfield = take(4 * P.pt_field.size());
  P.o_cfield = take(4 * P.pc_field.size());
  P.o_pdiff = take(P.esz * P.pt_val.size());
  P.o_cptr = take(4 * P.pc_ptr.size());
  P.o_ccell = take(4 * P.pc_cell.size());
  P.o_cbeg = take(4 * P.pc_beg.size());
  P.o_erec = take(4 * P.pe_rec.size());
  P.o_ew = take(P.esz * P.pe_w.size());
  P.o_inst = take(sizeof(DevInst) * n);
  P.o_st = take(sizeof(InstState) * n);
  P.o_cnt = take(sizeof(int) * n);
  P.o_q = take(2 * sizeof(int));
  for (int l = 0; l < MODIL_MAXL; ++l) P.o_ti[l] = take(4 * P.tile_inst[l].size());
  for (int l = 0; l < MODIL_MAXL; ++l) {
    P.o_cbi[l] = take(4 * P.cblk_inst[l].size());
    P.o_cbf[l] = take(4 * P.cblk_first[l].size());
  }
  P.o_csm = take(4 * P.csmall_inst.size());
  P.total = o;
  return MODIL_OK;
}

}  // namespace

struct modil_problem {
  Plan plan;
  void* arena = nullptr;
  bool own_arena = false;
  cudaStream_t stream = nullptr;
  Arena<float> A32{};
  Arena<double> A64{};
  long long steps = 0;  // host mirror of the device step counter (all instances)
  cudaGraph_t graph[2] = {nullptr, nullptr};       // one step reading p[0] / p[1]
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  bool use_graph = true;
  Ns3Maps maps;  // 3-D single instance: TMA maps of the composed fields
};

namespace {

template <class T>
void fill_arena(modil_problem* p, Arena<T>& A) {
  const Plan& P = p->plan;
  char* b = static_cast<char*>(p->arena);
  A.p[0] = reinterpret_cast<T*>(b + P.o_p0);
  A.p[1] = reinterpret_cast<T*>(b + P.o_p1);
  A.m = reinterpret_cast<T*>(b + P.o_m);
  A.v = reinterpret_cast<double*>(b + P.o_v);
  A.g = reinterpret_cast<T*>(b + P.o_g);
  A.ufine = reinterpret_cast<T*>(b + P.o_uf);
  A.wl = reinterpret_cast<T*>(b + P.o_wl);
  A.kq = reinterpret_cast<T*>(b + P.o_kq);
  A.km = reinterpret_cast<T*>(b + P.o_km);
  A.kv = reinterpret_cast<double*>(b + P.o_kv);
  A.kg = reinterpret_cast<T*>(b + P.o_kg);
  A.aux = reinterpret_cast<const T*>(b + P.o_aux);
  A.part = reinterpret_cast<double*>(b + P.o_part);
  A.run_ptr = reinterpret_cast<const int*>(b + P.o_rptr);
  A.run_cell = reinterpret_cast<const int*>(b + P.o_rcell);
  A.run_field = reinterpret_cast<const int*>(b + P.o_rfield);
  A.run_beg = reinterpret_cast<const int*>(b + P.o_rbeg);
  A.meas_val = reinterpret_cast<const T*>(b + P.o_mval);
  A.run_v0 = reinterpret_cast<const T*>(b + P.o_rv0);
  const bool pts = !P.pt_ptr.empty();
  A.pt_ptr = pts ? reinterpret_cast<const int*>(b + P.o_pptr) : nullptr;
  A.pt_cell = reinterpret_cast<const int*>(b + P.o_pcell);
  A.pt_w = reinterpret_cast<const T*>(b + P.o_pw);
  A.pt_val = reinterpret_cast<const T*>(b + P.o_pval);
  A.pt_own = reinterpret_cast<const int*>(b + P.o_pown);
  A.pt_field = reinterpret_cast<const int*>(b + P.o_pfield);
  A.pc_field = reinterpret_cast<const int*>(b + P.o_cfield);
  A.pt_diff = reinterpret_cast<T*>(b + P.o_pdiff);
  A.pc_ptr = pts ? reinterpret_cast<const int*>(b + P.o_cptr) : nullptr;
  A.pc_cell = reinterpret_cast<const int*>(b + P.o_ccell);
  A.pc_beg = reinterpret_cast<const int*>(b + P.o_cbeg);
  A.pe_rec = reinterpret_cast<const int*>(b + P.o_erec);
  A.pe_w = reinterpret_cast<const T*>(b + P.o_ew);
  A.inst = reinterpret_cast<const DevInst*>(b + P.o_inst);
  A.st = reinterpret_cast<InstState*>(b + P.o_st);
  A.counter = reinterpret_cast<int*>(b + P.o_cnt);
  A.queue = reinterpret_cast<int*>(b + P.o_q);
  A.persistent = 0;
  for (int l = 0; l < MODIL_MAXL; ++l) {
    A.tile_inst[l] = reinterpret_cast<const int*>(b + P.o_ti[l]);
    A.ntiles[l] = (int)P.tile_inst[l].size();
    A.cblk_inst[l] = reinterpret_cast<const int*>(b + P.o_cbi[l]);
    A.cblk_first[l] = reinterpret_cast<const int*>(b + P.o_cbf[l]);
    A.ncblk[l] = (int)P.cblk_inst[l].size();
  }
  A.csmall_inst = reinterpret_cast<const int*>(b + P.o_csm);
  A.ncsmall = (int)P.csmall_inst.size();
  A.npart = P.npart;
  A.n_inst = P.n_inst;
  A.gscale = 1.0f;
  A.inst0 = P.dev[0];
}

template <class T>
std::vector<T> convert(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

modil_status upload(modil_problem* p, size_t off, const void* src, size_t bytes) {
  if (bytes == 0) return MODIL_OK;
  CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(p->arena) + off, src, bytes, cudaMemcpyHostToDevice,
                           p->stream));
  return MODIL_OK;
}

// One pass of the method: the fused fine-tile kernel (which also finalises the
// loss), the restriction/Adam kernel of each larger coarse level, and the
// per-instance tail kernel for the small levels.  cur selects the parameter
// buffer the pass reads.  With ev != NULL an event is recorded after every
// launch (ev[0] before the first).
template <class T>
modil_status run_pass_t(modil_problem* p, Arena<T>& A, int mode, int cur, cudaEvent_t* ev,
                        int* nev) {
  const Plan& P = p->plan;
  int k = 0;
  if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
  if (P.grid) {
    // compose w_{L-2} .. w_0 (level 0: the composed field), the fine kernel,
    // the restriction chain, the loss terms
    for (int l = std::max(P.max_lev - 2, 0); l >= 0; --l) {
      CUDA_TRY(launch_gcompose<T>(A, l, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
    if (mode != MODE_COMPOSE) {
      CUDA_TRY(launch_gresid<T>(A, mode, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
      if (mode == MODE_GRAD || mode == MODE_STEP)
        for (int l = 1; l < P.max_lev; ++l) {
          CUDA_TRY(launch_grestrict<T>(A, l, mode, cur, p->stream));
          if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
        }
      CUDA_TRY(launch_gfinal<T>(A, mode, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
    if (nev) *nev = k;
    return MODIL_OK;
  }
  if (P.pde == MODIL_PDE_NS3D) {
    // compose level by level (coarse to fine), then the fused residual pass
    // (level -1: copy of single-level instances, launched only if the batch has one)
    const int lo = P.min_lev == 1 ? -1 : 0;
    for (int l = P.max_lev - 2; l >= lo; --l) {
      CUDA_TRY(launch_prolong3<T>(A, l, P.nfield, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
    if (mode == MODE_COMPOSE) {
      if (nev) *nev = k;
      return MODIL_OK;
    }
    // the TMA maps address the arena's composed-field buffer (a single instance)
    const bool own_uf = A.ufine == reinterpret_cast<T*>(static_cast<char*>(p->arena) + P.o_uf);
    CUDA_TRY(launch_resid3<T>(A, mode, cur, own_uf ? &p->maps : nullptr, p->stream));
  } else if (P.pde == MODIL_PDE_NS2D) {
    CUDA_TRY(launch_fine_ns2d<T>(A, P.cfg, mode, cur, P.pyr_elems, p->stream));
  } else if (P.stream) {
    // compose w_{L-2} .. w_2 (one launch), w_1, then the streaming fine kernel
    if (P.max_lev >= 4) {
      CUDA_TRY(launch_compose2<T>(A, 2, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
    if (P.max_lev >= 3) {
      CUDA_TRY(launch_compose2<T>(A, 1, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
    CUDA_TRY(launch_fine_stream<T>(A, mode, cur, p->stream));
  } else {
    CUDA_TRY(launch_fine_st<T>(A, P.pde, P.cfg, mode, cur, P.pyr_elems, p->stream));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
  if (mode == MODE_GRAD || mode == MODE_STEP)
    for (int l = 1; l < P.max_tail; ++l) {
      if (P.pde == MODIL_PDE_NS3D)
        CUDA_TRY(launch_level3<T>(A, l, P.nfield, mode, cur, p->stream));
      else
        CUDA_TRY(launch_level<T>(A, P.nfield, l, mode, cur, p->stream));
      if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
    }
  if (mode != MODE_COMPOSE) {
    CUDA_TRY(launch_tail<T>(A, mode, cur, P.tail, p->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[k++], p->stream));
  }
  if (nev) *nev = k;
  return MODIL_OK;
}

modil_status run_pass(modil_problem* p, int mode, cudaEvent_t* ev = nullptr, int* nev = nullptr) {
  const int cur = (int)(p->steps & 1);
  return p->plan.dtype == MODIL_F64 ? run_pass_t<double>(p, p->A64, mode, cur, ev, nev)
                                    : run_pass_t<float>(p, p->A32, mode, cur, ev, nev);
}

int kernels_per_step(const Plan& P) {
  const int compose3 = (P.max_lev - 1) + (P.min_lev == 1 ? 1 : 0);
  const int compose2 = P.stream ? (P.max_lev >= 4 ? 1 : 0) + (P.max_lev >= 3 ? 1 : 0) : 0;
  if (P.grid) return std::max(P.max_lev - 1, 1) + 1 + (P.max_lev - 1) + 1;
  return (P.pde == MODIL_PDE_NS3D ? compose3 + 1 : 1 + compose2) + (P.max_tail - 1) + 1;
}

modil_status read_terms(modil_problem* p, double* terms) {
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  const Plan& P = p->plan;
  std::vector<InstState> st(P.n_inst);
  CUDA_TRY(cudaMemcpy(st.data(), static_cast<char*>(p->arena) + P.o_st,
                      sizeof(InstState) * P.n_inst, cudaMemcpyDeviceToHost));
  bool bad = false, late = false;
  for (int i = 0; i < P.n_inst; ++i) {
    if (terms)
      for (int j = 0; j < MODIL_NTERMS; ++j) terms[i * MODIL_NTERMS + j] = st[i].terms[j];
    bad |= (st[i].nonfinite & kStatusNonfinite) != 0;
    late |= (st[i].nonfinite & kStatusTimeout) != 0;
  }
  if (late) {
    // reported once: clear the timeout bits, keep the non-finite latch
    for (int i = 0; i < P.n_inst; ++i) {
      if (!(st[i].nonfinite & kStatusTimeout)) continue;
      const int v = st[i].nonfinite & ~kStatusTimeout;
      CUDA_TRY(cudaMemcpy(static_cast<char*>(p->arena) + P.o_st + sizeof(InstState) * i +
                              offsetof(InstState, nonfinite),
                          &v, sizeof(int), cudaMemcpyHostToDevice));
    }
    return fail(MODIL_ERR_TIMEOUT, "a bounded wait inside a kernel ran out; the pass skipped the "
                "affected tiles, so its loss, gradient and step are incomplete");
  }
  if (bad) return fail(MODIL_ERR_NONFINITE, "loss became non-finite");
  return MODIL_OK;
}

modil_status check_level(const modil_problem* p, int inst, int field, int level, size_t bytes,
                         long long* off, long long* count) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  const Plan& P = p->plan;
  if (inst < 0 || inst >= P.n_inst) return fail(MODIL_ERR_ARG, "instance out of range");
  if (field < 0 || field >= P.nfield) return fail(MODIL_ERR_ARG, "field out of range");
  if (level < 0 || level >= P.inst[inst].nlev) return fail(MODIL_ERR_ARG, "level out of range");
  const long long cnt = P.inst[inst].lev_size[level];
  if (bytes != (size_t)cnt * P.esz) return fail(MODIL_ERR_ARG, "byte count does not match the level");
  *off = P.dev[inst].off[field][level];
  *count = cnt;
  return MODIL_OK;
}

modil_status copy_dev(modil_problem* p, void* dst, const void* src, size_t bytes, cudaMemcpyKind k) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, k, p->stream));
  if (k == cudaMemcpyDeviceToHost || k == cudaMemcpyHostToDevice) CUDA_TRY(cudaStreamSynchronize(p->stream));
  return MODIL_OK;
}

void drop_graph(modil_problem* p) {
  for (int c = 0; c < 2; ++c) {
    if (p->gexec[c]) cudaGraphExecDestroy(p->gexec[c]);
    if (p->graph[c]) cudaGraphDestroy(p->graph[c]);
    p->gexec[c] = nullptr;
    p->graph[c] = nullptr;
  }
}

}  // namespace

namespace {
// A pass over caller-owned levels (and gradient buffer), scaled gradient.
template <class T>
modil_status external_pass(modil_problem* p, Arena<T> A, const void* levels, void* grads,
                                  double scale, int mode) {
  A.p[0] = const_cast<T*>(static_cast<const T*>(levels));
  A.p[1] = nullptr;
  if (grads) A.g = static_cast<T*>(grads);
  A.gscale = (float)scale;
  return run_pass_t<T>(p, A, mode, 0, nullptr, nullptr);
}

}  // namespace

namespace {

// Checkpoint file: a fixed header, then the optimiser state in arena order.
struct CkptHeader {
  char magic[8];           // "MODILCK1"
  int32_t version, n_inst, pde, dtype, nfield, pad;
  int64_t n_param, n_k, steps;
  uint64_t shape_hash;     // FNV-1a over every instance's level shapes
};

uint64_t shape_hash(const Plan& P) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](long long v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (uint64_t)((v >> (8 * k)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  for (const DevInst& D : P.dev) {
    mix(D.nlev);
    for (int l = 0; l < D.nlev; ++l)
      for (int a = 0; a < 3; ++a) mix(D.n[l][a]);
  }
  return h;
}

// The regions a checkpoint holds: current levels, Adam moments, conductivity
// nodes and their moments, per-instance step state.
struct CkptRegion { size_t off, bytes; };

std::vector<CkptRegion> ckpt_regions(const modil_problem* p) {
  const Plan& P = p->plan;
  const size_t cur = (p->steps & 1) ? P.o_p1 : P.o_p0;
  return {{cur, P.esz * P.n_param},      {P.o_m, P.esz * P.n_param},
          {P.o_v, 8 * (size_t)P.n_param}, {P.o_kq, P.esz * P.n_k},
          {P.o_km, P.esz * P.n_k},        {P.o_kv, 8 * (size_t)P.n_k},
          {P.o_st, sizeof(InstState) * P.n_inst}};
}

}  // namespace

extern "C" {

modil_status modil_arena_bytes(const modil_desc* descs, int n, size_t* bytes) {
  if (!bytes) return fail(MODIL_ERR_ARG, "bytes is NULL");
  Plan P;
  modil_status s = make_plan(descs, n, P);
  if (s != MODIL_OK) return s;
  *bytes = P.total;
  return MODIL_OK;
}

modil_status modil_create(const modil_desc* descs, int n, void* arena, size_t arena_bytes,
                          void* stream, modil_problem** out) {
  if (!out) return fail(MODIL_ERR_ARG, "out is NULL");
  *out = nullptr;
  modil_problem* p = new (std::nothrow) modil_problem();
  if (!p) return fail(MODIL_ERR_OOM, "host allocation");
  modil_status s = make_plan(descs, n, p->plan);
  if (s != MODIL_OK) { delete p; return s; }
  Plan& P = p->plan;
  p->stream = static_cast<cudaStream_t>(stream);
  p->use_graph = (stream != nullptr) && !std::getenv("MODIL_NO_GRAPH");
  if (arena) {
    if (arena_bytes < P.total) { delete p; return fail(MODIL_ERR_ARG, "arena too small"); }
    if (reinterpret_cast<uintptr_t>(arena) & 255) { delete p; return fail(MODIL_ERR_ARG, "arena not 256-byte aligned"); }
    p->arena = arena;
  } else {
    cudaError_t e = cudaMalloc(&p->arena, P.total);
    if (e != cudaSuccess) { delete p; return fail(MODIL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
    p->own_arena = true;
  }
  fill_arena(p, p->A32);
  fill_arena(p, p->A64);
  auto bail = [&](modil_status st) { modil_destroy(p); return st; };
  cudaError_t e = cudaMemsetAsync(p->arena, 0, P.total, p->stream);
  if (e != cudaSuccess) return bail(fail(MODIL_ERR_CUDA, cudaGetErrorString(e)));
  // host-side staging of the read-only tables
  std::vector<double> kq, aux;
  for (int i = 0; i < n; ++i) {
    if (P.inst[i].nk) kq.insert(kq.end(), descs[i].knodes, descs[i].knodes + P.inst[i].nk);
    if (P.pde == MODIL_PDE_HEAT || P.pde == MODIL_PDE_POISSON)
      aux.insert(aux.end(), descs[i].aux, descs[i].aux + descs[i].n_aux);
  }
  modil_status st = MODIL_OK;
  if (P.dtype == MODIL_F64) {
    st = upload(p, P.o_kq, kq.data(), 8 * kq.size());
    if (st == MODIL_OK) st = upload(p, P.o_aux, aux.data(), 8 * aux.size());
    if (st == MODIL_OK) st = upload(p, P.o_mval, P.meas_val.data(), 8 * P.meas_val.size());
    if (st == MODIL_OK) st = upload(p, P.o_rv0, P.run_v0.data(), 8 * P.run_v0.size());
    if (st == MODIL_OK) st = upload(p, P.o_pw, P.pt_w.data(), 8 * P.pt_w.size());
    if (st == MODIL_OK) st = upload(p, P.o_pval, P.pt_val.data(), 8 * P.pt_val.size());
    if (st == MODIL_OK) st = upload(p, P.o_ew, P.pe_w.data(), 8 * P.pe_w.size());
  } else {
    auto kq32 = convert<float>(kq), aux32 = convert<float>(aux), mv32 = convert<float>(P.meas_val);
    auto rv32 = convert<float>(P.run_v0);
    st = upload(p, P.o_kq, kq32.data(), 4 * kq32.size());
    if (st == MODIL_OK) st = upload(p, P.o_aux, aux32.data(), 4 * aux32.size());
    if (st == MODIL_OK) st = upload(p, P.o_mval, mv32.data(), 4 * mv32.size());
    if (st == MODIL_OK) st = upload(p, P.o_rv0, rv32.data(), 4 * rv32.size());
    auto pw32 = convert<float>(P.pt_w), pv32 = convert<float>(P.pt_val), ew32 = convert<float>(P.pe_w);
    if (st == MODIL_OK) st = upload(p, P.o_pw, pw32.data(), 4 * pw32.size());
    if (st == MODIL_OK) st = upload(p, P.o_pval, pv32.data(), 4 * pv32.size());
    if (st == MODIL_OK) st = upload(p, P.o_ew, ew32.data(), 4 * ew32.size());
    if (st == MODIL_OK) {
      e = cudaStreamSynchronize(p->stream);
      if (e != cudaSuccess) st = fail(MODIL_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (st == MODIL_OK) st = upload(p, P.o_rptr, P.run_ptr.data(), 4 * P.run_ptr.size());
  if (st == MODIL_OK) st = upload(p, P.o_pptr, P.pt_ptr.data(), 4 * P.pt_ptr.size());
  if (st == MODIL_OK) st = upload(p, P.o_pcell, P.pt_cell.data(), 4 * P.pt_cell.size());
  if (st == MODIL_OK) st = upload(p, P.o_pown, P.pt_own.data(), 4 * P.pt_own.size());
  if (st == MODIL_OK) st = upload(p, P.o_pfield, P.pt_field.data(), 4 * P.pt_field.size());
  if (st == MODIL_OK) st = upload(p, P.o_cfield, P.pc_field.data(), 4 * P.pc_field.size());
  if (st == MODIL_OK) st = upload(p, P.o_cptr, P.pc_ptr.data(), 4 * P.pc_ptr.size());
  if (st == MODIL_OK) st = upload(p, P.o_ccell, P.pc_cell.data(), 4 * P.pc_cell.size());
  if (st == MODIL_OK) st = upload(p, P.o_cbeg, P.pc_beg.data(), 4 * P.pc_beg.size());
  if (st == MODIL_OK) st = upload(p, P.o_erec, P.pe_rec.data(), 4 * P.pe_rec.size());
  if (st == MODIL_OK) st = upload(p, P.o_rcell, P.run_cell.data(), 4 * P.run_cell.size());
  if (st == MODIL_OK) st = upload(p, P.o_rfield, P.run_field.data(), 4 * P.run_field.size());
  if (st == MODIL_OK) st = upload(p, P.o_rbeg, P.run_beg.data(), 4 * P.run_beg.size());
  if (st == MODIL_OK) st = upload(p, P.o_inst, P.dev.data(), sizeof(DevInst) * n);
  for (int l = 0; l < MODIL_MAXL && st == MODIL_OK; ++l)
    st = upload(p, P.o_ti[l], P.tile_inst[l].data(), 4 * P.tile_inst[l].size());
  for (int l = 0; l < MODIL_MAXL && st == MODIL_OK; ++l) {
    st = upload(p, P.o_cbi[l], P.cblk_inst[l].data(), 4 * P.cblk_inst[l].size());
    if (st == MODIL_OK) st = upload(p, P.o_cbf[l], P.cblk_first[l].data(), 4 * P.cblk_first[l].size());
  }
  if (st == MODIL_OK) st = upload(p, P.o_csm, P.csmall_inst.data(), 4 * P.csmall_inst.size());
  if (st != MODIL_OK) return bail(st);
  e = P.dtype == MODIL_F64 ? launch_reset<double>(p->A64, p->stream) : launch_reset<float>(p->A32, p->stream);
  if (e != cudaSuccess) return bail(fail(MODIL_ERR_CUDA, cudaGetErrorString(e)));
  if (P.pde == MODIL_PDE_NS3D)
    e = P.dtype == MODIL_F64 ? prepare_ns3d<double>(P.pyr_elems) : prepare_ns3d<float>(P.pyr_elems);
  else if (P.pde == MODIL_PDE_NS2D)
    e = P.dtype == MODIL_F64 ? prepare_fine_ns2d<double>(P.cfg, P.pyr_elems)
                             : prepare_fine_ns2d<float>(P.cfg, P.pyr_elems);
  else if (!P.stream && !P.grid)
    e = P.dtype == MODIL_F64 ? prepare_fine_st<double>(P.pde, P.cfg, P.pyr_elems)
                             : prepare_fine_st<float>(P.pde, P.cfg, P.pyr_elems);
  if (e == cudaSuccess)
    e = P.dtype == MODIL_F64 ? prepare_tail<double>(P.tail) : prepare_tail<float>(P.tail);
  if (e != cudaSuccess) return bail(fail(MODIL_ERR_CUDA, std::string("kernel setup: ") + cudaGetErrorString(e)));
  if (P.pde == MODIL_PDE_NS3D && P.n_inst == 1) {
    const InstPlan& ip = P.inst[0];
    if (make_ns3_maps(&p->maps, static_cast<char*>(p->arena) + P.o_uf, ip.n[0][0], ip.n[0][1], ip.n[0][2],
                      (int)P.esz) < 0)
      p->maps.ok = false;  // staged with cp.async instead
  }
  e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return bail(fail(MODIL_ERR_CUDA, cudaGetErrorString(e)));
  *out = p;
  return MODIL_OK;
}

void modil_destroy(modil_problem* p) {
  if (!p) return;
  drop_graph(p);
  cudaStreamSynchronize(p->stream);  // no kernel may still use the arena
  if (p->own_arena && p->arena) cudaFree(p->arena);
  delete p;
}

modil_status modil_set_stream(modil_problem* p, void* stream) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  drop_graph(p);
  p->stream = static_cast<cudaStream_t>(stream);
  p->use_graph = (stream != nullptr) && !std::getenv("MODIL_NO_GRAPH");
  return MODIL_OK;
}

modil_status modil_level_shape(const modil_problem* p, int instance, int level, int shape[3]) {
  if (!p || !shape) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  if (instance < 0 || instance >= P.n_inst) return fail(MODIL_ERR_ARG, "instance out of range");
  if (level < 0 || level >= P.inst[instance].nlev) return fail(MODIL_ERR_ARG, "level out of range");
  if (P.ndim == 3) {
    for (int a = 0; a < 3; ++a) shape[a] = P.inst[instance].n[level][a];
  } else if (P.ndim == 1) {
    shape[0] = P.inst[instance].n[level][2];
    shape[1] = 0;
    shape[2] = 0;
  } else {
    shape[0] = P.inst[instance].n[level][1];
    shape[1] = P.inst[instance].n[level][2];
    shape[2] = 0;
  }
  return MODIL_OK;
}

modil_status modil_write_level(modil_problem* p, int instance, int field, int level,
                               const void* src, size_t bytes, int src_on_device) {
  long long off, cnt;
  modil_status s = check_level(p, instance, field, level, bytes, &off, &cnt);
  if (s != MODIL_OK) return s;
  if (!src) return fail(MODIL_ERR_ARG, "src is NULL");
  const int cur = (int)(p->steps & 1);
  char* dst = static_cast<char*>(p->arena) + (cur ? p->plan.o_p1 : p->plan.o_p0) + off * p->plan.esz;
  return copy_dev(p, dst, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
}

static modil_status read_arr(modil_problem* p, size_t base, int instance, int field, int level,
                             void* dst, size_t bytes, int dst_on_device) {
  long long off, cnt;
  modil_status s = check_level(p, instance, field, level, bytes, &off, &cnt);
  if (s != MODIL_OK) return s;
  if (!dst) return fail(MODIL_ERR_ARG, "dst is NULL");
  const char* src = static_cast<const char*>(p->arena) + base + off * p->plan.esz;
  return copy_dev(p, dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
}

modil_status modil_read_level(modil_problem* p, int instance, int field, int level, void* dst,
                              size_t bytes, int dst_on_device) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  const int cur = (int)(p->steps & 1);
  return read_arr(p, cur ? p->plan.o_p1 : p->plan.o_p0, instance, field, level, dst, bytes, dst_on_device);
}

modil_status modil_read_grad(modil_problem* p, int instance, int field, int level, void* dst,
                             size_t bytes, int dst_on_device) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  return read_arr(p, p->plan.o_g, instance, field, level, dst, bytes, dst_on_device);
}

modil_status modil_read_field(modil_problem* p, int instance, int field, void* dst, size_t bytes,
                              int dst_on_device) {
  long long off, cnt;
  modil_status s = check_level(p, instance, field, 0, bytes, &off, &cnt);
  if (s != MODIL_OK) return s;
  if (!dst) return fail(MODIL_ERR_ARG, "dst is NULL");
  s = run_pass(p, MODE_COMPOSE);
  if (s != MODIL_OK) return s;
  const char* src = static_cast<const char*>(p->arena) + p->plan.o_uf +
                    p->plan.dev[instance].fine_off[field] * p->plan.esz;
  return copy_dev(p, dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
}

static modil_status knode_io(modil_problem* p, int instance, double* q, int n, size_t base, bool write) {
  if (!p || !q) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  if (instance < 0 || instance >= P.n_inst) return fail(MODIL_ERR_ARG, "instance out of range");
  if (n != P.inst[instance].nk || n == 0) return fail(MODIL_ERR_ARG, "node count does not match");
  char* dev = static_cast<char*>(p->arena) + base + P.dev[instance].k_off * P.esz;
  if (P.dtype == MODIL_F64) {
    return copy_dev(p, write ? (void*)dev : (void*)q, write ? (const void*)q : (const void*)dev, 8 * n,
                    write ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  }
  std::vector<float> tmp(n);
  if (write) {
    for (int j = 0; j < n; ++j) tmp[j] = (float)q[j];
    return copy_dev(p, dev, tmp.data(), 4 * n, cudaMemcpyHostToDevice);
  }
  modil_status s = copy_dev(p, tmp.data(), dev, 4 * n, cudaMemcpyDeviceToHost);
  for (int j = 0; j < n; ++j) q[j] = tmp[j];
  return s;
}

modil_status modil_write_knodes(modil_problem* p, int instance, const double* q, int n) {
  return knode_io(p, instance, const_cast<double*>(q), n, p ? p->plan.o_kq : 0, true);
}
modil_status modil_read_knodes(modil_problem* p, int instance, double* q, int n) {
  return knode_io(p, instance, q, n, p ? p->plan.o_kq : 0, false);
}
modil_status modil_read_kgrad(modil_problem* p, int instance, double* gq, int n) {
  return knode_io(p, instance, gq, n, p ? p->plan.o_kg : 0, false);
}

modil_status modil_eval_loss(modil_problem* p, double* terms) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  modil_status s = run_pass(p, MODE_LOSS);
  if (s != MODIL_OK) return s;
  return terms ? read_terms(p, terms) : MODIL_OK;
}

modil_status modil_eval_grad(modil_problem* p, double* terms) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  modil_status s = run_pass(p, MODE_GRAD);
  if (s != MODIL_OK) return s;
  return terms ? read_terms(p, terms) : MODIL_OK;
}

modil_status modil_step(modil_problem* p, int n_steps, double* terms) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  if (n_steps < 0) return fail(MODIL_ERR_ARG, "n_steps < 0");
  for (int i = 0; i < n_steps; ++i) {
    const int cur = (int)(p->steps & 1);
    if (p->use_graph) {
      if (!p->gexec[cur]) {
        CUDA_TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        modil_status s = run_pass(p, MODE_STEP);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->stream, &g);
        if (s != MODIL_OK) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) return fail(MODIL_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        p->graph[cur] = g;
        e = cudaGraphInstantiate(&p->gexec[cur], g, 0);
        if (e != cudaSuccess) { drop_graph(p); return fail(MODIL_ERR_CUDA, cudaGetErrorString(e)); }
      }
      CUDA_TRY(cudaGraphLaunch(p->gexec[cur], p->stream));
    } else {
      modil_status s = run_pass(p, MODE_STEP);
      if (s != MODIL_OK) return s;
    }
    p->steps++;
  }
  return terms ? read_terms(p, terms) : MODIL_OK;
}

modil_status modil_launches_per_step(const modil_problem* p, int* n) {
  if (!p || !n) return fail(MODIL_ERR_ARG, "NULL argument");
  *n = kernels_per_step(p->plan);
  return MODIL_OK;
}

modil_status modil_profile_labels(const modil_problem* p, int* kind, int* level, int max_kernels,
                                  int* n_kernels) {
  if (!p || !kind || !level || !n_kernels) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  const int nk = kernels_per_step(P);
  if (max_kernels < nk) return fail(MODIL_ERR_ARG, "arrays too short");
  int k = 0;
  auto put = [&](int kd, int lv) { kind[k] = kd; level[k] = lv; ++k; };
  if (P.grid) {
    for (int l = std::max(P.max_lev - 2, 0); l >= 0; --l) put(0, l);
    put(1, 0);
    for (int l = 1; l < P.max_lev; ++l) put(2, l);
    put(3, P.max_lev);
    *n_kernels = k;
    return MODIL_OK;
  }
  if (P.pde == MODIL_PDE_NS3D) {
    const int lo = P.min_lev == 1 ? -1 : 0;
    for (int l = P.max_lev - 2; l >= lo; --l) put(0, l);
  } else if (P.stream) {
    if (P.max_lev >= 4) put(0, 2);  // levels 2 .. L-2
    if (P.max_lev >= 3) put(0, 1);
  }
  put(1, 0);
  for (int l = 1; l < P.max_tail; ++l) put(2, l);
  put(3, P.max_tail);
  *n_kernels = k;
  return MODIL_OK;
}

modil_status modil_profile_step(modil_problem* p, float* ms, int max_kernels, int* n_kernels) {
  if (!p || !ms || !n_kernels) return fail(MODIL_ERR_ARG, "NULL argument");
  const int nk = kernels_per_step(p->plan);
  if (max_kernels < nk) return fail(MODIL_ERR_ARG, "ms[] too short");
  std::vector<cudaEvent_t> ev(nk + 1, nullptr);
  for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
  int nev = 0;
  // queue the timed launches behind a short delay so they run back to back
  CUDA_TRY(launch_delay(300000, p->stream));
  modil_status s = run_pass(p, MODE_STEP, ev.data(), &nev);
  if (s == MODIL_OK) {
    p->steps++;
    cudaError_t e = cudaEventSynchronize(ev[nev - 1]);
    for (int k = 0; k + 1 < nev && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    if (e != cudaSuccess) s = fail(MODIL_ERR_CUDA, cudaGetErrorString(e));
    *n_kernels = nev - 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return s;
}

modil_status modil_loss_fwd(modil_problem* p, const void* levels, double* terms) {
  if (!p || !levels) return fail(MODIL_ERR_ARG, "NULL argument");
  modil_status s = p->plan.dtype == MODIL_F64
                       ? external_pass<double>(p, p->A64, levels, nullptr, 1.0, MODE_LOSS)
                       : external_pass<float>(p, p->A32, levels, nullptr, 1.0, MODE_LOSS);
  if (s != MODIL_OK) return s;
  return terms ? read_terms(p, terms) : MODIL_OK;
}

modil_status modil_loss_bwd(modil_problem* p, const void* levels, double grad_out, void* grads) {
  if (!p || !levels || !grads) return fail(MODIL_ERR_ARG, "NULL argument");
  return p->plan.dtype == MODIL_F64
             ? external_pass<double>(p, p->A64, levels, grads, grad_out, MODE_GRAD)
             : external_pass<float>(p, p->A32, levels, grads, grad_out, MODE_GRAD);
}

modil_status modil_terms_device(const modil_problem* p, const double** terms, int* stride) {
  if (!p || !terms || !stride) return fail(MODIL_ERR_ARG, "NULL argument");
  static_assert(sizeof(InstState) % sizeof(double) == 0, "InstState layout");
  const InstState* st = reinterpret_cast<const InstState*>(static_cast<const char*>(p->arena) + p->plan.o_st);
  *terms = st->terms;  // device address (no dereference on the host)
  *stride = (int)(sizeof(InstState) / sizeof(double));
  return MODIL_OK;
}

modil_status modil_set_persistent(modil_problem* p, int on) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  const Plan& P = p->plan;
  if ((P.pde == MODIL_PDE_NS2D || P.pde == MODIL_PDE_NS3D) && on)
    return fail(MODIL_ERR_UNSUPPORTED, "persistent launch: Burgers/heat only");
  if (P.stream || P.grid) return MODIL_OK;  // equal work units: nothing to balance
  int grid = 0;
  if (on) {
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    CUDA_TRY(fine_st_blocks_per_sm(P.pde, P.cfg, P.pyr_elems, (int)P.esz, &per_sm));
    grid = std::max(1, per_sm) * sms;
  }
  drop_graph(p);  // the launch configuration is part of the captured graph
  p->A32.persistent = grid;
  p->A64.persistent = grid;
  return MODIL_OK;
}

modil_status modil_param_count(const modil_problem* p, long long* n) {
  if (!p || !n) return fail(MODIL_ERR_ARG, "NULL argument");
  *n = p->plan.n_param;
  return MODIL_OK;
}

modil_status modil_level_offset(const modil_problem* p, int instance, int field, int level,
                                long long* offset) {
  if (!p || !offset) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  if (instance < 0 || instance >= P.n_inst) return fail(MODIL_ERR_ARG, "instance out of range");
  if (field < 0 || field >= P.nfield) return fail(MODIL_ERR_ARG, "field out of range");
  if (level < 0 || level >= P.inst[instance].nlev) return fail(MODIL_ERR_ARG, "level out of range");
  *offset = P.dev[instance].off[field][level];
  return MODIL_OK;
}

modil_status modil_step_count(const modil_problem* p, long long* t) {
  if (!p || !t) return fail(MODIL_ERR_ARG, "NULL argument");
  *t = p->steps;
  return MODIL_OK;
}

modil_status modil_save(modil_problem* p, const char* path) {
  if (!p || !path) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  CkptHeader h{};
  std::memcpy(h.magic, "MODILCK1", 8);
  h.version = 1;
  h.n_inst = P.n_inst; h.pde = P.pde; h.dtype = P.dtype; h.nfield = P.nfield;
  h.n_param = P.n_param; h.n_k = P.n_k; h.steps = p->steps;
  h.shape_hash = shape_hash(P);
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MODIL_ERR_ARG, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
  std::vector<char> buf;
  for (const CkptRegion& r : ckpt_regions(p)) {
    if (!ok || r.bytes == 0) continue;
    buf.resize(r.bytes);
    cudaError_t e = cudaMemcpy(buf.data(), static_cast<char*>(p->arena) + r.off, r.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      std::fclose(f);
      return fail(MODIL_ERR_CUDA, cudaGetErrorString(e));
    }
    ok = std::fwrite(buf.data(), 1, r.bytes, f) == r.bytes;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(MODIL_ERR_ARG, std::string("writing ") + path + " failed");
  return MODIL_OK;
}

modil_status modil_load(modil_problem* p, const char* path) {
  if (!p || !path) return fail(MODIL_ERR_ARG, "NULL argument");
  const Plan& P = p->plan;
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MODIL_ERR_ARG, std::string("cannot open ") + path);
  CkptHeader h{};
  if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "MODILCK1", 8) != 0 || h.version != 1) {
    std::fclose(f);
    return fail(MODIL_ERR_ARG, std::string(path) + " is not a checkpoint of this library");
  }
  if (h.n_inst != P.n_inst || h.pde != P.pde || h.dtype != P.dtype || h.nfield != P.nfield ||
      h.n_param != P.n_param || h.n_k != P.n_k || h.shape_hash != shape_hash(P) || h.steps < 0) {
    std::fclose(f);
    return fail(MODIL_ERR_ARG, "the checkpoint was written by a problem of another shape");
  }
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  const long long old = p->steps;
  p->steps = h.steps;  // selects the level buffer the next step reads
  std::vector<char> buf;
  for (const CkptRegion& r : ckpt_regions(p)) {
    if (r.bytes == 0) continue;
    buf.resize(r.bytes);
    if (std::fread(buf.data(), 1, r.bytes, f) != r.bytes) {
      std::fclose(f);
      p->steps = old;
      return fail(MODIL_ERR_ARG, std::string(path) + " is truncated");
    }
    CUDA_TRY(cudaMemcpy(static_cast<char*>(p->arena) + r.off, buf.data(), r.bytes, cudaMemcpyHostToDevice));
  }
  std::fclose(f);
  return MODIL_OK;
}

modil_status modil_reset_optimizer(modil_problem* p) {
  if (!p) return fail(MODIL_ERR_ARG, "problem is NULL");
  const Plan& P = p->plan;
  char* b = static_cast<char*>(p->arena);
  // keep the current levels: move them into buffer 0 if they live in buffer 1
  if (p->steps & 1) CUDA_TRY(cudaMemcpyAsync(b + P.o_p0, b + P.o_p1, P.esz * P.n_param, cudaMemcpyDeviceToDevice, p->stream));
  CUDA_TRY(cudaMemsetAsync(b + P.o_m, 0, P.esz * P.n_param, p->stream));
  CUDA_TRY(cudaMemsetAsync(b + P.o_v, 0, 8 * P.n_param, p->stream));
  CUDA_TRY(cudaMemsetAsync(b + P.o_km, 0, P.esz * P.n_k, p->stream));
  CUDA_TRY(cudaMemsetAsync(b + P.o_kv, 0, 8 * P.n_k, p->stream));
  cudaError_t e = P.dtype == MODIL_F64 ? launch_reset<double>(p->A64, p->stream) : launch_reset<float>(p->A32, p->stream);
  if (e != cudaSuccess) return fail(MODIL_ERR_CUDA, cudaGetErrorString(e));
  p->steps = 0;
  return MODIL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Limited-memory BFGS over the level arena of a single-instance problem
// ---------------------------------------------------------------------------
struct modil_lbfgs {
  modil_problem* p = nullptr;
  int m = 0;                 // pairs kept
  long long n = 0;           // unknowns: the levels, then the heat conductivity nodes
  long long nl = 0;          // of which the levels (all fields)
  int nk = 0;                // and the conductivity nodes (heat without k_fixed; else 0)
  double ks = 1.0;           // the vector holds the nodes in units of k_scale
  void* vec = nullptr;       // device: S[m], Y[m], then 7 work vectors, problem dtype
  double* dsc = nullptr;     // device: dot partials, batched-dot partials and results, coefficients, scratch
  void** ptrs = nullptr;     // device: vector-pointer arrays of the batched dots and of the combination
  std::vector<int> order;    // slots of the stored pairs, oldest first
  std::vector<double> SY, YY;  // host, m x m by slot: s_i . y_j and y_i . y_j of stored pairs
  std::vector<double> a, b;    // host, by slot: s_i . g and y_i . g at the current gradient
  long long iters = 0;       // iterations completed over the optimiser's life
};

namespace {

int lbfgs_max_dots(int m) { return 5 + 4 * m; }

template <class T>
Arena<T>& arena_of(modil_problem* p);
template <>
Arena<float>& arena_of<float>(modil_problem* p) { return p->A32; }
template <>
Arena<double>& arena_of<double>(modil_problem* p) { return p->A64; }

// L-BFGS in the compact representation (Byrd, Nocedal and Schnabel 1994):
// with the stored pairs oldest first as the columns of S and Y, R the upper
// triangle of S^T Y, D its diagonal and gamma = s.y / y.y of the newest pair,
//   H g = gamma g + S u + gamma Y w,  w = -R^{-1} S^T g,
//   u = R^{-T} ((D + gamma Y^T Y) R^{-1} S^T g - gamma Y^T g),
// the same H g as the two-loop recursion (H0 = gamma I).  The products S^T g,
// Y^T g and the new entries of S^T Y and Y^T Y are batched dot products, the
// small triangular solves run on the host, and H g is one pass over the
// vectors: a few launches per iteration instead of four per stored pair.
template <class T>
modil_status lbfgs_run_t(modil_lbfgs* o, int iters, double* loss, int* done) {
  constexpr double kC1 = 1e-4, kCurv = 1e-12;
  constexpr int kTrials = 40;
  modil_problem* p = o->p;
  cudaStream_t s = p->stream;
  const long long n = o->n;
  const int m = o->m;
  const size_t vb = sizeof(T) * (size_t)n;
  T* base = static_cast<T*>(o->vec);
  auto Sv = [&](int i) { return base + (size_t)i * n; };
  auto Yv = [&](int i) { return base + (size_t)(m + i) * n; };
  T* x = base + (size_t)(2 * m) * n;
  T* xt = x + n;
  T* g = xt + n;
  T* gn = g + n;
  T* q = gn + n;  // s of the candidate pair
  T* r = q + n;   // H g
  T* yv = r + n;  // y of the candidate pair
  const int maxd = lbfgs_max_dots(m);
  double* part = o->dsc;
  double* mpart = part + lb_dot_partials();
  double* mout = mpart + lb_mdot_partials(maxd);
  double* coef = mout + maxd;
  double* tmp = coef + 2 * m;
  const T** dva = reinterpret_cast<const T**>(static_cast<void*>(o->ptrs));
  const T** dvb = dva + maxd;
  const T** dvc = dvb + maxd;
  Arena<T>& A = arena_of<T>(p);
  T* pc = A.p[p->steps & 1];  // the problem's current levels
  const long long nl = o->nl;
  const size_t kb = sizeof(T) * (size_t)o->nk;
  const double ks = o->ks;
  double terms[MODIL_NTERMS];
  // loss (and gradient) at lv; a non-finite loss of a trial point counts as
  // +inf (the line search backs off) and the problem's latch is cleared.  The
  // conductivity nodes (the vector's tail) go through the problem's own node
  // array: written before the pass, their gradient read after it.
  auto eval = [&](T* lv, T* gr, double* f) -> modil_status {
    if (kb) CUDA_TRY(lb_mul<T>(A.kq, lv + nl, ks, o->nk, s));
    modil_status st = external_pass<T>(p, A, lv, gr, 1.0, gr ? MODE_GRAD : MODE_LOSS);
    if (st == MODIL_OK && gr && kb) CUDA_TRY(lb_mul<T>(gr + nl, A.kg, ks, o->nk, s));
    if (st == MODIL_OK) st = read_terms(p, terms);
    *f = terms[0];
    if (st == MODIL_ERR_NONFINITE) {
      CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(A.st) + offsetof(InstState, nonfinite), 0, sizeof(int), s));
      *f = HUGE_VAL;
      return gr ? MODIL_ERR_NONFINITE : MODIL_OK;
    }
    return st;
  };
  auto dot_host = [&](const T* a, const T* b, double* out) -> modil_status {
    CUDA_TRY(lb_dot<T>(a, b, n, part, nullptr, tmp, s));
    CUDA_TRY(cudaMemcpyAsync(out, tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MODIL_OK;
  };
  // batched dots of the listed vector pairs (enqueued; results in mout)
  std::vector<const T*> la, lb;
  auto mdot = [&]() -> modil_status {
    CUDA_TRY(cudaMemcpyAsync(dva, la.data(), sizeof(T*) * la.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dvb, lb.data(), sizeof(T*) * lb.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(lb_mdot<T>(dva, dvb, (int)la.size(), n, mpart, mout, s));
    return MODIL_OK;
  };
  std::vector<double> h;
  auto read_mout = [&]() -> modil_status {  // on the problem's stream (it may not block the legacy one)
    h.resize(la.size());
    CUDA_TRY(cudaMemcpyAsync(h.data(), mout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MODIL_OK;
  };
  // the dots of a trial point: g.r; the candidate pair's s.y, y.y; the new
  // column of S^T Y and row of Y^T Y; S^T gn, Y^T gn of the stored pairs and
  // of the candidate
  auto trial_list = [&]() {
    la.clear();
    lb.clear();
    la.push_back(g); lb.push_back(r);
    la.push_back(q); lb.push_back(yv);
    la.push_back(yv); lb.push_back(yv);
    for (int i : o->order) { la.push_back(Sv(i)); lb.push_back(yv); la.push_back(Yv(i)); lb.push_back(yv); }
    for (int i : o->order) { la.push_back(Sv(i)); lb.push_back(gn); la.push_back(Yv(i)); lb.push_back(gn); }
    la.push_back(q); lb.push_back(gn);
    la.push_back(yv); lb.push_back(gn);
  };
  modil_status st;
  CUDA_TRY(cudaMemcpyAsync(x, pc, sizeof(T) * (size_t)nl, cudaMemcpyDeviceToDevice, s));
  if (kb) CUDA_TRY(lb_mul<T>(x + nl, A.kq, 1.0 / ks, o->nk, s));
  double fx = 0.0;
  if ((st = eval(x, g, &fx)) != MODIL_OK) return st;
  if (loss) loss[0] = fx;
  if (!o->order.empty()) {  // S^T g and Y^T g at this run's starting point
    la.clear();
    lb.clear();
    for (int i : o->order) { la.push_back(Sv(i)); lb.push_back(g); la.push_back(Yv(i)); lb.push_back(g); }
    if ((st = mdot()) != MODIL_OK) return st;
    if ((st = read_mout()) != MODIL_OK) return st;
    for (size_t j = 0; j < o->order.size(); ++j) {
      o->a[o->order[j]] = h[2 * j];
      o->b[o->order[j]] = h[2 * j + 1];
    }
  }
  std::vector<double> R, t, z, cu;
  std::vector<const T*> vecs;
  int k = 0;
  for (; k < iters; ++k) {
    const int np = (int)o->order.size();
    if (np == 0) {
      CUDA_TRY(cudaMemcpyAsync(r, g, vb, cudaMemcpyDeviceToDevice, s));
    } else {
      // coefficients of H g on the host (np <= m small triangular systems)
      const std::vector<int>& od = o->order;
      auto SYo = [&](int i, int j) { return o->SY[(size_t)od[i] * m + od[j]]; };
      auto YYo = [&](int i, int j) { return o->YY[(size_t)od[i] * m + od[j]]; };
      const int nw = od.back();
      const double gamma = o->SY[(size_t)nw * m + nw] / o->YY[(size_t)nw * m + nw];
      t.assign(np, 0.0);
      for (int i = np - 1; i >= 0; --i) {  // R t = S^T g
        double v = o->a[od[i]];
        for (int j = i + 1; j < np; ++j) v -= SYo(i, j) * t[j];
        t[i] = v / SYo(i, i);
      }
      z.assign(np, 0.0);
      for (int i = 0; i < np; ++i) {  // z = (D + gamma Y^T Y) t - gamma Y^T g
        double v = SYo(i, i) * t[i] - gamma * o->b[od[i]];
        for (int j = 0; j < np; ++j) v += gamma * YYo(i, j) * t[j];
        z[i] = v;
      }
      cu.assign(2 * np, 0.0);
      for (int i = 0; i < np; ++i) {  // R^T u = z
        double v = z[i];
        for (int j = 0; j < i; ++j) v -= SYo(j, i) * cu[j];
        cu[i] = v / SYo(i, i);
      }
      for (int i = 0; i < np; ++i) cu[np + i] = -gamma * t[i];  // gamma w
      vecs.clear();
      for (int i = 0; i < np; ++i) vecs.push_back(Sv(od[i]));
      for (int i = 0; i < np; ++i) vecs.push_back(Yv(od[i]));
      CUDA_TRY(cudaMemcpyAsync(coef, cu.data(), sizeof(double) * cu.size(), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(dvc, vecs.data(), sizeof(T*) * vecs.size(), cudaMemcpyHostToDevice, s));
      CUDA_TRY(lb_combine<T>(r, g, gamma, dvc, coef, 2 * np, n, s));
    }
    double step = 1.0;
    if (o->iters == 0) {
      double gg = 0.0;
      if ((st = dot_host(g, g, &gg)) != MODIL_OK) return st;
      step = 1.0 / std::sqrt(gg);
    }
    // The first trial point with its gradient and every dot product the
    // iteration needs, read back once: the first trial is accepted in most
    // iterations, and then one loss-and-gradient pass and one host round trip
    // make the iteration.
    CUDA_TRY(lb_axpby<T>(xt, x, r, -step, n, s));  // xt = x + step d
    double ft = 0.0;
    st = eval(xt, gn, &ft);
    if (st != MODIL_OK && st != MODIL_ERR_NONFINITE) return st;
    CUDA_TRY(lb_sub<T>(q, xt, x, n, s));
    CUDA_TRY(lb_sub<T>(yv, gn, g, n, s));
    trial_list();
    if ((st = mdot()) != MODIL_OK) return st;
    if ((st = read_mout()) != MODIL_OK) return st;
    const double gd = -h[0];  // g.d
    if (!(gd < 0.0)) break;
    if (!(ft <= fx + kC1 * step * gd)) {
      // backtracking on the Armijo condition (loss only), then the gradient
      // and the dots at the accepted point
      bool ok = false;
      for (int trial = 1; trial < kTrials; ++trial) {
        step *= 0.5;
        CUDA_TRY(lb_axpby<T>(xt, x, r, -step, n, s));
        if ((st = eval(xt, nullptr, &ft)) != MODIL_OK) return st;
        if (ft <= fx + kC1 * step * gd) { ok = true; break; }
      }
      if (!ok) break;
      if ((st = eval(xt, gn, &ft)) != MODIL_OK) return st;
      CUDA_TRY(lb_sub<T>(q, xt, x, n, s));
      CUDA_TRY(lb_sub<T>(yv, gn, g, n, s));
      trial_list();
      if ((st = mdot()) != MODIL_OK) return st;
      if ((st = read_mout()) != MODIL_OK) return st;
    }
    // the new point; the candidate pair if its curvature is positive
    const double sy_h = h[1], yy_h = h[2];
    const std::vector<int> old = o->order;
    const int no = (int)old.size();
    for (int j = 0; j < no; ++j) {  // S^T g and Y^T g at the new point
      o->a[old[j]] = h[3 + 2 * no + 2 * j];
      o->b[old[j]] = h[4 + 2 * no + 2 * j];
    }
    if (sy_h > kCurv * yy_h) {
      int slot, first = 0;
      if (no < m) {
        slot = no;
      } else {
        slot = o->order.front();  // the oldest pair makes room
        o->order.erase(o->order.begin());
        first = 1;
      }
      CUDA_TRY(cudaMemcpyAsync(Sv(slot), q, vb, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(Yv(slot), yv, vb, cudaMemcpyDeviceToDevice, s));
      for (int j = first; j < no; ++j) {
        const int i = old[j];
        o->SY[(size_t)i * m + slot] = h[3 + 2 * j];
        o->YY[(size_t)i * m + slot] = h[4 + 2 * j];
        o->YY[(size_t)slot * m + i] = h[4 + 2 * j];
      }
      o->SY[(size_t)slot * m + slot] = sy_h;
      o->YY[(size_t)slot * m + slot] = yy_h;
      o->a[slot] = h[3 + 4 * no];
      o->b[slot] = h[4 + 4 * no];
      o->order.push_back(slot);
    }
    std::swap(x, xt);
    std::swap(g, gn);
    fx = ft;
    if (loss) loss[k + 1] = fx;
    o->iters++;
  }
  // the result and its gradient become the problem's levels (and nodes) and gradient
  CUDA_TRY(cudaMemcpyAsync(pc, x, sizeof(T) * (size_t)nl, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(A.g, g, sizeof(T) * (size_t)nl, cudaMemcpyDeviceToDevice, s));
  if (kb) {
    CUDA_TRY(lb_mul<T>(A.kq, x + nl, ks, o->nk, s));
    CUDA_TRY(lb_mul<T>(A.kg, g + nl, 1.0 / ks, o->nk, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  if (done) *done = k;
  return MODIL_OK;
}

}  // namespace

extern "C" {

modil_status modil_lbfgs_create(modil_problem* p, int history, modil_lbfgs** out) {
  if (!p || !out) return fail(MODIL_ERR_ARG, "NULL argument");
  *out = nullptr;
  const Plan& P = p->plan;
  if (history < 1) return fail(MODIL_ERR_ARG, "history < 1");
  if (P.n_inst != 1) return fail(MODIL_ERR_UNSUPPORTED, "L-BFGS: single-instance problems only");
  modil_lbfgs* o = new (std::nothrow) modil_lbfgs();
  if (!o) return fail(MODIL_ERR_ARG, "out of host memory");
  o->p = p;
  o->m = history;
  o->nl = P.n_param;
  o->nk = (P.pde == MODIL_PDE_HEAT && !P.dev[0].k_fixed) ? P.dev[0].nk : 0;
  o->n = o->nl + o->nk;
  o->ks = P.dev[0].k_scale;
  o->SY.assign((size_t)history * history, 0.0);
  o->YY.assign((size_t)history * history, 0.0);
  o->a.assign(history, 0.0);
  o->b.assign(history, 0.0);
  const int maxd = lbfgs_max_dots(history);
  cudaError_t e = cudaMalloc(&o->vec, P.esz * (size_t)o->n * (2 * (size_t)history + 7));
  if (e == cudaSuccess)
    e = cudaMalloc(&o->dsc, sizeof(double) * ((size_t)lb_dot_partials() + (size_t)lb_mdot_partials(maxd) + maxd +
                                              2 * (size_t)history + 1));
  if (e == cudaSuccess) e = cudaMalloc(&o->ptrs, sizeof(void*) * (2 * (size_t)maxd + 2 * (size_t)history));
  if (e != cudaSuccess) {
    modil_lbfgs_destroy(o);
    return fail(MODIL_ERR_CUDA, std::string("L-BFGS buffers: ") + cudaGetErrorString(e));
  }
  *out = o;
  return MODIL_OK;
}

modil_status modil_lbfgs_run(modil_lbfgs* o, int iterations, double* loss, int* done) {
  if (!o) return fail(MODIL_ERR_ARG, "optimiser is NULL");
  if (iterations < 0) return fail(MODIL_ERR_ARG, "iterations < 0");
  if (done) *done = 0;
  return o->p->plan.dtype == MODIL_F64 ? lbfgs_run_t<double>(o, iterations, loss, done)
                                       : lbfgs_run_t<float>(o, iterations, loss, done);
}

void modil_lbfgs_destroy(modil_lbfgs* o) {
  if (!o) return;
  if (o->vec) cudaFree(o->vec);
  if (o->dsc) cudaFree(o->dsc);
  if (o->ptrs) cudaFree(o->ptrs);
  delete o;
}

const char* modil_last_error(void) { return g_err.c_str(); }

const char* modil_version(void) { return "modil-gb300 0.1 (sm_103a)"; }

size_t modil_desc_size(void) { return sizeof(modil_desc); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Loss and gradient without any device allocation.
//
// Some callers cannot allocate device memory: a host application or framework
// that owns every device allocation through its own pool (and forbids raw
// cudaMalloc from plug-ins), code that must not allocate once it is running
// (real-time loops, which cudaMalloc would stall by synchronising the device),
// or a caller that holds only the buffers it was handed.  For them this entry
// point keeps its working memory -- the per-tile partial sums, the problem
// tables and the measurement runs -- in one file-scope __device__ array of
// kNoAllocScratchBytes.  Every GPU that loads the library holds the array until
// the process exits.  In host code the array's name is only a host-side
// stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

modil_status noalloc_scratch(void** out) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MODIL_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MODIL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MODIL_OK;
}

template <class T>
modil_status noalloc_run(const Plan& P, const modil_desc* d, const void* levels, void* grads,
                         double* terms, double* kgrad, cudaStream_t s) {
  void* base = nullptr;
  modil_status st = noalloc_scratch(&base);
  if (st != MODIL_OK) return st;
  // compact layout of what the kernels read or write besides levels and grads
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t r = o; o = align256(o + std::max<size_t>(bytes, 1)); return r; };
  const size_t nft = P.tile_inst[0].size();
  const size_t o_kq = take(sizeof(T) * P.n_k), o_kg = take(sizeof(T) * P.n_k);
  const size_t o_aux = take(sizeof(T) * P.n_aux);
  const size_t o_part = take(8 * nft * P.npart);
  const size_t o_rptr = take(4 * P.run_ptr.size()), o_rcell = take(4 * P.run_cell.size());
  const size_t o_rfield = take(4 * P.run_field.size()), o_rbeg = take(4 * P.run_beg.size());
  const size_t o_mval = take(sizeof(T) * P.meas_val.size());
  const size_t o_rv0 = take(sizeof(T) * P.run_v0.size());
  const size_t o_inst = take(sizeof(DevInst)), o_st = take(sizeof(InstState));
  const size_t o_cnt = take(sizeof(int));
  const size_t o_q = take(2 * sizeof(int));
  size_t o_ti[MODIL_MAXL];
  for (int l = 0; l < MODIL_MAXL; ++l) o_ti[l] = take(4 * P.tile_inst[l].size());
  if (o > kNoAllocScratchBytes)
    return fail(MODIL_ERR_ARG, "problem needs " + std::to_string(o) + " scratch bytes; the allocation-free "
                "entry point holds at most " + std::to_string(kNoAllocScratchBytes));
  char* b = static_cast<char*>(base);
  auto up = [&](size_t off, const void* src, size_t bytes) -> modil_status {
    if (bytes) CUDA_TRY(cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, s));
    return MODIL_OK;
  };
  std::vector<T> kq(d->n_knodes > 0 && P.nk ? d->knodes : nullptr,
                    d->n_knodes > 0 && P.nk ? d->knodes + P.nk : nullptr);
  std::vector<T> aux(P.n_aux ? d->aux : nullptr, P.n_aux ? d->aux + P.n_aux : nullptr);
  std::vector<T> mv(P.meas_val.begin(), P.meas_val.end());
  std::vector<T> rv(P.run_v0.begin(), P.run_v0.end());
  InstState st0;
  std::memset(&st0, 0, sizeof(st0));
  st0.b1t = 1.0;
  st0.b2t = 1.0;
  st0.c1 = 1.0 / (1.0 - d->adam_beta1);
  st0.c2 = 1.0 / (1.0 - d->adam_beta2);
  if ((st = up(o_kq, kq.data(), sizeof(T) * kq.size())) != MODIL_OK) return st;
  if ((st = up(o_aux, aux.data(), sizeof(T) * aux.size())) != MODIL_OK) return st;
  if ((st = up(o_rptr, P.run_ptr.data(), 4 * P.run_ptr.size())) != MODIL_OK) return st;
  if ((st = up(o_rcell, P.run_cell.data(), 4 * P.run_cell.size())) != MODIL_OK) return st;
  if ((st = up(o_rfield, P.run_field.data(), 4 * P.run_field.size())) != MODIL_OK) return st;
  if ((st = up(o_rbeg, P.run_beg.data(), 4 * P.run_beg.size())) != MODIL_OK) return st;
  if ((st = up(o_mval, mv.data(), sizeof(T) * mv.size())) != MODIL_OK) return st;
  if ((st = up(o_rv0, rv.data(), sizeof(T) * rv.size())) != MODIL_OK) return st;
  if ((st = up(o_inst, P.dev.data(), sizeof(DevInst))) != MODIL_OK) return st;
  if ((st = up(o_st, &st0, sizeof(st0))) != MODIL_OK) return st;
  CUDA_TRY(cudaMemsetAsync(b + o_cnt, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(b + o_q, 0, 2 * sizeof(int), s));
  for (int l = 0; l < MODIL_MAXL; ++l)
    if ((st = up(o_ti[l], P.tile_inst[l].data(), 4 * P.tile_inst[l].size())) != MODIL_OK) return st;
  Arena<T> A{};
  A.p[0] = const_cast<T*>(static_cast<const T*>(levels));
  A.p[1] = nullptr;
  A.g = static_cast<T*>(grads);
  A.kq = reinterpret_cast<T*>(b + o_kq);
  A.kg = reinterpret_cast<T*>(b + o_kg);
  A.aux = reinterpret_cast<const T*>(b + o_aux);
  A.part = reinterpret_cast<double*>(b + o_part);
  A.run_ptr = reinterpret_cast<const int*>(b + o_rptr);
  A.run_cell = reinterpret_cast<const int*>(b + o_rcell);
  A.run_field = reinterpret_cast<const int*>(b + o_rfield);
  A.run_beg = reinterpret_cast<const int*>(b + o_rbeg);
  A.meas_val = reinterpret_cast<const T*>(b + o_mval);
  A.run_v0 = reinterpret_cast<const T*>(b + o_rv0);
  A.inst = reinterpret_cast<const DevInst*>(b + o_inst);
  A.st = reinterpret_cast<InstState*>(b + o_st);
  A.counter = reinterpret_cast<int*>(b + o_cnt);
  A.queue = reinterpret_cast<int*>(b + o_q);
  A.persistent = 0;
  for (int l = 0; l < MODIL_MAXL; ++l) {
    A.tile_inst[l] = reinterpret_cast<const int*>(b + o_ti[l]);
    A.ntiles[l] = (int)P.tile_inst[l].size();
  }
  A.npart = P.npart;
  A.n_inst = 1;
  A.gscale = 1.0f;
  A.inst0 = P.dev[0];
  if (P.pde == MODIL_PDE_NS2D) CUDA_TRY((prepare_fine_ns2d<T>(P.cfg, P.pyr_elems)));
  else CUDA_TRY((prepare_fine_st<T>(P.pde, P.cfg, P.pyr_elems)));
  CUDA_TRY(prepare_tail<T>(P.tail));
  if (P.pde == MODIL_PDE_NS2D) CUDA_TRY(launch_fine_ns2d<T>(A, P.cfg, MODE_GRAD, 0, P.pyr_elems, s));
  else CUDA_TRY(launch_fine_st<T>(A, P.pde, P.cfg, MODE_GRAD, 0, P.pyr_elems, s));
  for (int l = 1; l < P.max_tail; ++l) CUDA_TRY(launch_level<T>(A, P.nfield, l, MODE_GRAD, 0, s));
  CUDA_TRY(launch_tail<T>(A, MODE_GRAD, 0, P.tail, s));
  InstState out;
  CUDA_TRY(cudaMemcpyAsync(&out, b + o_st, sizeof(out), cudaMemcpyDeviceToHost, s));
  std::vector<T> kg(P.nk);
  if (kgrad && P.nk) CUDA_TRY(cudaMemcpyAsync(kg.data(), b + o_kg, sizeof(T) * P.nk, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int j = 0; j < MODIL_NTERMS; ++j) terms[j] = out.terms[j];
  if (kgrad)
    for (int j = 0; j < P.nk; ++j) kgrad[j] = (double)kg[j];
  if (out.nonfinite & kStatusTimeout)
    return fail(MODIL_ERR_TIMEOUT, "a bounded wait inside a kernel ran out");
  if (out.nonfinite) return fail(MODIL_ERR_NONFINITE, "loss became non-finite");
  return MODIL_OK;
}

}  // namespace

extern "C" modil_status modil_test_set_spin_limit(long long polls) {
  CUDA_TRY(set_spin_limit(polls));
  return MODIL_OK;
}

extern "C" modil_status modil_eval_grad_noalloc(const modil_desc* desc, const void* levels,
                                                void* grads, double* terms, double* kgrad,
                                                void* stream) {
  if (!desc || !levels || !grads || !terms) return fail(MODIL_ERR_ARG, "NULL argument");
  // the kernels move aligned runs of 4 elements with 16-byte accesses
  if ((reinterpret_cast<uintptr_t>(levels) | reinterpret_cast<uintptr_t>(grads)) & 15)
    return fail(MODIL_ERR_ARG, "levels and grads must start on 16-byte boundaries");
  Plan P;
  modil_status s = make_plan(desc, 1, P, /*allow_stream=*/false);
  if (s != MODIL_OK) return s;
  if (P.pde == MODIL_PDE_NS3D || P.grid)
    return fail(MODIL_ERR_UNSUPPORTED, "the allocation-free entry point takes the 2-D families "
                "(the Poisson family in its 2-D cell layout)");
  if (P.n_points > 0)
    return fail(MODIL_ERR_UNSUPPORTED, "the allocation-free entry point takes no off-grid points");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return P.dtype == MODIL_F64 ? noalloc_run<double>(P, desc, levels, grads, terms, kgrad, st)
                              : noalloc_run<float>(P, desc, levels, grads, terms, kgrad, st);
}
