// Device-side data structures and helpers of the mODIL library.
//
// Memory model.  One arena holds every instance of a batch:
//   p[2]  level values, ping-pong: step t reads p[t & 1] and writes p[(t+1) & 1]
//         so that tiles composing the field never see a half-updated level
//         (the buffer index is a kernel argument; the host keeps t);
//   m     Adam first moment (storage type T);
//   v     Adam second moment, always FP64;
//   g     dL/du per level (also the input of the next level's restriction);
// all four indexed by DevInst::off[field][level] (element offsets, row-major,
// last axis fastest).  Conductivity nodes (heat) have their own small arrays.
// Per fine tile the kernels write FP64 partial sums (residual, data and the
// conductivity-node gradient) that one finalising block per instance adds in
// a fixed order, so every result is bit-reproducible run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MODIL_MAXL 10
#define MODIL_MAXF 5
#define MODIL_MAXK 64
#define MODIL_NT 256  // threads per block of the tile kernels

namespace modil {

enum Mode { MODE_LOSS = 0, MODE_GRAD = 1, MODE_STEP = 2, MODE_COMPOSE = 3 };
enum Pde { PDE_BURGERS = 1, PDE_HEAT = 2, PDE_NS2D = 3, PDE_NS3D = 4, PDE_POISSON = 5 };

// Per-instance description (read-only on the device).
struct DevInst {
  int nlev, nfield, nk, ndim;
  int tail;                    // first level finished by the per-instance tail kernel
  int ntile0;                  // fine tiles of this instance
  int layout;                  // Poisson: 0 cell, 1 node (n[][] count the nodes)
  int n[MODIL_MAXL][3];        // cells per axis per level, slowest first (2-D: n[l][0] = 1)
  int nt[MODIL_MAXL][3];       // tiles per axis per level
  int tile_base[MODIL_MAXL];   // global tile index of this instance's first tile per level
  long long off[MODIL_MAXF][MODIL_MAXL];  // element offsets of (field, level) arrays
  long long fine_off[MODIL_MAXF];         // offset in the composed-field scratch
  long long k_off;             // offset of the conductivity nodes
  long long aux_off;           // offset of the heat initial profile
  double h[3];                 // spacing per axis (same order as n)
  double coef[4];              // PDE coefficients (Burgers: nu)
  double w_res_dV;             // w_res * cell volume
  double w_data_n;             // w_data / n_meas
  double w_reg;                // regulariser weight (heat)
  int k_fixed;                 // heat: conductivity nodes known (dL/dq = 0, not stepped)
  double k_scale;              // heat: unit of the nodes' optimiser steps (Adam lr * k_scale)
  double lr, b1, b2, eps;      // Adam
};

// Bits of InstState::nonfinite.
constexpr int kStatusNonfinite = 1;
constexpr int kStatusTimeout = 2;

// Per-instance mutable state.
struct InstState {
  long long t;        // completed Adam steps
  double b1t, b2t;    // beta1^t, beta2^t
  double c1, c2;      // bias corrections of step t+1: 1/(1-beta1^(t+1)), 1/(1-beta2^(t+1))
  double terms[4];    // total, residual, data, regulariser of the last evaluation
  int nonfinite;      // status bits: kStatusNonfinite (a loss was NaN/Inf, latched),
                      // kStatusTimeout (a bounded wait ran out; cleared when reported)
  int pad;
};

// Advance the step counter and precompute the next step's bias corrections
// (one thread; keeps FP64 divisions out of the per-cell code).
__device__ __forceinline__ void advance_step(InstState& S, double b1, double b2) {
  S.t += 1;
  S.b1t *= b1;
  S.b2t *= b2;
  S.c1 = 1.0 / (1.0 - S.b1t * b1);
  S.c2 = 1.0 / (1.0 - S.b2t * b2);
}

template <class T>
struct Arena {
  T* p[2];
  T* m;
  double* v;
  T* g;
  T* ufine;            // composed-field scratch (MODE_COMPOSE; every pass of the 3-D family)
  T* wl;               // 3-D family: composed coarse levels w_l (l >= 1), same offsets as p
  T* kq;               // conductivity nodes (heat), Adam moments and gradient
  T* km;
  double* kv;
  T* kg;
  const T* aux;        // heat initial profiles
  double* part;        // per fine tile partial sums, npart each
  const int* run_ptr;  // per global fine tile: first measurement run
  const int* run_cell; // flat fine cell of each run (within its instance)
  const int* run_field;
  const int* run_beg;  // first value of each run; run r spans [run_beg[r], run_beg[r+1])
  const T* meas_val;
  const T* run_v0;     // first value of each run (meas_val[run_beg[r]])
  // off-grid points (NULL when a batch has none): per global fine tile the
  // records of the points one of whose four corner cells it owns, and the
  // runs of (record, weight) entries adding to each owned corner cell
  const int* pt_ptr;   // per tile: first record
  const int* pt_cell;  // 4 (2-D) or 8 (3-D) corner cells per record (flat, within the instance)
  const T* pt_w;       // as many weights per record
  const T* pt_val;     // measured value per record
  const int* pt_own;   // 1 where this record's tile counts the point's misfit
  const int* pt_field; // field each record samples
  const int* pc_field; // field of each run's target cell
  T* pt_diff;          // scratch: sample - value per record
  const int* pc_ptr;   // per tile: first run of corner contributions
  const int* pc_cell;  // target cell of each run
  const int* pc_beg;   // first entry of each run (one past the last after it)
  const int* pe_rec;   // record of each entry
  const T* pe_w;       // weight of each entry
  const DevInst* inst;
  DevInst inst0;       // copy of instance 0 in the kernel parameters (read when n_inst == 1)
  InstState* st;
  int* counter;        // per instance: fine tiles done in the current launch
  const int* tile_inst[MODIL_MAXL];  // instance owning each global tile of level l
  int ntiles[MODIL_MAXL];
  // 2-D composition pass (streaming path): per block of level l its instance
  // and the first cell (within the instance's level) it composes
  const int* cblk_inst[MODIL_MAXL];
  const int* cblk_first[MODIL_MAXL];
  int ncblk[MODIL_MAXL];
  const int* csmall_inst;  // instances with levels >= 2 to compose (L >= 4)
  int ncsmall;
  int npart;
  int n_inst;
  float gscale;        // factor on the written fine gradient (d loss / d output), 1 normally
  int persistent;      // 0: one fine block per tile; > 0: grid size of the persistent launch
  int* queue;          // persistent launch: next tile, blocks finished
};

// Minimum, maximum and floor in the working precision (FP32 arguments take the
// FP32 instructions, never a round trip through FP64).
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tfloor(float a) { return floorf(a); }
__device__ __forceinline__ double tfloor(double a) { return floor(a); }
__device__ __forceinline__ float texp(float a) { return expf(a); }
__device__ __forceinline__ double texp(double a) { return exp(a); }

// ---------------------------------------------------------------------------
// Interpolation taps (cell-based linear interpolation, printed 1-D matrices)
// ---------------------------------------------------------------------------

// Fine cell i of a grid refined from nc coarse cells takes w0*c[j0] + w1*c[j1]:
// 3/4 of its parent j = i/2 and 1/4 of the nearer neighbour; past the first
// or last coarse centre the line through the two outermost centres is
// extended (5/4 and -1/4 of the parent and its inner neighbour); a single
// coarse cell is copied.  Written with selects only (no divergent branches).
template <class T>
__device__ __forceinline__ void prolong_taps(int i, int nc, int& j0, int& j1, T& w0, T& w1) {
  const int j = i >> 1;
  const int s = (i & 1) ? 1 : -1;
  const int jn = j + s;
  const bool out = (jn < 0) || (jn >= nc);
  const bool one = (nc == 1);
  j0 = j;
  j1 = one ? 0 : (out ? j - s : jn);
  w0 = one ? T(1) : (out ? T(1.25) : T(0.75));
  w1 = one ? T(0) : (out ? T(-0.25) : T(0.25));
}

// Column j of the interpolation matrix (coarse j <- fine cells): the transposed
// operator gathers at most six fine values (nc = 3, j = 1).  Returns the tap count.
template <class T>
__device__ __forceinline__ int restrict_taps(int j, int nc, int* idx, T* w) {
  if (nc == 1) { idx[0] = 0; w[0] = T(1); idx[1] = 1; w[1] = T(1); return 2; }
  int c = 0;
  // even fine cell 2j: parent j (weight 5/4 at the first coarse cell, else 3/4)
  idx[c] = 2 * j; w[c] = (j == 0) ? T(1.25) : T(0.75); ++c;
  // odd fine cell 2j+1: parent j (5/4 at the last coarse cell, else 3/4)
  idx[c] = 2 * j + 1; w[c] = (j == nc - 1) ? T(1.25) : T(0.75); ++c;
  // odd fine cell 2j-1 has parent j-1 and neighbour j
  if (j >= 1) { idx[c] = 2 * j - 1; w[c] = T(0.25); ++c; }
  // even fine cell 2j+2 has parent j+1 and neighbour j
  if (j <= nc - 2) { idx[c] = 2 * j + 2; w[c] = T(0.25); ++c; }
  // boundary extrapolation rows reach one cell further
  if (j == 1) { idx[c] = 0; w[c] = T(-0.25); ++c; }
  if (j == nc - 2) { idx[c] = 2 * nc - 1; w[c] = T(-0.25); ++c; }
  return c;
}

// ---------------------------------------------------------------------------
// Adam.  The second moment is accumulated in FP64; the rest in T.
// ---------------------------------------------------------------------------
struct AdamCoef {
  double lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
  float lrf, b1f, omb1f, omb2f, epsf, c1f, c2f;
};

// FP32 <-> FP64 of a non-negative value with integer operations only (IEEE-754
// binary32 / binary64 layouts: rebias the exponent by 1023 - 127 = 896 and
// move the mantissa by 52 - 23 = 29 bits).  On GB300 every FP64-pipe
// instruction, conversions included, costs about one SM cycle per lane, so
// Adam's second moment keeps exactly one (the FMA).  Widening is exact for
// normal values and keeps Inf and NaN; values below the FP32 normal range
// become 0.  Narrowing truncates the mantissa (relative error below 2^-23);
// values below the FP32 normal range become 0, values of 2^128 and more
// become Inf, NaN stays NaN.  Branch-free: no conversion instruction is ever
// issued.
__device__ __forceinline__ double widen_nonneg(float x) {
  const unsigned b = __float_as_uint(x);
  const bool nz = b >= 0x00800000u, special = b >= 0x7f800000u;
  const unsigned hi = special ? (0x7ff00000u | ((b >> 3) & 0x000fffffu)) : (nz ? (b >> 3) + (896u << 20) : 0u);
  const unsigned lo = nz ? (b << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float narrow_nonneg(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned ah = hi & 0x7fffffffu;
  const bool nan = ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u);
  const unsigned big = nan ? 0x7fc00000u : 0x7f800000u;
  const unsigned b = __funnelshift_l(lo, hi, 3) - (896u << 23);
  return __uint_as_float(hi >= 0x47f00000u ? big : (hi >= 0x38100000u ? b : 0u));
}

// The second moment is accumulated in FP64 (one FMA per cell: GB300 runs FP64
// at 1/64 of the FP32 rate); the square of the gradient, the first moment and
// the update are FP32, the square root and the division by the hardware's
// approximate reciprocal square root and reciprocal (relative error of a few
// 2^-23).  Where a sum has two products, which one is fused is fixed
// explicitly, so that every kernel that applies Adam to a level (the fine
// kernels, the restriction kernels, the tail) rounds identically.
__device__ __forceinline__ void adam_update(float& p, float& m, double& v, float g,
                                            const AdamCoef& c) {
  m = fmaf(c.b1f, m, __fmul_rn(c.omb1f, g));
  v = fma(c.b2, v, widen_nonneg(__fmul_rn(c.omb2f, __fmul_rn(g, g))));
  const float s = __fmul_rn(narrow_nonneg(v), c.c2f);
  const float den = (s > 0.f ? __fmul_rn(s, rsqrtf(s)) : 0.f) + c.epsf;
  p = fmaf(-c.lrf, __fdividef(__fmul_rn(m, c.c1f), den), p);
}

__device__ __forceinline__ void adam_update(double& p, double& m, double& v, double g,
                                            const AdamCoef& c) {
  m = fma(c.b1, m, __dmul_rn(1.0 - c.b1, g));
  v = fma(c.b2, v, __dmul_rn(1.0 - c.b2, __dmul_rn(g, g)));
  const double mh = m * c.c1;
  const double den = sqrt(v * c.c2) + c.eps;
  p = fma(-c.lr, mh / den, p);
}

__device__ __forceinline__ AdamCoef adam_coef(const DevInst& D, const InstState& S) {
  AdamCoef c;
  c.lr = D.lr; c.b1 = D.b1; c.b2 = D.b2; c.eps = D.eps;
  c.c1 = S.c1;
  c.c2 = S.c2;
  c.lrf = (float)c.lr; c.b1f = (float)c.b1; c.omb1f = (float)(1.0 - c.b1);
  c.omb2f = (float)(1.0 - c.b2); c.epsf = (float)c.eps; c.c1f = (float)c.c1; c.c2f = (float)c.c2;
  return c;
}

// Compensated FP32 sum of two (hi, lo) pairs (Knuth's two-sum on the high
// parts, low parts added): about 48 significant bits with FP32 instructions.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bp = s - hi;
  float e = (hi - (s - bp)) + (bh - bp);
  e += lo + bl;
  const float t = s + e;
  lo = e - (t - s);
  hi = t;
}

// Warp sum in compensated FP32; lane 0's result is the deterministic one.
__device__ __forceinline__ double warp_sum_ff(float x) {
  float hi = x, lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, bh, bl);
  }
  return (double)hi + (double)lo;
}

// ---------------------------------------------------------------------------
// Reductions (fixed order: deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the block; every thread gets the result.  scratch: >= NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* scratch) {
  x = warp_sum(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += scratch[i];
  return s;
}

// Raise (never lower) a kernel's dynamic shared-memory limit.  The limit is
// a property of the kernel for the whole process, shared by every problem
// that launches it, so a smaller problem created later must not cut it
// below what an earlier, larger problem launches with.
template <class K>
inline cudaError_t raise_smem_limit(K kernel, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel of a step is launched with
// programmatic stream serialisation.  Protocol: a kernel may read, before
// pdl_wait(), only data that no kernel writes or that was last written two or
// more launches earlier; it calls pdl_wait() and then pdl_trigger(), so its
// successor's prologue starts only after this kernel's predecessor finished.
// Without the launch attribute both instructions are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous global -> shared copies (4 or 8 bytes, any aligned element).
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Block sum of per-thread FP32 values in compensated FP32, fixed order;
// every thread gets the result.  scratch: >= NT/16 floats.
template <int NT>
__device__ __forceinline__ double block_sum_ff(float x, float* scratch) {
  float hi = x, lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, bh, bl);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { scratch[2 * w] = hi; scratch[2 * w + 1] = lo; }
  __syncthreads();
  float sh = scratch[0], sl = scratch[1];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) ff_add(sh, sl, scratch[2 * i], scratch[2 * i + 1]);
  return (double)sh + (double)sl;
}

// The descriptor of instance ii into shared memory: from the kernel
// parameters for a single instance (no global-memory round trip), else from
// the descriptor table.
template <class AR>
__device__ __forceinline__ void load_inst(DevInst* dst, const AR& A, int ii);

// Copy a POD struct from global to shared memory with the whole block.
template <class S>
__device__ __forceinline__ void block_copy(S* dst, const S* src) {
  static_assert(sizeof(S) % 4 == 0, "POD size");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(S) / 4); i += blockDim.x) d[i] = s[i];
}

template <class AR>
__device__ __forceinline__ void load_inst(DevInst* dst, const AR& A, int ii) {
  if (A.n_inst == 1) block_copy(dst, &A.inst0);
  else block_copy(dst, A.inst + ii);
}

}  // namespace modil
