// Host-side launch interface between the C ABI layer and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>

#include "modil_dev.cuh"

namespace modil {

// Tile configurations of the fused fine kernel: (rows, cols).  The last one
// is the strip of the warp-streaming Burgers kernel (kSR rows, kSW owned
// columns per warp).
constexpr int kNumTileCfg = 7;
constexpr int kTileCfg[kNumTileCfg][2] = {{16, 32}, {16, 64}, {8, 64}, {32, 32}, {8, 128}, {8, 32}, {32, 60}};
constexpr int kStreamCfg = 6;
constexpr int kSR = 32, kSW = 60;
constexpr int kStreamNT = 128;   // threads per block of the streaming kernel (one strip per warp)
constexpr int kStreamBlocksF32 = 4, kStreamBlocksF64 = 3;  // its resident blocks per SM (register cap)
constexpr int kStreamMinStrips = 4 * 152;  // default to the streaming kernel from this many strips
constexpr int kComposeNT = 256;  // threads per block of the level-1 composition (4 cells each)
constexpr int kComposeSmallNT = 512;  // threads per block composing levels >= 2 of one instance
constexpr int kGridNT = 256;     // threads (cells) per block of the d-dimensional Poisson kernels
// Tile of the restriction kernels (coarse levels), rows x cols.
constexpr int kLevTY = 32, kLevTX = 32;  // four coarse cells per thread of k_level

// Levels with at most this many cells are finished by the per-instance tail
// kernel (FP32 / FP64 problems).
constexpr int kTailCellsF32 = 4096;
constexpr int kTailCellsF64 = 1024;

// What the tail kernel of a batch needs (maxima over the instances).
struct TailPlan {
  int level_kernels = 0;     // restriction kernels between the fine kernel and the tail
  size_t prev_cells = 0;     // cells of the level just above the tail levels
  size_t tail_cells = 0;     // cells of the tail levels
  size_t smem_bytes = 0;     // dynamic shared memory of a tail block
  int cluster = 8;           // blocks per instance (one thread-block cluster)
};
// Most blocks per instance of the tail kernel.
constexpr int kTailC = 8;

size_t fine_st_smem_bytes(int pde, int cfg, size_t pyr_elems, int elem_bytes);
cudaError_t fine_st_blocks_per_sm(int pde, int cfg, size_t pyr_elems, int elem_bytes, int* n);
template <class T>
cudaError_t prepare_fine_st(int pde, int cfg, size_t pyr_elems);
template <class T>
cudaError_t launch_fine_st(const Arena<T>& A, int pde, int cfg, int mode, int cur,
                           size_t pyr_elems, cudaStream_t s);
size_t fine_ns2d_smem_bytes(int cfg, size_t pyr_elems, int elem_bytes);
template <class T>
cudaError_t prepare_fine_ns2d(int cfg, size_t pyr_elems);
template <class T>
cudaError_t launch_fine_ns2d(const Arena<T>& A, int cfg, int mode, int cur, size_t pyr_elems,
                             cudaStream_t s);
template <class T>
cudaError_t launch_level(const Arena<T>& A, int nf, int level, int mode, int cur, cudaStream_t s);
// Warp-streaming Burgers kernel and the composition pass it reads (w_l of
// levels 1 .. L-2 into the scratch wl).
template <class T>
cudaError_t launch_compose2(const Arena<T>& A, int level, int cur, cudaStream_t s);
template <class T>
cudaError_t launch_fine_stream(const Arena<T>& A, int mode, int cur, cudaStream_t s);
// The Poisson family in d = 1, 2, 3, node or cell layout: composition of a
// level, fine residual/adjoint/Adam, restriction/Adam of a level, loss terms.
template <class T>
cudaError_t launch_gcompose(const Arena<T>& A, int level, int cur, cudaStream_t s);
template <class T>
cudaError_t launch_gresid(const Arena<T>& A, int mode, int cur, cudaStream_t s);
template <class T>
cudaError_t launch_grestrict(const Arena<T>& A, int level, int mode, int cur, cudaStream_t s);
template <class T>
cudaError_t launch_gfinal(const Arena<T>& A, int mode, cudaStream_t s);
// 3-D penalised Navier-Stokes: fine tile 4 x 8 x 16 cells, coarse tile 2 x 8 x 16.
constexpr int k3TZ = 4, k3TY = 8, k3TX = 16;
constexpr int k3LZ = 2, k3LY = 8, k3LX = 16;
template <class T>
cudaError_t prepare_ns3d(size_t pyr_elems);
// Polls of the 3-D kernel's bounded copy wait (negative: the default); for
// tests that make a wait run out.
cudaError_t set_spin_limit(long long polls);
template <class T>
cudaError_t launch_prolong3(const Arena<T>& A, int level, int nfield, int cur, cudaStream_t s);
struct Ns3Maps {
  CUtensorMap u, c;
  bool ok = false;
};
int make_ns3_maps(Ns3Maps* m, const void* ufine, int nz, int ny, int nx, int elem);
template <class T>
cudaError_t launch_resid3(const Arena<T>& A, int mode, int cur, const Ns3Maps* maps, cudaStream_t s);
template <class T>
cudaError_t launch_level3(const Arena<T>& A, int level, int nfield, int mode, int cur, cudaStream_t s);
size_t tail_smem_bytes(const TailPlan& tp, int elem_bytes);
size_t tail_instance_bytes(int L, int ts, const int (*n)[3], int nf, int C, int elem_bytes);
template <class T>
cudaError_t prepare_tail(const TailPlan& tp);
template <class T>
cudaError_t launch_tail(const Arena<T>& A, int mode, int cur, const TailPlan& tp, cudaStream_t s);
template <class T>
cudaError_t launch_reset(const Arena<T>& A, cudaStream_t s);
cudaError_t launch_delay(long long ns, cudaStream_t s);

}  // namespace modil
