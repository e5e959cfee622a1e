// Host-side launch interface between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "modil_dev.cuh"

namespace modil {

// Tile configurations of the fused fine kernel: (rows, cols).
constexpr int kNumTileCfg = 5;
constexpr int kTileCfg[kNumTileCfg][2] = {{16, 32}, {16, 64}, {8, 64}, {32, 32}, {8, 128}};
// Tile of the restriction kernels (coarse levels), rows x cols.
constexpr int kLevTY = 8, kLevTX = 64;

size_t fine_st_smem_bytes(int cfg, size_t pyr_elems, int elem_bytes);
template <class T>
cudaError_t prepare_fine_st(int pde, int cfg, size_t pyr_elems);
template <class T>
cudaError_t launch_fine_st(const Arena<T>& A, int pde, int cfg, int mode, size_t pyr_elems,
                           cudaStream_t s);
template <class T>
cudaError_t launch_level(const Arena<T>& A, int level, int mode, cudaStream_t s);
template <class T>
cudaError_t launch_finalize(const Arena<T>& A, int mode, cudaStream_t s);
template <class T>
cudaError_t launch_reset(const Arena<T>& A, cudaStream_t s);

}  // namespace modil
