// Host interface of the tcgen05 BF16 GEMM (tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace modil_tc {

enum GemmMode { GEMM_STORE_BF16 = 0, GEMM_STORE_F32 = 1, GEMM_ATOMIC_F32 = 2, GEMM_STORE_BF16_MASK = 3 };

struct GemmArgs {
  int M, N, K;        // D is M x N, the contraction runs over K
  int kchunks;        // 64-wide K chunks per split (blockIdx.z)
  int mode;           // GemmMode
  int relu;           // BF16 store: max(x, 0) after the bias
  const float* bias;  // N values or nullptr (store modes)
  void* D;            // row-major output, ldd elements per row
  int ldd;
  int* err;           // device word: set non-zero when a wait timed out
  // BF16_MASK store: D = (act > 0 ? acc : 0) as BF16, act row-major like D
  const void* act;
  // Implicit 3x3x3 convolution (conv == 1): A is a 5-D activation map
  // (channels, x, y, z, sample) of S^3-voxel samples, a tile of 128 output
  // voxels its box; K chunk i is tap i / cc, channels 64 (i % cc) ..; the A box
  // sits at voxel + sign * tap offset (zero outside the grid).  B is a 3-D
  // weight map: b_tap_mid ? (channels, tap, row) : (channels, row, tap).
  int conv, S, cc, sign, b_tap_mid;
  // Its weight gradient (conv == 2): blockIdx.z = tap * wsplits + split; A is
  // the 4-D map (x and y flattened, z, sample, row) of three x-shifted
  // transposed copies of the input (row = (dx + 1) * wC + channel), a K chunk
  // 64 voxels; B the 2-D map of the transposed output gradient; D rows
  // tap * wC + channel (M = wC).
  int wsplits, wC;
};

// Tensor map of BF16 activations [B][S][S][S][C] (channels innermost) in
// boxes of 64 channels x 128 voxels (x fastest; 128B swizzle; channels past C
// and voxels outside the grid read as zero).  C % 8 == 0, S >= 8.  0 on success.
int make_act_map(CUtensorMap* m, const void* base, int C, int S, int B);

// Tensor map of three x-shifted transposed copies of BF16 activations,
// [3 C][B][S][S][S] (x innermost), x and y flattened into one axis, in boxes
// of 64 voxels x 128 rows (128B swizzle; voxels off the y range of a plane and
// rows past 3 C read as zero).  S >= 8.  0 on success.
int make_shift3_map(CUtensorMap* m, const void* base, int C, int S, int B);

// Tensor map of a BF16 3-D array (d0 innermost, strides in elements) in boxes
// of 64 x b1 x b2 (128B swizzle; reads past d0 are zero).  0 on success.
int make_3d_map(CUtensorMap* m, const void* base, long long d0, long long d1, long long d2, long long s1,
                long long s2, int b1, int b2);

// Tensor map of a row-major BF16 matrix (rows x k used, row pitch ld
// elements) in 64-column tiles of box_rows rows.  0 on success.
int make_kmajor_map(CUtensorMap* m, const void* base, long long rows, long long k, long long ld, int box_rows);

// Sets the kernels' shared-memory attributes (once per process) so that later
// launches, also inside a stream capture, make no attribute calls.
cudaError_t prepare_gemm();

// D (+)= A B^T with A: M x K map (box 128 rows), B: N x K map (box bn rows);
// bn in {16, 32, 64, 128, 256}; splits = gridDim.z (K split).
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int bn, int splits,
                        cudaStream_t s);

}  // namespace modil_tc
