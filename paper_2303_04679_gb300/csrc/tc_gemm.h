// Host interface of the tcgen05 BF16 GEMM (tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace modil_tc {

enum GemmMode { GEMM_STORE_BF16 = 0, GEMM_STORE_F32 = 1, GEMM_ATOMIC_F32 = 2 };

struct GemmArgs {
  int M, N, K;        // D is M x N, the contraction runs over K
  int kchunks;        // 64-wide K chunks per split (blockIdx.z)
  int mode;           // GemmMode
  int relu;           // BF16 store: max(x, 0) after the bias
  const float* bias;  // N values or nullptr (store modes)
  void* D;            // row-major output, ldd elements per row
  int ldd;
  int* err;           // device word: set non-zero when a wait timed out
};

// Tensor map of a row-major BF16 matrix (rows x k used, row pitch ld
// elements) in 64-column tiles of box_rows rows.  0 on success.
int make_kmajor_map(CUtensorMap* m, const void* base, long long rows, long long k, long long ld, int box_rows);

// D (+)= A B^T with A: M x K map (box 128 rows), B: N x K map (box bn rows);
// bn in {16, 32, 64, 128, 256}; splits = gridDim.z (K split).
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int bn, int splits,
                        cudaStream_t s);

}  // namespace modil_tc
