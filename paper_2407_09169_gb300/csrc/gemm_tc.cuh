// Tensor-core (tcgen05) GEMM of the reduced-precision contraction forms.
#pragma once

#include "kernels.cuh"

namespace qtt {

enum TcMode { TC_BF16X3 = 0, TC_TF32 = 1, TC_TF32X3 = 2, TC_BF16 = 3 };

// Packed K-major operand buffers of one product.
struct TcPacked {
  void *a0 = nullptr, *a1 = nullptr, *b0 = nullptr, *b1 = nullptr;
  int m_pad = 0, n_pad = 0, k_pad = 0;
};

// Bytes of packing workspace gemm_tc needs for this product.
size_t tc_workspace_bytes(int M, int N, int K, long long batch, int mode);

// Same contract as gemm_f64 (FP64 views in and out), computed on the tensor
// cores in the given mode with FP32 accumulation.  max_kb_per_split > 0 caps
// the k-blocks one accumulator sums (the rest is summed in FP64 by the split-K
// reduction).  Returns false (launching
// nothing) when the product does not fit the packing workspace or the grid
// limits; *err receives nonzero bits when a bounded wait gives up.
bool gemm_tc(cudaStream_t st, int mode, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
             double beta, OutView C, void* pack_ws, size_t pack_bytes, double* ws, size_t ws_elems, int* err,
             int max_kb_per_split = 0);

}  // namespace qtt
