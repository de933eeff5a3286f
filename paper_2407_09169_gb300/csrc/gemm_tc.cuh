// Tensor-core (tcgen05) GEMM of the reduced-precision contraction forms.
#pragma once

#include "kernels.cuh"

namespace qtt {

// BF16X6: exact 8-bit integer slices of row-scaled operands (3 x 3 slices,
// 6 slice products), exact FP32 accumulation per chunk of K, FP64 combination
// -- unbiased, ~2^-24 relative to the row and column maxima.  BF16X3 / TF32 /
// TF32X3 / BF16: floating-point operands (hi+lo 3-pass, 1-pass, hi+lo 3-pass,
// 1-pass) accumulated by the tensor cores in FP32, which rounds toward zero.
// BF16X10: 4 x 4 exact slices taken from the FP64 mantissa by integer
// arithmetic (each element to 2^-31 of its row's largest power of two), the
// 10 slice products of weight >= 2^-30 in four exact accumulators, ~2^-31
// relative to the row and column maxima.
enum TcMode { TC_BF16X3 = 0, TC_TF32 = 1, TC_TF32X3 = 2, TC_BF16 = 3, TC_BF16X6 = 4, TC_BF16X10 = 5 };

// Packed K-major operand buffers of one product.
struct TcPacked {
  void* a[4] = {nullptr, nullptr, nullptr, nullptr};
  void* b[4] = {nullptr, nullptr, nullptr, nullptr};
  int* ea = nullptr;  // per-row power-of-two exponents (sliced modes)
  int* eb = nullptr;
  int m_pad = 0, n_pad = 0, k_pad = 0;
};

// Bytes of packing workspace gemm_tc needs for this product.
size_t tc_workspace_bytes(int M, int N, int K, long long batch, int mode);

// Same contract as gemm_f64 (FP64 views in and out), computed on the tensor
// cores in the given mode.  max_kb_per_split > 0 caps the k-blocks (of 128
// bytes) one accumulator sums; the chunks are summed in FP64 by the split-K
// reduction.  Returns false (launching nothing) when the product does not fit
// the packing workspace, the FP64 split-K workspace (exact-slice modes) or the
// grid limits; *err receives nonzero bits when a bounded wait gives up.
bool gemm_tc(cudaStream_t st, int mode, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
             double beta, OutView C, void* pack_ws, size_t pack_bytes, double* ws, size_t ws_elems, int* err,
             int max_kb_per_split = 0);

}  // namespace qtt
