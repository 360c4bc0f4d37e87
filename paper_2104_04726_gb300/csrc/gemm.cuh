// Descriptor of a batched strided product C(m, n) = alpha * sum_k A(m, k) B(n, k)
// (+ C(m, n) when accumulate).  Every tensor contraction of the Tucker-ALS
// sweep is written as one of these, with layouts chosen so that no transpose
// pass is needed:
//
//   A(m, k) at A + m*a_m + k_lo*a_k + k_hi*a_kh + b*a_b,  k = k_lo + K_lo*k_hi
//   B(n, k) at B + n*b_n + k_lo*b_k + k_hi*b_kh + b*b_b
//   C(m, n) at C + m_lo*c_m + m_hi*c_mh + n_lo*c_n + n_hi*c_nh + b*c_b,
//            m = m_lo + M_lo*m_hi,  n = n_lo + N_lo*n_hi
#pragma once

#include <cstdint>

#include "common.cuh"

namespace mes {

struct Gemm {
  int64_t M = 0, N = 0, K_lo = 0, K_hi = 1;
  int batch = 1;
  const float* A = nullptr;
  int64_t a_m = 0, a_k = 0, a_kh = 0, a_b = 0;
  const float* B = nullptr;
  int64_t b_n = 0, b_k = 0, b_kh = 0, b_b = 0;
  // low parts of A and B for the three-term TF32 tensor-core product (kind 2
  // of gemm_tc): A = A + A2 and B = B + B2, all four exactly TF32, same strides
  const float* A2 = nullptr;
  const float* B2 = nullptr;
  float* C = nullptr;
  int64_t M_lo = 0, c_m = 0, c_mh = 0, N_lo = 0, c_n = 0, c_nh = 0, c_b = 0;
  // optional second output (same values, another layout), strides as for C
  float* C2 = nullptr;
  int64_t c2_m = 0, c2_mh = 0, c2_n = 0, c2_nh = 0, c2_b = 0;
  float alpha = 1.f;
  bool accumulate = false;
  bool round_tf32 = false;        // store C (and C2) rounded to TF32 (operands of later kind::tf32 products)
  const int* skip = nullptr;      // device flag: when non-zero the launch is a no-op
  // C is symmetric and its consumer reads only m >= n: tiles wholly above the
  // diagonal are not computed (their elements of C are left as they were).
  bool lower = false;
  // Residual mode: accumulate sum((ref - alpha*AB)^2) in FP64 (and store
  // alpha*AB to C when C is given, without accumulate or rounding); ref is
  // addressed like C.  partials needs gemm_partials(g) doubles.
  const float* ref = nullptr;
  double* partials = nullptr;
  // Optional FP32 workspace for split-K (deterministic: partial tiles are
  // summed in a fixed order).  Used when the tile grid leaves most SMs idle.
  float* split_ws = nullptr;
  int64_t split_elems = 0;
  // Bound of each pipeline wait of the tensor-core kernel in ns (0: 2 s).
  uint64_t wait_ns = 0;
  // Tensor-core kinds 0 and 1 only, C with m contiguous (c_m == 1): also
  // write the three BF16 parts of every stored value (as split_bf16x3 makes
  // them) to Cp[part * cp_plane + offset of C], the operand of a six-term
  // product that follows.
  uint16_t* Cp = nullptr;
  int64_t cp_plane = 0;
  // CTA slots the split-K rule fills (0: the SM count).  A caller that runs
  // several decompositions side by side gives each a share, trading the
  // latency of one product for less SM time (partials, reduction pass).
  int64_t fill = 0;
};

// FP32 CUDA-core path.
mes_status gemm_f32(const Gemm& g, cudaStream_t st);
// Number of per-block partial sums the residual mode writes.
int64_t gemm_partials(const Gemm& g);
// Sums n doubles in a fixed order into *out (one block).
mes_status sum_doubles(const double* partials, int64_t n, double* out, const int* skip,
                       cudaStream_t st);

}  // namespace mes
