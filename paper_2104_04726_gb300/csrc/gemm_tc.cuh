// Tensor-core (tcgen05 + TMA) GEMM over the descriptor of gemm.cuh.
#pragma once

#include "gemm.cuh"

namespace mes {

// kind: 0 = kind::tf32 on FP32 operands, 1 = kind::f16 on BF16 operands,
// 2 = three-term TF32 split (g.A/g.B the high parts, g.A2/g.B2 the low parts,
// all TF32-exact; FP32-level accuracy), 3 = six-term BF16 split (each operand
// as three BF16 parts in K_hi planes: g.K_hi = 3, g.a_kh / g.b_kh the part
// strides, from split_bf16x3; FP32-level accuracy; no residual, accumulate).
// True when both operands are K-major and satisfy the TMA alignment rules.
bool tc_eligible(const Gemm& g, int kind);
// split_ws (nullable) holds FP32 split-K partial tiles; err receives bit
// flags when a bounded pipeline wait gives up.
mes_status gemm_tc(const Gemm& g, int kind, float* split_ws, int64_t split_ws_elems, int* err,
                   cudaStream_t st);
// out[i], out[plane + i], out[2 plane + i] = the three BF16 parts of in[i]
// (x = x1 + x2 + x3 to ~2^-24 relative); a no-op when *skip != 0.
mes_status split_bf16x3(const float* in, uint16_t* out, int64_t n, int64_t plane, const int* skip,
                        cudaStream_t st);

}  // namespace mes
