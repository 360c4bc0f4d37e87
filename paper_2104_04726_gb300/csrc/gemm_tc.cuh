// Tensor-core (tcgen05 + TMA) GEMM over the descriptor of gemm.cuh.
#pragma once

#include "gemm.cuh"

namespace mes {

// kind: 0 = kind::tf32 on FP32 operands, 1 = kind::f16 on BF16 operands,
// 2 = three-term TF32 split (g.A/g.B the high parts, g.A2/g.B2 the low parts,
// all TF32-exact; FP32-level accuracy).
// True when both operands are K-major and satisfy the TMA alignment rules.
bool tc_eligible(const Gemm& g, int kind);
// split_ws (nullable) holds FP32 split-K partial tiles; err receives bit
// flags when a bounded pipeline wait gives up.
mes_status gemm_tc(const Gemm& g, int kind, float* split_ws, int64_t split_ws_elems, int* err,
                   cudaStream_t st);

}  // namespace mes
