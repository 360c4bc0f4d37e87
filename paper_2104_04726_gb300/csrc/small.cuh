// Declarations of the bandwidth and small-solver kernels used by the driver.
#pragma once

#include "common.cuh"

namespace mes {

// A set of fibres over the trailing small modes: fibre f = f_lo + F_lo*f_hi,
// element l of fibre f at in + f_lo*in_lo + f_hi*in_hi + l*in_l (and the
// same for `out` with its own strides).
struct Fibres {
  int64_t F_lo = 1, F_hi = 1;
  const float* in = nullptr;
  int64_t in_lo = 0, in_hi = 0, in_l = 0;
  float* out = nullptr;
  int64_t out_lo = 0, out_hi = 0, out_l = 0;
};

// Kronecker product of per-mode small matrices.  op: 'T' = U^T (r x s),
// 'N' = U (s x r), 'I' = identity (s x s).  Row index and column index are
// multi-indices with the first small mode fastest.  K is row-major (rows x cols).
struct KronDesc {
  int nm = 0;
  const float* U[6] = {nullptr};
  int s[6] = {0};
  int r[6] = {0};
  char op[6] = {0};
  int rows() const;
  int cols() const;
};
mes_status kron_build(const KronDesc& d, float* K, const int* skip, cudaStream_t st);

// XB = per-slice transpose of X (and ||X||^2 partials); with `round`, XB and
// the optional copy Xr hold X rounded to TF32.  X16 / XB16 (nullable)
// receive X and its per-slice transpose rounded to BF16.  XB is nullable.
mes_status slice_transpose(const float* X, int64_t s1, int64_t s2, int64_t L, float* XB,
                           double* partials, int nblocks, cudaStream_t st, float* Xr = nullptr,
                           bool round = false, uint16_t* X16 = nullptr, uint16_t* XB16 = nullptr);
// hi = round_tf32(in), lo = round_tf32(in - hi): the two terms of the
// three-term TF32 tensor-core product (x = hi + lo to ~2^-22 relative)
mes_status split_tf32(const float* in, float* hi, float* lo, int64_t n, cudaStream_t st, const int* skip = nullptr);
// out = bits of round_bf16(in), elementwise; a no-op when *skip != 0
mes_status to_bf16(const float* in, uint16_t* out, int64_t n, const int* skip, cudaStream_t st);
// out = round_tf32(in), elementwise
mes_status round_copy(const float* in, float* out, int64_t n, const int* skip, cudaStream_t st);
// out = in, elementwise; a no-op when *skip != 0
mes_status copy_if(const float* in, float* out, int64_t n, const int* skip, cudaStream_t st);
// U (s x r, column-major) = the first r columns of the identity
mes_status identity_fill(float* U, int64_t s, int r, cudaStream_t st);
mes_status sumsq(const float* x, int64_t n, double* partials, int nblocks, const int* skip,
                 cudaStream_t st);
mes_status uniform_fill(float* out, int64_t n, uint64_t seed, cudaStream_t st);
mes_status mix_fibres(const Fibres& fb, const float* Kmat, int L, int L2, const int* skip,
                      cudaStream_t st);
int small_gram_blocks(int64_t F);
mes_status small_gram(const Fibres& fb, const float* Kmat, int L, int L2, int sn, int inner,
                      double* partials, double* G, const int* skip, cudaStream_t st);
mes_status fit_flag(const double* normX, const double* normQ, int sweep, double tol, double* hist,
                    double* last, int* done, int* iters, cudaStream_t st);
mes_status final_fit(const double* normX, const double* sse, double* fit, cudaStream_t st);
// status (nullable device int) = MES_OK, MES_ERR_TIMEOUT (pipeline wait
// bits in flags[0]) or MES_ERR_NONFINITE (||T||^2 or fit not finite); the
// fit (nullable) becomes NaN on failure
mes_status finish_status(const int* flags, const double* normX, double* fit, int* status, cudaStream_t st);
// *x = NaN when flags[0] holds a pipeline-wait bit (x: an FP64 result such as a residual)
mes_status nan_on_timeout(const int* flags, double* x, cudaStream_t st);
mes_status col_signs(const float* U, int64_t s, int r, float* sign, cudaStream_t st);
mes_status diag_order(const float* H, int r, int* src_of, cudaStream_t st);
mes_status permute_cols(const float* Uin, int64_t s, int r, const int* src_of, const float* sign,
                        float* Uout, cudaStream_t st);
mes_status permute_core(const float* in, int64_t total, int64_t stride, int r, const int* src_of,
                        const float* sign, float* out, cudaStream_t st);

// dense.cu
// Shifted Cholesky of an r x r Gram: L, dinv and the inverses of the 32 x 32
// diagonal blocks of L (Linv_blk: ceil(r/32) row-major 32 x 32 blocks), and
// the right-side solve V = W D^-1 L^-T that completes one CholeskyQR pass.
// clean (nullable device int) receives 1 when the factorization kept its
// starting shift (or was skipped), 0 when a bad pivot forced a larger one.
mes_status chol(const float* M, int r, float shift_rel, float* L, float* dinv, float* Linv_blk, int* flags,
                const int* skip, cudaStream_t st, int* clean = nullptr);
mes_status trsm(const float* W, int64_t s, int r, const float* L, const float* dinv, const float* Linv_blk,
                float* V, bool round, const int* skip, cudaStream_t st);
mes_status eig_small(const double* G, int n, int r, float* U, double* evals, const int* skip,
                     cudaStream_t st);
mes_status eig_mid(const float* H, int r, float* Z, const int* skip, cudaStream_t st);
// One refinement step of approximate eigenvectors X of a symmetric A from
// G = X^T X and S = X^T A X: E with X (I + E) the refined vectors (r x r,
// column-major).
mes_status rr_update(const float* S, const float* G, int r, float* E, cudaStream_t st);

// colour.cu / quant.cu
mes_status colour_launch(const uint8_t* rgb8, int64_t s1, int64_t s2, int64_t K, int space,
                         float gamma, float* out, double* partials, double* norm2, cudaStream_t st);
unsigned colour_grid(int64_t npix, int64_t K);
// Validated plane geometry of the quantiser (plane_size = r1 r2, planes =
// prod_{n>=3} r_n <= max_planes), without int64 overflow.
mes_status quant_plane_shape(int N, const int64_t* ranks, int64_t max_planes, int64_t* plane_size,
                             int64_t* planes, const char* who);
mes_status quantize_launch(const float* core, int64_t plane_size, int64_t planes, int bits,
                           int16_t* q, float* scales, unsigned* maxbits, cudaStream_t st);

}  // namespace mes
