// Tucker-ALS / HOOI driver (Section III-B) and reconstruction (Eq. 1).
//
// Data layout.  The stack T (s1 x s2 x small modes) is first-mode fastest;
// l indexes the trailing small modes jointly (L = prod s_n, n >= 3).  A second
// copy XB has, per l, mode 2 fastest.  Intermediates:
//   P  [x][q2 + r2*l]      = T x_2 S2^T             (mode-1 partial contraction)
//   Ca [y][q1 + r1*l]      = T x_1 S1^T             (mode-2 partial contraction)
//   B  [q1 + r1*l + r1*L*q2] = Ca x_2 S2^T          (shared by the small modes)
// so every product below reads its operands along their contiguous index.
//
// Factor update of a large mode n (Eq. 8 and the text after it).  The paper
// takes S^(n) as the leading eigenvectors of G = Y_(n) Y_(n)^T.  Forming G in
// FP32 squares the condition number of Y_(n) and loses the trailing singular
// directions (their eigenvalues sit below the FP32 resolution of G at these
// sizes), so the Gram is applied in factored form: one step of block
// subspace iteration on G is
//     Z  = Y_(n)^T S          (the partial core),
//     Zh = Z R_z^-1           (R_z from a shifted Cholesky of Z^T Z: keeps the
//                              next product well conditioned),
//     W  = Y_(n) Zh           (= G S R_z^-1: same column space as G S),
//     S  = orth(W)            (shifted CholeskyQR, three passes),
// warm-started from the previous sweep's factor.  Repeated steps converge to
// the leading eigenvectors of G; the column space is what HOOI carries to the
// next mode, and the basis is made canonical at the end.
//
// Small modes (colour, view x exposure) use the paper's route literally: the
// Gram of the mode-n unfolding of Y^(n), accumulated in FP64, and its exact
// eigenvectors (FP64 Jacobi).
//
// Stopping (the paper is silent): after sweep t the fit
// 1 - sqrt(||T||^2 - ||Q||^2)/||T|| is compared with the previous one; a
// device flag set when |change| < tol turns every later sweep's kernels into
// no-ops, so the host enqueues max_iters sweeps without reading anything back.
// With tol = 0 (a fixed number of sweeps), no fit history asked for and every
// small mode at full rank, the per-sweep core and fit serve nothing and are
// formed in the last sweep only.
// The returned fit is recomputed from the explicit residual ||T - T_hat||,
// which does not suffer the cancellation of ||T||^2 - ||Q||^2 in FP32.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "gemm.cuh"
#include "gemm_tc.cuh"
#include "small.cuh"

namespace {

using mes::Gemm;
using mes::Fibres;
using mes::KronDesc;

// Starting relative shifts of the Z-preconditioning Cholesky and of the
// first CholeskyQR pass (the Cholesky kernel raises them on breakdown).
constexpr float kShiftZ = 1e-5f;
constexpr float kShiftW = 1e-5f;
// Refinement steps of the Rayleigh-Ritz rotation for ranks above 128.
constexpr int kRRSteps = 3;

struct Shape {
  int N = 0;
  int64_t s[8] = {0}, r[8] = {0};
  int64_t s1 = 1, s2 = 1, r1 = 1, r2 = 1;
  int nsm = 0;
  int64_t L = 1, Lr = 1;
  bool small_full = true;
};

mes_status make_shape(int N, const int64_t* dims, const int64_t* ranks, Shape* sh, const char* who) {
  if (N < 2 || N > 8) return mes::fail(MES_ERR_INVALID_ARG, "%s: N must be 2..8 (got %d)", who, N);
  if (!dims || !ranks) return mes::fail(MES_ERR_INVALID_ARG, "%s: null dims or ranks", who);
  sh->N = N;
  for (int n = 0; n < N; ++n) {
    sh->s[n] = dims[n];
    sh->r[n] = ranks[n];
    if (dims[n] < 1) return mes::fail(MES_ERR_INVALID_ARG, "%s: dims[%d] < 1", who, n);
    if (ranks[n] < 1 || ranks[n] > dims[n])
      return mes::fail(MES_ERR_RANK, "%s: ranks[%d]=%lld outside 1..%lld", who, n, (long long)ranks[n],
                       (long long)dims[n]);
  }
  for (int n = 0; n < N; ++n) {
    double prod = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) prod *= (double)ranks[m];
    if ((double)ranks[n] > prod)
      return mes::fail(MES_ERR_RANK, "%s: ranks[%d] exceeds the product of the other ranks", who, n);
  }
  sh->s1 = dims[0];
  sh->s2 = dims[1];
  sh->r1 = ranks[0];
  sh->r2 = ranks[1];
  sh->nsm = N - 2;
  sh->L = 1;
  sh->Lr = 1;
  sh->small_full = true;
  for (int n = 2; n < N; ++n) {
    if (dims[n] > 32) return mes::fail(MES_ERR_INVALID_ARG, "%s: modes 3..N must have size <= 32", who);
    sh->L *= dims[n];
    sh->Lr *= ranks[n];
    if (ranks[n] != dims[n]) sh->small_full = false;
  }
  if (sh->L > 1024) return mes::fail(MES_ERR_INVALID_ARG, "%s: product of modes 3..N above 1024", who);
  if (sh->L * sh->L > 16384)
    return mes::fail(MES_ERR_NOT_IMPLEMENTED, "%s: product of modes 3..N above 128", who);
  if (sh->r1 > 1024 || sh->r2 > 1024)
    return mes::fail(MES_ERR_NOT_IMPLEMENTED, "%s: ranks of modes 1, 2 above 1024", who);
  return MES_OK;
}

Gemm base() { return Gemm(); }

struct Driver {
  Shape sh;
  cudaStream_t st;
  mes::Scratch* scr;
  const int* skip = nullptr;       // device stop flag, null outside the sweeps
  int* flags = nullptr;            // numerics flags (Cholesky pivots, pipeline waits)
  int* clean = nullptr;            // 1 when the last fast CholeskyQR pass kept its shift

  float *cwA = nullptr, *cwX = nullptr, *H = nullptr, *Rinv = nullptr;
  float* dinv = nullptr;                    // equilibration of chol
  float* linv = nullptr;                    // inverted diagonal blocks of L
  float *W = nullptr, *W2 = nullptr, *Z = nullptr, *Zh = nullptr, *Kmat = nullptr;
  double *gpart = nullptr, *G64 = nullptr;

  int prec = MES_PREC_FP32;
  uint64_t wait_ns = 0;                     // bound of the tensor-core pipeline waits (0: default)
  int64_t fill = 0;                         // CTA slots for split-K (0: all SMs)
  float* split_ws = nullptr;
  int64_t split_elems = 0;
  uint16_t* Zh16 = nullptr;                 // BF16 copy of Zh (BF16 form, T-side steps)
  uint16_t* gparts = nullptr;               // three BF16 parts of a Gram operand (tensor-core forms)

  // tensor-core forms: operands of the Y-side products stored TF32-rounded
  bool tc() const { return prec != MES_PREC_FP32; }

  // precision-critical products (Grams of the factor update): FP32 CUDA cores
  mes_status gemm(const Gemm& g) {
    Gemm h = g;
    h.skip = skip;
    h.fill = fill;
    h.split_ws = split_ws;
    h.split_elems = split_elems;
    return mes::gemm_f32(h, st);
  }

  // the large contractions: tensor cores in the TF32 form when the operands
  // are K-major and TMA-addressable, CUDA cores otherwise
  mes_status big(const Gemm& g) {
    Gemm h = g;
    h.skip = skip;
    h.wait_ns = wait_ns;
    h.fill = fill;
    if (tc() && mes::tc_eligible(h, 0))
      return mes::gemm_tc(h, 0, split_ws, split_elems, flags, st);
    h.split_ws = split_ws;
    h.split_elems = split_elems;
    return mes::gemm_f32(h, st);
  }

  // a T-side product of the BF16 form: both operands BF16 (kind::f16),
  // FP32 accumulation; the caller guarantees TMA eligibility
  mes_status big16(const Gemm& g) {
    Gemm h = g;
    h.skip = skip;
    h.wait_ns = wait_ns;
    h.fill = fill;
    return mes::gemm_tc(h, 1, split_ws, split_elems, flags, st);
  }

  // same, with an explicit skip flag (e.g. the conditional second pass of orth)
  mes_status gemm_if(const Gemm& g, const int* skipf) {
    Gemm h = g;
    h.skip = skipf;
    h.fill = fill;
    h.split_ws = split_ws;
    h.split_elems = split_elems;
    return mes::gemm_f32(h, st);
  }

  // H = A^T A for a column-major s x r matrix A (the Grams of the factor
  // update); chol reads the lower triangle.  They need FP32-level accuracy
  // (Z^T Z feeds a Cholesky of condition up to ~1e8; the three-term TF32
  // product, ~12 ulp per term, failed the rank-520-of-600 scene).  The
  // tensor-core forms run the six-term BF16 split (A as three BF16 parts,
  // 24 significant bits, every part product down to 2^-16 of the leading
  // one: ~3 ulp per term) on the tensor cores; the FP32 form, and operands
  // whose rows TMA cannot address, run FP32 on CUDA cores.
  // True when gram(A, s, r) runs on the tensor cores, so the product that
  // makes A can write its BF16 parts to gparts (Gemm::Cp) instead of a split
  // pass over A.
  bool gram_tc(int64_t s) const { return tc() && gparts && s % 8 == 0; }

  // parts_ready: A's three BF16 parts are already in gparts (written by the
  // product that made A)
  mes_status gram(const float* A, int64_t s, int64_t r, const int* skipf, bool parts_ready = false) {
    if (gram_tc(s)) {
      Gemm t = base();
      t.M = r; t.N = r; t.K_lo = s; t.K_hi = 3;
      t.A = reinterpret_cast<const float*>(gparts); t.a_m = s; t.a_k = 1; t.a_kh = s * r;
      t.B = t.A; t.b_n = s; t.b_k = 1; t.b_kh = s * r;
      t.C = H; t.c_m = 1; t.c_n = r;
      t.lower = true;
      t.skip = skipf;
      t.wait_ns = wait_ns;
      // four times the concurrency share: un-split, a few CTAs stream all of
      // K (145 us for K = 7680 on six CTAs); four splits take about the same
      // SM time at a quarter of the latency, on the decomposition's chain
      t.fill = fill > 0 ? 4 * fill : 0;
      if (mes::tc_eligible(t, 3)) {
        if (!parts_ready) MES_TRY(mes::split_bf16x3(A, gparts, s * r, s * r, skipf, st));
        return mes::gemm_tc(t, 3, split_ws, split_elems, flags, st);
      }
      if (parts_ready) return mes::fail(MES_ERR_INVALID_ARG, "gram: parts written for an ineligible Gram");
    }
    Gemm g = base();
    g.M = r; g.N = r; g.K_lo = s;
    g.A = A; g.a_m = s; g.a_k = 1;
    g.B = A; g.b_n = s; g.b_k = 1;
    g.C = H; g.c_m = 1; g.c_n = r;
    g.lower = true;
    return gemm_if(g, skipf);
  }

  // One CholeskyQR pass dst = src R^-1 with R^T R = src^T src (equilibrated,
  // starting shift `shift`); every kernel is a no-op when *skipf != 0.
  mes_status cholqr_pass(const float* src, int64_t s, int64_t r, float shift, float* dst, const int* skipf,
                         int* clean, bool parts_ready = false) {
    MES_TRY(gram(src, s, r, skipf, parts_ready));
    MES_TRY(mes::chol(H, (int)r, shift, cwA, dinv, linv, flags, skipf, st, clean));
    return mes::trsm(src, s, (int)r, cwA, dinv, linv, dst, false, skipf, st);
  }

  // S (s x r) := orth(W); in the TF32 form Srnd receives S rounded to TF32
  // (the tensor-core operand).
  //  robust: three passes of CholeskyQR, the first shifted: any start (the
  //          random block of the initialisation, the first subspace steps).
  //  fast:   one unshifted pass, and a second one only when that pass had to
  //          raise its shift (a device flag decides, nothing is read back).
  //          Inside the sweeps W arrives preconditioned by Z^T Z (subspace
  //          step below) with an equilibrated condition number of a few
  //          units, where one pass is orthonormal to FP32 precision.
  // parts_ready: Win's BF16 parts are in gparts (see gram)
  mes_status orth(float* Win, int64_t s, int64_t r, float* Sout, float* Srnd, bool robust, bool parts_ready = false) {
    if (robust) {
      float* src = Win;
      float* bufs[2] = {W2, Win};
      for (int pass = 0; pass < 3; ++pass) {
        float* dst = (pass == 2) ? Sout : bufs[pass & 1];
        MES_TRY(cholqr_pass(src, s, r, pass == 0 ? kShiftW : 0.f, dst, skip, nullptr, pass == 0 && parts_ready));
        src = dst;
      }
    } else {
      MES_TRY(cholqr_pass(Win, s, r, 0.f, Sout, skip, clean, parts_ready));
      MES_TRY(cholqr_pass(Sout, s, r, 0.f, Win, clean, nullptr));   // only if pass 1 restarted
      MES_TRY(mes::copy_if(Win, Sout, s * r, clean, st));
    }
    if (tc() && Srnd) MES_TRY(mes::round_copy(Sout, Srnd, s * r, skip, st));
    return MES_OK;
  }

  // One subspace step for a large mode: Y is given through two GEMM operand
  // descriptions (Yt: Z = Y^T S,  Yn: W = Y Zh), J = number of columns of Y_(n).
  // In the BF16 form, z16 / w16 (nullable) describe the same products with
  // Y = T in BF16: then S16 is the BF16 copy of S (read by Z = Y^T S and
  // refreshed after the update) and Zh goes through a BF16 copy.
  mes_status subspace_step(const Gemm& zdesc, const Gemm& wdesc, int64_t J, int64_t s, int64_t r,
                           float* S, float* Srnd, bool robust, const Gemm* z16 = nullptr,
                           const Gemm* w16 = nullptr, uint16_t* S16 = nullptr) {
    // Z = Y^T S   (J x r, stored Z[j + J*q])
    Gemm gz = z16 ? *z16 : zdesc;
    gz.B = z16 ? reinterpret_cast<const float*>(S16) : (tc() ? Srnd : S); gz.b_n = s; gz.b_k = 1;
    gz.C = Z; gz.c_m = 1; gz.c_n = J;
    // the Gram's BF16 parts straight from the product's epilogue
    const bool zparts = gram_tc(J) && (z16 || mes::tc_eligible(gz, 0));
    if (zparts) { gz.Cp = gparts; gz.cp_plane = J * r; }
    MES_TRY(z16 ? big16(gz) : big(gz));
    // H = Z^T Z, R_z, Zh = Z R_z^-1
    MES_TRY(gram(Z, J, r, skip, zparts));
    MES_TRY(mes::chol(H, (int)r, kShiftZ, cwA, dinv, linv, flags, skip, st));
    // Zh = Z R_z^-1, an operand of the next product: TF32-rounded in those forms
    MES_TRY(mes::trsm(Z, J, (int)r, cwA, dinv, linv, Zh, tc(), skip, st));
    // W = Y Zh   (s x r)
    Gemm gw = w16 ? *w16 : wdesc;
    gw.C = W; gw.c_m = 1; gw.c_n = s;
    bool wparts = false;
    if (w16) {
      MES_TRY(mes::to_bf16(Zh, Zh16, J * r, skip, st));
      gw.B = reinterpret_cast<const float*>(Zh16);
      wparts = gram_tc(s);
      if (wparts) { gw.Cp = gparts; gw.cp_plane = s * r; }
      MES_TRY(big16(gw));
    } else {
      wparts = gram_tc(s) && mes::tc_eligible(gw, 0);
      if (wparts) { gw.Cp = gparts; gw.cp_plane = s * r; }
      MES_TRY(big(gw));
    }
    MES_TRY(orth(W, s, r, S, Srnd, robust, wparts));
    if (S16) MES_TRY(mes::to_bf16(S, S16, s * r, skip, st));
    return MES_OK;
  }

  // Small-mode Gram (FP64) of fibres projected by the Kronecker matrix built
  // from `kd`, then its leading eigenvectors into U (s_n x r_n).
  mes_status small_update(const Fibres& fb, const KronDesc& kd, int which, float* U) {
    MES_TRY(mes::kron_build(kd, Kmat, skip, st));
    int inner = 1;
    for (int m = 0; m < which; ++m) inner *= (kd.op[m] == 'T') ? kd.r[m] : kd.s[m];
    const int sn = kd.s[which];
    MES_TRY(mes::small_gram(fb, Kmat, kd.cols(), kd.rows(), sn, inner, gpart, G64, skip, st));
    return mes::eig_small(G64, sn, kd.r[which], U, nullptr, skip, st);
  }
};

// Reconstruction T_hat = Q x_1 S1 x_2 S2 x_{n>=3} S_n (Eq. 1): the small
// modes by fibre mixing, then mode 2, then mode 1 with an optional fused
// residual against `ref`.  Every workspace request comes before the first
// launch, so with a dry Scratch the call only counts bytes (no pointer is
// read).
mes_status mes_reconstruct_impl(const Shape& sh, const float* core, const float* const* fac, float* out,
                                const float* ref, double* sse, mes::Scratch& scr, float* T1, float* T2,
                                float* Kmat, cudaStream_t st, int prec = MES_PREC_FP32, int* err = nullptr,
                                uint64_t wait_ns = 0) {
  const int64_t s1 = sh.s1, s2 = sh.s2, r1 = sh.r1, r2 = sh.r2, L = sh.L, Lr = sh.Lr;
  auto small_modes = [&](float* dst) -> mes_status {   // T1[q2 + r2 q1 + r1 r2 l] = Q x_{n>=3} S_n
    KronDesc kd;
    kd.nm = sh.nsm;
    for (int m = 0; m < sh.nsm; ++m) {
      kd.s[m] = (int)sh.s[m + 2]; kd.r[m] = (int)sh.r[m + 2]; kd.op[m] = 'N'; kd.U[m] = fac[m + 2];
    }
    MES_TRY(mes::kron_build(kd, Kmat, nullptr, st));
    Fibres fb;
    fb.F_lo = r1; fb.F_hi = r2;
    fb.in = core; fb.in_lo = 1; fb.in_hi = r1; fb.in_l = r1 * r2;
    fb.out = dst; fb.out_lo = r2; fb.out_hi = 1; fb.out_l = r1 * r2;
    return mes::mix_fibres(fb, Kmat, (int)Lr, (int)L, nullptr, st);
  };
  if (prec != MES_PREC_FP32 && r1 % 4 == 0 && r2 % 4 == 0) {
    // tensor-core form: the same two products with K-major operands (the
    // factors transposed to rank-fastest copies), every operand split into
    // two TF32 terms and multiplied by the three-term product, which keeps
    // FP32-level accuracy: a plain TF32 product would add ~1e-3 relative
    // error to every entry of T_hat, more than the residual being measured
    float *U0t = nullptr, *U1t = nullptr, *U0h = nullptr, *U0l = nullptr, *U1h = nullptr, *U1l = nullptr;
    float *T1h = nullptr, *T1l = nullptr, *T2h = nullptr, *T2l = nullptr;
    MES_TRY(scr.alloc(&U0t, s1 * r1));
    MES_TRY(scr.alloc(&U1t, s2 * r2));
    MES_TRY(scr.alloc(&U0h, s1 * r1));
    MES_TRY(scr.alloc(&U0l, s1 * r1));
    MES_TRY(scr.alloc(&U1h, s2 * r2));
    MES_TRY(scr.alloc(&U1l, s2 * r2));
    MES_TRY(scr.alloc(&T1h, r1 * r2 * L));
    MES_TRY(scr.alloc(&T1l, r1 * r2 * L));
    MES_TRY(scr.alloc(&T2h, r1 * s2 * L));
    MES_TRY(scr.alloc(&T2l, r1 * s2 * L));
    Gemm g = Gemm();   // T2[q1 + r1 y + r1 s2 l] = sum_q2 T1[q2 + r2 q1 + r1 r2 l] S2t[q2 + r2 y]
    g.M = r1; g.N = s2; g.K_lo = r2; g.batch = (int)L;
    g.A = T1h; g.A2 = T1l; g.a_m = r2; g.a_k = 1; g.a_b = r1 * r2;
    g.B = U1h; g.B2 = U1l; g.b_n = r2; g.b_k = 1; g.b_b = 0;
    g.C = T2; g.c_m = 1; g.c_n = r1; g.c_b = r1 * s2;
    Gemm h = Gemm();   // out[x + s1 n] = sum_q1 S1t[q1 + r1 x] T2[q1 + r1 n]
    h.M = s1; h.N = s2 * L; h.K_lo = r1;
    h.A = U0h; h.A2 = U0l; h.a_m = r1; h.a_k = 1;
    h.B = T2h; h.B2 = T2l; h.b_n = r1; h.b_k = 1;
    h.C = out; h.c_m = 1; h.c_n = s1;
    g.wait_ns = h.wait_ns = wait_ns;
    if (mes::tc_eligible(g, 2) && mes::tc_eligible(h, 2)) {
      double* part = nullptr;
      const int64_t np = mes::gemm_partials(h) * 2 + 16;   // TC tiles are 128 x 128 or 128 x 256
      if (ref && sse) MES_TRY(scr.alloc(&part, np));
      if (scr.dry) return MES_OK;
      MES_TRY(mes::slice_transpose(fac[0], s1, r1, 1, U0t, nullptr, 64, st));
      MES_TRY(mes::slice_transpose(fac[1], s2, r2, 1, U1t, nullptr, 64, st));
      MES_TRY(mes::split_tf32(U0t, U0h, U0l, s1 * r1, st));
      MES_TRY(mes::split_tf32(U1t, U1h, U1l, s2 * r2, st));
      MES_TRY(small_modes(T1));
      MES_TRY(mes::split_tf32(T1, T1h, T1l, r1 * r2 * L, st));
      MES_TRY(mes::gemm_tc(g, 2, nullptr, 0, err, st));
      MES_TRY(mes::split_tf32(T2, T2h, T2l, r1 * s2 * L, st));
      if (ref && sse) {
        // one pass stores the product (when out is given) and accumulates the residual
        MES_CUDA_TRY(cudaMemsetAsync(part, 0, np * sizeof(double), st));
        h.ref = ref;
        h.partials = part;
        MES_TRY(mes::gemm_tc(h, 2, nullptr, 0, err, st));
        MES_TRY(mes::sum_doubles(part, np, sse, nullptr, st));
      } else if (out) {
        MES_TRY(mes::gemm_tc(h, 2, nullptr, 0, err, st));
      }
      return MES_OK;
    }
  }
  // CUDA-core form.  T2[q1 + r1 y + r1 s2 l] = sum_q2 T1[q2 + r2 q1 + r1 r2 l] S2[y + s2 q2]
  Gemm g = Gemm();
  g.M = r1; g.N = s2; g.K_lo = r2; g.batch = (int)L;
  g.A = T1; g.a_m = r2; g.a_k = 1; g.a_b = r1 * r2;
  g.b_n = 1; g.b_k = s2; g.b_b = 0;
  g.C = T2; g.c_m = 1; g.c_n = r1; g.c_b = r1 * s2;
  // out[x + s1 n] = sum_q1 S1[x + s1 q1] T2[q1 + r1 n],  n = y + s2 l
  Gemm h = Gemm();
  h.M = s1; h.N = s2 * L; h.K_lo = r1;
  h.a_m = 1; h.a_k = s1;
  h.B = T2; h.b_n = r1; h.b_k = 1;
  h.C = out; h.c_m = 1; h.c_n = s1;
  double* part = nullptr;
  const int64_t np = mes::gemm_partials(h);
  if (ref && sse) MES_TRY(scr.alloc(&part, np));
  if (scr.dry) return MES_OK;
  g.B = fac[1];
  h.A = fac[0];
  MES_TRY(small_modes(T1));
  MES_TRY(mes::gemm_f32(g, st));
  if (ref && sse) {
    // one pass stores the product (when out is given) and accumulates the residual
    h.ref = ref;
    h.partials = part;
    MES_TRY(mes::gemm_f32(h, st));
    MES_TRY(mes::sum_doubles(part, np, sse, nullptr, st));
    return MES_OK;
  }
  return mes::gemm_f32(h, st);
}

}  // namespace

// The decomposition; with ws_bytes non-null only the workspace it would take
// from the stream-ordered allocator is computed (no pointer is used).
static mes_status tucker_als_impl(const float* X, int N, const int64_t* dims, const int64_t* ranks,
                                  int max_iters, double tol, float* core, float* const* factors,
                                  double* fit, const mes_als_opts* opts, void* stream, size_t* ws_bytes) {
  Shape sh;
  MES_TRY(make_shape(N, dims, ranks, &sh, "mes_tucker_als"));
  if (!ws_bytes) {
    if (!X || !core || !factors) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: null pointer");
    for (int n = 0; n < N; ++n)
      if (!factors[n]) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: factors[%d] is null", n);
  }
  if (max_iters < 1) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: max_iters must be >= 1");
  if (!(tol >= 0.0)) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: tol must be >= 0");
  mes_als_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const int precision = o.precision;
  if (precision != MES_PREC_FP32 && precision != MES_PREC_BF16 && precision != MES_PREC_TF32)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: unknown precision %d", precision);
  // Default subspace steps.  With three or more sweeps every update starts
  // from the previous sweep's factor, so the sweeps keep refining the
  // subspaces: 2 steps for the start and 1 per factor update reach the same
  // fixed point as exact HOOI (fit within 1e-6 of the FP64 oracle on the
  // 1024x768 scene after 20 sweeps).  A run of 1 or 2 sweeps is read after
  // so few updates that each must be close to the exact eigenvectors of Eq.
  // 6, 7 and 8: 24 and 12 steps (an FP64 emulation of this iteration put the
  // fit after 1 and 2 sweeps within 4e-6 of exact HOOI on the 64x48 and
  // 1024x768 scenes, against 1.5e-4 with 2 and 1).
  const bool few = max_iters <= 2;
  const int init_iters = o.init_iters > 0 ? o.init_iters : (few ? 24 : 2);
  const int inner_iters = o.inner_iters > 0 ? o.inner_iters : (few ? 12 : 1);
  const uint64_t seed = o.seed ? o.seed : 1;
  const bool canonical = o.canonical >= 0;
  if (o.init_iters < 0 || o.inner_iters < 0)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: negative iteration option");
  if (o.init != MES_INIT_THOSVD && o.init != MES_INIT_INTERLACED)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: unknown init %d", o.init);
  if (o.wait_ns < 0) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: wait_ns must be >= 0");
  if (o.concurrency < 0) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: concurrency must be >= 0");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::Trace trace(ws_bytes ? nullptr : "mes_tucker_als", st);
  mes::AuditScope audit_scope;
  if (!ws_bytes) {
    int64_t nX = 1, nQ = 1;
    for (int n = 0; n < N; ++n) { nX *= sh.s[n]; nQ *= sh.r[n]; }
    mes::audit_register(X, (size_t)nX * 4);
    mes::audit_register(core, (size_t)nQ * 4);
    for (int n = 0; n < N; ++n) mes::audit_register(factors[n], (size_t)(sh.s[n] * sh.r[n]) * 4);
    if (o.reconstruction) mes::audit_register(o.reconstruction, (size_t)nX * 4);
    if (o.status) mes::audit_register(o.status, sizeof(int));
  }
  mes::Scratch scr(st, ws_bytes != nullptr);
  Driver d;
  d.sh = sh;
  d.st = st;
  d.scr = &scr;
  d.wait_ns = (uint64_t)o.wait_ns;
  if (o.concurrency > 1) {
    // each decomposition's share of the SMs (at least 4 CTA slots)
    const int64_t share = mes::sm_count() / o.concurrency;
    d.fill = share > 4 ? share : 4;
  }

  const int64_t s1 = sh.s1, s2 = sh.s2, r1 = sh.r1, r2 = sh.r2, L = sh.L, Lr = sh.Lr;
  const int64_t rmax = r1 > r2 ? r1 : r2;
  const int64_t nel = s1 * s2 * L;
  const int64_t J0 = r2 * Lr, J1 = r1 * Lr;     // columns of Y^(1)_(1), Y^(2)_(2)
  int64_t zsz = s2 * L * r1;
  if (s1 * L * r2 > zsz) zsz = s1 * L * r2;
  if (r1 * r2 * Lr > zsz) zsz = r1 * r2 * Lr;

  float *XB = nullptr, *P = nullptr, *Ca = nullptr, *Bt = nullptr, *Y0 = nullptr, *Y1 = nullptr, *ctmp = nullptr;
  float *T1 = nullptr, *T2 = nullptr;
  double *normX = nullptr, *normQ = nullptr, *sse = nullptr, *xpart = nullptr, *qpart = nullptr, *fitlast = nullptr;
  int *done = nullptr, *flags = nullptr;
  float* sign = nullptr;
  int* order = nullptr;
  const int nblk = (int)mes::grid_for(nel, 256, (int64_t)mes::sm_count() * 4);
  float *Pt = nullptr, *Cat = nullptr, *Xr = nullptr, *Ur[2] = {nullptr, nullptr};
  // BF16 form: the T-side products (P, Ca and the T-HOSVD products, whose
  // operands are T and the factors) run on BF16 copies with FP32
  // accumulation; the Y-side products (Z, W, B) run as in the TF32 form.
  // BF16 rows must be 16-byte aligned for TMA (s1, s2 multiples of 8);
  // otherwise the TF32 form runs.
  const bool bf = precision == MES_PREC_BF16 && s1 % 8 == 0 && s2 % 8 == 0;
  const bool tf32 = precision != MES_PREC_FP32;   // tensor-core forms
  uint16_t *X16 = nullptr, *XB16 = nullptr, *U16[2] = {nullptr, nullptr};
  if (!bf) MES_TRY(scr.alloc(&XB, nel));
  if (tf32) {
    // operands of the kind::tf32 products, pre-rounded to nearest TF32
    MES_TRY(scr.alloc(&Xr, nel));
    MES_TRY(scr.alloc(&Ur[0], s1 * r1));
    MES_TRY(scr.alloc(&Ur[1], s2 * r2));
  }
  if (bf) {
    MES_TRY(scr.alloc(&X16, nel));
    MES_TRY(scr.alloc(&XB16, nel));
    MES_TRY(scr.alloc(&U16[0], s1 * r1));
    MES_TRY(scr.alloc(&U16[1], s2 * r2));
    MES_TRY(scr.alloc(&d.Zh16, zsz));
  }
  MES_TRY(scr.alloc(&P, s1 * r2 * L));
  MES_TRY(scr.alloc(&Ca, s2 * r1 * L));
  MES_TRY(scr.alloc(&Pt, s1 * r2 * L));
  MES_TRY(scr.alloc(&Cat, s2 * r1 * L));
  d.prec = bf ? MES_PREC_BF16 : precision == MES_PREC_BF16 ? MES_PREC_TF32 : precision;
  {
    int64_t ws = s1 * r1 > s2 * r2 ? s1 * r1 : s2 * r2;
    d.split_elems = 16 * ws;
    MES_TRY(scr.alloc(&d.split_ws, d.split_elems));
  }
  MES_TRY(scr.alloc(&Bt, r1 * L * r2));
  if (!sh.small_full) {
    MES_TRY(scr.alloc(&Y0, s1 * J0));
    MES_TRY(scr.alloc(&Y1, s2 * J1));
  }
  MES_TRY(scr.alloc(&ctmp, r1 * r2 * Lr));
  MES_TRY(scr.alloc(&T1, r1 * r2 * L));
  MES_TRY(scr.alloc(&T2, r1 * s2 * L));
  MES_TRY(scr.alloc(&d.Z, zsz));
  MES_TRY(scr.alloc(&d.Zh, zsz));
  if (tf32) {
    int64_t gsz = zsz;
    if (s1 * r1 > gsz) gsz = s1 * r1;
    if (s2 * r2 > gsz) gsz = s2 * r2;
    MES_TRY(scr.alloc(&d.gparts, 3 * gsz));
  }
  MES_TRY(scr.alloc(&d.W, (s1 * r1 > s2 * r2 ? s1 * r1 : s2 * r2)));
  MES_TRY(scr.alloc(&d.W2, (s1 * r1 > s2 * r2 ? s1 * r1 : s2 * r2)));
  MES_TRY(scr.alloc(&d.H, rmax * rmax));
  MES_TRY(scr.alloc(&d.Rinv, rmax * rmax));
  MES_TRY(scr.alloc(&d.cwA, rmax * rmax));
  MES_TRY(scr.alloc(&d.cwX, rmax * rmax));
  MES_TRY(scr.alloc(&d.dinv, rmax));
  MES_TRY(scr.alloc(&d.linv, (rmax + 31) / 32 * 1024));
  MES_TRY(scr.alloc(&d.Kmat, 16384));
  MES_TRY(scr.alloc(&d.gpart, (size_t)mes::small_gram_blocks(s1 * s2) * 1024));
  MES_TRY(scr.alloc(&d.G64, 1024));
  MES_TRY(scr.alloc(&normX, 1));
  MES_TRY(scr.alloc(&normQ, 1));
  MES_TRY(scr.alloc(&sse, 1));
  MES_TRY(scr.alloc(&fitlast, 1));
  MES_TRY(scr.alloc(&xpart, nblk));
  MES_TRY(scr.alloc(&qpart, nblk));
  MES_TRY(scr.alloc(&done, 8));
  flags = done + 1;   // flags[0] error bits, flags[1] Cholesky calls, flags[2] shift restarts
  d.clean = done + 4;
  MES_TRY(scr.alloc(&sign, rmax));
  MES_TRY(scr.alloc(&order, rmax));
  float* rrw = nullptr;   // Rayleigh-Ritz refinement workspace (r > 128): G, HX, S, E, X'
  if (canonical && rmax > 128) MES_TRY(scr.alloc(&rrw, 5 * rmax * rmax));
  d.flags = flags;
  if (ws_bytes) {
    // the fit's reconstruction with fused residual draws from the same
    // workspace (counted, nothing enqueued: the Scratch is dry)
    // (T1 stands in for the reference tensor: any non-null pointer, unread)
    MES_TRY(mes_reconstruct_impl(sh, core, factors, nullptr, T1, sse, scr, T1, T2, d.Kmat, st,
                                 tf32 ? MES_PREC_TF32 : MES_PREC_FP32, flags));
    *ws_bytes = scr.total;
    return MES_OK;
  }
  MES_CUDA_TRY(cudaMemsetAsync(done, 0, 8 * sizeof(int), st));
  if (o.iters_done) MES_CUDA_TRY(cudaMemsetAsync(o.iters_done, 0, sizeof(int), st));

  float* U0 = factors[0];
  float* U1 = factors[1];

  // ---- second layout of T and ||T||^2 ----
  trace.phase("layout");
  MES_TRY(mes::slice_transpose(X, s1, s2, L, XB, xpart, nblk, st, Xr, tf32, X16, XB16));
  const float* Xop = tf32 ? Xr : X;    // T as an operand of the large products
  MES_TRY(mes::sum_doubles(xpart, nblk, normX, nullptr, st));

  // factor of small mode n from the Gram of B x_{m != n, m >= 3} S_m^T; in
  // the interlaced initialisation only the modes before n are truncated
  auto small_mode_update = [&](int n, bool interlaced) -> mes_status {
    KronDesc kd;
    kd.nm = sh.nsm;
    for (int m = 0; m < sh.nsm; ++m) {
      kd.s[m] = (int)sh.s[m + 2]; kd.r[m] = (int)sh.r[m + 2];
      kd.op[m] = (m + 2 == n || (interlaced && m + 2 > n)) ? 'I' : 'T';
      kd.U[m] = factors[m + 2];
    }
    Fibres fb;
    fb.F_lo = r1; fb.F_hi = r2;
    fb.in = Bt; fb.in_lo = 1; fb.in_hi = r1 * L; fb.in_l = r1;
    return d.small_update(fb, kd, n - 2, factors[n]);
  };
  // core = B x_{n>=3} S_n^T
  auto core_from_B = [&](const int* skipf) -> mes_status {
    KronDesc kd;
    kd.nm = sh.nsm;
    for (int m = 0; m < sh.nsm; ++m) {
      kd.s[m] = (int)sh.s[m + 2]; kd.r[m] = (int)sh.r[m + 2]; kd.op[m] = 'T'; kd.U[m] = factors[m + 2];
    }
    MES_TRY(mes::kron_build(kd, d.Kmat, skipf, st));
    Fibres fb;
    fb.F_lo = r1; fb.F_hi = r2;
    fb.in = Bt; fb.in_lo = 1; fb.in_hi = r1 * L; fb.in_l = r1;
    fb.out = core; fb.out_lo = 1; fb.out_hi = r1; fb.out_l = r1 * r2;
    return mes::mix_fibres(fb, d.Kmat, (int)L, (int)Lr, skipf, st);
  };
  // Q <- Q x_n M^T for an r_n x r_n column-major M (n = 0, 1): every mode-n
  // fibre q of the core becomes sum_p M[p + r_n q] Q(.. p ..)
  auto core_apply = [&](int n, const float* M) -> mes_status {
    Gemm gq = base();
    if (n == 0) {
      gq.M = r1; gq.N = r2 * Lr; gq.K_lo = r1;
      gq.A = M; gq.a_m = r1; gq.a_k = 1;
      gq.B = core; gq.b_n = r1; gq.b_k = 1;
      gq.C = ctmp; gq.c_m = 1; gq.c_n = r1;
    } else {
      gq.M = r1; gq.N = r2; gq.K_lo = r2; gq.batch = (int)Lr;
      gq.A = core; gq.a_m = 1; gq.a_k = r1; gq.a_b = r1 * r2;
      gq.B = M; gq.b_n = r2; gq.b_k = 1;
      gq.C = ctmp; gq.c_m = 1; gq.c_n = r1; gq.c_b = r1 * r2;
    }
    MES_TRY(d.gemm(gq));
    MES_CUDA_TRY(cudaMemcpyAsync(core, ctmp, sizeof(float) * r1 * r2 * Lr, cudaMemcpyDeviceToDevice, st));
    return MES_OK;
  };
  // Ca = T x_1 S1^T: Ca[(q1 + r1 l) + r1 L y] = sum_x U0[x + s1 q1] X[x + s1 (y + s2 l)],
  // on the BF16 copies when use16
  auto ca_product = [&](bool use16) -> mes_status {
    Gemm g = base();
    g.M = r1; g.N = s2 * L; g.K_lo = s1;
    g.A = tf32 ? Ur[0] : U0; g.a_m = s1; g.a_k = 1;
    g.B = Xop; g.b_n = s1; g.b_k = 1;
    g.C = Ca; g.c_m = 1; g.N_lo = s2; g.c_n = r1 * L; g.c_nh = r1;
    g.round_tf32 = tf32;
    // second layout Cat[y + s2 (q1 + r1 l)]: K-major operand of Z and B
    g.C2 = Cat; g.c2_m = s2; g.c2_n = 1; g.c2_nh = s2 * r1;
    if (!use16) return d.big(g);
    g.A = reinterpret_cast<const float*>(U16[0]);
    g.B = reinterpret_cast<const float*>(X16);
    return d.big16(g);
  };
  // B = Ca x_2 S2^T: B[(q1 + r1 l) + r1 L q2] = sum_y Cat[y + s2 (q1 + r1 l)] U1[y + s2 q2]
  auto b_product = [&]() -> mes_status {
    Gemm g = base();
    g.M = r1 * L; g.N = r2; g.K_lo = s2;
    g.A = Cat; g.a_m = s2; g.a_k = 1;
    g.B = tf32 ? Ur[1] : U1; g.b_n = s2; g.b_k = 1;
    g.C = Bt; g.c_m = 1; g.c_n = r1 * L;
    return d.big(g);
  };
  // ---- initialisation: truncated or interlaced HOSVD (Eq. 6, Eq. 7) or given factors ----
  trace.phase("init");
  if (o.init_factors) {
    for (int n = 0; n < N; ++n) {
      if (!o.init_factors[n]) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als: init_factors[%d] null", n);
      MES_CUDA_TRY(cudaMemcpyAsync(factors[n], o.init_factors[n], sizeof(float) * sh.s[n] * sh.r[n],
                                   cudaMemcpyDeviceToDevice, st));
      if (tf32 && n < 2) MES_TRY(mes::round_copy(factors[n], Ur[n], sh.s[n] * sh.r[n], nullptr, st));
      if (bf && n < 2) MES_TRY(mes::to_bf16(factors[n], U16[n], sh.s[n] * sh.r[n], nullptr, st));
    }
  } else {
    const bool interlaced = o.init == MES_INIT_INTERLACED;
    // small modes: exact eigenvectors of the unfolding Grams of T (of the
    // truncated tensor, below, in the interlaced form).  A small mode at
    // full rank has an orthogonal factor: it changes neither the other
    // modes' Grams nor the core norm, and its eigenvectors are taken from
    // the last sweep's B, so until then it starts as the identity.
    for (int n = 2; n < N; ++n) {
      if (sh.r[n] == sh.s[n]) {
        MES_TRY(mes::identity_fill(factors[n], sh.s[n], (int)sh.r[n], st));
        continue;
      }
      if (interlaced) continue;
      KronDesc kd;
      kd.nm = sh.nsm;
      for (int m = 0; m < sh.nsm; ++m) {
        kd.s[m] = (int)sh.s[m + 2];
        kd.r[m] = (int)sh.r[m + 2];
        kd.op[m] = 'I';
        kd.U[m] = nullptr;
      }
      Fibres fb;
      fb.F_lo = s1 * s2; fb.F_hi = 1;
      fb.in = X; fb.in_lo = 1; fb.in_hi = 0; fb.in_l = s1 * s2;
      MES_TRY(d.small_update(fb, kd, n - 2, factors[n]));
    }
    // mode 1: T_(1) = rows x, columns (y, l); mode 2: rows y, columns (x, l)
    // (the interlaced form takes only mode 1 from T itself)
    for (int n = 0; n < (interlaced ? 1 : 2); ++n) {
      const int64_t s = n == 0 ? s1 : s2, r = n == 0 ? r1 : r2;
      float* S = factors[n];
      MES_TRY(mes::uniform_fill(d.W, s * r, seed * 2 + n, st));
      MES_TRY(d.orth(d.W, s, r, S, Ur[n], true));
      if (bf) MES_TRY(mes::to_bf16(S, U16[n], s * r, nullptr, st));
      Gemm gz = base(), gw = base();
      int64_t J;
      if (n == 0) {
        J = s2 * L;   // Z[(y,l)][q] = sum_x T[x + s1*(y,l)] S[x,q]
        gz.M = J; gz.N = r; gz.K_lo = s1;
        gz.A = Xop; gz.a_m = s1; gz.a_k = 1;
        // W[x][q] = sum_{y,l} XB[y + s2*x + s1*s2*l] Zh[(y + s2*l) + J*q]
        gw.M = s1; gw.N = r; gw.K_lo = s2; gw.K_hi = L;
        gw.A = XB; gw.a_m = s2; gw.a_k = 1; gw.a_kh = s1 * s2;
        gw.B = d.Zh; gw.b_n = J; gw.b_k = 1; gw.b_kh = s2;
      } else {
        J = s1 * L;   // Z[(x,l)][q] = sum_y XB[y + s2*(x + s1*l)] S[y,q]
        gz.M = J; gz.N = r; gz.K_lo = s2;
        gz.A = XB; gz.a_m = s2; gz.a_k = 1;
        // W[y][q] = sum_{x,l} X[x + s1*y + s1*s2*l] Zh[(x + s1*l) + J*q]
        gw.M = s2; gw.N = r; gw.K_lo = s1; gw.K_hi = L;
        gw.A = Xop; gw.a_m = s1; gw.a_k = 1; gw.a_kh = s1 * s2;
        gw.B = d.Zh; gw.b_n = J; gw.b_k = 1; gw.b_kh = s1;
      }
      // BF16 form: the same products on the BF16 copies of T
      Gemm gz16 = gz, gw16 = gw;
      if (bf) {
        gz16.A = reinterpret_cast<const float*>(n == 0 ? X16 : XB16);
        gw16.A = reinterpret_cast<const float*>(n == 0 ? XB16 : X16);
      }
      for (int it = 0; it < init_iters; ++it)
        MES_TRY(d.subspace_step(gz, gw, J, s, r, S, Ur[n], true, bf ? &gz16 : nullptr, bf ? &gw16 : nullptr,
                                bf ? U16[n] : nullptr));
    }
    if (interlaced) {
      // mode 2 from the tensor truncated in mode 1, Ca = T x_1 S1^T (rows y,
      // J = r1 L columns instead of s1 L):
      //   Z[j][q] = sum_y Cat[y + s2 j] S[y][q],  W[y][q] = sum_j Ca[j + J y] Zh[j + J q]
      MES_TRY(ca_product(bf));
      const int64_t J = r1 * L;
      MES_TRY(mes::uniform_fill(d.W, s2 * r2, seed * 2 + 1, st));
      MES_TRY(d.orth(d.W, s2, r2, U1, Ur[1], true));
      if (bf) MES_TRY(mes::to_bf16(U1, U16[1], s2 * r2, nullptr, st));
      Gemm gz = base(), gw = base();
      gz.M = J; gz.N = r2; gz.K_lo = s2;
      gz.A = Cat; gz.a_m = s2; gz.a_k = 1;
      gw.M = s2; gw.N = r2; gw.K_lo = J;
      gw.A = Ca; gw.a_m = J; gw.a_k = 1;
      gw.B = d.Zh; gw.b_n = J; gw.b_k = 1;
      for (int it = 0; it < init_iters; ++it)
        MES_TRY(d.subspace_step(gz, gw, J, s2, r2, U1, Ur[1], true, nullptr, nullptr, bf ? U16[1] : nullptr));
      // small modes n = 3..N in order, each from B = Ca x_2 S2^T truncated in
      // the small modes before n
      if (!sh.small_full) {
        MES_TRY(b_product());
        for (int n = 2; n < N; ++n)
          if (sh.r[n] < sh.s[n]) MES_TRY(small_mode_update(n, true));
      }
    }
  }

  // ---- sweeps (Eq. 8), n = 1..N ----
  d.skip = done;
  for (int sweep = 1; sweep <= max_iters; ++sweep) {
    trace.phase("sweep", sweep);
    // mode 1: P = T x_2 S2^T, per l: P[x][q2 + r2 l] = sum_y XB[y + s2 x + s1 s2 l] U1[y + s2 q2]
    {
      Gemm g = base();
      g.M = s1; g.N = r2; g.K_lo = s2; g.batch = (int)L;
      g.A = XB; g.a_m = s2; g.a_k = 1; g.a_b = s1 * s2;
      g.B = tf32 ? Ur[1] : U1; g.b_n = s2; g.b_k = 1; g.b_b = 0;
      g.C = P; g.c_m = r2 * L; g.c_n = 1; g.c_b = r2;
      g.round_tf32 = tf32;
      // second layout Pt[x + s1 (q2 + r2 l)]: the K-major operand of Z below
      g.C2 = Pt; g.c2_m = 1; g.c2_n = s1; g.c2_b = s1 * r2;
      if (bf) {
        g.A = reinterpret_cast<const float*>(XB16);
        g.B = reinterpret_cast<const float*>(U16[1]);
        MES_TRY(d.big16(g));
      } else {
        MES_TRY(d.big(g));
      }
      const float* Y = P;
      if (!sh.small_full) {
        KronDesc kd;
        kd.nm = sh.nsm;
        for (int m = 0; m < sh.nsm; ++m) {
          kd.s[m] = (int)sh.s[m + 2]; kd.r[m] = (int)sh.r[m + 2]; kd.op[m] = 'T'; kd.U[m] = factors[m + 2];
        }
        MES_TRY(mes::kron_build(kd, d.Kmat, done, st));
        Fibres fb;
        fb.F_lo = r2; fb.F_hi = s1;
        fb.in = P; fb.in_lo = 1; fb.in_hi = r2 * L; fb.in_l = r2;
        fb.out = Y0; fb.out_lo = 1; fb.out_hi = J0; fb.out_l = r2;
        MES_TRY(mes::mix_fibres(fb, d.Kmat, (int)L, (int)Lr, done, st));
        Y = Y0;
      }
      const int64_t J = sh.small_full ? r2 * L : J0;
      Gemm gz = base(), gw = base();
      gz.M = J; gz.N = r1; gz.K_lo = s1;          // Z[j][q] = sum_x Y[j + J x] S[x][q]
      if (sh.small_full) {
        gz.A = Pt; gz.a_m = s1; gz.a_k = 1;
      } else {
        gz.A = Y; gz.a_m = 1; gz.a_k = J;
      }
      gw.M = s1; gw.N = r1; gw.K_lo = J;          // W[x][q] = sum_j Y[j + J x] Zh[j + J q]
      gw.A = Y; gw.a_m = J; gw.a_k = 1;
      gw.B = d.Zh; gw.b_n = J; gw.b_k = 1;
      for (int it = 0; it < inner_iters; ++it)
        MES_TRY(d.subspace_step(gz, gw, J, s1, r1, U0, Ur[0], false, nullptr, nullptr, U16[0]));
    }
    // mode 2: Ca = T x_1 S1^T
    {
      MES_TRY(ca_product(bf));
      const float* Y = Ca;
      if (!sh.small_full) {
        KronDesc kd;
        kd.nm = sh.nsm;
        for (int m = 0; m < sh.nsm; ++m) {
          kd.s[m] = (int)sh.s[m + 2]; kd.r[m] = (int)sh.r[m + 2]; kd.op[m] = 'T'; kd.U[m] = factors[m + 2];
        }
        MES_TRY(mes::kron_build(kd, d.Kmat, done, st));
        Fibres fb;
        fb.F_lo = r1; fb.F_hi = s2;
        fb.in = Ca; fb.in_lo = 1; fb.in_hi = r1 * L; fb.in_l = r1;
        fb.out = Y1; fb.out_lo = 1; fb.out_hi = J1; fb.out_l = r1;
        MES_TRY(mes::mix_fibres(fb, d.Kmat, (int)L, (int)Lr, done, st));
        Y = Y1;
      }
      const int64_t J = sh.small_full ? r1 * L : J1;
      Gemm gz = base(), gw = base();
      gz.M = J; gz.N = r2; gz.K_lo = s2;         // Z[j][q] = sum_y Y[j + J y] S[y][q]
      if (sh.small_full) {
        gz.A = Cat; gz.a_m = s2; gz.a_k = 1;
      } else {
        gz.A = Y; gz.a_m = 1; gz.a_k = J;
      }
      gw.M = s2; gw.N = r2; gw.K_lo = J;
      gw.A = Y; gw.a_m = J; gw.a_k = 1;
      gw.B = d.Zh; gw.b_n = J; gw.b_k = 1;
      for (int it = 0; it < inner_iters; ++it)
        MES_TRY(d.subspace_step(gz, gw, J, s2, r2, U1, Ur[1], false, nullptr, nullptr, U16[1]));
    }
    // B, the small modes and the core of this sweep.  With every small mode
    // at full rank nothing in the next sweep reads them: they serve the
    // stopping test and the fit history only, so with tol = 0 (a fixed sweep
    // count) and no history asked for they are formed in the last sweep
    // alone (the results are the same bit for bit)
    if (tol > 0.0 || o.fit_history || !sh.small_full || sweep == max_iters) {
      MES_TRY(b_product());
      // small modes n = 3..N with r_n < s_n: Gram of B x_{m != n} S_m^T, exact
      // eigenvectors.  A full-rank small mode's factor is orthogonal: it leaves
      // every other mode's Gram and the core norm unchanged, so its
      // eigenvectors are taken once, after the last sweep.
      for (int n = 2; n < N; ++n)
        if (sh.r[n] < sh.s[n]) MES_TRY(small_mode_update(n, false));
      // core Q = B x_{n>=3} S_n^T (Eq. 5 / Eq. 7 with the current factors)
      MES_TRY(core_from_B(done));
      MES_TRY(mes::sumsq(core, r1 * r2 * Lr, qpart, nblk, done, st));
      MES_TRY(mes::sum_doubles(qpart, nblk, normQ, done, st));
      MES_TRY(mes::fit_flag(normX, normQ, sweep, tol, o.fit_history, fitlast, done, o.iters_done, st));
    }
  }
  d.skip = nullptr;

  trace.phase("core");
  // ---- BF16 form: B and the core from T itself (TF32-rounded), so the
  // returned core carries no BF16 rounding of T ----
  if (bf) {
    MES_TRY(ca_product(false));
    MES_TRY(b_product());
    MES_TRY(core_from_B(nullptr));
  }

  // ---- full-rank small modes: eigenvectors from the last sweep's B ----
  {
    bool any_full = false;
    for (int n = 2; n < N; ++n)
      if (sh.r[n] == sh.s[n]) {
        MES_TRY(small_mode_update(n, false));
        any_full = true;
      }
    if (any_full) MES_TRY(core_from_B(nullptr));
  }

  // The end of the decomposition (the extra CholeskyQR pass, the canonical
  // basis, the fit) is a short chain of small products run once: its
  // CUDA-core products split over all SMs whatever the concurrency hint
  // (un-split, the 384 x 384 core Gram took 1.1 ms on nine CTAs against
  // ~30 us split, and more SM time, not less).
  d.fill = 0;

  // ---- one more CholeskyQR pass on each large factor ----
  trace.phase("orthonormalise");
  // The sweeps orthonormalise with one pass (enough for the iteration); the
  // returned factors get a second one, S <- S R^-1, and the core follows
  // exactly: Q x_n S^T = (Q x_n R^-T) for the new S, i.e. Q <- Q x_n R^-T.
  for (int n = 0; n < 2; ++n) {
    const int64_t s = n == 0 ? s1 : s2, r = n == 0 ? r1 : r2;
    float* S = factors[n];
    MES_TRY(d.cholqr_pass(S, s, r, 0.f, d.W, nullptr, nullptr));
    MES_CUDA_TRY(cudaMemcpyAsync(S, d.W, sizeof(float) * s * r, cudaMemcpyDeviceToDevice, st));
    // R^-1 = D^-1 L^-T of that pass: the solve applied to the identity
    MES_TRY(mes::identity_fill(d.cwX, r, (int)r, st));
    MES_TRY(mes::trsm(d.cwX, r, (int)r, d.cwA, d.dinv, d.linv, d.Rinv, false, nullptr, st));
    MES_TRY(core_apply(n, d.Rinv));
  }

  // ---- canonical basis of the large modes ----
  trace.phase("canonical");
  if (canonical) {
    const int64_t ncore = r1 * r2 * Lr;
    for (int n = 0; n < 2; ++n) {
      const int64_t s = n == 0 ? s1 : s2, r = n == 0 ? r1 : r2;
      float* S = factors[n];
      Gemm gh = base();   // H = Q_(n) Q_(n)^T
      gh.M = r; gh.N = r; gh.C = d.H; gh.c_m = 1; gh.c_n = r;
      if (n == 0) {
        gh.K_lo = r2 * Lr;
        gh.A = core; gh.a_m = 1; gh.a_k = r1;
        gh.B = core; gh.b_n = 1; gh.b_k = r1;
      } else {
        gh.K_lo = r1; gh.K_hi = Lr;
        gh.A = core; gh.a_m = r1; gh.a_k = 1; gh.a_kh = r1 * r2;
        gh.B = core; gh.b_n = r1; gh.b_k = 1; gh.b_kh = r1 * r2;
      }
      MES_TRY(d.gemm(gh));
      const int64_t stride = n == 0 ? 1 : r1;
      if (r <= 128) {
        // Z = eigenvectors of H (FP32 Jacobi, sorted by decreasing eigenvalue)
        MES_TRY(mes::eig_mid(d.H, (int)r, d.cwX, nullptr, st));
      } else {
        // Rayleigh-Ritz for r > 128 by refinement: the sweeps' orthogonal
        // iteration (every factor update orthonormalises with triangular
        // factors, so the leading columns converge to the leading
        // eigenvectors) leaves H nearly diagonal, and X <- X (I + E) with E
        // from rr_update converges from X = I (quadratically once the
        // rotations are small); pairs closer than the current accuracy stay
        // unrotated.  Three steps of four r x r products each (a float32
        // emulation with the 1024x768 scene's spectrum converged in two).
        float *Gm = rrw, *HX = rrw + r * r, *Sm = rrw + 2 * r * r, *E = rrw + 3 * r * r, *Xn = rrw + 4 * r * r;
        float* Xc = d.cwX;
        MES_TRY(mes::identity_fill(Xc, r, (int)r, st));
        for (int it = 0; it < kRRSteps; ++it) {
          Gemm gg = base();   // Gm = X^T X
          gg.M = r; gg.N = r; gg.K_lo = r;
          gg.A = Xc; gg.a_m = r; gg.a_k = 1;
          gg.B = Xc; gg.b_n = r; gg.b_k = 1;
          gg.C = Gm; gg.c_m = 1; gg.c_n = r;
          MES_TRY(d.gemm(gg));
          Gemm ga = base();   // HX = H X
          ga.M = r; ga.N = r; ga.K_lo = r;
          ga.A = d.H; ga.a_m = 1; ga.a_k = r;
          ga.B = Xc; ga.b_n = r; ga.b_k = 1;
          ga.C = HX; ga.c_m = 1; ga.c_n = r;
          MES_TRY(d.gemm(ga));
          Gemm gs = base();   // Sm = X^T H X
          gs.M = r; gs.N = r; gs.K_lo = r;
          gs.A = Xc; gs.a_m = r; gs.a_k = 1;
          gs.B = HX; gs.b_n = r; gs.b_k = 1;
          gs.C = Sm; gs.c_m = 1; gs.c_n = r;
          MES_TRY(d.gemm(gs));
          MES_TRY(mes::rr_update(Sm, Gm, (int)r, E, st));
          MES_CUDA_TRY(cudaMemcpyAsync(Xn, Xc, sizeof(float) * r * r, cudaMemcpyDeviceToDevice, st));
          Gemm ge = base();   // Xn = X + X E, then X = Xn
          ge.M = r; ge.N = r; ge.K_lo = r;
          ge.A = Xc; ge.a_m = 1; ge.a_k = r;
          ge.B = E; ge.b_n = r; ge.b_k = 1;
          ge.C = Xn; ge.c_m = 1; ge.c_n = r;
          ge.accumulate = true;
          MES_TRY(d.gemm(ge));
          MES_CUDA_TRY(cudaMemcpyAsync(Xc, Xn, sizeof(float) * r * r, cudaMemcpyDeviceToDevice, st));
        }
      }
      {
        // one CholeskyQR pass on Z so the rotation is orthogonal to FP32
        // precision (accumulated Jacobi rotations drift by ~sqrt(#rotations)
        // ulp; the refinement is orthonormal to first order only)
        Gemm gzz = base();
        gzz.M = r; gzz.N = r; gzz.K_lo = r;
        gzz.A = d.cwX; gzz.a_m = r; gzz.a_k = 1;
        gzz.B = d.cwX; gzz.b_n = r; gzz.b_k = 1;
        gzz.C = d.H; gzz.c_m = 1; gzz.c_n = r;
        MES_TRY(d.gemm(gzz));
        MES_TRY(mes::chol(d.H, (int)r, 0.f, d.cwA, d.dinv, d.linv, flags, nullptr, st));
        MES_TRY(mes::trsm(d.cwX, r, (int)r, d.cwA, d.dinv, d.linv, d.Rinv, false, nullptr, st));   // Z in Rinv
        Gemm gu = base();  // W = S Z
        gu.M = s; gu.N = r; gu.K_lo = r;
        gu.A = S; gu.a_m = 1; gu.a_k = s;
        gu.B = d.Rinv; gu.b_n = r; gu.b_k = 1;
        gu.C = d.W; gu.c_m = 1; gu.c_n = s;
        MES_TRY(d.gemm(gu));
        MES_CUDA_TRY(cudaMemcpyAsync(S, d.W, sizeof(float) * s * r, cudaMemcpyDeviceToDevice, st));
        MES_TRY(core_apply(n, d.Rinv));   // Q <- Q x_n Z^T
      }
      if (r > 128) {
        // the refinement does not sort: order by the rotated core's mode-n
        // Gram diagonal (the Ritz values), decreasing
        MES_TRY(d.gemm(gh));
        MES_TRY(mes::diag_order(d.H, (int)r, order, st));
        MES_TRY(mes::permute_cols(S, s, (int)r, order, nullptr, d.W, st));
        MES_CUDA_TRY(cudaMemcpyAsync(S, d.W, sizeof(float) * s * r, cudaMemcpyDeviceToDevice, st));
        MES_TRY(mes::permute_core(core, ncore, stride, (int)r, order, nullptr, ctmp, st));
        MES_CUDA_TRY(cudaMemcpyAsync(core, ctmp, sizeof(float) * ncore, cudaMemcpyDeviceToDevice, st));
      }
      MES_TRY(mes::col_signs(S, s, (int)r, sign, st));
      MES_TRY(mes::permute_cols(S, s, (int)r, nullptr, sign, d.W, st));
      MES_CUDA_TRY(cudaMemcpyAsync(S, d.W, sizeof(float) * s * r, cudaMemcpyDeviceToDevice, st));
      MES_TRY(mes::permute_core(core, ncore, stride, (int)r, nullptr, sign, ctmp, st));
      MES_CUDA_TRY(cudaMemcpyAsync(core, ctmp, sizeof(float) * ncore, cudaMemcpyDeviceToDevice, st));
    }
  }

  // ---- fit from the explicit residual (and T_hat when asked for) ----
  trace.phase("fit");
  if (fit || o.reconstruction) {
    const float* fac[8];
    for (int n = 0; n < N; ++n) fac[n] = factors[n];
    // evaluated at FP32-level accuracy in every form: CUDA cores in the FP32
    // form, the three-term TF32 tensor-core product in the tensor-core forms
    // (a plain TF32 reconstruction would add ~1e-3 relative rounding per entry
    // to the residual being measured); the same pass stores T_hat
    MES_TRY(mes_reconstruct_impl(sh, core, fac, o.reconstruction, fit ? X : nullptr, fit ? sse : nullptr, scr, T1,
                                 T2, d.Kmat, st, tf32 ? MES_PREC_TF32 : MES_PREC_FP32, flags, d.wait_ns));
    if (fit) MES_TRY(mes::final_fit(normX, sse, fit, st));
  }
  // ---- device-side failures: status word, NaN fit ----
  if (fit || o.status) MES_TRY(mes::finish_status(flags, normX, fit, o.status, st));
  return MES_OK;
}

extern "C" mes_status mes_reconstruct(const float* core, const float* const* factors, int N,
                                      const int64_t* dims, const int64_t* ranks, float* out,
                                      const float* ref, double* sse, int precision, void* stream) {
  mes::clear_error();
  Shape sh;
  MES_TRY(make_shape(N, dims, ranks, &sh, "mes_reconstruct"));
  if (!core || !factors || !out) return mes::fail(MES_ERR_INVALID_ARG, "mes_reconstruct: null pointer");
  for (int n = 0; n < N; ++n)
    if (!factors[n]) return mes::fail(MES_ERR_INVALID_ARG, "mes_reconstruct: factors[%d] is null", n);
  if ((ref == nullptr) != (sse == nullptr))
    return mes::fail(MES_ERR_INVALID_ARG, "mes_reconstruct: ref and sse go together");
  if (precision != MES_PREC_FP32 && precision != MES_PREC_BF16 && precision != MES_PREC_TF32)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_reconstruct: unknown precision %d", precision);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::Trace trace("mes_reconstruct", st);
  trace.phase("reconstruct");
  mes::AuditScope audit_scope;
  {
    int64_t nX = 1, nQ = 1;
    for (int n = 0; n < N; ++n) { nX *= sh.s[n]; nQ *= sh.r[n]; }
    mes::audit_register(out, (size_t)nX * 4);
    if (ref) mes::audit_register(ref, (size_t)nX * 4);
    mes::audit_register(core, (size_t)nQ * 4);
    for (int n = 0; n < N; ++n) mes::audit_register(factors[n], (size_t)(sh.s[n] * sh.r[n]) * 4);
  }
  mes::Scratch scr(st);
  float *T1 = nullptr, *T2 = nullptr, *Kmat = nullptr;
  MES_TRY(scr.alloc(&T1, sh.r1 * sh.r2 * sh.L));
  MES_TRY(scr.alloc(&T2, sh.r1 * sh.s2 * sh.L));
  MES_TRY(scr.alloc(&Kmat, 16384));
  int* err = nullptr;
  MES_TRY(scr.alloc(&err, 1));
  MES_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  MES_TRY(mes_reconstruct_impl(sh, core, factors, out, ref, sse, scr, T1, T2, Kmat, st,
                               precision == MES_PREC_FP32 ? MES_PREC_FP32 : MES_PREC_TF32, err));
  if (sse) MES_TRY(mes::nan_on_timeout(err, sse, st));
  return MES_OK;
}

extern "C" mes_status mes_tucker_als(const float* X, int N, const int64_t* dims, const int64_t* ranks,
                                     int max_iters, double tol, float* core, float* const* factors,
                                     double* fit, const mes_als_opts* opts, void* stream) {
  mes::clear_error();
  return tucker_als_impl(X, N, dims, ranks, max_iters, tol, core, factors, fit, opts, stream, nullptr);
}

extern "C" mes_status mes_tucker_als_workspace_size(int N, const int64_t* dims, const int64_t* ranks,
                                                    const mes_als_opts* opts, size_t* bytes) {
  mes::clear_error();
  if (!bytes) return mes::fail(MES_ERR_INVALID_ARG, "mes_tucker_als_workspace_size: null pointer");
  *bytes = 0;
  return tucker_als_impl(nullptr, N, dims, ranks, 1, 0.0, nullptr, nullptr, nullptr, opts, nullptr, bytes);
}
