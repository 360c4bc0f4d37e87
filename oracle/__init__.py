"""FP64 CPU oracle for the multi-exposure stereo Tucker-ALS path.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them: the two
sides share no code.  Only the seeded scene generator (`synth`), which holds
none of the method's arithmetic, feeds both.

Contents, each following the paper (Sharma & Grover, arXiv 2104.04726):

* `colour`  -- Section III-A: R'G'B' -> Y'CbCr (ITU-R BT.601, non-constant
  luminance) and R'G'B' -> IPT (Ebner & Fairchild), plus stacking the
  multi-exposure stereo images into the order-4 tensor of Section III-B.
* `tucker`  -- Section III-B: mode-n products, Tucker model (Eq. 1, Eq. 2),
  truncated HOSVD initialisation (Eq. 3 to Eq. 7), Tucker-ALS / HOOI sweeps
  with the factor taken from the leading eigenvectors of the Gram of the
  partial contraction (Eq. 8), core, fit, reconstruction and PSNR.
* `quant`   -- the core quantiser used as the rate knob (abstract and
  Section I mention "the rank of core tensor and its quantization"; the paper
  never defines the quantiser, see the module docstring for the reading).

Every function is written in plain numpy, FP64 unless stated (the quantiser
is FP32 by definition of its reading), with library primitives (matmul,
tensordot, eigh, sort) as single steps and no blocking or reordering beyond
the definitions.  Pins that tie these functions to the mathematics live in
`tests/test_oracle_*.py`.
"""
