"""FP64 CPU oracle for the HSDE-ADMM of chordally sparse SDPs (test infrastructure).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, deliberately literal
restatement of the method of Zheng, Fantuzzi, Papachristodoulou, Goulart and
Wynn, "Fast ADMM for homogeneous self-dual embedding of sparse SDPs"
(arXiv:1611.01828), written in NumPy/SciPy FP64.  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
product (the CUDA library and its Python binding) never does, and it shares no
code with it.

Modules
-------
symbolic  Section 2.1-2.2: aggregate sparsity pattern, chordal extension by
          exact minimum degree, maximal cliques in natural order, the entry
          selectors H_k = E_Ck (x) E_Ck and D = H^T H (Section 4.3).
hsde      Section 3 (vectorised decomposed pair, embedding matrix Q) and
          Section 4 (the three ADMM steps, the block eliminations of Sections
          4.2-4.3 and the matrix inversion lemma), plus the stopping rule and
          the infeasibility certificates.
dense     A literal dense (I+Q)^{-1} on tiny instances, used to pin the
          block-eliminated affine step.
adjoint   Reverse mode through K unrolled iterations (Eqs. Step1-Step3):
          the adjoint affine solve with the literal I - Q and the
          Daleckii-Krein derivative of the psd projection; pinned by
          central differences.

Readings where the paper is silent or garbled are listed in each function's
docstring; all of them are pinned by tests under ``tests/`` except the ADMM
iterate sequence itself, which only this oracle defines ("parity unpinned"
for the iterate trajectory beyond what the closed forms and fixed-point
invariants fix).
"""
from . import symbolic, hsde, dense  # noqa: F401
