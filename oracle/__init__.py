"""CPU oracle for DA-CSR sparse matrix-vector products (Saak & Schulze,
"Diagonally-Addressed Matrix Nicknack", arXiv 2307.06305).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call, link or execute anything in this directory.  The product path (the CUDA
library and its Python binding) never does, and this package never imports
the product path: the two share nothing but the seeded input generators in
``workloads``.

Everything here is plain and slow on purpose, written from the paper in its
order and notation so that a reader can check it by eye:

* ``traffic``  -- Eq. (1), Eq. (3), the SpMV work and traffic definitions of
  Section 4 and the ratio lattice of Fig. 3.
* ``dacsr``    -- the matrix bandwidth w of Eq. (2) and the CSR -> DA-CSR index
  translation of Section 2 (Example 1), with the 16-bit fit check.
* ``rcm``      -- reverse Cuthill-McKee ordering and the symmetric
  permutation P A P^T (Section 2, Example 2; Section 3).
* ``spmv``     -- y <- alpha A x + beta y in the row order of Listing 2, the
  exact (rational) reference, the componentwise error bound, the reduced
  precision variants (FP32 / BF16 values, FP32 accumulation) and the
  multi-right-hand-side product.
* ``cg``       -- FP64 conjugate gradients and mixed-precision iterative
  refinement around a low-precision CG.
* ``bsr``      -- block CSR and its diagonally-addressed form (DA-BSR),
  expanded to scalar CSR so the SpMV definitions above apply.
* ``spmv_listing2.c`` -- a plain C restatement of Listing 2 (CSR-32 and
  DA-CSR-16, FP64, OpenMP row partition), used as the timed CPU baseline.

Parity pins live in ``tests/test_oracle_*.py``.
"""
