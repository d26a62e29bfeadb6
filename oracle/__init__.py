"""Plain FP64 CPU oracle for the DMK Stokes near-field pass (arXiv 2509.21471).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library under
``paper_2509_21471_gb300/``; both sides only receive the same seeded inputs.

Every function here is written for a reader checking it against the paper by
eye: plain numpy/scipy in float64, no blocking, fusion or reordering beyond
what the cited definition states.

Modules
  window    -- PSWF psi_0^c, window phi, Phi, phi-hat, gamma-hat (Sec. 2.3, Eq. 4.1,
               Cor. 4.1); the Gaussian window for special-case pins.
  kernels3d -- residual biharmonic B_R (Thm 4.1), residual Stokeslet / stresslet
               and their self terms in 3D (Sec. 5.2), their gradients.
  kernels2d -- 2D residual kernels by the numerical Fourier route of App. B.
  params    -- the PSWF bandlimit c from the tolerance (Table 2).
  tree      -- adaptive level-restricted quad/oct-tree and near lists (Sec. 6.1 Step 1).
  near      -- the near (residual + self) component, Sec. 5.3 / Step 4.
  direct    -- O(N^2) free-space sums (Eq. 1.6) and the periodic zero mode (Sec. 5.3).
  ewald     -- single-level periodic Ewald sums with Gaussian or PSWF split (Sec. 5.3).

Parity status: every function listed above is pinned by a ``-m "not gpu"``
test in ``tests/test_oracle_*.py`` against something other than itself
(library routines, closed forms, invariants, brute force); none is
"parity unpinned".
"""
