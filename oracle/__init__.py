"""Plain FP64 CPU oracle for the ETD + embedded-boundary + level-set method of
Liu & Liu, "Integration factor combined with level set method for
reaction-diffusion systems with free boundary in high spatial dimensions"
(arXiv 2209.15095).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA path; the only module
both sides read is the seeded input generator ``paper_2209_15095_gb300.inputs``,
which holds none of the method's arithmetic.

Every function is written for clarity, not speed: numpy whole-array
operations, scipy for library primitives (sparse matvec, dense expm,
symmetric eigendecomposition), no blocking or fusion.  Each module names the
section / equation of the paper it restates.

Modules
  grid      -- node grid (Sec. 2)
  eb        -- point classification, ghost-point rules (cases 1-3), the
               discrete operator C (Sec. 2)
  phi       -- scalar phi_k, exact phi-combination via the augmented matrix
               exponential and via symmetric eigendecomposition (Eq. 3.7-3.10)
  krylov    -- adaptive Krylov (Lanczos / IOM2) phi-combination with
               time-substepping (Sec. 3.3)
  etd       -- reaction terms and the ETD1 / ETD2 steps (Sec. 3.1)
  levelset  -- level-set step: extension, Stefan speed, HJ-WENO5 + TVD-RK3,
               reinitialisation (Sec. 4.3 Algorithm)
  adjoint   -- adjoint of the ETD2 step on a frozen domain

Parity status: every public function is pinned by a test in
tests/test_oracle_*.py against closed forms, brute force, invariants or the
paper's Table 1 -- except where a module header says "parity unpinned".
"""
