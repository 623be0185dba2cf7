"""Oracle: plain, slow, obviously correct CPU implementation of the hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2602_14167_b300``) and never imports it.

Modules:
  sv     -- complex128 state-vector simulator in C (gate application by
            definition, Pauli expectations, H|psi>, energy, parameter-shift and
            finite-difference gradients), Sec. I.B of the paper;
  dense  -- full-matrix Kronecker checker, exact diagonalisation and the
            free-fermion TFIM ground energy (Sec. IV.C formalism);
  adam   -- the Adam update (the optimiser of the paper's training listings);
  mlp    -- float64 forward/backward of the warm-start MLP with BF16 rounding
            at the points where the kernels round (no paper counterpart:
            parity for the warm-start network is checked against this oracle,
            whose own gradients are pinned by finite differences).
"""
