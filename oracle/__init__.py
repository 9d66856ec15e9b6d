"""CPU oracle for the loop-hafnian hot path of arXiv:2108.01622.

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct restatement of the
paper's definitions and formulas in numpy / Python (complex128, exact summation with
``math.fsum``, optional mpmath high precision). Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import it. The product path (the CUDA library and
its Python binding) never imports, calls or links anything in here, and this package imports
nothing from the product.

Modules:
  lhaf_oracle  -- loop hafnian: definition (App. B), eigenvalue-trace (Eq. ET_loop), finite
                  difference sieve (Eq. fdsieve), repeated pairs (App. B.2, B.4), greedy pairing
                  (App. B.3), gradients by the minor identity.
  gbs_oracle   -- Gaussian state -> GBS kernel and pattern probability (App. A, Eq. mixed_prob).

Parity status: every function is pinned by tests/test_oracle_pins.py against closed forms, brute
force, the paper's worked example and identities of the definition, except where a docstring says
"parity unpinned".
"""
