"""Reference oracle for the chromatic-polynomial transfer matrix (Jacobsen, arXiv:1005.3609).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, link or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` use it.  It shares no code, table or helper
with the CUDA library under ``paper_1005_3609_gb300/``.

Everything here is plain and slow on purpose:

* ``graphs``      -- the L x N square / triangular rectangles (Sec. 3.2-3.3).
* ``brute``       -- proper-colouring counts and interpolation (definition, Sec. 1).
* ``delcon``      -- deletion-contraction (textbook recursion, independent pin).
* ``fk``          -- the Fortuin-Kasteleyn subset expansion, eqs. (Z2), (Z_modified).
* ``partitions``  -- canonical set partitions, the NCNNN state space and the
                     paper's ordering of it (Sec. 3.4, eq. (M_recurs)).
* ``tm_exact``    -- the paper's projected sparse factorisation, applied literally
                     operator by operator on a hash map of partitions, exact Python
                     integers (Sec. 3.1-3.3, eqs. (T_sq_decomp), (T_sq_proj),
                     (T_last), (T_last_i)).
* ``tm_generic``  -- the plain any-v transfer matrix T = (prod V)(prod H) on
                     non-crossing partitions (Sec. 3.2), evaluated at v = -1.
* ``modp``        -- the same projected factorisation in plain C, modulo one
                     31-bit prime at a time (Sec. 3.5), with a ctypes wrapper.
* ``crt``         -- primes (trial division) and Chinese remaindering (Sec. 3.5).
* ``flm``         -- the finite-lattice method and the series checks
                     (Sec. 4.1-4.3, eqs. (fb)-(fc), (efb), (efs), (efc)).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, the paper's printed orderings and Table 1.
"""
