"""CPU FP64 oracle for the alpha-circulant preconditioned Richardson method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only the test suite, the smoke check of
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA library; inputs reach
both sides from the seeded generators in ``paper_2103_12571_gb300.workloads``,
which the caller passes in as plain arrays.

Everything is plain numpy / scipy in float64 (complex128), written to be read
against the paper (Caklovic, Speck & Frank, "A parallel-in-time collocation
method using diagonalization", arXiv 2103.12571):

* ``collocation``  - Radau IIA nodes and the collocation matrix Q (Sec. 2.1,
                     eq. (collocation); node polynomial of Sec. 2.3).
* ``stencils``     - finite-difference weights of the centred (orders 2, 4,
                     6) and upwind (orders 1..5) schemes of Sec. 5, from their
                     moment conditions in exact rational arithmetic.
* ``operators``    - periodic stencil operators A, C_coll, H and the
                     all-at-once matrices C and C_alpha (eqs. (Hm),
                     (globalsys), (prec)), and the forcing term v_l.
* ``sequential``   - the sequential collocation time-stepper (eq.
                     (seq_collocation_problem)), its discrete adjoint and the
                     gradient contractions.  This is THE oracle: the unique
                     solution of C u = w.
* ``paradiag``     - Lemma 1, the three-step preconditioner solve
                     (eqs. (s1)-(s3), (inner1)), Lemma 2's characteristic
                     polynomial and the Richardson iteration (eq. (Riteration))
                     on small problems.
* ``alpha_rule``   - Algorithm 2's adaptive alpha sequence.
* ``fourier``      - stencil symbols and the closed-form Fourier-mode solution
                     of the collocation stepping (an independent second oracle
                     for periodic constant-coefficient problems).

Pins: every function is checked in ``tests/test_oracle_*.py`` against values
printed in the paper, closed forms, textbook special cases, invariants or a
brute-force dense solve.  Functions without such a pin are marked
"parity unpinned" in their docstring (none at present).
"""

from . import collocation, stencils, operators, sequential, paradiag, alpha_rule, fourier  # noqa: F401
