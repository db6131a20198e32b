"""FP64 CPU oracle for the ProxSkip / PDHGSkip hot path (test infrastructure only).

A plain, slow, direct numpy transcription of what the solvers compute, written from
the paper's definitions: the TV problem (Eq. 5), Dual-ROF and its projected-gradient
solver (Eq. 6-7, Section 2.1), the accelerated variant used as the inner TV prox
(Sections 2.2 and 3.1), PGD (Algorithm 2), FISTA (Algorithm 3), ProxSkip
(Algorithm 4) and PDHGSkip-2 (Algorithm 6), with the forward operators of Section 3
(blur, parallel-beam projector).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA path never calls it and shares no
code with it; the only module both sides use is ``synth`` (seeded inputs).

Every function computes in float64.  Pins (checks against facts fixed by the paper or
by the mathematics, not by this code) live in ``tests/test_oracle_*.py``.
"""

from . import tv, operators, coin, solvers, power  # noqa: F401
