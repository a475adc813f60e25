"""FP64 CPU oracle for the graded-material BEM hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import, call, link or run anything
under oracle/.  The product library (paper_1612_08395_gb300) never touches it,
and it never imports the product: the two share no code.

Parity status: every function is pinned by the tests in tests/test_oracle_*.py.
alpha(k, nu) is pinned on three families independent of Eq. 3: k = 0
(Boussinesq), nu = 1/(2+k) (the purely radial Frohlich-Holl field, alpha =
(2+k) / (2 pi (1+k)^2)) and the limit k -> 1 at nu = 0.5 (Gibson's
incompressible soil, alpha / (1 - k) -> 1 / pi); off them it rests on Eq. 3
as printed.
"""
from .bem_oracle import *  # noqa: F401,F403
from . import closed_forms  # noqa: F401
