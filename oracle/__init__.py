"""FP64 CPU oracle of the three-weight ADMM (TWA) trajectory planner.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  It shares no
code with the CUDA path (``paper_1311_4527_gb300``); the two meet only at the
seeded input generators in ``workloads``.

Contents:

* ``oracle.prox`` -- the minimizers (proximal operators) of every factor of the
  planning graph, written from their definitions (Section 3.3 and
  Appendices C-I of Bento, Derbinsky, Alonso-Mora and Yedidia, "A
  message-passing algorithm for multi-agent trajectory planning", NIPS 2013).
* ``oracle.twa`` -- the seven-step TWA iteration of Appendix B over the factor
  graph of Section 3.3, plus the stopping rule, total cost and feasibility
  measures used by the tests.
* ``oracle.adjoint`` -- the reference gradient of a loss on z^K after K
  unrolled iterations with respect to starts, goals, radii and cost weights,
  branch choices frozen; per-factor Jacobians by central differences of
  ``oracle.prox``, pinned by central differences of the whole K-iteration map.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, brute force on tiny inputs, invariants); see ``tests/``.
"""

from . import adjoint, prox, twa  # noqa: F401
