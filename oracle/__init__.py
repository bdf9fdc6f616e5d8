"""Plain CPU float64 oracle for BLIP / CoverBLIP matched-filtering reconstruction.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg
of ``bench.py`` (including its ``--impl reference`` arm) may import or call anything here.  The
product path (``paper_1810_01967_gb300``) never imports this package and shares no code with it.

Modules
  mrf_oracle  forward/adjoint operator, gradient step, exact cone projection, BLIP iteration,
              adaptive step rule, look-up table, error metrics (§3.2, Algorithm 2, §6)
  covertree   textbook cover tree built from the nesting/covering/separation invariants and
              the (1+eps)-ANNS branch and bound (§4.1, Algorithm 1)
  mlp         the learned-proposal network 2L -> 512 -> 512 -> 3 (GELU): forward, backward,
              Adam, input canonicalisation
Everything is float64 / complex128 (inputs stored in complex64 are upcast first).
"""
