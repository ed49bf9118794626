"""CPU oracle for the upwind-SBP elastic-wave method of Duru, Fung & Williams
(arXiv 2011.02600): a plain, slow, FP64 restatement of the method used ONLY
to check the CUDA path.

This package is test infrastructure.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path
(``paper_2011_02600_gb300``) never imports it and shares no code with it:
no kernels, headers, helpers, tables or constant generators.  The only code
both sides use is the seeded input generators in ``workloads/``, which hold
none of the method's arithmetic.

Modules
  operators  exact rational upwind SBP dual pairs of orders 2 to 9 (Section 4.1,
             Table 1) and the traditional central operators of orders 2, 4, 6, 8
             (Table 2)
  rk         Carpenter-Kennedy 2N-storage RK4 (cited in Sections 1 and 7)
  metrics    Jacobian and metric terms (Section 2.2)
  elastic    semi-discrete RHS, SATs, energy, boundary terms (Sections 4-5,
             Appendix A), on either operator family
  pointwise  the same right-hand side at single nodes (sampled checks of large grids)
  adjoint    receiver misfit, complex-step derivatives, assembled operator
  surrogate_net  the surrogate network in FP64 (with optional BF16 rounding points)
  source     discrete moment-tensor point source (Section 7.1)
  solver     time loop, receivers, energy history
  closure_search  how the free closure entries of upwind orders 8, 9 and traditional
             order 8 were chosen (run by hand; its output is in operators' tables)

Where the paper is silent, garbled or ambiguous, the reading taken is stated
in the docstring of the function that depends on it.
"""
