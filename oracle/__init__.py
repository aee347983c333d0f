"""Plain complex128 CPU oracle of the diagonal sweeping source-transfer DDM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product (the CUDA library and its Python binding) never calls into this package
and shares no code with it; both sides only read the seeded inputs of
``workloads``.

Modules, each a direct restatement of the paper (Leng & Ju, "A diagonal
sweeping domain decomposition method with source transfer for the Helmholtz
equation"):
  * ``helmholtz``  -- PML stretching (Eq. 2.1, Eq. 2.3 shifted profile), the
                      J-multiplied PML operator (Eq. 2.2) on any window, global
                      direct solve.
  * ``ddm``        -- checkerboard partition, cutoffs and truncations
                      (Section 2.2), transfer operator Psi, routing by Rules
                      3.1/3.2 and 4.1/4.2, Algorithm 3.1 / 4.1, Algorithm 2.1/2.2.
  * ``krylov``     -- right-preconditioned restarted GMRES in float64 (Remark 1).
  * ``adjoint``    -- adjoint solve and the receiver-misfit gradient w.r.t. m.

Where the paper is silent or garbled, the reading taken is stated at the
point of use.
"""
