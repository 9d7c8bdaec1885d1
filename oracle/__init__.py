"""Plain, slow FP64 CPU oracle for the aMFP phonon BTE (OpenBTE, arXiv 2106.02764).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA library: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
leg and its ``--impl reference`` arm) may import or run it.  The product path
(``paper_2106_02764_gb300.binding`` and the CUDA library) never imports it, and
this package imports nothing from the product except the seeded input
generators in ``paper_2106_02764_gb300.inputs``, which hold no solver
arithmetic.

Modules
  bte      -- discretisation (App. A) and the per-ordinate sparse solves;
              Algorithm 1 source iteration (mode A) and GMRES on the reduced
              unknowns (mode B)
  fourier  -- the heat-conduction first guess and kappa_fourier (App. B, the
              orthogonal-grid subset)
  dense    -- brute-force dense solve of the whole discrete system (tiny meshes)
  adjoint  -- transposed solves and d kappa_eff / d s(x)
  pool     -- worker processes over ordinate chunks (timed CPU baseline)

Every function names the passage of the paper it follows.  The readings taken
where the paper is silent or garbled are listed in the module docstrings.
"""
