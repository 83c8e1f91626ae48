"""CPU oracle for the SMC hot path (Emmett, Zhang & Bell, arXiv 1309.7327).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or run anything in this package.  The CUDA library never calls it and
shares no code, constants table or helper with it.

Plain, slow, FP64 NumPy restatement of what the paper's method computes:

* ``stencil``   -- 8th-order first derivative D and the 8th/6th-order narrow
                   stencils for (a u_x)_x (Sec. 2.2, eqs. DaDu and H, the two
                   M matrices).
* ``thermo``    -- NASA-7 ideal-gas mixture thermodynamics, the Newton
                   inversion e -> T, and the primitive variables (Sec. 2.1).
* ``transport`` -- power-law viscosity / constant-Lewis-number transport
                   (stands in for EGLIB, Sec. 5).
* ``chem``      -- mass-action reversible Arrhenius production rates (the
                   rho*omega_k source of eq. NS:rY).
* ``rhs``       -- the full right-hand side of eq. cns on a ghosted box or a
                   periodic domain, in both species-diffusion modes (Sec. 2.1
                   and Sec. 2.4).
* ``sdc``       -- Gauss-Lobatto collocation, the Q and S integration
                   matrices, the SDC sweep (Sec. 3.1, eq. expsdc) and the
                   mode-1 and mode-2 multirate sweeps (Sec. 3.2, eqs.
                   mrupdate and mrupdate2).
* ``bdf``       -- a variable-order, variable-step BDF integrator (the
                   implicit reaction integration of mode 2).
* ``react``     -- the reaction ODE of one cell with constant forcing, its
                   analytic Jacobian, and its integration by ``bdf``.
* ``heat2d``    -- the appendix heat-equation problems T1/T2 (App. A).

Where the paper is silent the reading taken is stated in the function that
uses it.
"""
