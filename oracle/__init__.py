"""Plain FP64 CPU oracle of the SDRT semi-discrete residual (arXiv 2105.08632).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link this package; only the tests, the smoke
check and the CPU-baseline leg of the benchmark use it.  It shares no code with
the GPU path: point sets, bases, operators, metrics, face pairing and fluxes are
all re-derived here, in plain NumPy, from the paper's equations.

Modules
-------
points     reference elements, solution points, flux points and their degrees of
           freedom (paper App. A, Tables "nsolpts_nfpts" / "nfpts_extra").
bases      monomial modal bases: the solution space and the Raviart-Thomas flux
           space of every element type (paper Sec. 2.1 and App. A).
operators  Vandermonde matrices, nodal bases and the matrix-form operators
           M0, M12, M13, M14, M15, M16, P (paper App. B).
mesh       affine metrics (Eqs. "mapping_jacobian", "transformed_quantities"),
           physical face normals and flux-point pairing across faces.
physics    physical fluxes (advection, Euler, Navier-Stokes) and common fluxes
           (upwind, Rusanov, Roe, LDG) (Sec. 2.1, Eqs. "flux_advection",
           "eulerConservativeVariables", "fluxOperatorNavierStokes").
residual   the SDRT residual dU/dt = R(U) (Eqs. "interpolate_sol_to_flux" to
           "divergence_sdrt"), the FR-SDRT residual (Eq. "divergence_fr"),
           classical RK4, complex-step JVP and Jacobian assembly.

Parity status of each function is stated in its module header.
"""
