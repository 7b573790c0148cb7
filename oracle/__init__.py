"""Plain CPU FP64 oracle for the FFT-based Poisson projection of Scapin, Costa & Brandt (§3.2, §3.6).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of ``bench.py`` use it.  It shares no code,
table or constant with the CUDA library: the separable solve takes the textbook orthonormal Fourier, cosine
and sine vectors of each x and y stencil matrix as dense basis matrices, with every eigenvalue computed as the
Rayleigh quotient of the stencil matrix itself (no closed-form eigenvalue table), transforms by plain matrix
products, and solves each z system by Thomas elimination (Sherman-Morrison around it for a periodic z axis, a
bordered dense solve for the singular mean mode).

What it computes (the plain definition of the method's result, because the paper's solver is a direct
solver for the second-order finite-difference Poisson equation, §3.2):

* ``mac``        MAC-grid stencils: divergence D, gradient G, Laplacian L = D G, 1-D operator matrices.
* ``poisson``    the exact solution of L p = f - fbar (zero volume-weighted mean gauge when L is singular),
                 the projection u <- u - (dt/rho0) G p (Eq. lap_p and the correction that follows it), and
                 the same step with the variable-density pressure-splitting terms of Eq. lap_p.
* ``interface``  |grad C| and n = -grad C/|grad C| (central or Youngs differences), the Stefan potential
                 solve (Eq. ext_div), u1e = u - grad(phi) (Eq. jump_subtr), uG = u1e - (mdot/rho1) n
                 (Eq. int_vel); the boiling variant with the vapour-velocity extension (Appendix A).
* ``vof``        the split VoF update with the interface velocity and its implicit volume deflation
                 (§3.1, Eqs. fluxes, final_corr_2; upwind fluxes in place of the MTHINC ones).

Every public function is pinned by the ``-m "not gpu"`` tests against closed forms, brute-force dense
LU solves and exact invariants; no function is "parity unpinned".
"""
from .mac import Grid, divergence, gradient, apply_laplacian, operator_matrix_1d, face_shape
from .poisson import poisson_solve, project, project_variable_density
from .interface import grad_c, delta_and_normal, stefan_source, extend_liquid_velocity, extend_vapour_velocity
from .vof import vof_update

__all__ = [
    "Grid", "divergence", "gradient", "apply_laplacian", "operator_matrix_1d", "face_shape",
    "poisson_solve", "project", "project_variable_density", "grad_c", "delta_and_normal", "stefan_source",
    "extend_liquid_velocity", "extend_vapour_velocity", "vof_update",
]
