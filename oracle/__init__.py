"""Plain FP64 CPU oracle of the CMCG hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import anything from this package.  The product path (the
CUDA library and its Python binding) never calls it; it shares no code,
tables or constants with the CUDA path.  Inputs come from the seeded
generators in ``paper_2106_02858_gb300.inputs``, which hold no numerics of the
method.

Modules (each function cites the part of the paper it follows):

* ``refelem``  -- nodal P_q basis on the reference tetrahedron built from an
  orthonormal (Dubiner) Vandermonde: mass, differentiation, face mass, lift.
* ``geometry`` -- face matching, node matching across faces, affine factors,
  normals, face areas, inscribed diameters (Section 5.2.2).
* ``dg``       -- the upwind DG operator Phi(t, U) = Re(J e^{i w t}) + B U
  (Eq. DG_semidiscrete and Eq. ode_system, extended to 3D).
* ``timestep`` -- CFL step choice (Eq. cfl), RK2 / RK4 (Algorithms rk2, rk4),
  propagators P_{psi,w}, P_w and the adjoint P*_w (Section 4.1.2).
* ``filtering`` -- trapezoid (Eq. filtering_RK2) and Hermite (Eq.
  filtering_RK4) discrete filters, with the 2/T of Eq. filter.
* ``cmcg``     -- Algorithms init, grad and cmcg (Section 2.2), residual form.
* ``dense``    -- brute-force dense matrices on tiny meshes (B, P, the
  frequency-domain solve (i w M + K) U = M J of Section 6).
"""
