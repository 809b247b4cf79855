"""Independent FP64 CPU oracle for the anisotropic Eulerian Gaussian beam hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its Python binding) may
import, call or link anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
path: its eigen-solver is LAPACK's ``eigh`` (the GPU uses a closed form), its stencils are written
out with numpy slicing, and it works in float64 throughout.

What it computes (X. Huang, "Eulerian Gaussian beams for high frequency wave propagation in
inhomogeneous media of arbitrary anisotropy", arXiv 2006.11945):

  medium.py       a_ijkl = c_ijkl / rho (Eq. 5), its spatial gradient, positive-definiteness check
  christoffel.py  Gamma_ik = a_ijkl p_j p_l (Eq. 4), qP eigenpair of (Gamma - I) U = 0 (Eq. 3),
                  phase-angle slowness p = n(theta)/v (Eq. 7), ray velocities of the Hamiltonian
                  system (the kinematic content of Eqs. 8-12)
  liouville.py    level sets and complex-traveltime carrier tau advected by the phase-space Liouville
                  equation (Eqs. 16 and 19) from coordinate initial data (Eq. 20), HJ-WENO3 in space
                  and angle, TVD-RK3 in pseudo-time
  superpose.py    Gaussian beams from the level-set Jacobian (Eqs. 21-26), summed over the phase
                  angle into the frequency-domain Green's function (Eqs. 33-35), plus arrival
                  extraction on the source manifold Gamma (Eq. 35)
  closed_forms.py exact references used to pin the above (isotropic and Thomsen VTI velocities,
                  the 2-D Hankel Green's function, homogeneous steady-state labels)
  shooter.py      Lagrangian ray + dynamic ray tracer (brute-force arrival counts and amplitudes)

Where the paper is garbled or silent the readings are listed in the design notes and restated in
the docstring of the function that takes them.
"""
