"""FP64 CPU oracle for the Hamiltonian ray tracing (HRT) hot path — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow restatement of the method of Zhou et al., "A Hamiltonian, post-Born,
three-dimensional, on-the-fly ray tracing algorithm for gravitational lensing" (arXiv 2405.12913), in
float64 with NumPy/SciPy and PyTorch-on-CPU.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does, and it shares no code with the
CUDA library (each side writes its own cosmology, deposit, Poisson kernel, gather and ray integrator).

Modules
  units      physical constants in code units (lengths Mpc/h, velocities 100 km/s, H0 = 1)
  cosmology  E(a), chi(a), D1(a), f(a), particle kick/drift time integrals, BBKS P(k), sigma8
  pm         lattice, CIC deposit, FFT Poisson gradient with sinc deconvolution, CIC gather, leapfrog, ICs
  rays       half-shell LOS quadrature, KDK ray step with the A/B recursion, readout (kappa, gamma, omega)
  power      convergence power spectrum in log-spaced multipole bins
  ewald      periodic point-mass fields (3D and 2D Ewald sums) used to pin the PM force and the lensing
  sim        the co-evolution driver: forward N-body, then reverse steps of particles and rays (Alg. 1)
"""
