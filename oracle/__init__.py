"""Plain FP64 CPU oracle of the DDA for EELS and CL in an arbitrary host
(Kichigin & Yurkin, arXiv:2208.01348).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import it.  The
product path (``paper_2208_01348_gb300``) never imports, links or executes
anything in here, and this package imports nothing from the product except
the seeded input generators in ``paper_2208_01348_gb300.inputs``.

Everything is SI, complex128, written for readability: dense Green's-tensor
assembly and LAPACK LU for small problems, and for large problems a plain
zero-padded FFT convolution (scipy.fft) driven by a library Krylov solver,
which the tests cross-check against the dense matrix.

Module map (each function cites the paper passage it follows):
  constants  -- physical constants (CODATA 2018)
  physics    -- electron speed, host index, beta_h/gamma_h (Eq. 24), polarizability
  field      -- incident field (Eq. 25) and auxiliary field (Eq. 34)
  green      -- Green's tensor (Eq. 5), dense DDA matrix, FFT matvec
  igt        -- cell-integrated Green's tensor and polarizability to second order in kd (Sec. S5)
  losses     -- P_EELS (Eq. 32, 37), P_ext (Eq. 17, 48), P_abs (Eq. 18), P_CL (Eq. 42)
  icosphere  -- far-field direction grid
  mie        -- plane-wave Lorenz-Mie cross sections (a pin for the DDA core)
  run        -- one (energy, beam) point end to end
"""
