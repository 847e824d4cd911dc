"""Plain FP64 CPU oracle for the NUFFT-based dipole-dipole interaction (DDI) solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` call it.  It shares no code with the
CUDA library (``paper_1504_02897_gb300/csrc``) and neither side imports the other.

Modules
-------
quadrature    spherical (3D) / polar (2D) Fourier quadrature and the DDI weights
              (Sec. 2.1, Eq. DDI-Trun1, symbol of Eq. DipKer / Eq. dipmn).
nudft         the discrete quadrature sum evaluated as a direct nonuniform DFT
              (type-2 grid->nodes, symbol x weights, type-1 nodes->grid).
closed_forms  closed-form dipolar potentials of Gaussian densities
              (Eq. extDensGausDipolar / Hessian_Ex1, the 2D Bessel form of
              Example 2d_exmp, and 1-D integral forms derived from the symbol).
gpe           TSFP step (Eq. tssp2; Case I and the general nonlinearity/damping
              of Sec. 5), energies (Sec. 3.2), normalised gradient flow with
              backward Euler (Eqs. gf-eq2..gffg33), the adjoint and the
              tangent-linear model of the TSFP step.
split         the improved split algorithm (Eq. 3.9): a padded-FFT convolution
              with the smooth part of the symbol plus a small-ball quadrature.
"""
