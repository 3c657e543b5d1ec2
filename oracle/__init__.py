"""FP64 CPU oracle for one Hessian-free ray-Born frequency-set update.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference that the CUDA library is checked against.  Only the tests, the
smoke check and the CPU-baseline timing of ``bench.py`` may import it; the
product path never does, and it shares no code with the CUDA library.

It follows the paper's statement of the problem step by step, in double
precision:

* geometry.py - ring, pixels and support (Sec. 4 acquisition);
* fields.py   - sound-speed derivative grids and bilinear sampling;
* rays.py     - ray fans: Eikonal characteristics and dynamic ray tracing
                (Eqs. 6-7), in the C file rb_oracle.c;
* grid.py     - first-arrival gridding of the fans onto pixels;
* green.py    - high-frequency 2-D Green's function (Eqs. 4-5) with
                absorption and power-law dispersion;
* link.py     - ray linking to receivers: the ray-model data p(c) of Eq. 8;
* born.py     - Born forward operator, its adjoint and the Gauss-Newton
                Hessian diagonal (the linearisation of Eqs. 9-10);
* update.py   - data weighting (75 % receiver mask, 1 % outlier zeroing),
                the diagonal one-step update, the frequency sweep and the
                CG variant of the linear solve;
* tof.py      - the time-of-flight initial guess (straight-ray SIRT,
                linearised about the current medium).

Parity status: every function is pinned by tests under tests/test_oracle_*.py
against closed forms, library routines or brute force.  The KMAH phase shift of
green.py and the KMAH index of the rays and the gridding are pinned past a caustic
against an independent finite-difference solution of the Helmholtz equation
(tests/test_oracle_kmah.py).  The sweep
(update.sweep) has no printed value to match; it is pinned by properties the
mathematics and the method fix: the true medium is a fixed point under its own
noise-free data, and on noise-free data the error to the phantom falls set by
set.
"""
