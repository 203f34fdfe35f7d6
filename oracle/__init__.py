"""Plain FP64 CPU oracle for the Zel'dovich initial-conditions path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and nothing here imports the product.

The oracle is the slow, obviously-correct statement of what the method
computes (Ginnungagap, arXiv:2511.10353):

* ``philox``    Philox4x32-10 counter-based generator (Salmon et al., SC'11),
                the stand-in for the paper's SPRNG white noise (Sec. 2.1).
* ``noise``     Gaussian white noise W(x) keyed by (seed, global cell index),
                Box-Muller on Philox uniforms (Sec. 2, step 1).
* ``cosmology`` BBKS / Eisenstein-Hu no-wiggle transfer functions, sigma_8
                normalisation, linear growth D(a) and f(a) (inputs named in
                Sec. 2.1: cosmological parameters and the power spectrum).
* ``fields``    Eq. 1 (delta = sqrt(P) W in Fourier space), Eq. 2
                (v_j = i delta k_j / k^2) and Eq. 3 (Zel'dovich positions),
                with numpy/scipy FFTs as the transform step.
* ``adjoint``   The transpose of the linear map W -> psi and of the CIC /
                smoothing chain used for gradient checks.
* ``refine``    Appendix A white-noise refinement (Eqs. A.1-A.28).
* ``particles`` Sec. 2.2 particle-set options (periodic shift, gas pairs,
                coordinate IDs) and the Sec. 2.4 degraded field.
* ``stats``     Sec. 2.1 diagnostics: shell-averaged power spectrum and
                moments of a field.
* ``merge``     Sec. 2.4: large scales of a coarse field (Eq. 5, with the
                cloud-in-cell deconvolution and interpolation) plus small
                scales of a fine one (Eq. 4), then Eq. 3.

Every function states the passage it follows. Where the paper is silent the
reading taken is stated at the function. Parity is pinned in
``tests/test_oracle_*.py`` against closed forms, brute-force sums and library
routines; functions with no such pin say "parity unpinned" in their docstring.
"""
