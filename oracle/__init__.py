"""FP64 CPU oracle for the long-range step of Ewald summation with prolates (ESP).

This package is TEST INFRASTRUCTURE.  Only the test suite, the smoke check of the
build entry point and the CPU-baseline / reference legs of the benchmark may import
it.  The CUDA library never imports, links or executes anything here, and nothing
here imports the CUDA library: the two share no code.  The only module both sides
use is the seeded input generator package ``synthetic`` (positions, charges and cells;
it holds none of the method's arithmetic).

Modules (each function cites the passage of the paper it follows):

* ``pswf``      - O-PSWF: the order-zero prolate spheroidal wave function psi_0^c,
                  its eigenvalue lambda_0, C_0 and derivatives (Appendix A.1,
                  eq. (formula)/(psidefinit)).
* ``ewald``     - O-EWALD: classical Ewald summation with an explicit k-sum
                  (Sec. 2.1), energy, forces and the full 3x3 virial tensor.
* ``esp_split`` - O-SPLIT: the PSWF kernel split with exact structure factors
                  (Sec. 3.1-3.4, eqs. (UN), (UF), (selfen), (PinsN), (Far), (Corr),
                  Appendix C eq. (Fc)).
* ``esp_grid``  - O-GRID: the gridded ESP quantity (Sec. 4.1 Algorithm 1, Sec. 4.2,
                  Sec. 4.3; Appendix C eq. (AD)) evaluated plainly: direct spreading,
                  a library FFT, mode-by-mode scaling, direct gathering.
* ``pressure``  - coupling projections of the 3x3 tensor (Sec. 2.2) and the paper's
                  error metrics (Sec. 5.1, eq. (ref_pres)).
"""
