"""FP64 CPU oracle for the block-floating-point FFT and SAR range-Doppler path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the CPU-baseline leg
of the benchmark do.  It shares no code with the CUDA library (no kernels,
headers, tables or helpers) and imports nothing from it.

Every function here is a plain, slow, obviously correct restatement of a
definition, in float64 / complex128:

* ``oracle.fft``       -- the DFT and its normalised inverse (Section III-B),
                          computed with a plain iterative radix-2 FFT and a
                          brute-force O(N^2) DFT for checking.
* ``oracle.sar``       -- matched-filter compression y = IDFT(DFT(x) . H)
                          along range lines and azimuth columns (Section III-B,
                          Fig. 1), and the stage magnitudes of the naive
                          (unshifted) FP16 pipeline (Section III-B, IV-A).
* ``oracle.quant``     -- IEEE binary16 and OCP FP8 (E4M3, E5M2) rounding,
                          round-to-nearest-even, written from the formats'
                          definitions (Section VII).
* ``oracle.metrics``   -- scale-aligned SQNR (Section IV-B) and point-target
                          PSLR / ISLR / 3 dB width / SNR (Section VI).
* ``oracle.autofocus`` -- image entropy of the azimuth-compressed image under
                          a per-pulse phase correction and its analytic
                          adjoint gradient.
* ``oracle.emulate``   -- a radix-2 FFT with rounding hooks at storage points,
                          products and sums: the precision modes of Tables I
                          and V and Section VI, and the error model that
                          predicts a storage schedule's SQNR.
* ``oracle.conv``      -- circular convolution and correlation by their
                          defining sums, and the forward-multiply-inverse
                          pipeline that computes them (Section VIII).
* ``oracle.bfp``       -- adaptive per-line block exponents (Section VIII).
* ``oracle.rda``       -- range-Doppler processing with range-cell migration
                          correction and a range-dependent azimuth filter
                          (Section VI's RCMC stage).

Pins: each function is checked by the ``-m "not gpu"`` tests against facts
fixed by the mathematics or printed in the paper (brute-force DFT, Parseval,
impulse / constant spectra, round trips, shift theorem, chirp closed forms,
format edge values, finite differences, the SQNRs of Tables I and V).  One
reading stays unpinned by the paper and says so in its docstring: the FP16
autofocus gradient tolerance.
"""

from . import fft, quant, sar, metrics, autofocus, emulate, conv, bfp, rda  # noqa: F401
