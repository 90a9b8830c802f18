"""FP64 CPU oracle for the scalar weak-object imaging model and its inverse.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
bench's CPU-baseline / reference legs may import or run anything in this
package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it.

It is a plain, slow, obviously-correct restatement of the method in numpy
float64, written from the paper's Methods section:

* ``optics``  - pupils, defocused arms, per-plane pupil correlations, the
  label-free [[1, 1], [i, -i]] combination and the fluorescence
  autocorrelation of Table 1 (scalar column), stacked into 3D transfer
  functions (Methods, "Summary of transfer functions").
* ``model``   - the linear shift-invariant forward model d = Hf + b
  (Eq. fwd, Eq. fwd_block and its Fourier form), its adjoint, and the
  per-contrast-mode Tikhonov reconstruction (Eq. recon, Eq. tls_solution),
  in 3D and in the 2D phase-from-defocus form.
* ``tiles``   - overlapping tiling and linear-ramp blending for shift-variant
  restoration (Results, "Physics-guided ML auto-tunes ..."; Methods,
  "Organelle-scale optical pooled screen data").
* ``dft``     - brute-force DFTs used to pin numpy's FFT and to take single
  Fourier coefficients of large volumes.

Pins that tie these functions to the paper and to closed forms live in
``tests/test_oracle_pins.py``.  Functions whose conventions the paper does not
fix say so in their docstrings; none is "parity unpinned".
"""
from . import dft, optics, model, tiles  # noqa: F401
