"""CPU oracle for the accelerated filtered back projection (IIR ramp filter + fast Hough
transform back projection) of Dolmatova, Chukalina and Nikolaev, arXiv 2007.06289.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct reference
that the CUDA path is checked against.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the library itself never does, and this
package imports nothing from the library.  It is written in numpy, in float64 unless a
function says otherwise, and each function cites the paper passage it follows.

Modules
-------
ramp       the band-limited ramp kernel h(n) and its causal/anticausal split (Eq. 6-7, 10)
iir        the causal and anticausal recursive filters and their sum (Eq. 9, 12-13), and the
           exact FIR ramp filter used by the direct reconstruction (Eq. 8)
geometry   the four line classes and the (r, theta) <-> (s, t) map (Sec. 4.1-4.2, Eq. 14-15)
linogram   bilinear resampling of the filtered sinogram into the four linogram quarters
dyadic     dyadic patterns, brute-force pattern back projection, the stage-by-stage fast
           Hough transform (float32 or float64) and the quarter sum (Sec. 4.3-4.5, Eq. 16-22)
fbp        the whole fast method, and the direct Theta(N^3) FBP used as the quality judge
           (Eq. 3-5)
adjoint    transposes of the filter, the resampling and the back projection (gradients of
           the fast method with respect to the sinogram)
sirt       algebraic reconstruction (SIRT) on the fast Hough operators and the Hough-space
           data of a sinogram (Sec. 4.4)
radon      the fast Radon transform: dyadic line sums (Eq. 17) resampled to (theta, r)
cnn        the learned corrector's network, loss and gradients (an extension beside the
           paper's method)

Readings of the paper that the oracle fixes where the text is silent or garbled are
listed in each module's docstring.
"""
from . import ramp, iir, geometry, linogram, dyadic, fbp, adjoint, sirt, radon  # noqa: F401
from .ramp import ramp_h, ramp_h_sinc, causal_part, anticausal_part  # noqa: F401
from .iir import (iir_causal, iir_anticausal, iir_filter, iir_impulse_response,  # noqa: F401
                  fir_ramp)
from .geometry import QUARTERS, slopes, quarter_angle, quarter_r, row_weights  # noqa: F401
from .linogram import sample_filtered, linogram_at, linogram  # noqa: F401
from .dyadic import (dyadic_pattern, pattern_backproject, fht_stages,  # noqa: F401
                     combine_quarters)
from .fbp import (fast_fbp, fast_backproject, fast_fbp_pixels, direct_fbp, direct_fbp_pixels,  # noqa: F401
                  fht_backproject)
from .adjoint import (quarter_gradients, pattern_backproject_adjoint,  # noqa: F401
                      fht_stages_adjoint, fht_backproject_adjoint, linogram_adjoint,
                      fast_fbp_adjoint)
