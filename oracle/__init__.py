"""CPU oracle for the multiple rank-1 lattice sparse FFT.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the CUDA library and its Python binding) never imports
or calls anything here, and this package imports nothing from the product.

The oracle is a plain, slow, fp64 restatement of the paper (Kaemmerer, Potts,
Volkmer, "High-dimensional sparse FFT based on sampling along multiple rank-1
lattices"):

* ``philox``  - Philox4x32-10 counter-based generator (Salmon et al., SC'11),
  written from its published definition, plus the draw conventions (uniform
  anchors, generating vectors, Box-Muller noise).
* ``lattice`` - rank-1 lattice residues, reconstruction property (Section 2.1),
  Algorithm 1 (randomized multiple rank-1 lattice construction with the prime
  set of Eq. 2.2), Algorithm 2 (inverse multiple rank-1 lattice FFT), lattice
  evaluation (Section 4.1 aliasing identity) and its adjoint.
* ``sfft``    - Algorithm 3 (dimension-incremental sparse FFT), its 1-D
  detection steps and thresholded top-s selection.
* ``bspline`` - the tensor-product B-spline test function of Section 5.3
  (spatial-domain evaluation, exact Fourier coefficients, L2 error).

Every function says which passage it follows.  Pins that tie the oracle to
the paper and to mathematics live in ``tests/test_oracle_*.py``.
"""

from . import philox, lattice, sfft, bspline  # noqa: F401
