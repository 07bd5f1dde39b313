"""FP64 CPU oracle for the fast-correlation matching-pursuit path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports it, and this package
imports nothing from the product: the two share no code.

Contents (each function cites the passage of the paper it follows):

* ``matrices``   explicit unitary A (Sylvester Hadamard, DFT) and Phi = S_Omega A
* ``omp``        Algorithm 1.1 (conventional OMP) with dense Phi^H r
* ``kernelsum``  the correlation kernel vector c, the permutations P_lambda of
                 Theorem 2-1 and the fast correlation of Eq. (kernelsum)
* ``transform``  Algorithm 1.1 for large N with Phi applied through FFT / FWHT
                 (pinned against ``omp`` at N <= 4096)
* ``pursuits``   subspace pursuit and CoSaMP in their standard forms (the
                 paper defines neither), pinned by iterates derived by hand
                 for tiny cases, the invariants each step defines, recovery
                 and OMP agreement on 1-sparse signals

Everything is plain numpy in float64 / complex128 with no blocking, fusion or
reordering beyond what the definitions state.
"""
from . import matrices, omp, kernelsum, pursuits, transform  # noqa: F401
