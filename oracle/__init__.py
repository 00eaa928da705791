"""Plain, slow FP64 CPU oracle for the Wilson / domain-wall Dirac operators,
the even-odd Schur complement, conjugate gradient, the fermion force, the
SU(3) x SU(3) field product, the Wilson gauge action with its force, the
HMC molecular-dynamics trajectory, the G-parity Wilson operator and the
multigrid aggregation and coarse-grid operator.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this package; only
the test suite, the smoke check and the CPU-baseline / reference leg of the
benchmark may use it. It shares no code with the CUDA path: it works on
full-lattice numpy arrays in the host layout of :mod:`synthetic`
(``psi[..., t, z, y, x, spin, colour]``, ``U[t, z, y, x, mu, row, col]``),
shifts fields with ``np.roll`` and multiplies full 4x4 spin matrices.

The paper (Grid, arXiv:1512.03487) names these operators and algorithms but
does not write them down ("Wilson and Domain Wall fermion operators", Sec. 3;
"Conjugate gradient", "HMC", "Wilson Fermion Action", "Five dimensional chiral
fermions", Sec. 4). Each module restates the textbook definition with the
convention chosen where the paper is silent, and each function is pinned by a
test against a closed form, an identity or brute force; see the module
headers. No function here is "parity unpinned".
"""
from . import gamma, wilson, dwf, cg, force, su3, gauge, hmc, gparity, mg  # noqa: F401
