"""CPU FP64 oracle for the FTH-MS per-(open arc, omega) hot path (arxiv 2507.05725).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or execute anything in this package.  The
product path (the CUDA library and its Python binding) never calls it and shares no code with it.

The oracle is a plain, slow, readable numpy/scipy restatement of the discrete method:

* ``geometry``   -- arcs, first-kind Chebyshev nodes, the boundary partition of unity chi_j
                    (Section 3.1, eqs. POU1 and eta), overlap masks (eq. vtilde).
* ``kernels``    -- the single-layer kernel Phi = (i/4) H0^(1) (Section 2.1), its log split and the
                    Chebyshev product-integration weights for the open-arc BIE (Section 4.2-4.3,
                    the endpoint weight of eq. singularity), cross-arc evaluation rows.
* ``transforms`` -- signal, incident fields, the time window of Section 5, the slow forward
                    transform (eq. Fourierk) and the recentred inverse transform (eq. TDsol).
* ``fthms``      -- the multiple-scattering driver of Algorithm 1 and eqs. criterion_int1/2.

Every function cites the passage it follows.  Readings of passages that the paper leaves open are
stated in the docstrings of the functions that take them.  Library primitives used as steps: scipy.special
Bessel functions, LAPACK LU (scipy.linalg.lu_factor), numpy matrix products.
"""
from .fthms import run_oracle, OracleResult  # noqa: F401
