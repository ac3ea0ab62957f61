"""CPU FP64 oracle for randomized QR with column pivoting (Duersch & Gu).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, header, table or helper with the CUDA path under
``paper_1509_06820_gb300/csrc``.

Every routine is a plain, slow, step-by-step restatement of the paper in numpy
float64.  numpy's matmul serves as a library primitive for the dense products
the algorithms name; nothing is blocked, fused or reordered beyond what the
algorithms themselves state.

Contents (paper sections in brackets):

* ``philox``      -- counter-based Philox4x32-10 generator (Salmon et al. SC'11)
                     and the Gaussian compression matrix Omega [Sec. 3, Alg. 3 / Alg. 4].
* ``householder`` -- Householder reflector, unblocked panel QR, compact-WY T
                     factor and block-reflector application [Sec. 2.1-2.2, Sec. 5.1].
* ``rqrcp``       -- partial QRCP on the sample [Alg. 1, Sec. 5], the full
                     deterministic QRCP it stands in for [Alg. 1], RQRCP with the
                     sample update formula [Alg. 4, Eq. (3)], repeated-sampling
                     RQRCP [Alg. 5], the unpivoted
                     blocked QR it reduces to [Table 3 note], TRQRCP [Alg. 6]
                     and TUXV [Alg. 7], with j_max iterations and the SVD of
                     the connection matrix X.

* ``selection``   -- the expected norm of the sample-selected column for
                     orthogonal columns with geometric norms [Sec. 3.2, sample
                     bias, Fig. selectExpect], by quadrature over chi variables;
                     the truncated chi-squared law of the trailing sample norms
                     after pivoting and the truncation bounds of a partial
                     sample factorization [Sec. 3.3, norm truncation].

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a library routine, a closed form, a
brute-force enumeration or a statistical law stated in the paper.
"""

from . import philox, householder, rqrcp, selection  # noqa: F401
from .rqrcp import (  # noqa: F401
    sample_qrcp,
    qrcp,
    rqrcp,
    rsrqrcp,
    qr_blocked,
    trqrcp,
    tuxv,
    tuxv_svd,
    PivotMismatch,
)
from .philox import philox4x32_10, gaussian_omega  # noqa: F401
