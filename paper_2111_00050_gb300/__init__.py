"""GB300 (sm_103a) solver for interacting bosonic momentum modes in sector-
restricted Fock space (arXiv:2111.00050).  The compute lives in libqb
(csrc/, C ABI in include/qb.h); this package is its thin Python binding."""
from ._lib import (QB_AT_START, QB_CROSSED, QB_EINTERNAL, QB_EUNSUPPORTED, QB_NOT_CROSSED, QbError,  # noqa: F401
                   lib)
from .api import AdjointLoss, Space, adjoint_loss, breaktime, meanfield  # noqa: F401
