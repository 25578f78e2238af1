"""GB300 (sm_103a) implementation of the stochastic-TDH action of W and the Tamm-Dancoff A of
arXiv 2205.06690 (Bradbury, Nguyen, Caram, Neuhauser). The compute path is libsbse.so (CUDA);
`binding` is its ctypes interface."""
from . import binding  # noqa: F401
from .binding import (  # noqa: F401
    Context,
    SbseError,
    TDHParams,
    SBSE_COEFF_GAUSSIAN,
    SBSE_COEFF_SIGN,
    SBSE_DIRECT,
    SBSE_EXCHANGE,
    SBSE_FP64,
    SBSE_MIXED,
)
