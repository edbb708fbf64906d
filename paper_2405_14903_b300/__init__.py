"""B300-native differentiable cut-cell fluid step (arXiv 2405.14903).

The compute path is ``libnf.so`` (hand-written CUDA for sm_103a behind the C
ABI in ``include/nf.h``); this package only marshals arguments. Importing it
fails if the library has not been built (``python
paper_2405_14903_b300/build.py``): there is no CPU fallback.
"""

from ._lib import LIB_PATH  # noqa: F401  (loads libnf.so or raises)
from .api import Context, Episode, NFError, NotConvergedWarning, Server, loss_noalloc  # noqa: F401
from .autograd import rollout_loss  # noqa: F401

__all__ = ["Context", "Episode", "NFError", "NotConvergedWarning", "Server", "rollout_loss",
           "loss_noalloc",
           "LIB_PATH"]
