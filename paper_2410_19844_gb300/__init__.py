"""GB300 engine for the over-parameterised sum-of-squares method of Keren,
Osadchy and Poranne (arXiv 2410.19844): the loss-and-gradient step of
1/2 ||c(A) - p||^2 and its first-order update, as hand-written sm_103a CUDA
behind the C ABI of ``include/sos_gb300.h``.
"""
from ._lib import SOSError, lib, library_path  # noqa: F401


def __getattr__(name):
    # torch-dependent front end, imported on first use
    if name in ("Plan", "Optimizer"):
        from . import engine
        return getattr(engine, name)
    if name in ("SOSLossGrad", "sos_loss"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
