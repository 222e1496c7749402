"""GB300 (sm_103a) implementation of randomized Tikhonov regularization
(Meier & Nakatsukasa): sketch A once, build a preconditioner per lambda from
the partly exact sketch, and run preconditioned LSQR for every lambda.

The numerical path lives in libtikhonov.so (CUDA, include/tikhonov.h);
``tikhonov`` is its ctypes binding and ``datagen`` builds seeded synthetic
problems shaped like the paper's experiments.
"""
from . import build  # noqa: F401

__all__ = ["build", "tikhonov", "datagen"]
