"""GB300-native dynamic-screening solver for the Lasso and Group-Lasso (arXiv 1412.4080).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/dscreen.h``); this package only marshals arguments to it.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import DscreenError, declared_functions, lib  # noqa: F401
from .build import build  # noqa: F401
