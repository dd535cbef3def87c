"""GB300-native QAOA MaxCut energy by lightcone bucket elimination.

``qtgb`` is the binding of the C ABI in ``include/qt.h``; ``synth`` draws the
seeded synthetic graphs and angles; ``build`` compiles ``libqtgb.so``.
"""
from . import synth  # noqa: F401
from .qtgb import Plan, QTError, plan, plan_batch  # noqa: F401
