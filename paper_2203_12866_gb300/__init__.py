"""GB300-native COSEnu RK4-stage engine (arXiv:2203.12866).

The compute path is the CUDA library ``libcosenu.so`` (sources in ``csrc/``,
C ABI in ``include/cosenu.h``); ``binding`` marshals arguments to it.
``inputs`` builds seeded synthetic initial states.
"""
__all__ = ["inputs", "binding"]
