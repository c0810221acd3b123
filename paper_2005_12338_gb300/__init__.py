"""GB300-native range-separated stochastic-RI GF2 self-energy (RS-SRI-GF2).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through its C ABI (``include/rssri.h``); ``binding`` marshals
arguments to it.  ``synth`` draws seeded synthetic inputs.  Submodules are
imported on demand so that input generation does not load the library.
"""
__all__ = ["binding", "synth", "build"]
