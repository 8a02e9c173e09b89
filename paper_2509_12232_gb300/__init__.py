"""GB300-native docking hot path (muDock method, arXiv 2509.12232).

``dock`` binds the CUDA library ``libdock.so`` (include/dock.h); ``synth``
draws the seeded synthetic workloads; ``build`` compiles the library.
"""
__all__ = ["dock", "synth", "build"]
