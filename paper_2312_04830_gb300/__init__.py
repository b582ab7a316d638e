"""GB300-native real-fluid (Peng-Robinson) property evaluation.

The compute path is the CUDA library ``libprgb300.so`` built from ``csrc/`` for
sm_103a; ``binding`` marshals arguments to its C ABI.  Importing this package
loads nothing: ``workloads`` (seeded synthetic inputs) is usable without a GPU
or a built library.
"""

__all__ = ["workloads", "binding"]
