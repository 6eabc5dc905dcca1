"""GB300-native CD-WAC (contour deformation with analytic continuation of W) for core-level G0W0.

The compute path lives in the CUDA library ``libcdwac.so`` (sources in ``csrc/``); ``cdwac`` is its thin
ctypes binding.  ``inputs`` builds seeded synthetic systems and holds none of the method's arithmetic.
Nothing here is imported eagerly, so ``import paper_2305_15955_gb300.inputs`` works without the library.
"""

__all__ = ["inputs", "cdwac", "build"]
