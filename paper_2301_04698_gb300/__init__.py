"""GB300-native LES time step (arXiv 2301.04698, Sec. 2.1-2.4 and App. A).

``paper_2301_04698_gb300.les`` is the Python binding of ``libles.so`` (the
C ABI in ``include/les.h``); ``build`` compiles it for sm_103a;
``inputs`` holds the seeded synthetic workloads.  Importing the package does
not load the CUDA library -- ``les.load_library()`` does, and raises if the
library is missing.
"""

__all__ = ["build", "inputs", "les"]
