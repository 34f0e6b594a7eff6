"""B300-native mixture-of-media random walk (sm_103a CUDA behind a C ABI).

Importing the package does not load the CUDA library; ``paper_2606_27604_b300.api``
does, and raises if it is missing.
"""
__version__ = "0.1.0"
