"""GB300-native 2D nonseparable discrete LCT (CM-CC-CM-CC chain).

The compute path is the C-ABI library ``libnslct.so`` (hand-written sm_103a
CUDA); ``paper_1707_03688_gb300.nslct`` is its thin Python binding. Importing
the package itself loads nothing: the binding loads the library on first use
and raises if it is missing.
"""
__all__ = ["inputs", "nslct"]
