"""GB300-native ILVES constraint solve: C-ABI CUDA library + thin Python binding.

Importing the package is cheap; the CUDA library is loaded on first use of
``paper_2503_13075_gb300.ilves`` (see ``binding.py``).
"""
__all__ = ["workloads", "binding"]
