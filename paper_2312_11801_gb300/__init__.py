"""USBS hot path on GB300 (sm_103a): C-ABI library ``libusbs`` and its Python binding.

Importing the package loads nothing native; ``paper_2312_11801_gb300.usbs`` opens the
shared library (and raises if it has not been built), ``instances`` builds inputs.
"""
__all__ = ["instances", "usbs"]
