"""GB300-native Jump Restore light transport (arXiv 2409.07148).

Importing the package loads nothing native; ``paper_2409_07148_gb300.jr``
loads the CUDA library and fails loudly when it is missing.
"""
__all__ = ["scenes", "jr"]
