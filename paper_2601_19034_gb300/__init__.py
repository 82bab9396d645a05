"""GB300-native qNEP force call (neuroevolution potential with dynamic charges).

Importing the package is cheap: the CUDA library is loaded on first use of
``paper_2601_19034_gb300.qnep`` (see ``_lib.load``).
"""
__all__ = ["workloads"]
