"""GB300 (sm_103a) implementation of the hybrid time-domain / spatial-frequency
3-D reconstruction for mechanically scanned polyline arrays (Wang, Li, Zhao,
Sun, arXiv 2109.02842), monostatic and multistatic.

The compute path is the CUDA shared library ``libpolyline.so`` behind the C
ABI declared in ``include/polyline.h``; ``binding`` marshals arguments to it.
Importing this package loads nothing; ``binding`` raises if the library has
not been built.
"""
__all__ = ["binding", "workloads"]
