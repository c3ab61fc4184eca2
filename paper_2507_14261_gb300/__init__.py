"""GB300-native FAMST: approximate Euclidean MST of large point clouds.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/famst.h``); ``famst`` is its Python binding.
"""
from .famst import (BatchInfo, BuildInfo, Context, Edges, FamstError, MSTWeight, Tree,  # noqa: F401
                    default_context, lib, library_path, mst_weight)

__all__ = ["BatchInfo", "BuildInfo", "Context", "Edges", "FamstError", "MSTWeight", "Tree",
           "default_context", "lib", "library_path", "mst_weight"]
