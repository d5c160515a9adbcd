"""B300-native (sm_103a) element assembly of the explicit momentum RHS.

Public pieces:
  paper_2005_05899_b300.fea      Python binding of libfea (include/fea.h)
  paper_2005_05899_b300.meshgen  seeded synthetic meshes and fields
  paper_2005_05899_b300.build    in-tree nvcc build of libfea.so

Importing the package loads nothing; the CUDA library is loaded on first use
and its absence is an error (there is no CPU fallback).
"""
__all__ = ["fea", "meshgen", "build"]
