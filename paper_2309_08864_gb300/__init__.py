"""SO2DR on one GB300: out-of-core stencil sweeps with on- and off-chip data
reuse (arxiv 2309.08864), as a C-ABI library (include/so2dr.h, libso2dr.so)
with a thin Python binding.  Importing the package loads nothing; the binding
loads the CUDA library on first use and raises if it is missing."""

__all__ = ["so2dr", "inputs", "build"]
