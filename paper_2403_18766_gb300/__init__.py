"""GB300 (sm_103a) competitive-sample-size Big-means (arXiv 2403.18766).

The compute path is the CUDA library libbigmeans.so (C ABI in
include/bigmeans.h); ``paper_2403_18766_gb300.native`` is its Python binding
and ``paper_2403_18766_gb300.synthetic`` draws the seeded synthetic inputs.
Importing the package itself loads neither, so the input generators stay
usable without a GPU.
"""
__all__ = ["native", "synthetic", "build"]
