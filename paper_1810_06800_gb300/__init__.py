"""GB300-native RSA of linear k-mers on an L x L torus: jamming count n_j and
first-wrap count n_c per sample (arXiv:1810.06800), computed by hand-written
sm_103a CUDA kernels behind a C ABI (``include/rsa.h``).

Importing the package is cheap; the CUDA library is loaded by
:mod:`paper_1810_06800_gb300.rsa` on first use and fails loudly if it is
missing."""

__all__ = ["rsa", "workloads", "study", "serve"]
