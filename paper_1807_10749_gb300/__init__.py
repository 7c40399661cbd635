"""GB300-native Schroedinger-Feynman simulator of random grid circuits
(arXiv:1807.10749). The compute path is the CUDA C-ABI library in csrc/;
`sfsim` is its Python binding and `inputs` writes seeded workloads."""
