"""GB300-native directionally unsplit Riemann-solver fluid update of batches of
AMR patch groups (Schive, Zhang & Chiueh 2011, arXiv:1103.3373).

The compute path is libhydro.so (hand-written sm_103a CUDA behind a C ABI,
include/hydro.h); `hydro` is its Python binding, `workloads` the seeded
synthetic inputs, `runtime` the batched / serving drivers built on the C ABI.
Importing the package does not load the library.
"""
