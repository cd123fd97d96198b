"""GB300 (sm_103a) interval-arithmetic Apollonius voting for a full-stereo drift chamber
(arXiv:2401.04576).  The CUDA kernels and the C ABI live in csrc/ and include/apo.h; apo.py
is the Python binding and build.py compiles the library in-tree."""
