"""GB300-native electromagnetic shower transport (arXiv:2203.09467 hot path).

The transport loop runs in libemt.so (hand-written CUDA for sm_103a behind
the C ABI in include/emt.h); `emt` is its Python binding and `workloads`
holds the seeded synthetic inputs.
"""
