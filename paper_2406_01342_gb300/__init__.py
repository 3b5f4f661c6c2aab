"""GB300 (sm_103a) implementation of the PolyCLEAN hot path (arXiv 2406.01342).

The compute path is the CUDA library libpolyclean.so (C ABI in
include/polyclean.h, sources in csrc/). `abi` is its thin Python binding,
`build` compiles it in-tree, `synth` generates seeded synthetic inputs.
"""
__all__ = ["abi", "build", "synth"]
