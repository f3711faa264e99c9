"""Zolo-PD / Zolo-SVD (arxiv 1806.06204) on one GB300: hand-written sm_103a CUDA
behind the C ABI of include/zolo.h.

`binding` loads libzolo.so (built by `build`) and fails loudly if it is missing;
`synth` draws the seeded synthetic inputs.  Importing the package loads neither.
"""
__all__ = ["binding", "build", "synth"]
