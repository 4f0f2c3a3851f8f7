"""GB300-native (sm_103a) engine for the SimInf split-step method
(arXiv 1605.01421): per-node direct SSA, scheduled events and the post time
step, as hand-written CUDA kernels behind the C ABI of include/siminf_gpu.h.

``binding`` is the thin ctypes layer over that library; ``workloads`` builds
seeded synthetic inputs; ``emulator`` trains and quantises the learned
one-day emulator of SISe3 nodes (an extension of the method) through the
library's own tensor-core kernels.  Importing the package does not load the
CUDA library; ``binding.lib()`` does, and fails loudly when it is missing.
"""
__all__ = ["binding", "workloads", "emulator"]
