"""GB300-native inter-agent relocalisation hot path (Golodetz et al., Sec. 3.3.1).

The compute path lives in ``csrc/`` (sm_103a CUDA behind a C ABI declared in
``include/relo.h``); ``binding`` loads that library with ctypes and passes raw
device pointers and streams.  Importing this package does not load the CUDA
library: ``binding.lib()`` does, and fails loudly when it is missing.
"""
__all__ = ["binding", "synth", "presets", "study", "checkpoint"]
