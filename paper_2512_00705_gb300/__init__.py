"""GB300-native engine for the per-step transition sampling of dynamic random
walks (node2vec, metapath, weighted) after FlexiWalker (arXiv 2512.00705).

The compute path is the CUDA library built from csrc/ (C ABI in
include/flexiwalk.h); `flexiwalk` is its thin Python binding (the library is
loaded on first use) and `synth` generates seeded synthetic inputs.
"""
from . import flexiwalk, synth  # noqa: F401

__all__ = ["synth", "flexiwalk"]
