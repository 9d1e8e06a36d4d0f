"""GB300 (sm_103a) block-local Discontinuous DLS compressor (arXiv 2601.20113).

``dls`` is the binding of the C ABI in include/dls.h; ``synth`` holds the
seeded synthetic field generators.  The CUDA library loads on first use.
"""
