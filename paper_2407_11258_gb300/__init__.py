"""GB300-native fragment CCSD(T) (LNO-CCSD(T) hot path): liblnocc (CUDA, sm_103a) and its binding.

Submodules: `lnocc` (ctypes binding of include/lnocc.h), `synth` (seeded synthetic inputs),
`build` (nvcc build of liblnocc.so). Importing the package loads nothing.
"""
__all__ = ["lnocc", "synth", "build"]
