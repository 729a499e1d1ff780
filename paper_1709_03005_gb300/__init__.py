"""GB300-native close-coupling Hamiltonian build (MPI-SCATCI's hot path).

The compute path lives in the CUDA library csrc/ (C ABI in include/hb.h);
`hb` is its Python binding and `synth` the seeded problem generator.
"""
__all__ = ["hb", "synth", "build_ext"]
