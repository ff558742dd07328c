"""GB300-native SparseStack sketching (Y = S A with FP32 / FP16 accumulation, sketch-and-solve,
batched launches and a serving loop). The compute path is libsk.so (CUDA, sm_103a); this package
holds its ctypes binding (`sk`), the seeded input generators (`inputs`), the tile autotuner
(`autotune`) and the continuous-batching serving loop (`serve`).

Submodules are imported on demand so that `inputs` can be used without loading the CUDA library.
"""

__all__ = ["sk", "inputs", "autotune", "serve"]
