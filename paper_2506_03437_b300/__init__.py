"""B300-native implementation of the query-time hot path of Quake's adaptive
partitioned vector index (Mohoney et al., OSDI'25).

The compute runs in the CUDA library libquake_b300.so (C ABI in
include/quake_b300.h); `paper_2506_03437_b300.index.Index` is its Python face.
Importing this package alone loads nothing, so the seeded input generators in
`paper_2506_03437_b300.synth` can be used without the library.
"""
