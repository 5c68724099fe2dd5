"""GB300-native preconditioned multigrid Landweber reconstruction for
cone-beam CT (Myers et al., arXiv 2103.10329).

The compute path is libmgct.so (CUDA, sm_103a; C ABI in include/mgct.h);
`mgct` is its Python binding and `synth` holds the seeded input generators.
"""
