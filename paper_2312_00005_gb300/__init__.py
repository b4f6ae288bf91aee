"""GB300-native (sm_103a) collocation BEM + FMM matrix-vector product for the
3D Helmholtz equation (Burton-Miller, constant triangles), after arXiv
2312.00005.  The compute path is the C-ABI library built from ``csrc/``;
``bemfmm`` is its thin Python binding.  ``inputs`` holds seeded synthetic
inputs only."""
