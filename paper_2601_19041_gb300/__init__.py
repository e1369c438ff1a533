"""GB300 (sm_103a) HeatACO decoder: heatmap-guided Max-Min Ant System (arXiv 2601.19041).

``heataco`` binds the CUDA library (libheataco.so, C ABI in include/heataco.h);
``synth`` draws seeded synthetic instances and heatmaps; ``build`` compiles the
library with nvcc.  Submodules are imported on demand so that the input
generators work on machines without a GPU.
"""
