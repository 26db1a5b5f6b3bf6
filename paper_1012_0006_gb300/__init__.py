"""GB300-native flow-based refinement of block pairs (Sanders & Schulz, Section 4.1 / 4.1.1).

The compute path lives in lib/libflowref.so (CUDA, sm_103a) behind include/flowref.h;
`flowref` is its Python binding and `inputs` builds seeded synthetic workloads.
"""
