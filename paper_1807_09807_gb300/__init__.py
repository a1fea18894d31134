"""GB300-native high-order TMOP (Target-Matrix Optimization Paradigm).

The compute path lives in ``libtmop_gb300.so`` (hand-written sm_103a CUDA
behind a C ABI declared in ``include/tmop.h``); this package only marshals
arguments to it. ``meshgen`` builds the seeded synthetic input meshes.
"""
