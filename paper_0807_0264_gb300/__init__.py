"""GB300-native Maximal Center Gauge fixing with stout / over-improved stout
preconditioning, Z3 center projection and P-vortex counting.

The compute path is the C-ABI library `libmcg.so` (hand-written CUDA for
sm_103a, declared in include/mcg.h); `paper_0807_0264_gb300.mcg` is its thin
Python binding.  `synth` builds seeded synthetic input fields.
"""
__all__ = ["synth"]
