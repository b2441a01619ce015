"""GB300-native parallel-tempering hardness engine for Chimera Ising instances.

Implements the hot path of "Practical engineering of hard spin-glass instances"
(arXiv:1605.03607): PT-based time-to-solution measurement of an instance, the random adaptive
optimisation loop (Algorithm 1) around it, and loop adaptive optimisation of
planted-solution instances (Algorithm 2).  The compute runs in
hand-written sm_103a kernels behind the C ABI of include/pt.h; this package is
the Python binding of that ABI.
"""
from ._lib import (PT_KMAX, PT_TARGET_BEST, PTError, PTHandle, load, pt_rule,  # noqa: F401
                   pt_step_result, SIGNATURES, LIB_PATH, select_device, PTBatch, Surrogate,
                   PT_LOOP_WORDS, pt_lao_result, lao_plant, int_issue_rate, INT_ISSUE_KINDS,
                   debug_enabled, debug_status)
