"""GB300-native particle-based BP update of "Soft-Coherent Direct Multipath SLAM".

The compute path is the CUDA library ``libbp`` (sm_103a) behind a C ABI
(``include/bp.h``); ``paper_2604_19723_gb300.bp`` is its thin ctypes binding.
"""
