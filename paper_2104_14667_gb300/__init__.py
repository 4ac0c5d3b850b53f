"""GB300-native iterative ensemble compositor (Johnson & Jankun-Kelly,
"Efficacy of Images Versus Data Buffers").

The compute path is the CUDA library ``libcomposite.so`` built from ``csrc/``
for sm_103a; ``binding`` is a thin ctypes layer over its C ABI.
"""
