"""GB300-native (sm_103a) hot path of WaveOrder's linear wave-optical model.

The compute path is the CUDA library behind include/wo.h; ``binding`` is its
ctypes binding (marshalling only).  Build the library with
``paper_2412_09775_gb300.build.build()``.
"""
