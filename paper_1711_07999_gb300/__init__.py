"""GB300 tracker for "Dynamic High Resolution Deformable Articulated Tracking" (Walsman et al., 3DV 2017).

Every step of a tracking iteration runs in the CUDA kernels of ``libtrk.so`` behind the C ABI of
``include/trk.h``; :mod:`paper_1711_07999_gb300.trk` is its ctypes binding and
:mod:`paper_1711_07999_gb300.synth` generates seeded synthetic inputs.
"""
