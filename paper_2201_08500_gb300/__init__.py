"""GB300-native two-beam FFT beam propagation method (BPM) for time-dependent
Bragg diffraction in deformed crystals (Krzywinski & Halavanau, arXiv:2201.08500).

The compute path is the C-ABI library ``libbpm.so`` (hand-written CUDA for
sm_103a); :mod:`paper_2201_08500_gb300.bpm` is its thin ctypes binding and
:mod:`paper_2201_08500_gb300.workloads` generates seeded synthetic inputs.
"""
