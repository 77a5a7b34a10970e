"""GB300-native El-WaveHoltz: WaveHoltz operator applies and the Krylov solve
of M (I - S) v = M Pi 0 on sm_103a, behind the C ABI of include/ewh.h.

``paper_2205_12344_gb300.api`` holds the user-facing Python wrapper,
``paper_2205_12344_gb300._lib`` the raw ctypes binding with the C names,
``paper_2205_12344_gb300.inputs`` the seeded synthetic problem generators.
"""
