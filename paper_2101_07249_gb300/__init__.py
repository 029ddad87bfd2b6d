"""GB300-native inner loop of forcing-formulation weak-constraint 4D-Var with
randomised spectral-LMP preconditioning.  The compute runs in libwc4d.so
(hand-written CUDA for sm_103a); this package is its thin ctypes binding."""
