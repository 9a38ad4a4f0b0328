"""GB300-native (sm_103a) evolutionary fitter for static binary-lens microlensing lightcurves
(Rajpaul 2012). The computation lives in the CUDA library ``libsblm.so`` (C ABI in
include/sblm.h); ``paper_1208_4830_gb300.sblm`` is its Python binding and
``paper_1208_4830_gb300.synth`` generates seeded synthetic inputs."""
