"""GB300-native Wallace normal generator (Brent's vectorised RANN4 form).

The compute lives in libwallace.so (CUDA, sm_103a) behind include/wallace.h;
`paper_1004_3114_gb300.wallace` is the thin ctypes binding over it.
"""
