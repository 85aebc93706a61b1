"""GB300 (sm_103a) implementation of the VMC energy / force / covariance hot path
and the accelerated Langevin step of Sorella & Mazzola (arXiv:1605.08423).

The compute lives in libqmcmd.so (CUDA kernels behind the C ABI of
include/qmcmd.h); :mod:`.qmcmd` is its Python binding and :mod:`.synth` makes
the seeded synthetic inputs.
"""
