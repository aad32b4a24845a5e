"""GB300-native (sm_103a) Metropolis-within-Gibbs sampler for single-plate hierarchical
models (arXiv:2105.08026, CUDAHM): per-member robust adaptive Metropolis, exact grid-wide
reduction for the population step, and the selection integral of the thinned
point-process likelihood, all in one persistent CUDA kernel behind a C ABI.

Modules: ``cudahm`` (ctypes binding of include/cudahm.h), ``build`` (nvcc build of
lib/libcudahm.so), ``synth`` (seeded synthetic catalogs).
"""
