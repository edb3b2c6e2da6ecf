"""GB300-native ray-parameterized reverberation hot path.

Backward path tracing with diffuse rain into low-rate spherical-harmonic energy
histograms, followed by per-band reverberation-parameter estimation (Schissler &
Manocha, Sections 4.2 and 5), as hand-written CUDA for sm_103a behind a C ABI.

``paper_1803_00430_gb300.rpr`` is the thin ctypes binding of that ABI; it loads the
compiled library on first use and raises if it is missing.  ``scenes`` builds the
seeded synthetic workloads.
"""
__all__ = ["rpr", "scenes"]
