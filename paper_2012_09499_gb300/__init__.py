"""GB300-native steered response power (SRP) mapping: conventional SRP and its
Nyquist-Shannon approximation (Dietzen, De Sena, van Waterschoot, WASPAA 2021),
computed by hand-written sm_103a CUDA kernels behind a small C ABI.

Importing the package loads nothing; ``paper_2012_09499_gb300.srp`` loads the
compiled library on first use and raises if it is missing.
"""
__all__ = ["srp", "synth"]
