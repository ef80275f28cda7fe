"""Measurement support of the benchmark (bench.py) and of the commands behind profiles/: probe kernels
that measure gather and FMA ceilings (their own library, libgkm_probes.so) and the profiling cases.
Nothing here is part of the clustering library or its C ABI."""
