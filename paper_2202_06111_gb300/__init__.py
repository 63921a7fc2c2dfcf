"""GB300-native graph-based invariant set (GIS) hot path.

The compute runs in the CUDA library ``libgis.so`` behind the C ABI declared in
``include/gis.h``; ``paper_2202_06111_gb300.gis`` is its thin ctypes binding.
``paper_2202_06111_gb300.workloads`` holds the seeded problem definitions.
"""
__all__ = ["gis", "workloads"]
