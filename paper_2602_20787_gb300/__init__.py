"""GB300-native (sm_103a) S1xR2 StePS hot path: direct softened image-sum
forces, finite-cylinder background and comoving KDK behind a C-ABI library.

The CUDA library is loaded lazily by ``paper_2602_20787_gb300.steps_cyl``; this
package import does not touch the GPU.
"""
__all__ = ["ics", "steps_cyl"]
