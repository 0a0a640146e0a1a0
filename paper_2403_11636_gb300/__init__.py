"""GB300-native restricted additive smoother and geometric multigrid for
finite cell Stokes problems (Saberi & Vogel, Sec. 3).

The CUDA library ``libfc`` (C-ABI, ``include/fc.h``) does all the numerical
work; ``paper_2403_11636_gb300.fc`` is its thin ctypes binding.  Importing the
package itself loads nothing; ``inputs`` holds the seeded workload generators.
"""
__all__ = ["fc", "inputs"]
