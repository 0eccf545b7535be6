"""GB300-native grouped-isochromat Bloch simulator (libmrsim + Python binding).

The CUDA library is built in-tree by ``paper_2508_03960_gb300.build``; the
binding lives in ``paper_2508_03960_gb300.mrsim``.
"""
