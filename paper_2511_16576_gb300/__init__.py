"""PolyMinHash on GB300: area-based MinHash signatures of polygons (arXiv 2511.16576).

The compute path is the C-ABI library ``libpolyminhash.so`` (hand-written CUDA for
sm_103a); :mod:`paper_2511_16576_gb300.binding` is its thin ctypes binding.
"""
