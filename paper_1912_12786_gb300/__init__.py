"""GB300-native custom-intersector BVH traversal (Zellmann, arXiv 1912.12786).

The GPU library lives in ``csrc/`` and is reached through the C ABI declared in
``include/vsr.h``; ``paper_1912_12786_gb300.vsr`` is the thin ctypes binding.
Importing this package does not load the CUDA library; ``vsr`` does, and fails
loudly when it is missing.
"""
