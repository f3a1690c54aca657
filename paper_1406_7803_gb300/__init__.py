"""GB300-native periodic frozen-density-embedding (subsystem DFT) hot path.

The CUDA library (``libfde.so``, built from ``csrc/``) is loaded by
``paper_1406_7803_gb300.fde`` on first use; ``workloads`` holds the seeded synthetic
inputs and no arithmetic of the method.
"""
