"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This package holds no arithmetic of the method: only the named configurations
and seeded random arrays of the right shapes.  Both the CUDA path and the
oracle consume these arrays through their own code.
"""
