"""GB300-native t-product regularization (RT-tSVD, tGKB, Tikhonov-tGKB).

The compute path is the CUDA library built from csrc/ (libtprod.so); the
Python module `tprod` only marshals arguments to its C entry points.
"""
