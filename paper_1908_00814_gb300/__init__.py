"""GB300-native k-NN graph merge (Zhao et al., "On the Merge of k-NN Graph").

The compute path is the C-ABI library ``libknnm.so`` (CUDA kernels for
sm_103a, declared in ``include/knnm.h``); :mod:`.knnm` is a thin ctypes
binding over it.  Importing this package does not load the library; the first
call into :mod:`.knnm` does, and fails loudly when it has not been built.
"""
