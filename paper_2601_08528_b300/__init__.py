"""B300-native (sm_103a) graph-ANNS hot path of SVFusion (arXiv 2601.08528).

The compute lives in ``libsvf.so`` (CUDA kernels behind the C ABI of
``include/svf.h``); this package is a thin binding that allocates device
buffers with torch and passes pointers.
"""
from ._lib import EMPTY, SvfError, load  # noqa: F401
from .index import Index, SearchConfig, Server, gather_probe, knn, knn_tc  # noqa: F401
