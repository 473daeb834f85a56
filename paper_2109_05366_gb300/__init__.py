"""GB300 GPU file-read path: GPU page cache + readahead prefetcher + streaming
replacement, served by host I/O threads over a request ring.

Method: "A readahead prefetcher for GPU file system layer" (Dimitsas and
Silberstein).  The compute path is libgfs.so (CUDA for sm_103a + C++ host
runtime) behind the C ABI in include/gfs.h; `gfs` is its ctypes binding.
"""
from . import gfs  # noqa: F401
from .gfs import Context, GfsError, load  # noqa: F401
