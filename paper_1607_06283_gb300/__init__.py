"""GB300-native event-camera intensity reconstruction on the event manifold.

Reinbacher, Graber, Pock, BMVC 2016 (arXiv:1607.06283), hot path: per event
packet, integrate the events into the time surface and the data image, then run
warm-started primal-dual TV-KL iterations on the event manifold.  The C ABI lives
in include/evr.h and libevr.so (built by ``build.build()``); ``evr`` is its thin
ctypes binding.
"""
__all__ = ["build", "evr"]
