"""FP64 CPU oracle of the event-manifold reconstruction (test infrastructure only).

Used by the test suite, the smoke check and the benchmark's CPU-baseline leg.
The CUDA library never imports it.
"""
