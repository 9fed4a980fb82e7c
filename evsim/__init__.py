"""Seeded synthetic event-camera streams.

This package only simulates a sensor: it renders a moving log-intensity scene and
emits an event whenever a pixel's log intensity has moved by the contrast
threshold C since its last event.  It holds none of the reconstruction method's
arithmetic and is the one module that both the FP64 oracle tests and the CUDA
path draw their inputs from.
"""
from .events import EventStream, simulate, packets
from .configs import CONFIGS, StreamConfig, make_stream

__all__ = ["EventStream", "simulate", "packets", "CONFIGS", "StreamConfig", "make_stream"]
