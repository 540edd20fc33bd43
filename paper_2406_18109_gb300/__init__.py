"""GB300-native task and kernel fusion (the hot path of Diffuse, arXiv 2406.18109).

  * ``binding``   -- ctypes binding of the C-ABI declared in include/diffuse.h
  * ``arrays``    -- NumPy-style front end issuing index tasks to the runtime
  * ``workloads`` -- Black-Scholes, CG, the Fig. 1 stencil and BiCGSTAB written
                     on the front end
  * ``_build``    -- builds the in-tree shared library for sm_103a
"""
from . import binding  # noqa: F401

__all__ = ["binding", "arrays", "workloads"]
