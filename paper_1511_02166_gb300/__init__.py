"""Batched 2D constant-strength vortex panel solver for GB300 (sm_103a).

The compute path is the C-ABI library built from ``csrc/`` (see
``include/panel.h``); ``binding`` marshals torch device tensors into it.
Importing this package loads nothing native; the library is loaded on the
first call and a missing library is an error, never a CPU fallback.
"""
__all__ = ["inputs"]
