"""Tile-wise LISI / augLISI IQA maps (arxiv 2501.10653) on GB300.

The compute path is the C-ABI library ``libiqa.so`` (hand-written CUDA for
sm_103a, declared in ``include/iqa.h``); ``paper_2501_10653_gb300.iqa`` is its
thin ctypes binding.  ``synth`` generates seeded synthetic sky pairs.
Importing this package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""
__all__ = ["iqa", "synth", "build"]
