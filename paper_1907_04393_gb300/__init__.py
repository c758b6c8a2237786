"""GB300-native hand-isolation path of arXiv 1907.04393 (Magoules & Zou).

The compute lives in ``libhmi.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/hmi.h``); ``paper_1907_04393_gb300.hmi`` is its Python binding.
``paper_1907_04393_gb300.synth`` makes seeded synthetic camera frames.
"""
__all__ = ["hmi", "synth", "build"]
