"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests."""
from .kikuchi import *  # noqa: F401,F403
