"""FP64 CPU oracle for the GIGA-Lens hot path (arXiv:2202.07663, Sec. 2.1-2.2).

TEST INFRASTRUCTURE ONLY. Importable by ``tests/``, the smoke check and the
CPU-baseline leg of ``bench.py``; never by the product package.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
