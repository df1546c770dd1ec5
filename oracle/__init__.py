"""FP64 CPU oracle for the HipFT surface-flux-transport (SFT) time step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously
correct restatement of the paper's method (Caplan et al., "Open-source Flux
Transport I. HipFT"), used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product library (``paper_2501_06377_gb300``) never imports
it and shares no code with it.

Every function cites the section / equation of the paper it restates.
Pins for each function live in ``tests/test_oracle_*.py``.
"""
from .sft_oracle import *  # noqa: F401,F403
