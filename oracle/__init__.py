"""FP64 CPU oracle of the NOLSM hot path -- test infrastructure only.

Importable only from ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.
The GPU library neither imports nor links anything here.
"""
from . import nolsm_oracle, mlp_oracle, combine_oracle, inverse_oracle  # noqa: F401
