"""FP64 CPU oracle for the DPM scoring path -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this package. It shares no
code with the CUDA library: it restates the paper's definitions in plain loops (``tdpm_oracle.c``), numpy
(``oracle.py``) and pure Python (``tiny.py``).
"""
