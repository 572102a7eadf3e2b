"""tdpm: tensor-decomposed DPM scoring on GB300 (sm_103a).

Importing the package loads nothing native; ``paper_1707_03268_gb300.tdpm`` is the ctypes binding of the C-ABI library
and loads ``libtdpm.so`` on first use, failing loudly when it is missing.
"""
