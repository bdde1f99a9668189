"""Compute-based point-cloud rendering on GB300 (sm_103a).

The product is the CUDA library libpcr.so behind the C interface in
include/pcr.h; ``paper_2104_07526_gb300.pcr`` is its Python binding and
``paper_2104_07526_gb300.scenes`` makes seeded synthetic inputs.
"""
