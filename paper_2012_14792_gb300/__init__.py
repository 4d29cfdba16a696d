"""GB300 library for dynamic tile / rectangular-slice (TRS) VVC frame
partitioning (Amestoy et al., "Quality-driven Dynamic VVC Frame Partitioning
for efficient Parallel Processing", ICIP 2020).

The hot path -- per-CTU texture map, region tables, the two-step exact search
and the decoding of the chosen partition -- runs in hand-written CUDA kernels
for sm_103a behind the C ABI of ``include/trs.h``; ``trs`` is its Python
binding and ``runtime`` a small torch-facing helper that owns device tensors.
"""

__all__ = ["build", "trs"]
