"""GB300-native Gauss-Newton hot path for sparse polynomial systems in complex
double, double double and quad double arithmetic (after Verschelde & Yu,
"GPU acceleration of Newton's method for large systems of polynomial
equations in double double and quad double arithmetic", 2014).

* ``paper_1402_2626_gb300.gn``     - binding of the C ABI (include/gn.h)
* ``paper_1402_2626_gb300.inputs`` - seeded synthetic workloads
* ``paper_1402_2626_gb300.build``  - in-tree nvcc build of libgn.so
"""

__all__ = ["gn", "inputs", "build"]
