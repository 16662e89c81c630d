"""GB300-native Kerr photon tracer (backward RK4 on null geodesics in
Boyer-Lindquist coordinates), after Chan, Psaltis & Ozel 2013 ("GRay").

The compute path is the CUDA library ``libgray.so`` (C ABI, ``include/gray.h``);
``paper_1303_5057_gb300.gray`` is its thin ctypes binding.  Importing this
package loads nothing; the library is loaded on first use and a missing
library is an error, never a fallback.
"""
__all__ = ["gray", "inputs"]
