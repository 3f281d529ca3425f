"""GB300-native spin-polarized XL-BOMD hot path (arXiv 2303.03529).

workload.py  seeded synthetic inputs (no method arithmetic)
sxl.py       ctypes binding of the C-ABI library libsxl.so (csrc/)
"""
