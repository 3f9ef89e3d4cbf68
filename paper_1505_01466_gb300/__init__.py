"""GB300-native batched list-CRC decoding of polar codes over an unrolled
Fast-SSC decoding tree ("Fast List Decoders for Polar Codes", Sarkis, Giard,
Vardy, Thibeault, Gross).

The decoder lives in the C-ABI library ``libpolar_gb300.so`` (CUDA, sm_103a);
``paper_1505_01466_gb300.polar`` is a thin ctypes binding over it. The
``inputs`` submodule generates seeded synthetic codes and channel LLRs.
"""

__all__ = ["inputs", "polar"]
