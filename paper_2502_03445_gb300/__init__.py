"""GB300-native cut-network reconstruction (TensorQC's classical hot path).

The compute path is libtqc.so (hand-written sm_103a kernels behind the C ABI
in include/tqc.h); :mod:`.tqc` is its ctypes binding."""
from . import tqc  # noqa: F401
