"""GB300-native line-opacity, ODF and spectrum synthesis (MPS-ATLAS hot path).

The compute runs in the sm_103a CUDA library ``_lib/libmpsa.so`` behind the C ABI
declared in ``include/mpsa.h``; ``binding`` marshals numpy arrays and torch CUDA
tensors into those calls.  Importing this package does not load the library;
``binding.Context`` does, and raises if it is missing (there is no CPU path).
"""
__all__ = ["binding"]
