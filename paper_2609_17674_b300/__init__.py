"""B300-native transdimensional SMC hot path (Demasi & Del Pozzo).

The compute path is the CUDA library ``libtsmc.so`` behind the C ABI declared
in ``include/tsmc.h``; ``capi`` is its thin ctypes binding.  Importing this
package loads nothing; ``capi.lib()`` loads the library and fails loudly when
it is missing.
"""
__all__ = ["capi", "synth"]
