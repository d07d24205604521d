"""GB300-native EMPSO fitness evaluation (arXiv 1905.12795).

The compute path lives in the CUDA shared library built from ``csrc/`` and
declared in ``include/empso.h``; :mod:`.binding` is the thin ctypes layer over
that C ABI and :mod:`.synth` draws seeded synthetic inputs.  Importing the
package loads nothing: the library is opened on first use of the binding and
raises if it has not been built.
"""
__all__ = ["binding", "synth"]
