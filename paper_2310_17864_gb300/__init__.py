"""GB300-native CTC forced alignment (Viterbi over the CTC trellis).

The compute path is the CUDA library ``libalign.so`` built from ``csrc/`` and
reached through the C ABI declared in ``include/align.h``; ``align`` is the thin
ctypes binding. ``synth`` generates seeded synthetic inputs. Importing this
package loads nothing: the library is loaded on first use of ``align``.
"""
__all__ = ["align", "synth"]
