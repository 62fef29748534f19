"""GB300-native backward-Euler Richards solver (arXiv 2112.05051 method).

The compute path lives in a C-ABI shared library built from ``csrc/`` (CUDA
for sm_103a); ``richards`` is its thin ctypes binding.  Importing this
package loads nothing: the library is loaded on first use of the binding.
"""
