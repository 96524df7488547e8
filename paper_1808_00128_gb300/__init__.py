"""GB300-native low-rank stabilizer-decomposition simulator.

The compute path lives in the C-ABI library ``liblrstab.so`` (CUDA, sm_103a);
``paper_1808_00128_gb300.lrstab`` is its thin ctypes binding.  Importing this
package loads nothing: the library is opened on first use of the binding.
"""
__all__ = ["workloads"]
