"""GB300-native Euclidean distance similarity self-join (grid index + distance
tiles as ||a||^2 + ||b||^2 - 2 a.b, FP64 and certified low-precision filter).

The compute path is the CUDA library ``libsj`` (C ABI, ``include/simjoin.h``);
``paper_2209_11287_gb300.binding`` marshals arguments to it.  Importing this
package does not load the library; ``binding`` does, and fails loudly when it
is missing.
"""

__all__ = ["binding", "workloads"]
