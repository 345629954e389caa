"""KADABRA on GB300: adaptive-sampling betweenness centrality, sm_103a.

The compute path is ``libkadabra.so`` (CUDA kernels behind a C ABI declared
in ``include/kadabra.h``); ``paper_1604_08553_gb300.kadabra`` is its thin
ctypes binding.  ``paper_1604_08553_gb300.graphgen`` builds the seeded input
graphs.  Submodules load lazily so that the input generators stay usable on
hosts without a GPU.
"""

__all__ = ["graphgen", "kadabra"]
