"""Incremental betweenness centrality on GB300 (Nasre, Pontecorvi, Ramachandran).

The compute path lives in the CUDA library ``libbcgpu.so`` (sources under ``csrc/``,
C-ABI in ``include/bcgpu.h``); ``binding`` marshals arguments to it.  ``synth`` draws
seeded synthetic graphs and update streams.  Importing the package loads nothing.
"""
