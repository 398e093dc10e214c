"""GB300-native multigrid pressure-Poisson solver (Neural Physics hot path).

The compute path is the C-ABI library ``libnpmg.so`` built from ``csrc/``;
``paper_2402_17913_gb300.lib`` is its thin ctypes binding.  Importing this
package does not load the library; ``lib.load()`` does, and raises if it has
not been built.
"""
