"""GB300-native Pauli-frame Monte Carlo sampler for distributed transversal
QEC operations (arXiv 2504.05611).

Submodules:
  * ``circuits`` -- circuit generator (codes, protocols, noise); pure Python.
  * ``tmcs``     -- ctypes binding of the CUDA library ``libtmcs.so``.

Importing the package loads nothing native; ``tmcs`` loads the library on
first use and raises if it is missing.
"""

__version__ = "0.1.0"
