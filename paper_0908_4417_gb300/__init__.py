"""GB300-native finite-size pencil beam D_ij engine.

``paper_0908_4417_gb300.dsc`` binds the C-ABI library ``libdsc.so`` (built
from ``csrc/`` for sm_103a); ``paper_0908_4417_gb300.phantoms`` generates the
seeded synthetic inputs.  Importing the package loads neither.
"""
