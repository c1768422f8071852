"""GB300-native echelle frame renderer (arXiv 2008.05858, Sec. 2.2 image simulator).

The compute path is the C-ABI library ``libe2e_render.so`` built from ``csrc/`` for
sm_103a; :mod:`paper_2008_05858_gb300.binding` is a thin ctypes layer over it, and
:mod:`paper_2008_05858_gb300.workloads` builds seeded synthetic optical models and spectra.
"""

__all__ = ["workloads"]
