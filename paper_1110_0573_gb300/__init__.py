"""GB300 (sm_103a) CUDA library for the QuTiP paper's open-system solvers.

* ``paper_1110_0573_gb300.qt``: the binding of libqt's C ABI (include/qt.h):
  qt_mesolve, qt_mcsolve, qt_expect and the device-resident System.
* ``paper_1110_0573_gb300.systems``: operator library and the synthetic
  systems shaped like the paper's examples (inputs only).
* ``paper_1110_0573_gb300.build``: compiles libqt.so in-tree with nvcc.
"""
