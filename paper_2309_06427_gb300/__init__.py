"""sspcg: symmetric stair preconditioned CG for trajectory-optimisation Schur
systems on GB300 (sm_103a).

* ``problems``: seeded synthetic QP inputs (no method arithmetic).
* ``build``: compiles the CUDA library (``csrc/``) in-tree for sm_103a.
* ``sspcg``: Python binding of the C ABI in ``include/sspcg.h``; importing it
  needs torch and a built library, and fails loudly without one.
"""
__all__ = ["problems", "build", "sspcg"]
