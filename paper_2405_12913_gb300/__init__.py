"""GB300 (sm_103a) hot path of Hamiltonian ray tracing (HRT, arXiv 2405.12913).

``hrt`` is the ctypes binding of ``libhrt.so`` (built in-tree by ``build.build()``); ``configs`` holds the
workload definitions.  Importing ``hrt`` requires the built library.
"""
__all__ = ["configs"]
