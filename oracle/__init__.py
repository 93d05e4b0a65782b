"""FP64 reference implementation of the SBS chemical stage and its fixed points.

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.
"""
