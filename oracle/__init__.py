"""FP64 reference implementation of the SBS chemical stage and its fixed points:
``sbs`` (the step-by-step stage), ``homogeneous`` (the beam-off stage of the rate
equations), ``kinetics`` (the rate equations in concentrations) and ``gillespie`` (a
well-mixed stochastic simulation for the volume-scaling study).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.
"""
