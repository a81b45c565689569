"""Plain FP64 CPU oracle for the IMEX RK / SDC incompressible-flow method.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
restatement of what the paper defines, written from the paper and sharing no
code with the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the library under ``paper_2112_04167_gb300/`` never does.
"""
