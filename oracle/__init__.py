"""FP64 CPU oracle for the CPQR -> ID -> CUR method of Voronin & Martinsson,
"Efficient Algorithms for CUR and Interpolative Matrix Decompositions".

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the paper in numpy float64.  It exists to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The library in
``paper_1412_8447_gb300`` never imports it and shares no code with it.

Pinning status of every function is stated in its docstring; each one is
pinned by the CPU tests in ``tests/test_oracle_pins.py`` against values fixed by
the paper's identities, library routines, closed forms or brute force.
"""
from .curid_oracle import *  # noqa: F401,F403
from .curid_oracle import __all__  # noqa: F401
