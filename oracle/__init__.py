"""Plain CPU oracle of the 3-D Yee leapfrog sweep (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library under
``paper_1301_4539_gb300`` never does, and shares no code with it.
"""

from .oracle import (  # noqa: F401
    C0,
    EPS0,
    OracleGrid,
    build,
    cfl_dt,
    load,
    round24,
    waveform,
)
