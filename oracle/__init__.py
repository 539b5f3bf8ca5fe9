"""FP64 CPU oracle for the H(curl) V-cycle of arXiv 2205.05840.

Test infrastructure, not product code: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` may
import it.  It is written from the paper (Sec. 2 and Sec. 3) and shares no
code, tables or constants with the CUDA library.

Parity unpinned: ``mg.Smoother(kind="edge")`` (edge-based smoother, eq.
Preconditioner E) is pinned only by invariants (symmetry, the interior
eigenmode, contraction < 1), not by the paper's Table 1.
"""
from . import hcurl, mg  # noqa: F401
