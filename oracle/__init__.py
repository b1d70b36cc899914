"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct CPU statement of what the sparse-permanent
path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path (the CUDA
library and its binding) never imports, calls or links anything here, and
nothing here imports the product path.

Contents, each following a passage of the paper (arXiv 1112.6072):

* ``per_bruteforce``   -- Eq. 1, the sum over all permutations (n <= 9).
* ``per_ryser_py``     -- Ryser's formula (Section 1) in Python integers.
* ``ryser`` / ``permanent`` / ``jobs`` / ``job_permanents`` -- the C oracle
  (``hybrid.c``): Algorithm H_per with the expansion of Eq. 2 (Section 2.1),
  the level-by-level pre-expansion of Algorithm PH, Step 2 (Section 2.2),
  exact big-integer results.
* ``kklll`` helpers    -- Algorithm KKLLL (Section 2.3) in fp64 with a
  counter-based SplitMix64 stream.
* ``schedule``         -- list scheduling LS / LPT (Section 2.4) and the
  parallel efficiency T1 / (m Tm) of Tables T5-T17.
* ``kendall_tau_b``    -- Eq. 7-10 (Section 3.2).
* ``mlp``              -- fp64 forward and backward of the job-cost network.
"""
from __future__ import annotations

from .exact import (  # noqa: F401
    per_bruteforce,
    per_ryser_py,
    ryser,
    permanent,
    jobs,
    job_permanents,
    rowcol_bound,
    bregman_bound,
    schrijver_lower_bound,
)
from .kklll import (  # noqa: F401
    splitmix64_mix,
    kklll_choice,
    kklll_log_ap,
    kklll_trial_log_abs2,
    det_partial_pivot,
    kklll_exact_mean,
)
from .schedule import (  # noqa: F401
    list_schedule,
    lpt_order,
    efficiency,
    kendall_tau_b,
)
