"""The oracle's results do not depend on the number of host threads.

hb_oracle.c runs the contraction of Eq. 8 over fixed chunks of bra
determinants (their count does not depend on the thread count), merged in chunk
order; every other parallel loop writes disjoint outputs.  So the whole matrix,
its condition scales and the sampled-element path give the same bits with 1, 2
or 5 OpenMP threads.  Each thread count runs in its own process (OpenMP reads
OMP_NUM_THREADS once)."""
import hashlib
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, {root!r})
from oracle import coracle
from paper_1709_03005_gb300 import synth
P = synth.make_tiny(611, n_to=10, n_co=6, n_elec=4, n_det=140, n_groups=2, n_state=[3, 2],
                    cont_ranges=[(0, 6), (1, 4)], n_l2=20, e_core=-2.5)
o = coracle.Oracle(P)
h = hashlib.sha256()
h.update(o.dense().tobytes())
h.update(np.ascontiguousarray(o.condition(full=True)).tobytes())
print(h.hexdigest())
"""


def _digest(threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-c", _SCRIPT.format(root=ROOT)], env=env, check=True,
                         capture_output=True, text=True, timeout=600)
    return out.stdout.strip().splitlines()[-1]


def test_oracle_bits_independent_of_thread_count():
    digests = {t: _digest(t) for t in (1, 2, 5)}
    assert len(set(digests.values())) == 1, digests
