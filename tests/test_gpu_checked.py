"""The checked diagnostic build of the library (-DWADG_CHECKED).

In that build the stage kernels check the indices of their scattered reads
(neighbour element, face code, neighbour face node) before using them; a
violation is recorded in the context's status word, the read is skipped and
the stepping call reports it.  This test builds the variant and, in a
separate process (the library is loaded once per process; WADG_LIB selects
the build), runs one-stage parity cases against the oracle in every
precision plus a few full steps: no check may fire and the results must
match the oracle as closely as the normal build's do."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
from paper_2006_02551_gb300 import wadg
assert wadg.LIB_PATH.endswith("libwadg_checked.so"), wadg.LIB_PATH
from oracle import lserk
from synthetic import PmlProfile
from tests.parity_util import make_pair, random_states, to_lib

PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
for precision, N, bound in (("fp64", 3, 1e-10), ("fp32", 3, 1e-4),
                            ("tf32", 4, 1e-2), ("bf16", 4, 3e-2)):
    s, sim, mask = make_pair(N, 3, 0.15, 4, PML3, precision, n_batch=2)
    st = random_states(sim.K, sim.Np, 2, 11, mask)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t = 0.01, 0.37
    s.rk_stage(1, t, dt)                 # raises if an index check fired
    q, _ = s.get_state()
    for b in range(2):
        rhs = sim.rhs(st[b], t + lserk.RK_C[1] * dt, b)
        for f in st[b]:
            st[b][f] = st[b][f] + lserk.RK_B[1] * dt * rhs[f]
    ref = to_lib(st)
    sel = np.ones(ref.shape[:3], bool)
    sel[:, ~mask, 6:] = False
    err = np.linalg.norm((q - ref)[sel]) / np.linalg.norm((ref - q0)[sel])
    assert err < bound, (precision, err)
    s.run_steps(3, s.stable_dt(0.5))     # raises if an index check fired
    s.close()
    print(precision, err)
print("checked build ok")
'''


def test_checked_build_runs_clean():
    from paper_2006_02551_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, WADG_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked build ok" in r.stdout, r.stdout + r.stderr
