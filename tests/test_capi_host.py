"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host-built reference operators agree with the
oracle's independent construction (no device work)."""
import os
import re

import numpy as np
import pytest

from oracle.refelem import RefElement

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_02551_gb300 import build
    build.build()
    from paper_2006_02551_gb300 import wadg
    return wadg.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wadg.h")).read()
    return sorted(set(re.findall(r"\b(wadg_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2006_02551_gb300 import wadg
    assert sorted(wadg.exported_symbols()) == declared_symbols()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_host_operators_match_oracle(lib, N):
    from paper_2006_02551_gb300 import reference_operator
    re_ = RefElement(N)
    Np, Nfp, Nq = re_.Np, re_.Nfp, re_.Nq
    cases = [(0, re_.Dr), (1, re_.Ds), (2, re_.Dt), (3, re_.LIFT), (4, re_.Vq),
             (5, re_.Pq), (7, re_.Minv),
             (6, np.stack([re_.rq, re_.sq, re_.tq, re_.wq], axis=1))]
    for which, ref in cases:
        got = reference_operator(N, which).reshape(ref.shape)
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err < 1e-13, (which, err)


def test_bad_order_rejected(lib):
    from paper_2006_02551_gb300 import wadg
    with pytest.raises(wadg.WadgError) as e:
        wadg.reference_operator(9, 0)
    assert e.value.status == wadg.WADG_EINVAL


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2006_02551_gb300 import wadg
    with pytest.raises(wadg.WadgError) as e:
        wadg.Solver(3)
    assert e.value.status == wadg.WADG_ECUDA
