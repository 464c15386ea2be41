"""A plan read back from a plan file (sht_plan_load) runs on the device with
outputs identical to the plan that wrote it, and matches the oracle; at the
bench configuration the file replaces the whole factorization."""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


def synth(sht, P, prec, beta):
    l = P.l
    dt = torch.complex64 if prec == 1 else torch.complex128
    b = torch.from_numpy(beta).to(dt).cuda()
    G = torch.full((2 * l, 2 * l), float("nan"), dtype=dt, device="cuda")
    sht.sht_legendre_synthesize(P, prec, b, G)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    return G.cpu().numpy()


def test_loaded_plan_outputs_are_identical(sht, tmp_path):
    l = 128
    P = sht.Plan(l, 1e-12, leaf_cols=16)
    P.prepare(1)
    path = str(tmp_path / "l128.plan")
    P.save(path)
    Q = sht.Plan.load(path)
    beta = inputs.random_beta(l, seed=21)
    for prec in (0, 2, 1):
        a, b = synth(sht, P, prec, beta), synth(sht, Q, prec, beta)
        assert np.array_equal(a, b), prec
    Go = oracle.legendre_synthesis(beta, l)
    assert np.linalg.norm(synth(sht, Q, 0, beta) - Go) / np.linalg.norm(Go) < 1e-10
    P.close()
    Q.close()


def test_bench_configuration_from_a_plan_file(sht, tmp_path):
    l = 1024
    path = str(tmp_path / "l1024.plan")
    P = sht.Plan(l, 1e-12, leaf_cols=32, device_build=True, plan_cache=path)
    Q = sht.Plan(l, 1e-12, leaf_cols=32, plan_cache=path)
    assert Q.stats()["t_factor"] == 0.0
    beta = inputs.random_beta(l, seed=3, decay=True)
    assert np.array_equal(synth(sht, P, 0, beta), synth(sht, Q, 0, beta))
    P.close()
    Q.close()
